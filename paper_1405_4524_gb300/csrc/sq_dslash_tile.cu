// G1, halo-tiled: the even-odd clover-Wilson hop (+ A^-1, xpay, fused
// reductions) for FP32 and FP16 (per-site norm) fields, with every source's
// input spinors staged in shared memory by bulk copies.
//
// Work unit = one site tile of the output parity times a group of source
// slots. The tile holds all X/2 checkerboard sites of by x bz x bt rows
// (y, z, t), one thread per output site. A thread keeps its eight
// reconstruct-12 links (the forward links of its site and the backward links
// of its four lower neighbours) and its two clover-inverse blocks in
// registers for the whole group, so the gauge data of a tile comes from HBM
// once per group. For every source of the group the tile's input spinors
// plus their y, z, t halo rows (each contiguous in the checkerboard order,
// x being complete inside the tile) are copied into a shared-memory ring
// with cp.async.bulk on an mbarrier transaction count; the copies of the
// next source(s) run while the current one is computed, and every neighbour
// spinor is read from shared memory instead of through L2 once per
// neighbouring site.
//
// Shared-memory rows of one source buffer (compact, in this order):
//   A: t in [t0, t0+bt), z in [z0, z0+bz), y in [y0-hy, y0+by-1+hy]
//   B: t in [t0, t0+bt), z in {z0-1, z0+bz},  y in [y0, y0+by)     (if hz)
//   C: t in {t0-1, t0+bt}, z in [z0, z0+bz),  y in [y0, y0+by)     (if ht)
// (hy, hz, ht: 1 when the tile is shorter than the lattice in y, z, t; a
// tile that spans a dimension wraps inside itself). One buffer holds the
// chunk planes [NC][S] of S = rows * X/2 sites (16 bytes per site and
// chunk) and, for FP16, the S site norms.
//
// Every wait on the ring is bounded: a timeout sets ERRBIT_TIMEOUT in the
// context's error word, the CTA waits (bounded) for the copies it issued
// and returns.
#include <cstdio>
#include <cstring>

#include "sq_async.cuh"
#include "sq_hop.cuh"
#include "sq_internal.h"

namespace sq {

constexpr int kTileMaxThreads = 256;
constexpr int kTileMaxSlots = 512;  // row segments of a tile (fixed slots)
constexpr int kTileBarBytes = 64;   // ring barriers (<= 3), a never-completed one at byte 56
constexpr long long kTileWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

struct TileArgs {
  Geom g;
  Field out, in, x, r1;
  const void* links;  // FP32 reconstruct-12
  const void* clov;   // FP32 A^-1 blocks
  int p_out;
  float a;            // xpay coefficient
  const int* list;
  const int* count;
  int n;
  int by, bz, bt;       // tile rows in y, z, t
  int nty, ntz;         // tiles along y and z
  int ngroups, sg;      // source groups per tile, source slots per group
  int nbuf;             // ring depth (2 or 3)
  int hy, hz, ht;       // halo rows needed in y, z, t
  int nyA, NA, NB;      // region A rows per (t, z); rows of regions A and B
  int nslot;            // segment slots: 3 bt bz (A) + 2 bt (B) + 2 bz (C)
  int S;                // staged sites per source buffer
  uint32_t buf_bytes;   // bytes of one source buffer = bytes copied per source
  long long wait_cycles;
  int stall;            // test: first wait on a barrier that nothing completes
  RedArgs ra;
  int* err;
};

// compact row of region A for (tr, zr, yy), yy in [-hy, by - 1 + hy]
__device__ __forceinline__ int rowA(const TileArgs& a, int tr, int zr, int yy) {
  return (tr * a.bz + zr) * a.nyA + yy + a.hy;
}

// Segment slot q -> (first compact row, rows, first global row index
// y + Y (z + Z t)); rows = 0 for an unused slot. Region A rows of one (t, z)
// split at the y wrap into at most three contiguous runs.
__device__ void tile_segment(const TileArgs& a, int y0, int z0, int t0, int q, int& srow, int& nrows, int& grow) {
  const Geom& g = a.g;
  nrows = 0;
  srow = 0;
  grow = 0;
  const int nA = 3 * a.bt * a.bz;
  if (q < nA) {
    const int pr = q / 3, piece = q - 3 * pr;
    const int tr = pr / a.bz, zr = pr - tr * a.bz;
    const int z = z0 + zr, t = t0 + tr;
    // runs of yy in [-hy, by-1+hy]: split where the global y wraps to 0
    int lo = -a.hy, hi = a.by - 1 + a.hy;
    int p = 0;
    int yy = lo;
    while (yy <= hi) {
      const int gy = (y0 + yy + g.Y) % g.Y;
      int len = 1;
      while (yy + len <= hi && (y0 + yy + len + g.Y) % g.Y == gy + len) len++;
      if (p == piece) {
        srow = rowA(a, tr, zr, yy);
        nrows = len;
        grow = gy + g.Y * (z + g.Z * t);
        return;
      }
      p++;
      yy += len;
    }
    return;
  }
  q -= nA;
  if (q < 2 * a.bt) {
    if (!a.hz) return;
    const int tr = q >> 1, side = q & 1;
    const int z = side ? (z0 + a.bz) % g.Z : (z0 - 1 + g.Z) % g.Z;
    srow = a.NA + (tr * 2 + side) * a.by;
    nrows = a.by;
    grow = y0 + g.Y * (z + g.Z * (t0 + tr));
    return;
  }
  q -= 2 * a.bt;
  if (q < 2 * a.bz) {
    if (!a.ht) return;
    const int side = q / a.bz, zr = q - side * a.bz;
    const int t = side ? (t0 + a.bt) % g.T : (t0 - 1 + g.T) % g.T;
    srow = a.NA + a.NB + (side * a.bz + zr) * a.by;
    nrows = a.by;
    grow = y0 + g.Y * (z0 + zr + g.Z * t);
  }
}

template <int P>
struct TileIO;

template <>
struct TileIO<P32> {
  static constexpr int NC = 6;
  static __device__ __forceinline__ float load(const unsigned char* buf, int S, int site, cx<float> v[12]) {
    const float4* p = (const float4*)buf + site;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 q = p[(size_t)c * S];
      v[2 * c] = mk(q.x, q.y);
      v[2 * c + 1] = mk(q.z, q.w);
    }
    return 1.0f;
  }
};

template <>
struct TileIO<P16> {
  static constexpr int NC = 3;
  // values as stored; returns the site norm (applied to the hop's result)
  static __device__ __forceinline__ float load(const unsigned char* buf, int S, int site, cx<float> v[12]) {
    const uint4* p = (const uint4*)buf + site;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint4 q = p[(size_t)c * S];
      const float2 e0 = h2f(q.x), e1 = h2f(q.y), e2 = h2f(q.z), e3 = h2f(q.w);
      v[4 * c + 0] = mk(e0.x, e0.y);
      v[4 * c + 1] = mk(e1.x, e1.y);
      v[4 * c + 2] = mk(e2.x, e2.y);
      v[4 * c + 3] = mk(e3.x, e3.y);
    }
    return ((const float*)(buf + (size_t)48 * S))[site];
  }
};

// reconstruct-12 link held as three float4 (rows 0, 1)
struct Link12 {
  float4 q[3];
};

__device__ __forceinline__ void load12(const void* base, int Vh, int p, int mu, int cb, Link12& u) {
  const float4* q = (const float4*)base + ((size_t)(p * 4 + mu) * 3) * Vh + cb;
#pragma unroll
  for (int c = 0; c < 3; c++) u.q[c] = __ldg(q + (size_t)c * Vh);
}

__device__ __forceinline__ void expand12(const Link12& s, Link<float>& u) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    u.e[2 * c] = mk(s.q[c].x, s.q[c].y);
    u.e[2 * c + 1] = mk(s.q[c].z, s.q[c].w);
  }
  reconstruct_row2(u);
}

// Warp 0 issues the bulk copies of source k into ring buffer b (lane 0
// first posts the byte count on the buffer's barrier).
template <int P>
__device__ __forceinline__ void tile_issue(const TileArgs& a, const int2* seg, unsigned char* ring, uint32_t bar, int k) {
  constexpr int NC = TileIO<P>::NC;
  constexpr int NCP = NC + (P == P16 ? 1 : 0);
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_expect_tx(bar, a.buf_bytes);
  __syncwarp();
  const int X2 = a.g.X2;
  const size_t Vh = (size_t)a.g.Vh;
  for (int q = lane; q < a.nslot * NCP; q += 32) {
    const int sl = q / NCP, c = q - sl * NCP;
    const int2 sg = seg[sl];
    const int nrows = sg.x >> 16, srow = sg.x & 0xFFFF;
    if (nrows == 0) continue;
    const size_t gcb = (size_t)sg.y * X2;
    if (c < NC) {
      const uint4* src = (const uint4*)a.in.data + ((size_t)k * NC + c) * Vh + gcb;
      bulk_load(smem_addr(ring + ((size_t)c * a.S + (size_t)srow * X2) * 16), src, (uint32_t)(nrows * X2 * 16), bar);
    } else {
      const float* src = a.in.norm + (size_t)k * Vh + gcb;
      bulk_load(smem_addr(ring + (size_t)NC * a.S * 16 + (size_t)srow * X2 * 4), src, (uint32_t)(nrows * X2 * 4), bar);
    }
  }
}

template <int P, int MU>
__device__ __forceinline__ void tile_hop(const unsigned char* buf, int S, int sf, int sb, const Link12& uf,
                                         const Link12& ub, float ff, float fb, cx<float> acc[12]) {
  {  // forward: (1 - g_mu) U_mu(x) psi(x + mu)
    cx<float> v[12], h[6], w[6];
    const float f = TileIO<P>::load(buf, S, sf, v) * ff;
    project<MU, -1>(v, h);
    Link<float> u;
    expand12(uf, u);
    mv(u, h, w);
    accum_f<MU, -1>(acc, w, f);
  }
  {  // backward: (1 + g_mu) U_mu(x - mu)^+ psi(x - mu)
    cx<float> v[12], h[6], w[6];
    const float f = TileIO<P>::load(buf, S, sb, v) * fb;
    project<MU, +1>(v, h);
    Link<float> u;
    expand12(ub, u);
    mv_dag(u, h, w);
    accum_f<MU, +1>(acc, w, f);
  }
}

template <int P, int CLOV, int XPAY, int FIN>
__global__ void __launch_bounds__(kTileMaxThreads, 1) k_dslash_tile(const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr int NRED = FIN == FIN_ALPHA ? 2 : FIN == FIN_OMEGA ? 3 : 1;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int grp = blockIdx.x % a.ngroups;
  const int tile = blockIdx.x / a.ngroups;
  const int cnt = a.list ? *a.count : a.n;
  const int s0 = grp * a.sg;
  if (s0 >= cnt) return;  // uniform in the CTA
  const int ns = min(cnt, s0 + a.sg) - s0;

  uint64_t* bars = (uint64_t*)sm;
  int2* seg = (int2*)(sm + kTileBarBytes);
  unsigned char* ring = sm + kTileBarBytes + 8 * kTileMaxSlots;

  // tile origin
  const int tt = tile / (a.nty * a.ntz);
  const int rem = tile - tt * a.nty * a.ntz;
  const int tz = rem / a.nty, ty = rem - tz * a.nty;
  const int y0 = ty * a.by, z0 = tz * a.bz, t0 = tt * a.bt;

  if (tid == 0) {
    for (int b = 0; b < a.nbuf; b++) mbar_init(smem_addr(bars + b), 1);
    mbar_init(smem_addr(bars + 7), 1);  // nothing arrives on it
    mbar_init_fence();
  }
  for (int q = tid; q < a.nslot; q += blockDim.x) {
    int srow, nrows, grow;
    tile_segment(a, y0, z0, t0, q, srow, nrows, grow);
    seg[q] = make_int2(srow | (nrows << 16), grow);
  }
  __syncthreads();
  // prefetch the first nbuf - 1 sources
  if (warp == 0)
    for (int i = 0; i < a.nbuf - 1 && i < ns; i++)
      tile_issue<P>(a, seg, ring + (size_t)i * a.buf_bytes, smem_addr(bars + i),
                    a.list ? a.list[s0 + i] : s0 + i);

  // this thread's output site
  const int X2 = g.X2;
  const int xh = tid % X2;
  int r = tid / X2;
  const int yr = r % a.by;
  r /= a.by;
  const int zr = r % a.bz, tr = r / a.bz;
  const int y = y0 + yr, z = z0 + zr, t = t0 + tr;
  const int cb = xh + X2 * (y + g.Y * (z + g.Z * t));
  const int bpar = (y + z + t + a.p_out) & 1;  // x = 2 xh + bpar
  // neighbour sites in the staged buffer
  const int own = rowA(a, tr, zr, yr);
  int sn[8];
  sn[0] = own * X2 + (bpar ? (xh + 1) % X2 : xh);       // x + 1
  sn[1] = own * X2 + (bpar ? xh : (xh - 1 + X2) % X2);  // x - 1
  sn[2] = (a.hy ? rowA(a, tr, zr, yr + 1) : rowA(a, tr, zr, (yr + 1) % a.by)) * X2 + xh;
  sn[3] = (a.hy ? rowA(a, tr, zr, yr - 1) : rowA(a, tr, zr, (yr - 1 + a.by) % a.by)) * X2 + xh;
  {
    int rz;
    if (zr + 1 < a.bz) rz = rowA(a, tr, zr + 1, yr);
    else if (a.hz) rz = a.NA + (tr * 2 + 1) * a.by + yr;
    else rz = rowA(a, tr, 0, yr);
    sn[4] = rz * X2 + xh;
    if (zr > 0) rz = rowA(a, tr, zr - 1, yr);
    else if (a.hz) rz = a.NA + (tr * 2 + 0) * a.by + yr;
    else rz = rowA(a, tr, a.bz - 1, yr);
    sn[5] = rz * X2 + xh;
    int rt;
    if (tr + 1 < a.bt) rt = rowA(a, tr + 1, zr, yr);
    else if (a.ht) rt = a.NA + a.NB + (1 * a.bz + zr) * a.by + yr;
    else rt = rowA(a, 0, zr, yr);
    sn[6] = rt * X2 + xh;
    if (tr > 0) rt = rowA(a, tr - 1, zr, yr);
    else if (a.ht) rt = a.NA + a.NB + (0 * a.bz + zr) * a.by + yr;
    else rt = rowA(a, a.bt - 1, zr, yr);
    sn[7] = rt * X2 + xh;
  }
  const float ftp = (t == g.T - 1) ? (float)g.tbc : 1.0f;  // time-boundary signs
  const float ftm = (t == 0) ? (float)g.tbc : 1.0f;

  // gauge data of this site, kept for the whole source group
  Link12 uf[4], ub[4];
  {
    const int x = 2 * xh + bpar;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      load12(a.links, g.Vh, a.p_out, mu, cb, uf[mu]);
      int nx = x, ny = y, nz = z, nt = t;
      if (mu == 0) nx = (x - 1 + g.X) % g.X;
      else if (mu == 1) ny = (y - 1 + g.Y) % g.Y;
      else if (mu == 2) nz = (z - 1 + g.Z) % g.Z;
      else nt = (t - 1 + g.T) % g.T;
      load12(a.links, g.Vh, 1 - a.p_out, mu, cb_of(g, nx, ny, nz, nt), ub[mu]);
    }
  }
  float blk0[36], blk1[36];
  if (CLOV) {
    CloverIO<P32>::template load_block<0>(a.clov, g.Vh, a.p_out, cb, blk0);
    CloverIO<P32>::template load_block<1>(a.clov, g.Vh, a.p_out, cb, blk1);
  }

  for (int i = 0; i < ns; i++) {
    const int b = i % a.nbuf;
    bool ok = !(a.stall && i == 0) || mbar_wait_bounded(smem_addr(bars + 7), 0u, a.wait_cycles);
    ok = ok && mbar_wait_bounded(smem_addr(bars + b), (uint32_t)((i / a.nbuf) & 1), a.wait_cycles);
    if (__syncthreads_or(!ok)) {
      // a copy did not land in time: record it, let the issued copies
      // drain (bounded) and stop
      if (tid == 0) {
        atomicOr(a.err, ERRBIT_TIMEOUT);
        const int issued = min(ns, i + a.nbuf - 1);
        for (int j = i; j < issued; j++)
          mbar_wait_bounded(smem_addr(bars + (j % a.nbuf)), (uint32_t)((j / a.nbuf) & 1), kTileWaitCycles);
      }
      return;
    }
    // the buffer of source i - 1 is free (every thread passed the barrier)
    if (warp == 0 && i + a.nbuf - 1 < ns) {
      const int j = i + a.nbuf - 1;
      tile_issue<P>(a, seg, ring + (size_t)(j % a.nbuf) * a.buf_bytes, smem_addr(bars + (j % a.nbuf)),
                    a.list ? a.list[s0 + j] : s0 + j);
    }
    const int k = a.list ? a.list[s0 + i] : s0 + i;
    const unsigned char* buf = ring + (size_t)b * a.buf_bytes;
    cx<float> acc[12];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[j] = zero<float>();
    tile_hop<P, 0>(buf, a.S, sn[0], sn[1], uf[0], ub[0], 1.0f, 1.0f, acc);
    tile_hop<P, 1>(buf, a.S, sn[2], sn[3], uf[1], ub[1], 1.0f, 1.0f, acc);
    tile_hop<P, 2>(buf, a.S, sn[4], sn[5], uf[2], ub[2], 1.0f, 1.0f, acc);
    tile_hop<P, 3>(buf, a.S, sn[6], sn[7], uf[3], ub[3], ftp, ftm, acc);
    if (CLOV) {
      cx<float> w[6];
      herm6_apply(blk0, acc, w);
#pragma unroll
      for (int j = 0; j < 6; j++) acc[j] = w[j];
      herm6_apply(blk1, acc + 6, w);
#pragma unroll
      for (int j = 0; j < 6; j++) acc[6 + j] = w[j];
    }
    cx<float> xv[12];
    if (XPAY) {
      SpinorIO<P>::load(a.x, k, cb, xv);
#pragma unroll
      for (int j = 0; j < 12; j++) acc[j] = mk(fmaf(a.a, acc[j].re, xv[j].re), fmaf(a.a, acc[j].im, xv[j].im));
    }
    SpinorIO<P>::store(a.out, k, cb, acc);
    if (FIN != FIN_NONE) {
      typedef SumOf<float>::T S;
      S red[NRED];
      if (FIN == FIN_ALPHA) {  // <r1, out>
        cx<float> rv[12];
        SpinorIO<ShadowPrec<P>::value>::load(a.r1, k, cb, rv);
        S sr = 0, si = 0;
#pragma unroll
        for (int j = 0; j < 12; j++) {
          sr += (S)rv[j].re * acc[j].re + (S)rv[j].im * acc[j].im;
          si += (S)rv[j].re * acc[j].im - (S)rv[j].im * acc[j].re;
        }
        red[0] = sr;
        red[1] = si;
      } else if (FIN == FIN_OMEGA) {  // <out, x>, <out, out>
        S sr = 0, si = 0, q2 = 0;
#pragma unroll
        for (int j = 0; j < 12; j++) {
          sr += (S)acc[j].re * xv[j].re + (S)acc[j].im * xv[j].im;
          si += (S)acc[j].re * xv[j].im - (S)acc[j].im * xv[j].re;
          q2 += (S)acc[j].re * acc[j].re + (S)acc[j].im * acc[j].im;
        }
        red[0] = sr;
        red[1] = si;
        red[2] = q2;
      } else {
        S q2 = 0;
#pragma unroll
        for (int j = 0; j < 12; j++) q2 += (S)acc[j].re * acc[j].re + (S)acc[j].im * acc[j].im;
        red[0] = q2;
      }
      warp_partials<NRED>(a.ra, red, k, tile * (int)(blockDim.x >> 5) + warp);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TilePlan {
  bool ok = false;
  int threads = 0;
  int nty = 0, ntz = 0, ntt = 0, ntiles = 0;
  int hy = 0, hz = 0, ht = 0, nyA = 0, NA = 0, NB = 0, NCr = 0, rows = 0, S = 0, nslot = 0;
  uint32_t buf_bytes = 0;
  size_t smem = 0;
};

static TilePlan tile_plan(const sq_ctx* c, int prec, const Shape& sh) {
  TilePlan p;
  const int X2 = c->dims[0] / 2, Y = c->dims[1], Z = c->dims[2], T = c->dims[3];
  const int by = sh.by, bz = sh.bz, bt = sh.bt;
  if (by <= 0 || bz <= 0 || bt <= 0 || Y % by || Z % bz || T % bt) return p;
  p.threads = X2 * by * bz * bt;
  if (p.threads > kTileMaxThreads || p.threads % 32) return p;
  if (prec == P16 && X2 % 4) return p;  // 16-byte norm rows
  if (sh.nbuf < 2 || sh.nbuf > 3 || sh.sg <= 0) return p;
  p.nty = Y / by;
  p.ntz = Z / bz;
  p.ntt = T / bt;
  p.ntiles = p.nty * p.ntz * p.ntt;
  p.hy = by < Y;
  p.hz = bz < Z;
  p.ht = bt < T;
  p.nyA = by + 2 * p.hy;
  p.NA = bt * bz * p.nyA;
  p.NB = p.hz ? 2 * bt * by : 0;
  p.NCr = p.ht ? 2 * bz * by : 0;
  p.rows = p.NA + p.NB + p.NCr;
  if (p.rows > 0xFFFF) return p;
  p.S = p.rows * X2;
  p.nslot = 3 * bt * bz + 2 * bt + 2 * bz;
  if (p.nslot > kTileMaxSlots) return p;
  p.buf_bytes = (uint32_t)((size_t)p.S * (prec == P16 ? 52 : 96));
  p.smem = kTileBarBytes + 8 * kTileMaxSlots + (size_t)sh.nbuf * p.buf_bytes;
  if (p.smem > 227 * 1024) return p;
  p.ok = true;
  return p;
}

bool tile_shape_ok(const sq_ctx* c, int prec, int recon, const Shape& sh) {
  if (prec != P32 && prec != P16) return false;
  if (recon != 12) return false;
  return tile_plan(c, prec, sh).ok;
}

template <int P, int CLOV, int XPAY, int FIN>
static void go_tile(const TileArgs& a, int grid, int threads, size_t smem, cudaStream_t s) {
  static int configured[64] = {0};  // per device: large dynamic shared memory allowed
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    cudaFuncSetAttribute(k_dslash_tile<P, CLOV, XPAY, FIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    configured[dev] = 1;
  }
  k_dslash_tile<P, CLOV, XPAY, FIN><<<grid, threads, smem, s>>>(a);
}

template <int P>
static bool dispatch_tile(const DslashCall& d, const TileArgs& a, int grid, int threads, size_t smem, cudaStream_t s) {
  const int m = (d.clover ? 1 : 0) | (d.xpay ? 2 : 0);
  if (d.fin == FIN_NONE) {
    switch (m) {
      case 0: go_tile<P, 0, 0, FIN_NONE>(a, grid, threads, smem, s); return true;
      case 1: go_tile<P, 1, 0, FIN_NONE>(a, grid, threads, smem, s); return true;
      case 2: go_tile<P, 0, 1, FIN_NONE>(a, grid, threads, smem, s); return true;
      case 3: go_tile<P, 1, 1, FIN_NONE>(a, grid, threads, smem, s); return true;
    }
  }
  if (m != 3) return false;
  if (d.fin == FIN_ALPHA) { go_tile<P, 1, 1, FIN_ALPHA>(a, grid, threads, smem, s); return true; }
  if (d.fin == FIN_OMEGA) { go_tile<P, 1, 1, FIN_OMEGA>(a, grid, threads, smem, s); return true; }
  if (d.fin == FIN_TRUE && P == P32) { go_tile<P32, 1, 1, FIN_TRUE>(a, grid, threads, smem, s); return true; }
  return false;
}

// Launch the tiled kernel for call d; false if the shape does not apply
// (the caller then uses the per-site kernel). Returns the number of
// per-warp partials per source in *nparts.
bool launch_dslash_tile(const sq_ctx* c, const DslashCall& d, cudaStream_t s, int* nparts) {
  const TilePlan p = tile_plan(c, d.prec, d.shape);
  if (!p.ok || d.recon != 12) return false;
  TileArgs a;
  memset(&a, 0, sizeof(a));
  a.g = geom_of(c);
  a.out = d.out;
  a.in = d.in;
  a.x = d.x;
  a.r1 = d.r1;
  a.links = c->U32;
  a.clov = (d.clover && d.cs) ? (const void*)d.cs->Ainv32 : nullptr;
  a.p_out = d.p_out;
  a.a = (float)d.a;
  a.list = d.list;
  a.count = d.count;
  a.n = d.n;
  a.by = d.shape.by;
  a.bz = d.shape.bz;
  a.bt = d.shape.bt;
  a.nty = p.nty;
  a.ntz = p.ntz;
  a.sg = d.shape.sg;
  a.ngroups = (d.n + a.sg - 1) / a.sg;
  a.nbuf = d.shape.nbuf;
  a.hy = p.hy;
  a.hz = p.hz;
  a.ht = p.ht;
  a.nyA = p.nyA;
  a.NA = p.NA;
  a.NB = p.NB;
  a.nslot = p.nslot;
  a.S = p.S;
  a.buf_bytes = p.buf_bytes;
  a.wait_cycles = c->wait_cycles > 0 ? c->wait_cycles : kTileWaitCycles;
  a.stall = c->wait_stall;
  a.ra = d.ra;
  a.err = c->d_err;
  const int grid = p.ntiles * a.ngroups;
  bool ok = d.prec == P32 ? dispatch_tile<P32>(d, a, grid, p.threads, p.smem, s)
                          : dispatch_tile<P16>(d, a, grid, p.threads, p.smem, s);
  if (nparts) *nparts = p.ntiles * (p.threads / 32);
  return ok;
}

}  // namespace sq

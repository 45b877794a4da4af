// G1: even-odd Wilson hopping term with fused clover inverse, xpay and
// reductions, for FP64 / FP32 / FP16 fields and many sources per CTA.
//
// Operator (the kappa-normalised clover-Wilson matrix M = A - kappa D, with
// D psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)),
// restricted to hops from parity 1-p onto parity p. Each hop is done on a
// half spinor: in the DeGrand-Rossi basis g_mu = [[0, B_mu], [B_mu^+, 0]] in
// 2x2 spin blocks, so (1 -+ g_mu) psi = [h; -+ B_mu^+ h] with
// h = psi_up -+ B_mu psi_dn: two SU(3) mat-vecs per hop instead of four.
//
// CTA = sx sites (threadIdx.x, consecutive checkerboard sites: every spinor
// and link chunk load of a warp is one contiguous 128-bit-per-lane segment)
// times ry sources (threadIdx.y). The ry sources of a CTA read the same
// links and clover blocks, so those come from HBM once per CTA and from L1
// for the other sources.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "sq_hop.cuh"
#include "sq_internal.h"

namespace sq {

struct KArgs {
  Geom g;
  Field out, in, x, r1;
  const void* links;
  const void* clov;
  int p_out;
  double a;
  const int* list;
  const int* count;
  int n;
  int nsb, nrb;  // site blocks, source blocks of the flattened grid
  int order;     // 0: source blocks fastest (a site tile's links are shared
                 //    through L2 by its source blocks); 1: site blocks fastest
  RedArgs ra;
};

// Register budget of the FP32 / FP16 kernels (per thread). Uncapped, the
// compiler takes ~200 registers for them (one 256-thread CTA per SM); with
// the cap two stay resident. Measured on GB300 (16^3x32, 16 sources): caps
// of 80..128 give 87..101 us per clover dslash, 128 the fastest. The FP64
// kernel is ALU-bound and stays uncapped (~146 registers).
#ifndef SQ_DSLASH_LP_REGS
#define SQ_DSLASH_LP_REGS 128
#endif

// precision of the links and clover blocks read by a dslash on fields of
// precision P: FP16 fields use the FP32 gauge data (per site, shared by the
// sources of a launch) and save the per-source half -> float conversions
__host__ __device__ constexpr int gauge_prec(int P) { return P == P16 ? P32 : P; }

template <int P, int RECON, int MU>
__device__ __forceinline__ void hop_dir(const KArgs& a, int k, int cb, Coord c,
                                        cx<typename Real<P>::T> acc[12]) {
  typedef typename Real<P>::T R;
  {  // forward: (1 - g_mu) U_mu(x) psi(x + mu)
    Coord n = step(a.g, c, MU, +1);
    int ncb = cb_of(a.g, n.x, n.y, n.z, n.t);
    cx<R> v[12], h[6], w[6];
    R f = (R)1;
    if (P == P16) f = SpinorIO<P16>::load_raw(a.in, k, ncb, (cx<float>*)v);  // norm applied to w
    else SpinorIO<P>::load(a.in, k, ncb, v);
    project<MU, -1>(v, h);
    Link<R> u;
    LinkIO<gauge_prec(P), RECON>::load(a.links, a.g.Vh, a.p_out, MU, cb, u);
    mv(u, h, w);
    if (P == P16) {  // site norm, and the time-boundary sign
      if (MU == 3 && c.t == a.g.T - 1) f *= (R)a.g.tbc;
#pragma unroll
      for (int j = 0; j < 6; j++) w[j] = f * w[j];
    } else if (MU == 3 && c.t == a.g.T - 1) {
      const R tb = (R)a.g.tbc;
#pragma unroll
      for (int j = 0; j < 6; j++) w[j] = tb * w[j];
    }
    accum<MU, -1>(acc, w);
  }
  {  // backward: (1 + g_mu) U_mu(x - mu)^+ psi(x - mu)
    Coord n = step(a.g, c, MU, -1);
    int ncb = cb_of(a.g, n.x, n.y, n.z, n.t);
    cx<R> v[12], h[6], w[6];
    R f = (R)1;
    if (P == P16) f = SpinorIO<P16>::load_raw(a.in, k, ncb, (cx<float>*)v);  // norm applied to w
    else SpinorIO<P>::load(a.in, k, ncb, v);
    project<MU, +1>(v, h);
    Link<R> u;
    LinkIO<gauge_prec(P), RECON>::load(a.links, a.g.Vh, 1 - a.p_out, MU, ncb, u);
    mv_dag(u, h, w);
    if (P == P16) {  // site norm, and the time-boundary sign
      if (MU == 3 && c.t == 0) f *= (R)a.g.tbc;
#pragma unroll
      for (int j = 0; j < 6; j++) w[j] = f * w[j];
    } else if (MU == 3 && c.t == 0) {
      const R tb = (R)a.g.tbc;
#pragma unroll
      for (int j = 0; j < 6; j++) w[j] = tb * w[j];
    }
    accum<MU, +1>(acc, w);
  }
}

// CTA coordinates of the flattened grid: site block sb, slot block rb
__device__ __forceinline__ void cta_blocks(const KArgs& a, int& sb, int& rb) {
  if (a.order == 0) {
    sb = blockIdx.x / a.nrb;
    rb = blockIdx.x - sb * a.nrb;
  } else {
    rb = blockIdx.x / a.nsb;
    sb = blockIdx.x - rb * a.nsb;
  }
}

// One pass over source slots slot0 .. slot0 + blockDim.y - 1 for the sites
// of site block sb. Every thread of the CTA calls it (reductions).
template <int P, int RECON, int CLOV, int XPAY, int FIN>
__device__ __forceinline__ void dslash_pass(const KArgs& a, int sb, int slot0, int cnt) {
  typedef typename Real<P>::T R;
  constexpr int NRED = FIN == FIN_ALPHA ? 2 : FIN == FIN_OMEGA ? 3 : 1;
  const int cb = sb * blockDim.x + threadIdx.x;
  const int slot = slot0 + threadIdx.y;
  const int k = slot < cnt ? (a.list ? a.list[slot] : slot) : -1;
  const bool ok = (k >= 0) && (cb < a.g.Vh);
  typedef typename SumOf<R>::T S;
  S red[NRED];
#pragma unroll
  for (int i = 0; i < NRED; i++) red[i] = (S)0;
  if (ok) {
    cx<R> acc[12];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[j] = zero<R>();
    const Coord c = cb_coords(a.g, cb, a.p_out);
    hop_dir<P, RECON, 0>(a, k, cb, c, acc);
    hop_dir<P, RECON, 1>(a, k, cb, c, acc);
    hop_dir<P, RECON, 2>(a, k, cb, c, acc);
    hop_dir<P, RECON, 3>(a, k, cb, c, acc);
    if (CLOV) {
      cx<R> w[6];
      R blk[36];
      CloverIO<gauge_prec(P)>::template load_block<0>(a.clov, a.g.Vh, a.p_out, cb, blk);
      herm6_apply(blk, acc, w);
#pragma unroll
      for (int j = 0; j < 6; j++) acc[j] = w[j];
      CloverIO<gauge_prec(P)>::template load_block<1>(a.clov, a.g.Vh, a.p_out, cb, blk);
      herm6_apply(blk, acc + 6, w);
#pragma unroll
      for (int j = 0; j < 6; j++) acc[6 + j] = w[j];
    }
    cx<R> xv[12];
    if (XPAY) {
      SpinorIO<P>::load(a.x, k, cb, xv);
      const R f = (R)a.a;
#pragma unroll
      for (int j = 0; j < 12; j++) acc[j] = mk(xv[j].re + f * acc[j].re, xv[j].im + f * acc[j].im);
    }
    SpinorIO<P>::store(a.out, k, cb, acc);
    if (FIN == FIN_ALPHA) {  // <r1, out>
      cx<R> rv[12];
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
      S sr = 0, si = 0, tt = 0;
#pragma unroll
      for (int j = 0; j < 12; j++) {
        sr += (S)acc[j].re * xv[j].re + (S)acc[j].im * xv[j].im;
        si += (S)acc[j].re * xv[j].im - (S)acc[j].im * xv[j].re;
        tt += (S)acc[j].re * acc[j].re + (S)acc[j].im * acc[j].im;
      }
      red[0] = sr;
      red[1] = si;
      red[2] = tt;
    } else if (FIN == FIN_TRUE) {
      S tt = 0;
#pragma unroll
      for (int j = 0; j < 12; j++) tt += (S)acc[j].re * acc[j].re + (S)acc[j].im * acc[j].im;
      red[0] = tt;
    }
  }
  if (FIN != FIN_NONE)  // per-warp partials, added up by k_finish
    warp_partials<NRED>(a.ra, red, k, sb * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5));

}

// FP32 / FP16: one pass, a CTA row per slot block
template <int P, int RECON, int CLOV, int XPAY, int FIN>
__global__ void __maxnreg__(SQ_DSLASH_LP_REGS) k_dslash(const KArgs a) {
  int sb, rb;
  cta_blocks(a, sb, rb);
  const int cnt = a.list ? *a.count : a.n;
  const int slot0 = rb * blockDim.y;
  if (slot0 >= cnt) return;  // whole CTA idle (uniform)
  dslash_pass<P, RECON, CLOV, XPAY, FIN>(a, sb, slot0, cnt);
}

// FP64: the CTA rows stride over the slots (a single pass with the usual
// one row per slot block)
template <int CLOV, int XPAY, int FIN>
__global__ void __launch_bounds__(256) k_dslash64(const KArgs a) {
  int sb, rb;
  cta_blocks(a, sb, rb);
  const int cnt = a.list ? *a.count : a.n;
  for (int slot0 = rb * blockDim.y; slot0 < cnt; slot0 += a.nrb * blockDim.y)
    dslash_pass<P64, 18, CLOV, XPAY, FIN>(a, sb, slot0, cnt);
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------
int dslash_nblk(const sq_ctx* c, Shape sh) { return (c->Vh + sh.sx - 1) / sh.sx; }

template <int P, int RECON, int CLOV, int XPAY, int FIN>
static void go(const KArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
  if (P == P64) k_dslash64<CLOV, XPAY, FIN><<<grid, block, 0, s>>>(a);
  else k_dslash<P, RECON, CLOV, XPAY, FIN><<<grid, block, 0, s>>>(a);
}

template <int P, int RECON>
static bool dispatch_mode(const DslashCall& d, const KArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
  const int m = (d.clover ? 1 : 0) | (d.xpay ? 2 : 0);
  if (d.fin == FIN_NONE) {
    switch (m) {
      case 0: go<P, RECON, 0, 0, FIN_NONE>(a, grid, block, s); return true;
      case 1: go<P, RECON, 1, 0, FIN_NONE>(a, grid, block, s); return true;
      case 2: go<P, RECON, 0, 1, FIN_NONE>(a, grid, block, s); return true;
      case 3: go<P, RECON, 1, 1, FIN_NONE>(a, grid, block, s); return true;
    }
  }
  if (m != 3) return false;
  if (d.fin == FIN_ALPHA) { go<P, RECON, 1, 1, FIN_ALPHA>(a, grid, block, s); return true; }
  if (d.fin == FIN_OMEGA) { go<P, RECON, 1, 1, FIN_OMEGA>(a, grid, block, s); return true; }
  if (d.fin == FIN_TRUE && P == P32) { go<P, RECON, 1, 1, FIN_TRUE>(a, grid, block, s); return true; }
  return false;
}

void launch_dslash(const sq_ctx* c, const DslashCall& d, cudaStream_t s) {
  KArgs a;
  a.g = geom_of(c);
  a.out = d.out;
  a.in = d.in;
  a.x = d.x;
  a.r1 = d.r1;
  a.p_out = d.p_out;
  a.a = d.a;
  a.list = d.list;
  a.count = d.count;
  a.n = d.n;
  a.ra = d.ra;
  a.clov = nullptr;
  if (d.clover && d.cs) {
    a.clov = d.prec == P64 ? (const void*)d.cs->Ainv64 : (const void*)d.cs->Ainv32;
  }
  a.links = d.prec == P64 ? (const void*)c->U64 : c->U32;
  dim3 block(d.shape.sx, d.shape.ry);
  a.nsb = (c->Vh + d.shape.sx - 1) / d.shape.sx;
  a.nrb = (d.n + d.shape.ry - 1) / d.shape.ry;
  a.order = d.shape.order;
  dim3 grid((unsigned)a.nsb * (unsigned)a.nrb);
  bool ok = false;
  int nparts = a.nsb * (int)(block.x >> 5);
  if (d.prec == P64 && d.emul) {
    ok = launch_dslash_df(c, d, d.out2, d.xfirst, s, &nparts);
  } else if (d.shape.kind == 1 && launch_dslash_tile(c, d, s, &nparts)) {
    ok = true;
  } else if (d.prec == P64) {
    if (d.fin == FIN_TRUE && d.clover && d.xpay) {
      go<P64, 18, 1, 1, FIN_TRUE>(a, grid, block, s);
      ok = true;
    } else {
      ok = dispatch_mode<P64, 18>(d, a, grid, block, s);
    }
  } else if (d.prec == P32) {
    ok = d.recon == 18 ? dispatch_mode<P32, 18>(d, a, grid, block, s)
                       : dispatch_mode<P32, 12>(d, a, grid, block, s);
  } else {
    ok = d.recon == 18 ? dispatch_mode<P16, 18>(d, a, grid, block, s) : dispatch_mode<P16, 12>(d, a, grid, block, s);
  }
  if (!ok) fprintf(stderr, "libstochq: internal error: no dslash variant for this call\n");
  if (d.fin != FIN_NONE) {  // per-source sums and scalars
    if (d.prec == P64) {
      if (d.fin == FIN_ALPHA) k_finish<double, 2, FIN_ALPHA><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
      else if (d.fin == FIN_OMEGA) k_finish<double, 3, FIN_OMEGA><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
      else if (d.fin == FIN_STORE) k_finish<double, 1, FIN_STORE><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
      else k_finish<double, 1, FIN_TRUE><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
    } else {
      if (d.fin == FIN_ALPHA) k_finish<SumOf<float>::T, 2, FIN_ALPHA><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
      else if (d.fin == FIN_OMEGA) k_finish<SumOf<float>::T, 3, FIN_OMEGA><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
      else k_finish<SumOf<float>::T, 1, FIN_TRUE><<<d.n, 256, 0, s>>>(a.ra, d.list, d.count, d.n, nparts);
    }
  }
}

bool dslash_tuned(const sq_ctx* c, int prec, int recon, int n) {
  const long long key = ((long long)prec << 56) ^ ((long long)recon << 48) ^ ((long long)c->Vh << 12) ^ n;
  return c->tuned.find(key) != c->tuned.end();
}

// Halo-tiled shapes for the tuner: the two tiles (all of x, by x bz x bt
// rows dividing the lattice, 128 to 256 sites) with the fewest staged rows
// per site, with a double-buffered ring and the largest source group that
// fills the machine. Measured on GB300 (16^3x32 .. 32^3x64, FP32 and FP16)
// the tiled kernel ran 1.4-2x slower than the per-site kernel: with links
// and clover blocks resident in registers (255 per thread) only 8 warps fit
// on an SM, so it issues half as often, although it moves 40% fewer bytes
// from L2. It stays a candidate for the lattices and source counts where
// that balance turns.
static void tile_candidates(const sq_ctx* c, int prec, int recon, int n, std::vector<Shape>& out) {
  if ((prec != P32 && prec != P16) || recon != 12) return;
  const int X2 = c->dims[0] / 2, Y = c->dims[1], Z = c->dims[2], T = c->dims[3];
  struct Cand {
    double halo;
    int by, bz, bt;
  };
  std::vector<Cand> tiles;
  for (int by = 1; by <= Y; by++)
    for (int bz = 1; bz <= Z; bz++)
      for (int bt = 1; bt <= T; bt++) {
        if (Y % by || Z % bz || T % bt) continue;
        const int th = X2 * by * bz * bt;
        if (th < 128 || th > 256 || th % 32) continue;
        const int hy = by < Y, hz = bz < Z, ht = bt < T;
        const int rows = bt * bz * (by + 2 * hy) + (hz ? 2 * bt * by : 0) + (ht ? 2 * bz * by : 0);
        tiles.push_back({(double)rows / (by * bz * bt), by, bz, bt});
      }
  std::sort(tiles.begin(), tiles.end(), [](const Cand& a, const Cand& b) { return a.halo < b.halo; });
  if (tiles.size() > 2) tiles.resize(2);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  for (const Cand& t : tiles) {
    // the largest group (fewest reloads of the gauge data) that still gives
    // at least four CTAs per SM
    const int ntiles = (Y / t.by) * (Z / t.bz) * (T / t.bt);
    int sg = n;
    while (sg > 2 && (long long)ntiles * ((n + sg - 1) / sg) < 4LL * (nsm > 0 ? nsm : 152)) sg = (sg + 1) / 2;
    Shape sh;
    sh.kind = 1;
    sh.by = t.by;
    sh.bz = t.bz;
    sh.bt = t.bt;
    sh.sg = sg;
    sh.nbuf = 2;
    if (tile_shape_ok(c, prec, recon, sh)) out.push_back(sh);
  }
}

// Pick the launch shape by timing the candidates on the call's own fields
// (no reduction). Results are cached per (precision, recon, Vh, n).
Shape tune_dslash(sq_ctx* c, DslashCall d, cudaStream_t s) {
  long long key = ((long long)d.prec << 56) ^ ((long long)d.recon << 48) ^ ((long long)c->Vh << 12) ^ d.n;
  auto it = c->tuned.find(key);
  if (it != c->tuned.end()) return it->second;
  static const int cand[][3] = {{32, 1, 0}, {32, 2, 0}, {32, 4, 0}, {32, 8, 0}, {64, 1, 0}, {64, 2, 0},
                                {64, 4, 0}, {128, 1, 0}, {128, 2, 0}, {256, 1, 0}, {64, 2, 1}, {32, 4, 1}};
  std::vector<Shape> shapes;
  for (auto& cd : cand) {
    if (cd[1] > 1 && cd[1] > d.n) continue;
    Shape sh;
    sh.sx = cd[0];
    sh.ry = cd[1];
    sh.order = cd[2];
    shapes.push_back(sh);
  }
  tile_candidates(c, d.prec, d.recon, d.n, shapes);
  d.fin = FIN_NONE;
  d.list = nullptr;
  d.count = nullptr;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Shape best;
  float best_ms = 1e30f;
  for (const Shape& sh : shapes) {
    d.shape = sh;
    for (int w = 0; w < 2; w++) launch_dslash(c, d, s);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 5; r++) launch_dslash(c, d, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaGetLastError() != cudaSuccess) continue;
    if (ms < best_ms) {
      best_ms = ms;
      best = d.shape;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tuned[key] = best;
  c->tuned_meta[key] = {d.prec, d.recon, d.n};
  return best;
}

}  // namespace sq

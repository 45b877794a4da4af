// FP64-accurate even-odd hop and clover applications in double-FP32
// arithmetic (sq_df32.cuh) for the solver's FP64 steps: the Schur source,
// the reliable-update residual, the reconstruction of the odd sites and the
// full-lattice residual check. GB300's FP64 pipe runs at 1/60 of its FP32
// rate; these kernels keep FP64 fields (double2) in memory and do the
// arithmetic on the FP32 pipe with about 46 correct bits:
//   * links and clover blocks come pre-split (float4 = re.h, im.h, re.l, im.l,
//     made once per gauge load / clover build), spinors are split from their
//     FP64 bits with integer operations, results are rounded back to FP64;
//   * every product of leading parts is exact (FMA), every sum of leading
//     parts is exact (TwoSum); trailing parts and cross terms add in FP32.
// Relative error per output component: a few times 2^-46 of the sum of the
// magnitudes of its terms (the splitting, 2^-47 per input, dominates).
//
// Operator as in sq_dslash.cu: D psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
// + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu) on half spinors, restricted to hops
// from parity 1-p onto p. Modes (out, out2: FP64 fields of parity p):
//   XFIRST = 0: w = D in; w <- A^-1 w (CLOV); out = x + a w (XPAY) or w
//   XFIRST = 1: w = x + a D in; out = A^-1 w; out2 = w (OUT2)
// FIN_TRUE and FIN_STORE add ||out||^2 per source (per-warp partials for
// k_finish: the solver's true residual, or a stored norm).
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "sq_df32.cuh"
#include "sq_internal.h"

namespace sq {

struct DfArgs {
  Geom g;
  Field out, out2, in, x;
  const float4* links;  // [p][mu][9][Vh]
  const float4* clov;   // [p][36][Vh]: 36 cdf per site, 18 per chirality block
  int p_out;
  df a;
  const int* list;
  const int* count;
  int n;
  int nsb, nrb;
  RedArgs ra;
};

__device__ __forceinline__ void load_link_df(const float4* base, int Vh, int p, int mu, int cb, cdf u[9]) {
  const float4* q = base + ((size_t)(p * 4 + mu) * 9) * Vh + cb;
#pragma unroll
  for (int e = 0; e < 9; e++) u[e] = cdf_of(__ldg(q + (size_t)e * Vh));
}

// acc + s * b for s = +1 or -1 (exact sign)
template <int S>
__device__ __forceinline__ cdf cpm(cdf acc, cdf b) {
  return S > 0 ? cadd(acc, b) : csub(acc, b);
}

// flip the sign of z when neg (runtime, exact)
__device__ __forceinline__ cdf csign(cdf z, bool neg) {
  const float s = neg ? -1.f : 1.f;
  return cdf{df{s * z.re.h, s * z.re.l}, df{s * z.im.h, s * z.im.l}};
}

// Two threads per site and source: lanes l and l ^ 16 of a warp, j = the
// upper lane bit. In each hop thread j forms row j of the spin projection,
// h_j = psi_j + SIGN c psi_dn, multiplies it by the link and scatters it
// back: w_j to spin j and SIGN conj(c) w_j to spin dn, where (rows of B_mu
// of sq_hop.cuh, chiral basis)
//   mu = 0: dn = 3 - j, c = i;   mu = 1: dn = 3 - j, c = -1 (j = 0), +1 (j = 1)
//   mu = 2: dn = 2 + j, c = i (j = 0), -i (j = 1);   mu = 3: dn = 2 + j, c = 1.
// Spin 3 - j is the partner's own lower spin: those contributions are kept
// apart and handed over by one shuffle after the eight hops. Each thread then
// holds one chirality block (spins 2j, 2j + 1) for the clover term, the xpay
// and the store, so a thread carries half the registers and half the code
// path of a whole site.

// three colour components of spin s of source k at site cb
__device__ __forceinline__ void load_spin_df(const Field& f, int k, int cb, int s, cdf v[3]) {
  const double2* p = (const double2*)f.data + ((size_t)k * 12 + 3 * s) * f.Vh + cb;
#pragma unroll
  for (int c = 0; c < 3; c++) v[c] = cdf_split(__ldg(p + (size_t)c * f.Vh));
}

// the six components of chirality block ch (spins 2 ch, 2 ch + 1)
__device__ __forceinline__ void load_block_df(const Field& f, int k, int cb, int ch, cdf v[6]) {
  const double2* p = (const double2*)f.data + ((size_t)k * 12 + 6 * ch) * f.Vh + cb;
#pragma unroll
  for (int c = 0; c < 6; c++) v[c] = cdf_split(__ldg(p + (size_t)c * f.Vh));
}

__device__ __forceinline__ void store_block_df(const Field& f, int k, int cb, int ch, const cdf v[6]) {
  double2* p = (double2*)f.data + ((size_t)k * 12 + 6 * ch) * f.Vh + cb;
#pragma unroll
  for (int c = 0; c < 6; c++) p[(size_t)c * f.Vh] = double2_of(v[c]);
}

// w = U h or U^+ h for one colour vector
template <bool DAG>
__device__ __forceinline__ void mv3_df(const cdf u[9], const cdf h[3], cdf w[3]) {
  const cdf z{df{0.f, 0.f}, df{0.f, 0.f}};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    cdf r;
    if (DAG) {
      r = cjfma_df(u[a], h[0], z);
      r = cjfma_df(u[3 + a], h[1], r);
      r = cjfma_df(u[6 + a], h[2], r);
    } else {
      r = cfma_df(u[3 * a], h[0], z);
      r = cfma_df(u[3 * a + 1], h[1], r);
      r = cfma_df(u[3 * a + 2], h[2], r);
    }
    w[a] = r;
  }
}

// One hop (MU, forward or backward) of thread j: up += w_j; dn_part (mu 0, 1)
// or dn_own (mu 2, 3) += SIGN conj(c) w_j
template <int MU, bool FWD>
__device__ __forceinline__ void hop_pair_df(const DfArgs& a, int k, int cb, Coord c, int j, cdf up[3],
                                            cdf dn_part[3], cdf dn_own[3]) {
  constexpr int SIGN = FWD ? -1 : +1;
  const Coord nb = step(a.g, c, MU, FWD ? +1 : -1);
  const int ncb = cb_of(a.g, nb.x, nb.y, nb.z, nb.t);
  const int dn = MU < 2 ? 3 - j : 2 + j;
  const bool flip = (MU == 1 && j == 0) || (MU == 2 && j == 1);  // the j-dependent sign of c
  cdf vu[3], vd[3], h[3], w[3], u[9];
  load_spin_df(a.in, k, ncb, j, vu);
  load_spin_df(a.in, k, ncb, dn, vd);
#pragma unroll
  for (int q = 0; q < 3; q++) {
    const cdf d = csign(MU == 0 || MU == 2 ? citimes(vd[q]) : vd[q], flip);
    h[q] = cpm<SIGN>(vu[q], d);
  }
  load_link_df(a.links, a.g.Vh, FWD ? a.p_out : 1 - a.p_out, MU, FWD ? cb : ncb, u);
  mv3_df<!FWD>(u, h, w);
  if (MU == 3 && a.g.tbc < 0 && (FWD ? c.t == a.g.T - 1 : c.t == 0)) {
#pragma unroll
    for (int q = 0; q < 3; q++) w[q] = cdf{df_neg(w[q].re), df_neg(w[q].im)};
  }
#pragma unroll
  for (int q = 0; q < 3; q++) {
    up[q] = cadd(up[q], w[q]);
    // conj(c) w, with conj(i) = -i
    const cdf e = csign(MU == 0 || MU == 2 ? cdf{w[q].im, df_neg(w[q].re)} : w[q], flip);
    if (MU < 2) dn_part[q] = cpm<SIGN>(dn_part[q], e);
    else dn_own[q] = cpm<SIGN>(dn_own[q], e);
  }
}

__device__ __forceinline__ cdf shfl16(cdf v) {
  return cdf{df{__shfl_xor_sync(0xffffffffu, v.re.h, 16), __shfl_xor_sync(0xffffffffu, v.re.l, 16)},
             df{__shfl_xor_sync(0xffffffffu, v.im.h, 16), __shfl_xor_sync(0xffffffffu, v.im.l, 16)}};
}

// w = B v for one packed Hermitian 6x6 block held as 18 cdf: the six real
// diagonals in entries 0..2 (re, im of each), then the 15 strictly-lower
// entries (i > j, row by row) in entries 3..17
__device__ __forceinline__ void herm6_apply_df(const float4* blk, int Vh, const cdf v[6], cdf w[6]) {
  const cdf d01 = cdf_of(__ldg(blk)), d23 = cdf_of(__ldg(blk + (size_t)Vh)), d45 = cdf_of(__ldg(blk + 2 * (size_t)Vh));
  w[0] = cscale(d01.re, v[0]);
  w[1] = cscale(d01.im, v[1]);
  w[2] = cscale(d23.re, v[2]);
  w[3] = cscale(d23.im, v[3]);
  w[4] = cscale(d45.re, v[4]);
  w[5] = cscale(d45.im, v[5]);
#pragma unroll
  for (int i = 1; i < 6; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      const cdf l = cdf_of(__ldg(blk + (size_t)(3 + tri(i, j)) * Vh));
      w[i] = cfma_df(l, v[j], w[i]);   // L_ij v_j
      w[j] = cjfma_df(l, v[i], w[j]);  // conj(L_ij) v_i
    }
  }
}

constexpr int kDfSites = 64;      // sites per CTA: 128 threads, two per site
constexpr int kDfMinBlocks = 6;   // resident CTAs per SM the register budget is cut for

template <int CLOV, int XPAY, int XFIRST, int FIN, int OUT2>
__global__ void __launch_bounds__(2 * kDfSites, kDfMinBlocks) k_dslash_df(const DfArgs a) {
  const int sb = blockIdx.x / a.nrb, rb = blockIdx.x - (blockIdx.x / a.nrb) * a.nrb;
  const int cnt = a.list ? *a.count : a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane >> 4;  // row of the projection; at the end, the chirality block
  const int cb = sb * kDfSites + warp * 16 + (lane & 15);
  const bool site_ok = cb < a.g.Vh;
  for (int slot = rb; slot < cnt; slot += a.nrb) {  // uniform over the CTA
    const int k = a.list ? a.list[slot] : slot;
    double red = 0.0;
    cdf blk[6];
    {
      const df z{0.f, 0.f};
      cdf up[3], dn_part[3], dn_own[3];
#pragma unroll
      for (int q = 0; q < 3; q++) up[q] = dn_part[q] = dn_own[q] = cdf{z, z};
      if (site_ok) {
        const Coord c = cb_coords(a.g, cb, a.p_out);
        hop_pair_df<0, true>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<0, false>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<1, true>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<1, false>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<2, true>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<2, false>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<3, true>(a, k, cb, c, j, up, dn_part, dn_own);
        hop_pair_df<3, false>(a, k, cb, c, j, up, dn_part, dn_own);
      }
      // lower spin 2 + j complete with the partner's part; then regroup by
      // chirality: thread 0 keeps spins 0, 1 and thread 1 spins 2, 3
#pragma unroll
      for (int q = 0; q < 3; q++) dn_own[q] = cadd(dn_own[q], shfl16(dn_part[q]));
#pragma unroll
      for (int q = 0; q < 3; q++) {
        const cdf got = shfl16(j ? up[q] : dn_own[q]);  // 0 hands over spin 2, 1 spin 1
        blk[q] = j ? got : up[q];
        blk[3 + q] = j ? dn_own[q] : got;
      }
    }
    if (site_ok) {
      const size_t cofs = ((size_t)a.p_out * 36 + 18 * j) * a.g.Vh + cb;
      if (XFIRST) {
        cdf xv[6], w[6];
        load_block_df(a.x, k, cb, j, xv);
#pragma unroll
        for (int q = 0; q < 6; q++) blk[q] = cdf{df_fma(a.a, blk[q].re, xv[q].re), df_fma(a.a, blk[q].im, xv[q].im)};
        if (OUT2) store_block_df(a.out2, k, cb, j, blk);
        herm6_apply_df(a.clov + cofs, a.g.Vh, blk, w);
#pragma unroll
        for (int q = 0; q < 6; q++) blk[q] = w[q];
      } else {
        if (CLOV) {
          cdf w[6];
          herm6_apply_df(a.clov + cofs, a.g.Vh, blk, w);
#pragma unroll
          for (int q = 0; q < 6; q++) blk[q] = w[q];
        }
        if (XPAY) {
          cdf xv[6];
          load_block_df(a.x, k, cb, j, xv);
#pragma unroll
          for (int q = 0; q < 6; q++)
            blk[q] = cdf{df_fma(a.a, blk[q].re, xv[q].re), df_fma(a.a, blk[q].im, xv[q].im)};
        }
      }
      store_block_df(a.out, k, cb, j, blk);
      if (FIN == FIN_TRUE || FIN == FIN_STORE) {
        // ||out||^2 to FP32 accuracy (a residual norm). A residual is the
        // cancellation of nearly equal terms, after which the leading float
        // of a pair need not carry the value: square the rounded h + l.
        typedef SumOf<float>::T S;
        S q2 = 0;
#pragma unroll
        for (int q = 0; q < 6; q++) {
          const S re = blk[q].re.h + blk[q].re.l, im = blk[q].im.h + blk[q].im.l;
          q2 = fma(re, re, fma(im, im, q2));
        }
        red = (double)q2;
      }
    }
    if (FIN == FIN_TRUE || FIN == FIN_STORE) {  // both threads of a site sit in one warp
      double r1[1] = {red};
      warp_partials<1>(a.ra, r1, k, sb * (2 * kDfSites / 32) + warp);
    }
  }
}

// one site and chirality block of k_clover_df; returns the block's
// ||out||^2 to FP32 accuracy
__device__ __forceinline__ double clover_df_site(int Vh, const Field& out, const Field& x, const Field& in,
                                                 const float4* C, int parity, df c1, df c2, int k, int cb, int ch) {
  cdf v[6], w[6];

  load_block_df(in, k, cb, ch, v);
  herm6_apply_df(C + ((size_t)parity * 36 + 18 * ch) * Vh + cb, Vh, v, w);
  if (x.data) {
    load_block_df(x, k, cb, ch, v);
    const df z{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 6; j++)
      w[j] = cdf{df_fma(c2, w[j].re, df_fma(c1, v[j].re, z)), df_fma(c2, w[j].im, df_fma(c1, v[j].im, z))};
  } else {
#pragma unroll
    for (int j = 0; j < 6; j++) w[j] = cscale(c2, w[j]);
  }
  store_block_df(out, k, cb, ch, w);
  typedef SumOf<float>::T S;
  S q2 = 0;
#pragma unroll
  for (int q = 0; q < 6; q++) {
    const S re = w[q].re.h + w[q].re.l, im = w[q].im.h + w[q].im.l;
    q2 = fma(re, re, fma(im, im, q2));
  }
  return (double)q2;
}

// out = c1 x + c2 (C in), C = A or A^{-1} (pre-split blocks); x may be
// absent. The two chirality blocks are independent: a CTA of 128 threads
// takes 64 sites, warps 0-1 block 0 and warps 2-3 block 1. NORM: per-warp
// partials of ||out||^2 (FP32-accurate squares, as in k_dslash_df) for a
// k_finish.
template <int NORM>
__global__ void __launch_bounds__(128) k_clover_df(int Vh, Field out, Field x, Field in, const float4* C, int parity,
                                                   df c1, df c2, int n, RedArgs ra) {
  const int ch = threadIdx.x >> 6;
  const int cb = blockIdx.x * 64 + (threadIdx.x & 63);
  const int k = blockIdx.y;
  if (NORM) {  // every thread reaches the warp sums
    double red[1] = {0.0};
    if (cb < Vh && k < n) red[0] = clover_df_site(Vh, out, x, in, C, parity, c1, c2, k, cb, ch);
    warp_partials<1>(ra, red, k < n ? k : -1, (int)blockIdx.x * 4 + (int)(threadIdx.x >> 5));
    return;
  }
  if (cb >= Vh || k >= n) return;
  clover_df_site(Vh, out, x, in, C, parity, c1, c2, k, cb, ch);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static df df_host(double v) {
  const float h = (float)v;
  return df{h, (float)(v - (double)h)};
}

void launch_clover_df(const sq_ctx* c, const CloverSet& cs, Field out, Field x, Field in, int parity, double c1,
                      double c2, int which, int n, cudaStream_t s, const RedArgs* norm) {
  dim3 grid((c->Vh + 63) / 64, n);
  const float4* C = which ? cs.Ainvdf : cs.Adf;
  if (norm && (int)grid.x * 4 <= norm->nblk_stride) {
    k_clover_df<1><<<grid, 128, 0, s>>>(c->Vh, out, x, in, C, parity, df_host(c1), df_host(c2), n, *norm);
    k_finish<double, 1, FIN_STORE><<<n, 256, 0, s>>>(*norm, nullptr, nullptr, n, (int)grid.x * 4);
  } else {
    RedArgs none;
    memset(&none, 0, sizeof(none));
    k_clover_df<0><<<grid, 128, 0, s>>>(c->Vh, out, x, in, C, parity, df_host(c1), df_host(c2), n, none);
    if (norm) fprintf(stderr, "libstochq: internal error: clover norm partials do not fit\n");
  }
}

template <int CLOV, int XPAY, int XFIRST, int FIN, int OUT2>
static void go_df(const DfArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
  k_dslash_df<CLOV, XPAY, XFIRST, FIN, OUT2><<<grid, block, 0, s>>>(a);
}

// emulated-FP64 dslash for a call with d.prec == P64; false if the mode has
// no kernel. out2 (XFIRST only) may be a null field.
bool launch_dslash_df(const sq_ctx* c, const DslashCall& d, Field out2, int xfirst, cudaStream_t s, int* nparts) {
  DfArgs a;
  memset(&a, 0, sizeof(a));
  a.g = geom_of(c);
  a.out = d.out;
  a.out2 = out2;
  a.in = d.in;
  a.x = d.x;
  a.links = (const float4*)c->Udf;
  a.clov = d.cs ? d.cs->Ainvdf : nullptr;
  a.p_out = d.p_out;
  a.a = df_host(d.a);
  a.list = d.list;
  a.count = d.count;
  a.n = d.n;
  a.ra = d.ra;
  a.nsb = (c->Vh + kDfSites - 1) / kDfSites;
  a.nrb = d.n;
  dim3 block(2 * kDfSites), grid((unsigned)a.nsb * (unsigned)a.nrb);
  *nparts = a.nsb * (2 * kDfSites / 32);
  if (d.fin != FIN_NONE && *nparts > d.ra.nblk_stride) return false;  // partials would not fit
  const int m = (d.clover ? 1 : 0) | (d.xpay ? 2 : 0);
  if (xfirst) {
    if (!d.clover || !d.xpay || d.fin != FIN_NONE) return false;
    if (out2.data) go_df<1, 1, 1, FIN_NONE, 1>(a, grid, block, s);
    else go_df<1, 1, 1, FIN_NONE, 0>(a, grid, block, s);
    return true;
  }
  if (d.fin == FIN_TRUE) {
    if (m != 3) return false;
    go_df<1, 1, 0, FIN_TRUE, 0>(a, grid, block, s);
    return true;
  }
  if (d.fin == FIN_STORE) {  // the full residual's even half: x + a D in, with its norm
    if (m != 2) return false;
    go_df<0, 1, 0, FIN_STORE, 0>(a, grid, block, s);
    return true;
  }
  if (d.fin != FIN_NONE) return false;
  switch (m) {
    case 0: go_df<0, 0, 0, FIN_NONE, 0>(a, grid, block, s); return true;
    case 1: go_df<1, 0, 0, FIN_NONE, 0>(a, grid, block, s); return true;
    case 2: go_df<0, 1, 0, FIN_NONE, 0>(a, grid, block, s); return true;
    default: go_df<1, 1, 0, FIN_NONE, 0>(a, grid, block, s); return true;
  }
}

}  // namespace sq

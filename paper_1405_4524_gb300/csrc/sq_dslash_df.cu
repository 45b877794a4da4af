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
// FIN_TRUE adds ||out||^2 per source (per-warp partials for k_finish).
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

__device__ __forceinline__ void load_spinor_df(const Field& f, int k, int cb, cdf v[12]) {
  const double2* p = (const double2*)f.data + (size_t)k * 12 * f.Vh + cb;
#pragma unroll
  for (int c = 0; c < 12; c++) v[c] = cdf_split(__ldg(p + (size_t)c * f.Vh));
}

__device__ __forceinline__ void store_spinor_df(const Field& f, int k, int cb, const cdf v[12]) {
  double2* p = (double2*)f.data + (size_t)k * 12 * f.Vh + cb;
#pragma unroll
  for (int c = 0; c < 12; c++) p[(size_t)c * f.Vh] = double2_of(v[c]);
}

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

// h = psi_up + SIGN * B_mu psi_dn (the projection of sq_hop.cuh in df32)
template <int MU, int SIGN>
__device__ __forceinline__ void project_df(const cdf v[12], cdf h[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cdf d0, d1;
    if (MU == 0) {  // B = [[0, i], [i, 0]]
      d0 = citimes(v[9 + c]);
      d1 = citimes(v[6 + c]);
    } else if (MU == 1) {  // B = [[0, -1], [1, 0]]
      d0 = cdf{df_neg(v[9 + c].re), df_neg(v[9 + c].im)};
      d1 = v[6 + c];
    } else if (MU == 2) {  // B = [[i, 0], [0, -i]]
      d0 = citimes(v[6 + c]);
      d1 = cdf{v[9 + c].im, df_neg(v[9 + c].re)};
    } else {  // B = 1
      d0 = v[6 + c];
      d1 = v[9 + c];
    }
    h[c] = cpm<SIGN>(v[c], d0);
    h[3 + c] = cpm<SIGN>(v[3 + c], d1);
  }
}

// acc_up += w ; acc_dn += SIGN * B_mu^+ w
template <int MU, int SIGN>
__device__ __forceinline__ void accum_df(cdf acc[12], const cdf w[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = cadd(acc[c], w[c]);
    acc[3 + c] = cadd(acc[3 + c], w[3 + c]);
    cdf e0, e1;
    if (MU == 0) {  // B^+ = [[0, -i], [-i, 0]]
      e0 = cdf{w[3 + c].im, df_neg(w[3 + c].re)};
      e1 = cdf{w[c].im, df_neg(w[c].re)};
    } else if (MU == 1) {  // B^+ = [[0, 1], [-1, 0]]
      e0 = w[3 + c];
      e1 = cdf{df_neg(w[c].re), df_neg(w[c].im)};
    } else if (MU == 2) {  // B^+ = [[-i, 0], [0, i]]
      e0 = cdf{w[c].im, df_neg(w[c].re)};
      e1 = citimes(w[3 + c]);
    } else {
      e0 = w[c];
      e1 = w[3 + c];
    }
    acc[6 + c] = cpm<SIGN>(acc[6 + c], e0);
    acc[9 + c] = cpm<SIGN>(acc[9 + c], e1);
  }
}

// w[s] = U h[s]
__device__ __forceinline__ void mv_df(const cdf u[9], const cdf h[6], cdf w[6]) {
  const cdf z{df{0.f, 0.f}, df{0.f, 0.f}};
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cdf r = cfma_df(u[3 * a], h[3 * s], z);
      r = cfma_df(u[3 * a + 1], h[3 * s + 1], r);
      r = cfma_df(u[3 * a + 2], h[3 * s + 2], r);
      w[3 * s + a] = r;
    }
}

// w[s] = U^+ h[s]
__device__ __forceinline__ void mv_dag_df(const cdf u[9], const cdf h[6], cdf w[6]) {
  const cdf z{df{0.f, 0.f}, df{0.f, 0.f}};
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cdf r = cjfma_df(u[a], h[3 * s], z);
      r = cjfma_df(u[3 + a], h[3 * s + 1], r);
      r = cjfma_df(u[6 + a], h[3 * s + 2], r);
      w[3 * s + a] = r;
    }
}

template <int MU>
__device__ __forceinline__ void hop_dir_df(const DfArgs& a, int k, int cb, Coord c, cdf acc[12]) {
  {  // forward: (1 - g_mu) U_mu(x) psi(x + mu)
    const Coord nb = step(a.g, c, MU, +1);
    cdf v[12], h[6], w[6], u[9];
    load_spinor_df(a.in, k, cb_of(a.g, nb.x, nb.y, nb.z, nb.t), v);
    project_df<MU, -1>(v, h);
    load_link_df(a.links, a.g.Vh, a.p_out, MU, cb, u);
    mv_df(u, h, w);
    if (MU == 3 && c.t == a.g.T - 1 && a.g.tbc < 0) {
#pragma unroll
      for (int j = 0; j < 6; j++) w[j] = cdf{df_neg(w[j].re), df_neg(w[j].im)};
    }
    accum_df<MU, -1>(acc, w);
  }
  {  // backward: (1 + g_mu) U_mu(x - mu)^+ psi(x - mu)
    const Coord nb = step(a.g, c, MU, -1);
    const int ncb = cb_of(a.g, nb.x, nb.y, nb.z, nb.t);
    cdf v[12], h[6], w[6], u[9];
    load_spinor_df(a.in, k, ncb, v);
    project_df<MU, +1>(v, h);
    load_link_df(a.links, a.g.Vh, 1 - a.p_out, MU, ncb, u);
    mv_dag_df(u, h, w);
    if (MU == 3 && c.t == 0 && a.g.tbc < 0) {
#pragma unroll
      for (int j = 0; j < 6; j++) w[j] = cdf{df_neg(w[j].re), df_neg(w[j].im)};
    }
    accum_df<MU, +1>(acc, w);
  }
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

__device__ __forceinline__ void clover_apply_df(const float4* clov, int Vh, int p, int cb, cdf v[12]) {
  cdf w[6];
  const float4* b0 = clov + (size_t)p * 36 * Vh + cb;
  herm6_apply_df(b0, Vh, v, w);
#pragma unroll
  for (int j = 0; j < 6; j++) v[j] = w[j];
  herm6_apply_df(b0 + (size_t)18 * Vh, Vh, v + 6, w);
#pragma unroll
  for (int j = 0; j < 6; j++) v[6 + j] = w[j];
}

template <int CLOV, int XPAY, int XFIRST, int FIN, int OUT2>
__global__ void __launch_bounds__(64) k_dslash_df(const DfArgs a) {
  const int sb = blockIdx.x / a.nrb, rb = blockIdx.x - (blockIdx.x / a.nrb) * a.nrb;
  const int cnt = a.list ? *a.count : a.n;
  const int cb = sb * blockDim.x + threadIdx.x;
  for (int slot0 = rb * blockDim.y; slot0 < cnt; slot0 += a.nrb * blockDim.y) {
    const int slot = slot0 + threadIdx.y;
    const int k = slot < cnt ? (a.list ? a.list[slot] : slot) : -1;
    double red = 0.0;
    if (k >= 0 && cb < a.g.Vh) {
      const df z{0.f, 0.f};
      cdf acc[12];
#pragma unroll
      for (int j = 0; j < 12; j++) acc[j] = cdf{z, z};
      const Coord c = cb_coords(a.g, cb, a.p_out);
      hop_dir_df<0>(a, k, cb, c, acc);
      hop_dir_df<1>(a, k, cb, c, acc);
      hop_dir_df<2>(a, k, cb, c, acc);
      hop_dir_df<3>(a, k, cb, c, acc);
      if (XFIRST) {
        cdf xv[12];
        load_spinor_df(a.x, k, cb, xv);
#pragma unroll
        for (int j = 0; j < 12; j++) acc[j] = cdf{df_fma(a.a, acc[j].re, xv[j].re), df_fma(a.a, acc[j].im, xv[j].im)};
        if (OUT2) store_spinor_df(a.out2, k, cb, acc);
        clover_apply_df(a.clov, a.g.Vh, a.p_out, cb, acc);
      } else {
        if (CLOV) clover_apply_df(a.clov, a.g.Vh, a.p_out, cb, acc);
        if (XPAY) {
          cdf xv[12];
          load_spinor_df(a.x, k, cb, xv);
#pragma unroll
          for (int j = 0; j < 12; j++)
            acc[j] = cdf{df_fma(a.a, acc[j].re, xv[j].re), df_fma(a.a, acc[j].im, xv[j].im)};
        }
      }
      store_spinor_df(a.out, k, cb, acc);
      if (FIN == FIN_TRUE) {
        // ||out||^2 to FP32 accuracy (a residual norm). A residual is the
        // cancellation of nearly equal terms, after which the leading float
        // of a pair need not carry the value: square the rounded h + l.
        typedef SumOf<float>::T S;
        S q = 0;
#pragma unroll
        for (int j = 0; j < 12; j++) {
          const S re = acc[j].re.h + acc[j].re.l, im = acc[j].im.h + acc[j].im.l;
          q = fma(re, re, fma(im, im, q));
        }
        red = (double)q;
      }
    }
    if (FIN == FIN_TRUE) {
      double r1[1] = {red};
      warp_partials<1>(a.ra, r1, k, sb * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5));
    }
  }
}

// out = c1 x + c2 (C in), C = A or A^{-1} (pre-split blocks); x may be absent
__global__ void __launch_bounds__(128) k_clover_df(int Vh, Field out, Field x, Field in, const float4* C, int parity,
                                                   df c1, df c2, int n) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (cb >= Vh || k >= n) return;
  cdf v[12];
  load_spinor_df(in, k, cb, v);
  clover_apply_df(C, Vh, parity, cb, v);
  if (x.data) {
    cdf xv[12];
    load_spinor_df(x, k, cb, xv);
    const df z{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 12; j++) {
      v[j] = cdf{df_fma(c2, v[j].re, df_fma(c1, xv[j].re, z)), df_fma(c2, v[j].im, df_fma(c1, xv[j].im, z))};
    }
  } else {
#pragma unroll
    for (int j = 0; j < 12; j++) v[j] = cscale(c2, v[j]);
  }
  store_spinor_df(out, k, cb, v);
}

// float4 (hi.re, hi.im, lo.re, lo.im) copies of n double2 values, rounded
// splits in FP64 (once per gauge load or clover build)
__global__ void k_split_copy(const double2* in, float4* out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 d = in[i];
    const float hr = __double2float_rn(d.x), hi = __double2float_rn(d.y);
    out[i] = make_float4(hr, hi, __double2float_rn(d.x - (double)hr), __double2float_rn(d.y - (double)hi));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static df df_host(double v) {
  const float h = (float)v;
  return df{h, (float)(v - (double)h)};
}

void launch_split_copy(const double2* in, float4* out, size_t n, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_split_copy<<<grid > 0 ? grid : 1, 256, 0, s>>>(in, out, n);
}

void launch_clover_df(const sq_ctx* c, const CloverSet& cs, Field out, Field x, Field in, int parity, double c1,
                      double c2, int which, int n, cudaStream_t s) {
  dim3 grid((c->Vh + 127) / 128, n);
  k_clover_df<<<grid, 128, 0, s>>>(c->Vh, out, x, in, which ? cs.Ainvdf : cs.Adf, parity, df_host(c1), df_host(c2),
                                   n);
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
  const int sx = 64, ry = 1;
  a.nsb = (c->Vh + sx - 1) / sx;
  a.nrb = (d.n + ry - 1) / ry;
  dim3 block(sx, ry), grid((unsigned)a.nsb * (unsigned)a.nrb);
  *nparts = a.nsb * (sx / 32);
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
  if (d.fin != FIN_NONE) return false;
  switch (m) {
    case 0: go_df<0, 0, 0, FIN_NONE, 0>(a, grid, block, s); return true;
    case 1: go_df<1, 0, 0, FIN_NONE, 0>(a, grid, block, s); return true;
    case 2: go_df<0, 1, 0, FIN_NONE, 0>(a, grid, block, s); return true;
    default: go_df<1, 1, 0, FIN_NONE, 0>(a, grid, block, s); return true;
  }
}

}  // namespace sq

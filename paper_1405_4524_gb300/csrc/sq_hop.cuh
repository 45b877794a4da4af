// Hop arithmetic of the even-odd Wilson stencil, shared by the dslash
// kernels: spin projection onto half spinors, SU(3) mat-vecs and the
// reconstruction of the full spinor. In the DeGrand-Rossi basis
// g_mu = [[0, B_mu], [B_mu^+, 0]] in 2x2 spin blocks, so
// (1 -+ g_mu) psi = [h; -+ B_mu^+ h] with h = psi_up -+ B_mu psi_dn: two
// SU(3) mat-vecs per hop instead of four.
#pragma once

#include "sq_device.cuh"

namespace sq {

// h = psi_up + SIGN * B_mu psi_dn   (SIGN = -1: forward hop, +1: backward)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void project(const cx<R> v[12], cx<R> h[6]) {
  const R sg = (R)SIGN;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cx<R> d0, d1;
    if (MU == 0) {  // B = [[0, i], [i, 0]]
      d0 = itimes(v[9 + c]);
      d1 = itimes(v[6 + c]);
    } else if (MU == 1) {  // B = [[0, -1], [1, 0]]
      d0 = mk(-v[9 + c].re, -v[9 + c].im);
      d1 = v[6 + c];
    } else if (MU == 2) {  // B = [[i, 0], [0, -i]]
      d0 = itimes(v[6 + c]);
      d1 = mk(v[9 + c].im, -v[9 + c].re);
    } else {  // B = 1
      d0 = v[6 + c];
      d1 = v[9 + c];
    }
    h[c] = mk(v[c].re + sg * d0.re, v[c].im + sg * d0.im);
    h[3 + c] = mk(v[3 + c].re + sg * d1.re, v[3 + c].im + sg * d1.im);
  }
}

// acc_up += w ; acc_dn += SIGN * B_mu^+ w
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void accum(cx<R> acc[12], const cx<R> w[6]) {
  const R sg = (R)SIGN;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = acc[c] + w[c];
    acc[3 + c] = acc[3 + c] + w[3 + c];
    cx<R> e0, e1;
    if (MU == 0) {  // B^+ = [[0, -i], [-i, 0]]
      e0 = mk(w[3 + c].im, -w[3 + c].re);
      e1 = mk(w[c].im, -w[c].re);
    } else if (MU == 1) {  // B^+ = [[0, 1], [-1, 0]]
      e0 = w[3 + c];
      e1 = mk(-w[c].re, -w[c].im);
    } else if (MU == 2) {  // B^+ = [[-i, 0], [0, i]]
      e0 = mk(w[c].im, -w[c].re);
      e1 = itimes(w[3 + c]);
    } else {
      e0 = w[c];
      e1 = w[3 + c];
    }
    acc[6 + c] = mk(acc[6 + c].re + sg * e0.re, acc[6 + c].im + sg * e0.im);
    acc[9 + c] = mk(acc[9 + c].re + sg * e1.re, acc[9 + c].im + sg * e1.im);
  }
}

// w[s] = U h[s]
template <typename R>
__device__ __forceinline__ void mv(const Link<R>& u, const cx<R> h[6], cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> r = u.e[3 * a] * h[3 * s];
      r = cfma(u.e[3 * a + 1], h[3 * s + 1], r);
      r = cfma(u.e[3 * a + 2], h[3 * s + 2], r);
      w[3 * s + a] = r;
    }
}

// w[s] = U^+ h[s]
template <typename R>
__device__ __forceinline__ void mv_dag(const Link<R>& u, const cx<R> h[6], cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> r = cmul(u.e[a], h[3 * s]);
      r = cjfma(u.e[3 + a], h[3 * s + 1], r);
      r = cjfma(u.e[6 + a], h[3 * s + 2], r);
      w[3 * s + a] = r;
    }
}

// acc_up += f w ; acc_dn += SIGN * f * B_mu^+ w  (f: a per-hop scalar such
// as the time-boundary sign or an FP16 site norm, folded into the adds)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void accum_f(cx<R> acc[12], const cx<R> w[6], R f) {
  const R g = (R)SIGN * f;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = mk(fma(f, w[c].re, acc[c].re), fma(f, w[c].im, acc[c].im));
    acc[3 + c] = mk(fma(f, w[3 + c].re, acc[3 + c].re), fma(f, w[3 + c].im, acc[3 + c].im));
    cx<R> e0, e1;
    if (MU == 0) {  // B^+ = [[0, -i], [-i, 0]]
      e0 = mk(w[3 + c].im, -w[3 + c].re);
      e1 = mk(w[c].im, -w[c].re);
    } else if (MU == 1) {  // B^+ = [[0, 1], [-1, 0]]
      e0 = w[3 + c];
      e1 = mk(-w[c].re, -w[c].im);
    } else if (MU == 2) {  // B^+ = [[-i, 0], [0, i]]
      e0 = mk(w[c].im, -w[c].re);
      e1 = itimes(w[3 + c]);
    } else {
      e0 = w[c];
      e1 = w[3 + c];
    }
    acc[6 + c] = mk(fma(g, e0.re, acc[6 + c].re), fma(g, e0.im, acc[6 + c].im));
    acc[9 + c] = mk(fma(g, e1.re, acc[9 + c].re), fma(g, e1.im, acc[9 + c].im));
  }
}

}  // namespace sq

// Per-source solver state kept on the device, the deterministic
// "last block finalises" reduction used by every reducing kernel, and the
// BiCGStab scalar updates that run in those last blocks.
//
// BiCGStab (van der Vorst 1992) per source k, on the even-odd Schur system
// Mhat x = bhat:  v = Mhat p; alpha = rho/<rhat,v>; s = r - alpha v;
// t = Mhat s; omega = <t,s>/<t,t>; x += alpha p + omega s; r = s - omega t;
// rho' = <rhat,r>; beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v).
// FP64 updates (reliable updates, Sleijpen & van der Vorst 1996, or
// defect-correction restarts) recompute r = bhat - Mhat x in FP64.
#pragma once

#include "sq_device.cuh"

namespace sq {

struct RhsState {
  double rho_re, rho_im;
  double alpha_re, alpha_im;
  double omega_re, omega_im;
  double beta_re, beta_im;
  double rnorm2;   // iterated (low-precision) residual norm^2
  double maxr2;    // max iterated ||r||^2 since the last FP64 update
  double rstart2;  // ||r||^2 at the last FP64 update
  double target2;  // stop when the FP64 Schur residual^2 <= target2
  double conv2;    // retire when the iterated residual^2 <= conv2 (target2
                   // times a safety margin for the inner precision); the
                   // full-lattice FP64 residual after the loop confirms it
  double true_r2;  // last FP64 Schur residual norm^2
  double delta2;   // update trigger (squared)
  int iter, updates, restarts, breakdowns;
  int status;        // sq_status value
  int active;        // 1 while iterating
  int want_update;   // FP64 residual requested
  int want_restart;  // BiCGStab restart requested with the update
  int max_iter;
  int defect;        // 1: restart at every FP64 update (defect correction)
  int pad[2];
};

// control block shared by all sources of a solve
struct Control {
  int n_active;   // length of the active list
  int n_update;   // length of the update list
  int err;        // sticky device error bits
  int pad;
};

enum FinKind {
  FIN_NONE = 0,
  FIN_ALPHA = 1,   // sums: <rhat,v> (re, im)
  FIN_OMEGA = 2,   // sums: <t,s> (re, im), <t,t>
  FIN_TRUE = 3,    // sums: ||r64||^2
  FIN_ITER = 4,    // sums: ||r||^2, <rhat,r> (re, im)
  FIN_UPDATE = 5,  // sums: <rhat,r> (re, im)
  FIN_STORE = 6    // sums stored to out[k*NRED + i]
};

struct RedArgs {
  double* partial;     // [k][block][NRED]
  unsigned* counter;   // [k], zero between uses
  RhsState* st;        // per-source state
  Control* ctl;        // lists and counts
  int* update_list;    // append target for FIN_ITER
  double* out;         // FIN_STORE target
  int nblk_stride;     // blocks per source in `partial`
};

template <int FIN>
__device__ __forceinline__ void finalize(const RedArgs& ra, int k, const double* s) {
  RhsState& q = ra.st[k];
  if (FIN == FIN_ALPHA) {
    double dr = s[0], di = s[1];
    double d2 = dr * dr + di * di;
    double rr = q.rho_re, ri = q.rho_im;
    if (!(d2 > 0.0) || !isfinite(d2)) {
      q.alpha_re = 0.0;
      q.alpha_im = 0.0;
      q.want_restart = 1;
      q.breakdowns++;
    } else {
      q.alpha_re = (rr * dr + ri * di) / d2;  // rho / d
      q.alpha_im = (ri * dr - rr * di) / d2;
    }
  } else if (FIN == FIN_OMEGA) {
    double tt = s[2];
    if (!(tt > 0.0) || !isfinite(tt)) {
      q.omega_re = 0.0;
      q.omega_im = 0.0;
    } else {
      q.omega_re = s[0] / tt;
      q.omega_im = s[1] / tt;
    }
  } else if (FIN == FIN_TRUE) {
    q.true_r2 = s[0];
  } else if (FIN == FIN_ITER) {
    double r2 = s[0];
    double nr = s[1], ni = s[2];  // rho'
    q.rnorm2 = r2;
    if (r2 > q.maxr2) q.maxr2 = r2;
    q.iter++;
    // beta = (rho'/rho) (alpha/omega)
    double rr = q.rho_re, ri = q.rho_im;
    double ar = q.alpha_re, ai = q.alpha_im, wr = q.omega_re, wi = q.omega_im;
    double den = (rr * rr + ri * ri) * (wr * wr + wi * wi);
    bool bad = !(den > 0.0) || !isfinite(r2) || q.want_restart;
    if (!bad) {
      // num = rho' * alpha ; dd = rho * omega
      double nre = nr * ar - ni * ai, nim = nr * ai + ni * ar;
      double dre = rr * wr - ri * wi, dim = rr * wi + ri * wr;
      q.beta_re = (nre * dre + nim * dim) / den;
      q.beta_im = (nim * dre - nre * dim) / den;
    } else {
      q.beta_re = 0.0;
      q.beta_im = 0.0;
    }
    q.rho_re = nr;
    q.rho_im = ni;
    // |rho'| negligible against ||rhat|| ||r||: near breakdown, restart
    if (!bad && (nr * nr + ni * ni) < 1e-28 * r2 * q.rstart2 && r2 > q.target2) {
      q.want_restart = 1;
      q.breakdowns++;
    }
    if (bad) q.want_restart = 1;
    if (!q.want_restart && r2 <= q.conv2) {
      // converged on the iterated residual: retire; x is flushed and the
      // FP64 full-lattice residual is checked after the loop
      q.active = 0;
      q.status = 0;
      q.true_r2 = r2;
      return;
    }
    bool upd = q.want_restart || q.iter >= q.max_iter;
    if (q.defect) {
      if (r2 < q.delta2 * q.rstart2) {
        upd = true;
        q.want_restart = 1;
      }
    } else if (r2 < q.delta2 * q.maxr2) {
      upd = true;
    }
    // the update list itself is planned for all sources at once (k_plan)
    if (upd) q.want_update = 1;
  } else if (FIN == FIN_UPDATE) {
    // r was replaced by the FP64 residual; rho = <rhat, r> with the rhat in
    // use (after a restart rhat = r, so rho = ||r||^2 up to rounding)
    q.rho_re = s[0];
    q.rho_im = s[1];
    q.rnorm2 = q.true_r2;
    q.maxr2 = q.true_r2;
    q.rstart2 = q.true_r2;
    q.updates++;
    if (q.want_restart) q.restarts++;
    q.want_restart = 0;
    q.want_update = 0;
    if (q.true_r2 <= q.target2) {
      q.active = 0;
      q.status = 0;
    } else if (!isfinite(q.true_r2)) {
      q.active = 0;
      q.status = 4;  // SQ_ERR_NONFINITE
    } else if (q.iter >= q.max_iter) {
      q.active = 0;
      q.status = 6;  // SQ_ERR_NOCONV
    } else if (q.breakdowns > 64) {
      q.active = 0;
      q.status = 7;  // SQ_ERR_BREAKDOWN
    }
  } else if (FIN == FIN_STORE) {
    // handled by the caller (needs NRED)
  }
}

// Block-level reduction of NRED doubles per source slot (threadIdx.y) over
// the sites of the block (threadIdx.x; blockDim.x is a multiple of 32), then
// across the nblk site blocks of the launch through `partial` (this block is
// site block bidx): the last block of a source (per-source arrival counter)
// sums the per-block partials in block order and runs the finaliser. The
// summation order is fixed for a fixed launch shape, so the result is
// bitwise reproducible. Every thread of the block must call this.
template <int NRED, int FIN>
__device__ __forceinline__ void reduce_finalize(const RedArgs& ra, double v[NRED], int k, int nblk, int bidx) {
  __shared__ double sm[32][NRED];  // one row per warp
  __shared__ int last[32];         // per slot: this block finishes source k
  const int lane = threadIdx.x & 31;
  const int wx = threadIdx.x >> 5;
  const int nwx = blockDim.x >> 5;
  const int ty = threadIdx.y;
#pragma unroll
  for (int i = 0; i < NRED; i++) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NRED; i++) sm[ty * nwx + wx][i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int is_last = 0;
    if (k >= 0) {
      double acc[NRED];
#pragma unroll
      for (int i = 0; i < NRED; i++) acc[i] = 0.0;
      for (int w = 0; w < nwx; w++)
#pragma unroll
        for (int i = 0; i < NRED; i++) acc[i] += sm[ty * nwx + w][i];
      double* dst = ra.partial + ((size_t)k * ra.nblk_stride + bidx) * NRED;
#pragma unroll
      for (int i = 0; i < NRED; i++) dst[i] = acc[i];
      __threadfence();
      unsigned prev = atomicAdd(ra.counter + k, 1u);
      is_last = (prev == (unsigned)nblk - 1u);
    }
    last[ty] = is_last;
  }
  __syncthreads();
  if (last[ty]) {
    __threadfence();
    double acc[NRED];
#pragma unroll
    for (int i = 0; i < NRED; i++) acc[i] = 0.0;
    const double* src = ra.partial + (size_t)k * ra.nblk_stride * NRED;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
      for (int i = 0; i < NRED; i++) acc[i] += __ldcg(src + (size_t)b * NRED + i);
#pragma unroll
    for (int i = 0; i < NRED; i++) acc[i] = warp_sum(acc[i]);
    // second level inside this slot's warps: reuse sm rows of this slot
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NRED; i++) sm[ty * nwx + wx][i] = acc[i];
    }
  }
  __syncthreads();
  if (last[ty] && threadIdx.x == 0) {
    double tot[NRED];
#pragma unroll
    for (int i = 0; i < NRED; i++) tot[i] = 0.0;
    for (int w = 0; w < nwx; w++)
#pragma unroll
      for (int i = 0; i < NRED; i++) tot[i] += sm[ty * nwx + w][i];
    if (FIN == FIN_STORE) {
#pragma unroll
      for (int i = 0; i < NRED; i++) ra.out[(size_t)k * NRED + i] = tot[i];
    } else {
      finalize<FIN>(ra, k, tot);
    }
    ra.counter[k] = 0u;
  }
}

}  // namespace sq

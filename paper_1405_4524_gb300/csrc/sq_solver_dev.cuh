// Per-source solver state kept on the device, the deterministic reductions
// (per-warp partials added up by a finishing kernel in the inner loop; a
// "last block finalises" scheme for the norms) and the BiCGStab scalar
// updates that run where a source's sums are complete.
//
// BiCGStab (van der Vorst 1992) per source k, on the even-odd Schur system
// Mhat x = bhat:  v = Mhat p; alpha = rho/<rhat,v>; s = r - alpha v;
// t = Mhat s; omega = <t,s>/<t,t>; x += alpha p + omega s; r = s - omega t;
// rho' = <rhat,r>; beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v).
// FP64 updates (reliable updates, Sleijpen & van der Vorst 1996, or
// defect-correction restarts) recompute r = bhat - Mhat x in FP64. With an
// FP16 inner recurrence the reliable updates whose residual is still far
// above the FP32 floor recompute it in FP32 instead (a refresh: same
// operator, FP32 fields, x = x64 + xs rounded once); below the floor they
// are FP64 updates.
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
  double ref2;     // residual^2 of the first FP64 update (the reference for
                   // FP32 refreshes)
  double bd2;      // near-breakdown threshold: restart when |rho'|^2 <
                   // bd2 ||rhat||^2 ||r||^2
  int iter, updates, restarts, breakdowns;
  int status;        // sq_status value
  int active;        // 1 while iterating
  int want_update;   // FP64 residual requested
  int want_restart;  // BiCGStab restart requested with the update
  int max_iter;
  int defect;        // 1: restart at every FP64 update (defect correction)
  int refresh;       // 1: updates above the FP32 floor are FP32 refreshes
  int refreshes;     // FP32 residual refreshes done
};

// control block shared by all sources of a solve
struct Control {
  int n_active;   // length of the active list
  int n_update;   // length of the update list
  int n_refresh;  // length of the refresh list
  int err;        // sticky device error bits
  int launched;   // kernels run inside conditional graph nodes (counted by
                  // k_plan when it switches a node on)
  int pad;
};

enum FinKind {
  FIN_NONE = 0,
  FIN_ALPHA = 1,   // sums: <rhat,v> (re, im)
  FIN_OMEGA = 2,   // sums: <t,s> (re, im), <t,t>
  FIN_TRUE = 3,    // sums: ||r64||^2
  FIN_ITER = 4,    // sums: ||r||^2, <rhat,r> (re, im)
  FIN_UPDATE = 5,  // sums: <rhat,r> (re, im)
  FIN_STORE = 6,   // sums stored to out[k*NRED + i]
  FIN_REFRESH = 7  // sums: <rhat,r> (re, im) after an FP32 refresh
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
    if (!bad && (nr * nr + ni * ni) < q.bd2 * r2 * q.rstart2 && r2 > q.target2) {
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
    if (q.updates == 0) q.ref2 = q.true_r2;
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
  } else if (FIN == FIN_REFRESH) {
    // r was replaced by the residual recomputed in FP32 (far above the
    // FP32 floor, so its rounding is negligible); the Krylov space is kept
    q.rho_re = s[0];
    q.rho_im = s[1];
    q.rnorm2 = q.true_r2;
    q.maxr2 = q.true_r2;
    q.rstart2 = q.true_r2;
    q.refreshes++;
    q.want_update = 0;
    if (!isfinite(q.true_r2)) {
      q.active = 0;
      q.status = 4;  // SQ_ERR_NONFINITE
    }
  } else if (FIN == FIN_STORE) {
    // handled by the caller (needs NRED)
  }
}

// Second half of every reduction: thread x = 0 of slot ty holds the block's
// NRED sums for source k (k < 0: idle slot). They go to `partial` (this is
// site block bidx of nblk); the last block of a source (per-source arrival
// counter) sums the per-block partials in block order in FP64 and runs the
// finaliser. The summation order is fixed for a fixed launch shape, so the
// result is bitwise reproducible. Every thread of the block must call this.
template <int NRED, int FIN>
__device__ __forceinline__ void reduce_across_blocks(const RedArgs& ra, const double blk[NRED], int k, int nblk,
                                                     int bidx) {
  __shared__ double sm[32][NRED];  // one row per warp
  __shared__ int last[32];         // per slot: this block finishes source k
  const int lane = threadIdx.x & 31;
  const int wx = threadIdx.x >> 5;
  const int nwx = blockDim.x >> 5;
  const int ty = threadIdx.y;
  if (threadIdx.x == 0) {
    int is_last = 0;
    if (k >= 0) {
      double* dst = ra.partial + ((size_t)k * ra.nblk_stride + bidx) * NRED;
#pragma unroll
      for (int i = 0; i < NRED; i++) dst[i] = blk[i];
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

// Block-level reduction of NRED doubles per source slot (threadIdx.y) over
// the sites of the block (threadIdx.x; blockDim.x is a multiple of 32),
// then across blocks (reduce_across_blocks). Used by the FP64 update path
// and the norms; the inner iteration uses warp_partials + k_finish.
template <int NRED, int FIN>
__device__ __forceinline__ void reduce_finalize(const RedArgs& ra, double v[NRED], int k, int nblk, int bidx) {
  __shared__ double sm[32][NRED];
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
  double blk[NRED];
#pragma unroll
  for (int i = 0; i < NRED; i++) blk[i] = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nwx; w++)
#pragma unroll
      for (int i = 0; i < NRED; i++) blk[i] += sm[ty * nwx + w][i];
  reduce_across_blocks<NRED, FIN>(ra, blk, k, nblk, bidx);
}

// FP32 per-thread values on the same path (the FP64 update path's
// reductions of FP32 fields): summed in FP64 from the warp level up.
template <int NRED, int FIN>
__device__ __forceinline__ void reduce_finalize(const RedArgs& ra, float v[NRED], int k, int nblk, int bidx) {
  double d[NRED];
#pragma unroll
  for (int i = 0; i < NRED; i++) d[i] = (double)v[i];
  reduce_finalize<NRED, FIN>(ra, d, k, nblk, bidx);
}

// Per-warp partial sums for the reductions of the inner iteration (no
// cross-block synchronisation in the producing kernel): warp j of source k
// writes its NRED sums to partial[(k * nblk_stride + j) * NRED + i], and
// k_finish adds them up per source in a fixed order in FP64 and runs the
// finaliser. A fence-and-counter "last block" scheme here made every CTA
// wait for its own output stores; the kernel boundary orders them for free.
// FP32 values (FP32 / FP16 fields) are summed across the warp in FP32 and
// stored as float (they are sums of FP32 products already); FP64 in FP64.
// All 32 lanes of the warp must call this.
template <int NRED>
__device__ __forceinline__ void warp_partials(const RedArgs& ra, float v[NRED], int k, int j) {
#pragma unroll
  for (int i = 0; i < NRED; i++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if ((threadIdx.x & 31) == 0 && k >= 0) {
    float* dst = (float*)ra.partial + ((size_t)k * ra.nblk_stride + j) * NRED;
#pragma unroll
    for (int i = 0; i < NRED; i++) dst[i] = v[i];
  }
}

template <int NRED>
__device__ __forceinline__ void warp_partials(const RedArgs& ra, double v[NRED], int k, int j) {
#pragma unroll
  for (int i = 0; i < NRED; i++) v[i] = warp_sum(v[i]);
  if ((threadIdx.x & 31) == 0 && k >= 0) {
    double* dst = ra.partial + ((size_t)k * ra.nblk_stride + j) * NRED;
#pragma unroll
    for (int i = 0; i < NRED; i++) dst[i] = v[i];
  }
}

// One CTA per source slot: sum the nparts per-warp partials of source k in
// FP64 (fixed thread assignment and tree: bitwise reproducible for a fixed
// launch shape) and run the finaliser. T is the partials' type.
template <typename T, int NRED, int FIN>
__global__ void __launch_bounds__(256) k_finish(const RedArgs ra, const int* list, const int* count, int n,
                                                int nparts) {
  __shared__ double sm[8][NRED];
  const int cnt = count ? *count : n;
  const int slot = blockIdx.x;
  if (slot >= cnt) return;
  const int k = list ? list[slot] : slot;
  const T* src = (const T*)ra.partial + (size_t)k * ra.nblk_stride * NRED;
  double acc[NRED];
#pragma unroll
  for (int i = 0; i < NRED; i++) acc[i] = 0.0;
  for (int j = threadIdx.x; j < nparts; j += blockDim.x)
#pragma unroll
    for (int i = 0; i < NRED; i++) acc[i] += (double)src[(size_t)j * NRED + i];
#pragma unroll
  for (int i = 0; i < NRED; i++) acc[i] = warp_sum(acc[i]);
  const int wx = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < NRED; i++) sm[wx][i] = acc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[NRED];
#pragma unroll
    for (int i = 0; i < NRED; i++) tot[i] = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++)
#pragma unroll
      for (int i = 0; i < NRED; i++) tot[i] += sm[w][i];
    if (FIN == FIN_STORE) {
#pragma unroll
      for (int i = 0; i < NRED; i++) ra.out[(size_t)k * NRED + i] = tot[i];
    } else {
      finalize<FIN>(ra, k, tot);
    }
  }
}

}  // namespace sq

// Batched even-odd BiCGStab for the clover-Wilson system M psi = eta, one
// Krylov recurrence per source, all sources advanced by the same kernels.
//
// Schur system on even sites (M = [[A_ee, -k D_eo], [-k D_oe, A_oo]]):
//   Mhat = 1 - k^2 A_ee^{-1} D_eo A_oo^{-1} D_oe,
//   bhat = A_ee^{-1} (eta_e + k D_eo A_oo^{-1} eta_o),
//   psi_o = A_oo^{-1} (eta_o + k D_oe psi_e).
// The full-lattice residual is r_e = A_ee (bhat - Mhat psi_e), r_o = 0, so
// ||r|| <= max||A|| ||bhat - Mhat psi_e||: the Schur target is
// tol ||eta|| / max||A||, and the full FP64 residual is checked at the end.
//
// Precision: the inner recurrence runs on FP32 or FP16 (per-site norm)
// fields with FP32 arithmetic; x accumulates in FP32; every FP64 update
// recomputes r = bhat - Mhat x in FP64 (reliable updates keep the Krylov
// space, defect correction restarts it). With inner FP64 the same loop is
// the plain FP64 solver (an FP64 update only to confirm convergence).
//
// One iteration = 12 kernels, all reading their per-source scalars and the
// active / update lists from device memory, so `chunk` iterations are
// captured once into a CUDA graph and replayed; the host reads one integer
// (sources still active) per graph launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sq_internal.h"

namespace sq {

static const Shape kBlasShape = {128, 2, 0};
// kernels of one inner iteration outside the update paths (two plain and
// two fused dslash, three k_finish, s / x,r / p updates, plan, control) and
// inside each update path (FP64 update or FP32 refresh: x, two operator
// launches, two k_finish, r)
static const int kChainLaunches = 12;
static const int kUpdateLaunches = 6;
// host sources are copied in this many groups, overlapped with the FP64
// Schur-source build of the previous group
static const int kSetupGroups = 4;
// FP64 dslash: ~146 registers per thread; 64-thread CTAs keep 7 per SM resident
static const Shape k64Shape = {64, 1, 0};

struct VArgs {
  int Vh;
  Field f0, f1, f2, f3, f4, f5;
  RhsState* st;
  const int* list;
  const int* count;
  int n;
  RedArgs ra;
};

// Source slots of a list: CTA row y covers slots blockIdx.y * blockDim.y +
// threadIdx.y, then strides by the grid's rows. The inner loop launches
// ceil(n / rows) CTA rows (one pass); the FP64 update path launches one CTA
// row that walks the list, so a launch with an empty list costs one row of
// CTAs instead of n / rows of them. The trip count is uniform in a CTA.
#define SLOT_LOOP_BEGIN                                                                   \
  const int cnt = *a.count;                                                               \
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;                                   \
  for (int slot0 = blockIdx.y * blockDim.y; slot0 < cnt; slot0 += gridDim.y * blockDim.y) { \
    const int slot = slot0 + threadIdx.y;                                                 \
    const int k = slot < cnt ? a.list[slot] : -1;                                         \
    const bool ok = (k >= 0) && (cb < a.Vh);
#define SLOT_LOOP_END }

// s = r - alpha v          f0 = r, f1 = v, f2 = s
template <int P>
__global__ void __launch_bounds__(256) k_s_update(const VArgs a) {
  typedef typename Real<P>::T R;
  SLOT_LOOP_BEGIN
    if (!ok) continue;
    const RhsState& q = a.st[k];
    const R ar = (R)q.alpha_re, ai = (R)q.alpha_im;
    cx<R> r[12], v[12];
    SpinorIO<P>::load(a.f0, k, cb, r);
    SpinorIO<P>::load(a.f1, k, cb, v);
#pragma unroll
    for (int j = 0; j < 12; j++)
      r[j] = mk(r[j].re - (ar * v[j].re - ai * v[j].im), r[j].im - (ar * v[j].im + ai * v[j].re));
    SpinorIO<P>::store(a.f2, k, cb, r);
  SLOT_LOOP_END
}

// x += alpha p + omega s ; r = s - omega t ; reduce ||r||^2, <rhat, r>
// f0 = x (PX), f1 = p, f2 = s, f3 = t, f4 = r, f5 = rhat
template <int P, int PX>
__global__ void __launch_bounds__(256) k_xr_update(const VArgs a) {
  typedef typename Real<P>::T R;
  typedef typename Real<PX>::T RX;
  SLOT_LOOP_BEGIN
    typedef typename SumOf<R>::T S;
    S red[3] = {(S)0, (S)0, (S)0};
    if (ok) {
      const RhsState& q = a.st[k];
      const R ar = (R)q.alpha_re, ai = (R)q.alpha_im, wr = (R)q.omega_re, wi = (R)q.omega_im;
      cx<R> p[12], s[12];
      cx<RX> x[12];
      SpinorIO<P>::load(a.f1, k, cb, p);
      SpinorIO<P>::load(a.f2, k, cb, s);
      SpinorIO<PX>::load(a.f0, k, cb, x);
#pragma unroll
      for (int j = 0; j < 12; j++) {
        R dr = ar * p[j].re - ai * p[j].im + wr * s[j].re - wi * s[j].im;
        R di = ar * p[j].im + ai * p[j].re + wr * s[j].im + wi * s[j].re;
        x[j] = mk((RX)(x[j].re + dr), (RX)(x[j].im + di));
      }
      SpinorIO<PX>::store(a.f0, k, cb, x);
      cx<R> t[12], rh[12];
      SpinorIO<P>::load(a.f3, k, cb, t);
#pragma unroll
      for (int j = 0; j < 12; j++)
        s[j] = mk(s[j].re - (wr * t[j].re - wi * t[j].im), s[j].im - (wr * t[j].im + wi * t[j].re));
      SpinorIO<P>::store(a.f4, k, cb, s);
      SpinorIO<ShadowPrec<P>::value>::load(a.f5, k, cb, rh);
      S n2 = 0, dr = 0, di = 0;
#pragma unroll
      for (int j = 0; j < 12; j++) {
        n2 += (S)s[j].re * s[j].re + (S)s[j].im * s[j].im;
        dr += (S)rh[j].re * s[j].re + (S)rh[j].im * s[j].im;
        di += (S)rh[j].re * s[j].im - (S)rh[j].im * s[j].re;
      }
      red[0] = n2;
      red[1] = dr;
      red[2] = di;
    }
    warp_partials<3>(a.ra, red, k, (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)));
  SLOT_LOOP_END
}

// p = r + beta (p - omega v)     f0 = r, f1 = p, f2 = v
template <int P>
__global__ void __launch_bounds__(256) k_p_update(const VArgs a) {
  typedef typename Real<P>::T R;
  SLOT_LOOP_BEGIN
    if (!ok) continue;
    const RhsState& q = a.st[k];
    const R br = (R)q.beta_re, bi = (R)q.beta_im, wr = (R)q.omega_re, wi = (R)q.omega_im;
    cx<R> r[12], p[12], v[12];
    SpinorIO<P>::load(a.f0, k, cb, r);
    SpinorIO<P>::load(a.f1, k, cb, p);
    SpinorIO<P>::load(a.f2, k, cb, v);
#pragma unroll
    for (int j = 0; j < 12; j++) {
      R ur = p[j].re - (wr * v[j].re - wi * v[j].im);
      R ui = p[j].im - (wr * v[j].im + wi * v[j].re);
      p[j] = mk(r[j].re + br * ur - bi * ui, r[j].im + br * ui + bi * ur);
    }
    SpinorIO<P>::store(a.f1, k, cb, p);
  SLOT_LOOP_END
}

// FP64 update, part 1: x64 += xs ; xs = 0 ; r64 = b64 - x64
// f0 = x64, f1 = xs (PX), f2 = b64, f3 = r64
template <int PX>
__global__ void __launch_bounds__(256) k_rel_x(const VArgs a) {
  typedef typename Real<PX>::T RX;
  SLOT_LOOP_BEGIN
    if (!ok) continue;
    cx<double> x[12], b[12];
    cx<RX> xs[12];
    SpinorIO<P64>::load(a.f0, k, cb, x);
    SpinorIO<PX>::load(a.f1, k, cb, xs);
    SpinorIO<P64>::load(a.f2, k, cb, b);
#pragma unroll
    for (int j = 0; j < 12; j++) {
      x[j] = mk(x[j].re + (double)xs[j].re, x[j].im + (double)xs[j].im);
      b[j] = b[j] - x[j];
      xs[j] = mk((RX)0, (RX)0);
    }
    SpinorIO<P64>::store(a.f0, k, cb, x);
    SpinorIO<PX>::store(a.f1, k, cb, xs);
    SpinorIO<P64>::store(a.f3, k, cb, b);
  SLOT_LOOP_END
}

// FP32 refresh, part 1: x32 = x64 + xs and r32 = bhat - x64 - xs, both
// formed in FP64 and rounded once.  f0 = x64, f1 = xs (PX), f2 = b64,
// f3 = x32 (FP32), f4 = r32 (FP32)
template <int PX>
__global__ void __launch_bounds__(256) k_ref_x(const VArgs a) {
  typedef typename Real<PX>::T RX;
  SLOT_LOOP_BEGIN
    if (!ok) continue;
    cx<double> x[12], b[12];
    cx<RX> xs[12];
    SpinorIO<P64>::load(a.f0, k, cb, x);
    SpinorIO<PX>::load(a.f1, k, cb, xs);
    SpinorIO<P64>::load(a.f2, k, cb, b);
    cx<float> x32[12], r32[12];
#pragma unroll
    for (int j = 0; j < 12; j++) {
      const double xr = x[j].re + (double)xs[j].re, xi = x[j].im + (double)xs[j].im;
      x32[j] = mk((float)xr, (float)xi);
      r32[j] = mk((float)(b[j].re - xr), (float)(b[j].im - xi));
    }
    SpinorIO<P32>::store(a.f3, k, cb, x32);
    SpinorIO<P32>::store(a.f4, k, cb, r32);
  SLOT_LOOP_END
}

// FP64 update (or FP32 refresh), part 2: r = r64 (r32) ; on restart
// rhat = r, p = r ; reduce <rhat, r>.  f0 = r64 (PS), f1 = r, f2 = rhat, f3 = p
template <int P, int PS>
__global__ void __launch_bounds__(256) k_rel_r(const VArgs a) {
  typedef typename Real<P>::T R;
  SLOT_LOOP_BEGIN
    typedef typename SumOf<R>::T S;
    S red[2] = {(S)0, (S)0};
    if (ok) {
      const bool restart = a.st[k].want_restart != 0;
      cx<typename Real<PS>::T> r64[12];
      SpinorIO<PS>::load(a.f0, k, cb, r64);
      cx<R> r[12], rh[12];
#pragma unroll
      for (int j = 0; j < 12; j++) r[j] = mk((R)r64[j].re, (R)r64[j].im);
      SpinorIO<P>::store(a.f1, k, cb, r);
      if (restart) {  // rhat = r as stored (rounded to its storage precision)
        SpinorIO<ShadowPrec<P>::value>::store(a.f2, k, cb, r);
        SpinorIO<P>::store(a.f3, k, cb, r);
#pragma unroll
        for (int j = 0; j < 12; j++) rh[j] = r[j];
        SpinorIO<ShadowPrec<P>::value>::round_trip(rh);
      } else {
        SpinorIO<ShadowPrec<P>::value>::load(a.f2, k, cb, rh);
      }
      S dr = 0, di = 0;
#pragma unroll
      for (int j = 0; j < 12; j++) {
        dr += (S)rh[j].re * r[j].re + (S)rh[j].im * r[j].im;
        di += (S)rh[j].re * r[j].im - (S)rh[j].im * r[j].re;
      }
      red[0] = dr;
      red[1] = di;
    }
    warp_partials<2>(a.ra, red, k, (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)));
  SLOT_LOOP_END
}

// ||r64||^2 into the sources' true residual (initial update with x = 0,
// where r64 = bhat exactly and no FP64 operator is needed).  f0 = r64
__global__ void __launch_bounds__(256) k_true_norm(const VArgs a) {
  SLOT_LOOP_BEGIN
    double red[1] = {0.0};
    if (ok) {
      cx<double> r[12];
      SpinorIO<P64>::load(a.f0, k, cb, r);
      double t = 0;
#pragma unroll
      for (int j = 0; j < 12; j++) t += r[j].re * r[j].re + r[j].im * r[j].im;
      red[0] = t;
    }
    reduce_finalize<1, FIN_TRUE>(a.ra, red, k, (int)gridDim.x, (int)blockIdx.x);
  SLOT_LOOP_END
}

// Rebuild the active list (ascending source index) and clear the update list.
// hist (optional) records the list lengths this iteration ran with.
__global__ void k_control(RhsState* st, Control* ctl, int* active_list, int n, int* hist, int it, int chunk) {
  const int lane = threadIdx.x;
  if (hist && lane == 0) {
    hist[it] = ctl->n_active;
    hist[chunk + it] = ctl->n_update;
  }
  __syncwarp();
  int base = 0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int k = k0 + lane;
    const bool on = k < n && st[k].active;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (on) active_list[base + __popc(m & ((1u << lane) - 1u))] = k;
    base += __popc(m);
  }
  if (lane == 0) {
    ctl->n_active = base;
    ctl->n_update = 0;
  }
}

// Plan the updates of this iteration for all sources at once. A source is
// updated when it asked for it, or - if any source asked - when its
// iterated residual is already within a factor 5 of its own trigger (a
// couple of iterations away): the updates of sources that converge at
// similar rates then share launches instead of each running an almost
// empty one, without adding updates. A joining source whose residual is
// still far above the FP32 floor (|r|^2 > kRefreshFloor * ref2, FP16 inner
// recurrence, no restart) gets an FP32 refresh, the others an FP64
// update. Lists are in ascending source order (deterministic). In a
// captured graph the two conditional nodes that hold the refresh and the
// FP64 update run only when their list is non-empty.
constexpr double kRefreshFloor = 1e-12;

__global__ void k_plan(RhsState* st, Control* ctl, int* update_list, int* refresh_list, int n,
                       cudaGraphConditionalHandle h_upd, cudaGraphConditionalHandle h_ref, int use_h) {
  const int lane = threadIdx.x;
  bool any = false;
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int k = k0 + lane;
    const bool w = k < n && st[k].active && st[k].want_update;
    any = __any_sync(0xffffffffu, w) || any;
  }
  int nu = 0, nr = 0;
  if (any) {
    for (int k0 = 0; k0 < n; k0 += 32) {
      const int k = k0 + lane;
      bool up = false, rf = false;
      if (k < n && st[k].active) {
        RhsState& q = st[k];
        const double ref = q.defect ? q.rstart2 : q.maxr2;
        if (q.want_update || q.rnorm2 < 25.0 * q.delta2 * ref) {
          q.want_update = 1;
          if (q.defect) q.want_restart = 1;
          rf = q.refresh && !q.defect && !q.want_restart && q.updates > 0 && q.iter < q.max_iter &&
               q.rnorm2 > kRefreshFloor * q.ref2;
          up = !rf;
        }
      }
      const unsigned mu = __ballot_sync(0xffffffffu, up), mr = __ballot_sync(0xffffffffu, rf);
      const unsigned below = (1u << lane) - 1u;
      if (up) update_list[nu + __popc(mu & below)] = k;
      if (rf) refresh_list[nr + __popc(mr & below)] = k;
      nu += __popc(mu);
      nr += __popc(mr);
    }
  }
  if (lane == 0) {
    ctl->n_update = nu;
    ctl->n_refresh = nr;
    if (use_h) {
      cudaGraphSetConditional(h_upd, nu > 0 ? 1u : 0u);
      if (h_ref) cudaGraphSetConditional(h_ref, nr > 0 ? 1u : 0u);
      ctl->launched += (nu > 0 ? kUpdateLaunches : 0) + (nr > 0 && h_ref ? kUpdateLaunches : 0);
    }
  }
}

// x64 += xs ; xs = 0 for every source (after the loop: sources that retired
// on their iterated residual still hold their last correction in xs).
// f0 = x64, f1 = xs (PX)
template <int PX>
__global__ void __launch_bounds__(256) k_flush(const VArgs a) {
  typedef typename Real<PX>::T RX;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (cb >= a.Vh || k >= a.n) return;
  cx<double> x[12];
  cx<RX> xs[12];
  SpinorIO<P64>::load(a.f0, k, cb, x);
  SpinorIO<PX>::load(a.f1, k, cb, xs);
#pragma unroll
  for (int j = 0; j < 12; j++) {
    x[j] = mk(x[j].re + (double)xs[j].re, x[j].im + (double)xs[j].im);
    xs[j] = mk((RX)0, (RX)0);
  }
  SpinorIO<P64>::store(a.f0, k, cb, x);
  SpinorIO<PX>::store(a.f1, k, cb, xs);
}

// Initial state: every source asks for an FP64 update with restart.
__global__ void k_init(RhsState* st, Control* ctl, int* update_list, const double* target2, double delta2,
                       double margin2, int max_iter, int defect, int refresh, double bd2, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    RhsState q;
    memset(&q, 0, sizeof(q));
    q.target2 = target2[k];
    q.conv2 = target2[k] * margin2;
    q.delta2 = delta2;
    q.max_iter = max_iter;
    q.defect = defect;
    q.refresh = refresh;
    q.bd2 = bd2;
    q.active = 1;
    q.want_update = 1;
    q.want_restart = 1;
    q.status = 0;
    q.rho_re = 1.0;
    q.alpha_re = 1.0;
    q.omega_re = 1.0;
    st[k] = q;
    update_list[k] = k;
  }
  if (k == 0) {
    ctl->n_update = n;
    ctl->n_refresh = 0;
    ctl->n_active = 0;
    ctl->launched = 0;
  }
}


// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static inline int px_of(int inner) { return inner == P64 ? P64 : P32; }

static void free_ws(Workspace& w) {
  if (w.aux) {
    cudaStreamSynchronize(w.aux);
    cudaStreamDestroy(w.aux);
  }
  if (w.ev_rec) cudaEventDestroy(w.ev_rec);
  if (w.ev_out) cudaEventDestroy(w.ev_out);
  for (auto ev : w.ev_in)
    if (ev) cudaEventDestroy(ev);
  if (w.graph) cudaGraphExecDestroy(w.graph);
  if (w.graph2) cudaGraphExecDestroy(w.graph2);
  for (auto e : w.pev) cudaEventDestroy(e);
  dev_free(w.mem, w.hist, 2 * (size_t)w.hist_chunk * sizeof(int));
  dev_free(w.mem, w.base, w.bytes);
  if (w.h_pin) cudaFreeHost(w.h_pin);
  w = Workspace();
}

void release_workspace(sq_ctx* c) {
  free_ws(c->ws);
  if (c->batch) {
    BatchCache* b = c->batch;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto* w : b->ws) {
      free_ws(*w);
      delete w;
    }
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->events) cudaEventDestroy(e);
    delete b;
    c->batch = nullptr;
  }
}

static sq_status alloc_ws(sq_ctx* c, Workspace& w, int n, int inner) {
  if (w.base && w.n_rhs == n && w.inner == inner && w.Vh == c->Vh) return SQ_OK;
  free_ws(w);
  const int Vh = c->Vh;
  const size_t f64 = field_bytes(Vh, P64, n), fin = field_bytes(Vh, inner, n);
  const size_t fx = field_bytes(Vh, px_of(inner), n);
  // per source: one partial per warp of the launch with the most warps per
  // site (the emulated-FP64 operator: two threads per site, 16 sites per
  // warp), rounded up per CTA of up to 32 warps
  const int nblk = (Vh + 15) / 16 + 32;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t tot = 0;
  size_t o_f64 = tot; tot += al(f64) * 7;
  size_t o_fin = tot; tot += al(fin) * 7;
  size_t o_fx = tot; tot += al(fx);
  size_t o_lex = tot; tot += al((size_t)n * c->V * 24 * sizeof(double));
  size_t o_part = tot; tot += al((size_t)n * nblk * 3 * sizeof(double));
  size_t o_cnt = tot; tot += al((size_t)n * sizeof(unsigned));
  size_t o_st = tot; tot += al((size_t)n * sizeof(RhsState));
  size_t o_ctl = tot; tot += al(sizeof(Control));
  size_t o_al = tot; tot += al((size_t)n * sizeof(int));
  size_t o_ul = tot; tot += al((size_t)n * sizeof(int));
  size_t o_rl = tot; tot += al((size_t)n * sizeof(int));
  size_t o_sc = tot; tot += al((size_t)n * 8 * sizeof(double));
  size_t o_pi = tot; tot += al((size_t)n * c->dims[3] * sizeof(double));
  size_t o_ts = tot; tot += al((size_t)n * sizeof(int));
  size_t o_fl = tot; tot += al(sizeof(int));
  void* base = nullptr;
  cudaError_t e = dev_alloc(c->mem, &base, tot);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, SQ_ERR_OOM, "workspace of %zu bytes for %d sources: %s", tot, n, cudaGetErrorString(e));
  }
  char* b = (char*)base;
  w.mem = c->mem;
  w.base = base;
  w.bytes = tot;
  w.n_rhs = n;
  w.inner = inner;
  w.Vh = Vh;
  Field* f64s[7] = {&w.b64, &w.x64, &w.r64, &w.t64o, &w.x64o, &w.eta_e, &w.eta_o};
  for (int i = 0; i < 7; i++) *f64s[i] = make_field(b + o_f64 + al(f64) * i, Vh, P64, n);
  Field* fins[7] = {&w.r, &w.rh, &w.p, &w.v, &w.s, &w.t, &w.to};
  for (int i = 0; i < 7; i++) *fins[i] = make_field(b + o_fin + al(fin) * i, Vh, inner, n);
  w.rh = make_field(w.rh.data, Vh, inner == P64 ? P64 : P16, n);  // the shadow residual (ShadowPrec)
  w.xs = make_field(b + o_fx, Vh, px_of(inner), n);
  w.lex = (double*)(b + o_lex);
  w.partial = (double*)(b + o_part);
  w.counter = (unsigned*)(b + o_cnt);
  w.st = (RhsState*)(b + o_st);
  w.ctl = (Control*)(b + o_ctl);
  w.active_list = (int*)(b + o_al);
  w.update_list = (int*)(b + o_ul);
  w.refresh_list = (int*)(b + o_rl);
  w.scal = (double*)(b + o_sc);
  w.pion = (double*)(b + o_pi);
  w.tsl = (int*)(b + o_ts);
  w.flag = (int*)(b + o_fl);
  w.nblk_stride = nblk;
  // highest priority: the output kernels are scheduled ahead of the pending
  // CTAs of the FP64 check, so the copy-out starts early
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  e = cudaStreamCreateWithPriority(&w.aux, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_rec, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_out, cudaEventDisableTiming);
  for (int g = 0; g < kSetupGroups && e == cudaSuccess; g++)
    e = cudaEventCreateWithFlags(&w.ev_in[g], cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_check(c, e, "workspace stream");
  e = cudaMemset(w.counter, 0, (size_t)n * sizeof(unsigned));
  return cuda_check(c, e, "workspace counters");
}

static RedArgs red_args(const Workspace& w) {
  RedArgs r;
  r.partial = w.partial;
  r.counter = w.counter;
  r.st = w.st;
  r.ctl = w.ctl;
  r.update_list = w.update_list;
  r.out = w.scal;
  r.nblk_stride = w.nblk_stride;
  return r;
}

static VArgs vargs(const sq_ctx* c, const Workspace& w, bool update_list) {
  VArgs a;
  memset(&a, 0, sizeof(a));
  a.Vh = c->Vh;
  a.st = w.st;
  a.list = update_list ? w.update_list : w.active_list;
  a.count = update_list ? &w.ctl->n_update : &w.ctl->n_active;
  a.n = w.n_rhs;
  a.ra = red_args(w);
  return a;
}

// Event marks between the kernels of one iteration (profiling only). Inside
// a stream capture the records become event-record graph nodes.
struct Marks {
  cudaEvent_t* ev = nullptr;  // KC_N + 1 events for this iteration
  unsigned mask = 0;          // marks that record (mark kc opens class kc)
  bool capture = false;
  bool cond = false;          // capturing: FP64 update path under an IF node
  bool* cond_failed = nullptr;  // set when a conditional node could not be added
  int i = 0;
  void mark(cudaStream_t s) {
    if (!ev) return;
    if ((mask >> i) & 1u) {
      if (capture) cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
      else cudaEventRecord(ev[i], s);
    }
    i++;
  }
};

// profile = 1: every class; profile = 2: the two clover dslash launches
// only (four event nodes per iteration instead of fourteen)
static unsigned profile_mask(int profile) {
  if (profile == 2)
    return (1u << KC_DSLASH_CLOVER) | (1u << (KC_DSLASH_CLOVER + 1)) | (1u << KC_DSLASH_CLOVER_2) |
           (1u << (KC_DSLASH_CLOVER_2 + 1));
  return (1u << (KC_N + 1)) - 1u;
}

// Stream capture of a conditional IF node: the node is added after the
// current dependencies of the capturing stream s, its body is captured on
// `body` (a second stream); cond_end makes the node the new dependency of s.
// Returns nullptr (and captures nothing on `body`) if the node could not be
// added; the caller then launches the body on s.
static cudaStream_t cond_begin(cudaStream_t s, cudaStream_t body, cudaGraphConditionalHandle h,
                               cudaGraphNode_t* node) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess ||
      cst != cudaStreamCaptureStatusActive || !cg)
    return nullptr;
  // (the union inside has no default constructor: zeroed storage)
  alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
  memset(cpbuf, 0, sizeof(cpbuf));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cpbuf);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  if (cudaGraphAddNode(node, cg, deps, nullptr, nd, &cp) != cudaSuccess || !cp.conditional.phGraph_out ||
      !cp.conditional.phGraph_out[0])
    return nullptr;
  if (cudaStreamBeginCaptureToGraph(body, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return nullptr;
  return body;
}

static void cond_end(cudaStream_t s, cudaStream_t body, cudaGraphNode_t node) {
  cudaGraph_t g = nullptr;
  cudaStreamEndCapture(body, &g);
  cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

template <int P, int PX>
static void launch_iteration(sq_ctx* c, Workspace& w, const CloverSet& cs, double kappa, Shape sh, cudaStream_t s,
                             Marks m, int it, int chunk) {
  typedef typename Real<P>::T R;
  const int n = w.n_rhs;
  dim3 bb(kBlasShape.sx, kBlasShape.ry);
  dim3 bg((c->Vh + kBlasShape.sx - 1) / kBlasShape.sx, (n + kBlasShape.ry - 1) / kBlasShape.ry);
  DslashCall d;
  memset(&d, 0, sizeof(d));
  d.prec = P;
  d.recon = P == P64 ? 18 : c->recon;  // FP16 fields use the FP32 links
  d.cs = &cs;
  d.list = w.active_list;
  d.count = &w.ctl->n_active;
  d.n = n;
  d.ra = red_args(w);
  d.shape = sh;
  d.clover = 1;
  m.mark(s);
  // v = Mhat p ; alpha
  d.out = w.to; d.in = w.p; d.p_out = 1; d.xpay = 0; d.fin = FIN_NONE;
  launch_dslash(c, d, s);
  m.mark(s);
  d.out = w.v; d.in = w.to; d.x = w.p; d.p_out = 0; d.xpay = 1; d.a = -kappa * kappa;
  d.fin = FIN_ALPHA; d.r1 = w.rh;
  launch_dslash(c, d, s);
  m.mark(s);
  VArgs a = vargs(c, w, false);
  a.f0 = w.r; a.f1 = w.v; a.f2 = w.s;
  k_s_update<P><<<bg, bb, 0, s>>>(a);
  m.mark(s);
  // t = Mhat s ; omega
  d.out = w.to; d.in = w.s; d.p_out = 1; d.xpay = 0; d.fin = FIN_NONE;
  launch_dslash(c, d, s);
  m.mark(s);
  d.out = w.t; d.in = w.to; d.x = w.s; d.p_out = 0; d.xpay = 1; d.fin = FIN_OMEGA;
  launch_dslash(c, d, s);
  m.mark(s);
  a.f0 = w.xs; a.f1 = w.p; a.f2 = w.s; a.f3 = w.t; a.f4 = w.r; a.f5 = w.rh;
  k_xr_update<P, PX><<<bg, bb, 0, s>>>(a);
  k_finish<typename SumOf<R>::T, 3, FIN_ITER><<<n, 256, 0, s>>>(a.ra, w.active_list, &w.ctl->n_active, n, (int)bg.x * (kBlasShape.sx / 32));
  m.mark(s);
  a.f0 = w.r; a.f1 = w.p; a.f2 = w.v;
  k_p_update<P><<<bg, bb, 0, s>>>(a);
  m.mark(s);
  // Updates: usually none this iteration. In a captured graph the FP32
  // refresh path and the FP64 update path each sit under an IF node that
  // k_plan switches on only when its list is non-empty; otherwise (no graph,
  // or profiling every kernel: event nodes may not sit inside a conditional
  // body) their launches see an empty list and exit.
  cudaGraphConditionalHandle h_upd = 0, h_ref = 0;
  bool cond = m.cond;
  if (cond) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    // (a handle must belong to a conditional node: h_ref only with refreshes)
    cond = cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, nullptr, nullptr, nullptr) == cudaSuccess &&
           cst == cudaStreamCaptureStatusActive &&
           cudaGraphConditionalHandleCreate(&h_upd, cg, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
           (!w.refresh || cudaGraphConditionalHandleCreate(&h_ref, cg, 0, cudaGraphCondAssignDefault) == cudaSuccess);
  }
  k_plan<<<1, 32, 0, s>>>(w.st, w.ctl, w.update_list, w.refresh_list, n, h_upd, h_ref, cond ? 1 : 0);
  m.mark(s);
  // the BLAS launches walk their list with a single CTA row; the operators
  // keep a row per source (measured faster for real updates)
  const dim3 bgu(bg.x, 1);
  cudaGraphNode_t cnode = nullptr;
  cudaStream_t us = s;
  if (w.refresh) {
    // FP32 refresh: r = bhat - Mhat (x64 + xs) in FP32 for the refresh list.
    // Its FP32 temporaries live in the FP64 update's buffers (the two paths
    // run one after the other)
    bool in_node = false;
    if (cond) {
      us = cond_begin(s, w.aux, h_ref, &cnode);
      in_node = us != nullptr;
      if (!in_node) {
        us = s;
        if (m.cond_failed) *m.cond_failed = true;
      }
    }
    const Field x32 = make_field(w.x64o.data, c->Vh, P32, n), r32 = make_field(w.r64.data, c->Vh, P32, n);
    const Field t32o = make_field(w.t64o.data, c->Vh, P32, n);
    VArgs rf = vargs(c, w, true);
    rf.list = w.refresh_list;
    rf.count = &w.ctl->n_refresh;
    rf.f0 = w.x64; rf.f1 = w.xs; rf.f2 = w.b64; rf.f3 = x32; rf.f4 = r32;
    k_ref_x<PX><<<bgu, bb, 0, us>>>(rf);
    DslashCall d32;
    memset(&d32, 0, sizeof(d32));
    d32.prec = P32;
    d32.recon = c->recon;
    d32.cs = &cs;
    d32.clover = 1;
    d32.list = w.refresh_list;
    d32.count = &w.ctl->n_refresh;
    d32.n = n;
    d32.ra = red_args(w);
    d32.shape = kBlasShape;
    d32.out = t32o; d32.in = x32; d32.p_out = 1; d32.xpay = 0; d32.fin = FIN_NONE;
    launch_dslash(c, d32, us);
    d32.out = r32; d32.in = t32o; d32.x = r32; d32.p_out = 0; d32.xpay = 1; d32.a = kappa * kappa;
    d32.fin = FIN_TRUE;
    launch_dslash(c, d32, us);
    rf.f0 = r32; rf.f1 = w.r; rf.f2 = w.rh; rf.f3 = w.p;
    k_rel_r<P, P32><<<bgu, bb, 0, us>>>(rf);
    k_finish<typename SumOf<R>::T, 2, FIN_REFRESH><<<n, 256, 0, us>>>(rf.ra, w.refresh_list, &w.ctl->n_refresh, n,
                                                    (int)bgu.x * (kBlasShape.sx / 32));
    if (in_node) cond_end(s, w.aux, cnode);
    us = s;
  }
  m.mark(s);
  // FP64 update
  bool in_node = false;
  if (cond) {
    us = cond_begin(s, w.aux, h_upd, &cnode);
    in_node = us != nullptr;
    if (!in_node) {
      us = s;
      if (m.cond_failed) *m.cond_failed = true;
    }
  }
  VArgs u = vargs(c, w, true);
  u.f0 = w.x64; u.f1 = w.xs; u.f2 = w.b64; u.f3 = w.r64;
  k_rel_x<PX><<<bgu, bb, 0, us>>>(u);
  m.mark(us);
  DslashCall d64 = d;
  d64.prec = P64;
  d64.recon = 18;
  d64.list = w.update_list;
  d64.count = &w.ctl->n_update;
  d64.shape = k64Shape;
  d64.emul = P != P64 ? 1 : 0;  // mixed solvers: FP64-accurate arithmetic on the FP32 pipe
  d64.out = w.t64o; d64.in = w.x64; d64.p_out = 1; d64.xpay = 0; d64.fin = FIN_NONE;
  launch_dslash(c, d64, us);
  m.mark(us);
  d64.out = w.r64; d64.in = w.t64o; d64.x = w.r64; d64.p_out = 0; d64.xpay = 1; d64.a = kappa * kappa;
  d64.fin = FIN_TRUE;
  launch_dslash(c, d64, us);
  m.mark(us);
  u.f0 = w.r64; u.f1 = w.r; u.f2 = w.rh; u.f3 = w.p;
  k_rel_r<P, P64><<<bgu, bb, 0, us>>>(u);
  k_finish<typename SumOf<R>::T, 2, FIN_UPDATE><<<n, 256, 0, us>>>(u.ra, w.update_list, &w.ctl->n_update, n, (int)bgu.x * (kBlasShape.sx / 32));
  m.mark(us);
  if (in_node) cond_end(s, w.aux, cnode);
  k_control<<<1, 32, 0, s>>>(w.st, w.ctl, w.active_list, n, m.ev ? w.hist : nullptr, it, chunk);
  m.mark(s);
}

// the FP64 update alone (used once at the start: r = bhat - Mhat x0; with
// x0 = 0 the residual is bhat itself and no operator is applied)
template <int P, int PX>
static void launch_update(sq_ctx* c, Workspace& w, const CloverSet& cs, double kappa, cudaStream_t s, bool zero_x) {
  typedef typename Real<P>::T R;
  const int n = w.n_rhs;
  dim3 bb(kBlasShape.sx, kBlasShape.ry);
  dim3 bg((c->Vh + kBlasShape.sx - 1) / kBlasShape.sx, (n + kBlasShape.ry - 1) / kBlasShape.ry);
  VArgs u = vargs(c, w, true);
  if (zero_x) {  // x64 = xs = 0 (set up so): the residual is bhat itself
    u.f0 = w.b64;
    k_true_norm<<<bg, bb, 0, s>>>(u);
    u.f0 = w.b64; u.f1 = w.r; u.f2 = w.rh; u.f3 = w.p;
    k_rel_r<P, P64><<<bg, bb, 0, s>>>(u);
    k_finish<typename SumOf<R>::T, 2, FIN_UPDATE><<<n, 256, 0, s>>>(u.ra, w.update_list, &w.ctl->n_update, n, (int)bg.x * (kBlasShape.sx / 32));
    k_control<<<1, 32, 0, s>>>(w.st, w.ctl, w.active_list, n, nullptr, 0, 0);
    c->launches += 4;
    return;
  }
  u.f0 = w.x64; u.f1 = w.xs; u.f2 = w.b64; u.f3 = w.r64;
  k_rel_x<PX><<<bg, bb, 0, s>>>(u);
  DslashCall d64;
  memset(&d64, 0, sizeof(d64));
  d64.prec = P64;
  d64.recon = 18;
  d64.cs = &cs;
  d64.clover = 1;
  d64.list = w.update_list;
  d64.count = &w.ctl->n_update;
  d64.n = n;
  d64.ra = red_args(w);
  d64.shape = k64Shape;
  d64.emul = P != P64 ? 1 : 0;
  d64.out = w.t64o; d64.in = w.x64; d64.p_out = 1;
  launch_dslash(c, d64, s);
  d64.out = w.r64; d64.in = w.t64o; d64.x = w.r64; d64.p_out = 0; d64.xpay = 1; d64.a = kappa * kappa;
  d64.fin = FIN_TRUE;
  launch_dslash(c, d64, s);
  u.f0 = w.r64; u.f1 = w.r; u.f2 = w.rh; u.f3 = w.p;
  k_rel_r<P, P64><<<bg, bb, 0, s>>>(u);
  k_finish<typename SumOf<R>::T, 2, FIN_UPDATE><<<n, 256, 0, s>>>(u.ra, w.update_list, &w.ctl->n_update, n, (int)bg.x * (kBlasShape.sx / 32));
  k_control<<<1, 32, 0, s>>>(w.st, w.ctl, w.active_list, n, nullptr, 0, 0);
  c->launches += 8;
}

typedef void (*IterFn)(sq_ctx*, Workspace&, const CloverSet&, double, Shape, cudaStream_t, Marks, int, int);
typedef void (*UpdFn)(sq_ctx*, Workspace&, const CloverSet&, double, cudaStream_t, bool);

static void fns_for(int inner, IterFn* it, UpdFn* up) {
  if (inner == P64) { *it = launch_iteration<P64, P64>; *up = launch_update<P64, P64>; }
  else if (inner == P32) { *it = launch_iteration<P32, P32>; *up = launch_update<P32, P32>; }
  else { *it = launch_iteration<P16, P32>; *up = launch_update<P16, P32>; }
}

sq_status find_clover(sq_ctx* c, double kappa, double csw, CloverSet** out);

// Algorithmic bytes and flops of one launch of class `kc` with na active
// and nu updating sources: every datum counted once, links and clover blocks
// once per launch (they are shared by the sources of a CTA).
struct Cost {
  double bytes, flops;
};
static Cost class_cost(int kc, int inner, int recon, double Vh, double na, double nu) {
  const double S = inner == P64 ? 192 : inner == P32 ? 96 : 52;  // spinor site
  const double SX = inner == P64 ? 192 : 96;                      // x accumulator
  const double SH = inner == P64 ? 192 : 52;                      // shadow residual (ShadowPrec)
  // links and clover blocks: FP64 for the FP64 operator, FP32 otherwise
  // (FP16 fields are hopped with the FP32 gauge data)
  const double L = inner == P64 ? 144 : (recon == 12 ? 48 : 72);
  const double Cl = inner == P64 ? 576 : 288;
  const double hop = 1320, clv = 504, xpay = 48;  // flops per site and source
  Cost r = {0, 0};
  switch (kc) {
    case KC_DSLASH_CLOVER:
    case KC_DSLASH_CLOVER_2:
      if (na > 0) r = {Vh * (8 * L + Cl) + na * Vh * 2 * S, na * Vh * (hop + clv)};
      break;
    case KC_DSLASH_XPAY_ALPHA:
      if (na > 0) r = {Vh * (8 * L + Cl) + na * Vh * (3 * S + SH), na * Vh * (hop + clv + xpay + 48)};
      break;
    case KC_DSLASH_XPAY_OMEGA:
      if (na > 0) r = {Vh * (8 * L + Cl) + na * Vh * 3 * S, na * Vh * (hop + clv + xpay + 96)};
      break;
    case KC_S_UPDATE: r = {na * Vh * 3 * S, na * Vh * 48}; break;
    case KC_XR_UPDATE: r = {na * Vh * (2 * SX + 4 * S + SH), na * Vh * 240}; break;
    case KC_P_UPDATE: r = {na * Vh * 4 * S, na * Vh * 96}; break;
    case KC_PLAN: break;
    case KC_REL_X: r = {nu * Vh * (4 * 192 + 2 * SX), nu * Vh * 48}; break;
    case KC_REL_DSLASH1:
      if (nu > 0) r = {Vh * (8 * 144 + 576) + nu * Vh * 2 * 192, nu * Vh * (hop + clv)};
      break;
    case KC_REL_DSLASH2:
      if (nu > 0) r = {Vh * (8 * 144 + 576) + nu * Vh * 3 * 192, nu * Vh * (hop + clv + xpay + 48)};
      break;
    case KC_REL_R: r = {nu * Vh * (192 + 2 * S), nu * Vh * 48}; break;
    default: break;
  }
  return r;
}

// FP64 full-lattice residual norms^2 of (x64 even, x64o odd) -> scal[0..n)
// even, scal[n..2n) odd. On entry t64o holds eta_o + k D_oe psi_e (the
// reconstruction's right-hand side), so the odd half needs no hop:
//   r_e = eta_e - A_ee psi_e + k D_eo psi_o,   r_o = t64o - A_oo psi_o.
static void launch_full_residual(sq_ctx* c, Workspace& w, const CloverSet& cs, double kappa, cudaStream_t s) {
  const int n = w.n_rhs;
  const bool emul = w.inner != P64;  // mixed solvers: emulated-FP64 arithmetic
  DslashCall d;
  memset(&d, 0, sizeof(d));
  d.prec = P64;
  d.recon = 18;
  d.cs = &cs;
  d.n = n;
  d.shape = kBlasShape;
  d.ra = red_args(w);
  d.emul = emul ? 1 : 0;
  RedArgs ra = red_args(w);
  if (emul) {  // the norms come with the last kernel of each half
    launch_clover_df(c, cs, w.r64, w.eta_e, w.x64, 0, 1.0, -1.0, 0, n, s);
    d.out = w.r64; d.in = w.x64o; d.x = w.r64; d.p_out = 0; d.xpay = 1; d.a = kappa;
    d.fin = FIN_STORE;  // ||r_e||^2 -> scal[0..n)
    launch_dslash(c, d, s);
    RedArgs ro = ra;
    ro.out = w.scal + n;  // ||r_o||^2
    launch_clover_df(c, cs, w.t64o, w.t64o, w.x64o, 1, 1.0, -1.0, 0, n, s, &ro);
    c->launches += 5;
    return;
  }
  launch_clover64(c, cs, w.r64, w.eta_e, w.x64, 0, 1.0, -1.0, 0, n, s);
  d.out = w.r64; d.in = w.x64o; d.x = w.r64; d.p_out = 0; d.xpay = 1; d.a = kappa;
  launch_dslash(c, d, s);
  launch_clover64(c, cs, w.t64o, w.t64o, w.x64o, 1, 1.0, -1.0, 0, n, s);
  launch_norm2(c, w.r64, P64, n, w.scal, ra, s);
  launch_norm2(c, w.t64o, P64, n, w.scal + n, ra, s);
  c->launches += 5;
}

// One problem of a solve: a lattice (context), kappa, its sources.
struct Prob {
  sq_ctx* c = nullptr;
  double kappa = 0, csw = 0, tol = 0;
  const double* src = nullptr;
  double* sol = nullptr;
  int n = 0;
  sq_solve_stats* stats = nullptr;
  CloverSet* cs = nullptr;
  Workspace* w = nullptr;
  cudaStream_t s = nullptr;
  Shape sh;
  IterFn iter = nullptr;
  UpdFn upd = nullptr;
  int recon_in = 12;
  std::vector<double> enorm2, target2;
};

static sq_status validate_params(sq_ctx* c, sq_solve_params& prm) {
  if (prm.inner_prec < P64 || prm.inner_prec > P16) return set_error(c, SQ_ERR_ARG, "sq_solve: bad inner_prec");
  if (prm.io != SQ_HOST && prm.io != SQ_DEVICE) return set_error(c, SQ_ERR_ARG, "sq_solve: bad io");
  if (prm.max_iter <= 0) return set_error(c, SQ_ERR_ARG, "sq_solve: max_iter must be > 0");
  if (!(prm.delta < 1.0)) return set_error(c, SQ_ERR_ARG, "sq_solve: delta must be < 1");
  // Defaults measured on GB300: FP32 3e-6 (16^3x32: one FP64 update
  // mid-solve; the full-lattice FP64 check catches any drift of the
  // iterated residual), FP16 3e-3 (11-bit mantissas drift sooner; 24^3x48
  // sweep 2e-3..5e-3), FP16 defect correction 1e-4 (32^3x64 sweep
  // 1e-4..1e-2: fewest outer cycles for a few more inner iterations)
  if (!(prm.delta > 0.0))
    prm.delta = prm.inner_prec == P16 ? (prm.outer == SQ_OUTER_DEFECT ? 1e-4 : 3e-3) : 3e-6;
  if (prm.chunk < 0) prm.chunk = 0;  // 0: sized automatically
  if (!(prm.breakdown_tol > 0.0)) prm.breakdown_tol = 1e-14;
  if (!std::isfinite(prm.breakdown_tol)) return set_error(c, SQ_ERR_ARG, "sq_solve: breakdown_tol must be finite");
  if (prm.fallback_max_iter < 0) return set_error(c, SQ_ERR_ARG, "sq_solve: fallback_max_iter must be >= 0");
  if (prm.chunk > 256) return set_error(c, SQ_ERR_ARG, "sq_solve: chunk must be <= 256");
  if (prm.sites_per_block > 0 || prm.rhs_per_block > 0) {
    if (prm.sites_per_block <= 0 || prm.rhs_per_block <= 0 || prm.sites_per_block % 32 ||
        prm.sites_per_block * prm.rhs_per_block > 256)
      return set_error(c, SQ_ERR_ARG, "sq_solve: bad CTA shape");
  }
  return SQ_OK;
}

// Per problem, on its stream: clover, workspace, sources, Schur source, norms,
// targets and the tuned dslash shape.
static sq_status setup_problem(Prob& p, const sq_solve_params& prm) {
  sq_ctx* c = p.c;
  const int inner = prm.inner_prec;
  if (!p.src || !p.sol || p.n <= 0) return set_error(c, SQ_ERR_ARG, "sq_solve: null buffer or n_rhs <= 0");
  if (!(p.tol > 0.0) || !std::isfinite(p.tol)) return set_error(c, SQ_ERR_ARG, "sq_solve: tol must be > 0");
  if (!std::isfinite(p.kappa) || !std::isfinite(p.csw))
    return set_error(c, SQ_ERR_ARG, "sq_solve: non-finite kappa/c_sw");
  if (!c->have_gauge) return set_error(c, SQ_ERR_STATE, "sq_solve: no gauge field loaded");
  sq_status st = find_clover(c, p.kappa, p.csw, &p.cs);
  if (st != SQ_OK) return st;
  st = alloc_ws(c, *p.w, p.n, inner);
  if (st != SQ_OK) return st;
  Workspace& w = *p.w;
  // FP32 refreshes pay off only for the FP16 recurrence (it drifts at the
  // 1e-3 level); defect correction restarts at every update instead
  w.refresh = inner == P16 && prm.outer != SQ_OUTER_DEFECT;
  cudaStream_t s = p.s;
  const int n = p.n;
  const size_t lex_src = (size_t)c->V * 24;  // doubles per source
  // Sources in groups: with host I/O the copy of group g + 1 (on the side
  // stream) overlaps the FP64 work on group g. Per group: finite check
  // (flag read once at the end), even / odd packing, norms and the Schur
  // source bhat = A_ee^{-1} (eta_e + k D_eo A_oo^{-1} eta_o).
  const int G = prm.io == SQ_HOST ? std::min(n, kSetupGroups) : 1;
  const double* dsrc = prm.io == SQ_HOST ? w.lex : p.src;
  if (prm.io == SQ_HOST && prm.pion && prm.pion_tslice)
    cudaMemcpyAsync(w.tsl, prm.pion_tslice, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s);
  // the side stream must not overwrite the staging buffer while an earlier
  // solve's output copy may still read it (it was synchronised, but keep
  // the order explicit)
  cudaEventRecord(w.ev_rec, s);
  cudaStreamWaitEvent(w.aux, w.ev_rec, 0);
  cudaMemsetAsync(w.flag, 0, sizeof(int), s);
  auto sub64 = [&](const Field& f, int k0) {
    return make_field((double2*)f.data + (size_t)k0 * 12 * c->Vh, c->Vh, P64, 0);
  };
  RedArgs ra = red_args(w);
  Field none = make_field(nullptr, c->Vh, P64, n);
  for (int g = 0; g < G; g++) {
    const int k0 = g * n / G, k1 = (g + 1) * n / G, ng = k1 - k0;
    if (ng <= 0) continue;
    const double* gsrc = dsrc + (size_t)k0 * lex_src;
    if (prm.io == SQ_HOST) {
      cudaMemcpyAsync(w.lex + (size_t)k0 * lex_src, p.src + (size_t)k0 * lex_src, ng * lex_src * sizeof(double),
                      cudaMemcpyHostToDevice, w.aux);
      cudaEventRecord(w.ev_in[g], w.aux);
      cudaStreamWaitEvent(s, w.ev_in[g], 0);
    }
    launch_finite(c, gsrc, ng * lex_src, w.flag, s);
    launch_pack_norm2(c, sub64(w.eta_e, k0), gsrc, 0, ng, w.scal + k0, ra, s);
    launch_pack_norm2(c, sub64(w.eta_o, k0), gsrc, 1, ng, w.scal + n + k0, ra, s);
    DslashCall d;
    memset(&d, 0, sizeof(d));
    d.prec = P64;
    d.recon = 18;
    d.cs = p.cs;
    d.n = ng;
    d.shape = kBlasShape;
    d.ra = ra;
    if (inner != P64) {
      // emulated-FP64 arithmetic, A_ee^{-1} fused after the xpay:
      // bhat = A_ee^{-1} (eta_e + k D_eo A_oo^{-1} eta_o)
      launch_clover_df(c, *p.cs, sub64(w.t64o, k0), none, sub64(w.eta_o, k0), 1, 0.0, 1.0, 1, ng, s);
      d.emul = 1;
      d.clover = 1;
      d.xfirst = 1;
      d.out = sub64(w.b64, k0); d.in = sub64(w.t64o, k0); d.x = sub64(w.eta_e, k0); d.p_out = 0; d.xpay = 1;
      d.a = p.kappa;
      launch_dslash(c, d, s);
      c->launches += 5;
    } else {
      launch_clover64(c, *p.cs, sub64(w.t64o, k0), none, sub64(w.eta_o, k0), 1, 0.0, 1.0, 1, ng, s);
      d.out = sub64(w.r64, k0); d.in = sub64(w.t64o, k0); d.x = sub64(w.eta_e, k0); d.p_out = 0; d.xpay = 1;
      d.a = p.kappa;
      launch_dslash(c, d, s);
      launch_clover64(c, *p.cs, sub64(w.b64, k0), none, sub64(w.r64, k0), 0, 0.0, 1.0, 1, ng, s);
      c->launches += 6;
    }
  }
  std::vector<double> eta2(2 * n);
  int bad = 0;
  cudaMemcpyAsync(eta2.data(), w.scal, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&bad, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(c, e, "sq_solve setup");
  if (bad) return set_error(c, SQ_ERR_NONFINITE, "sq_solve: NaN or Inf in the sources");
  if (prm.use_x0) {
    const double* dx0 = p.sol;
    if (prm.io == SQ_HOST) {
      cudaMemcpyAsync(w.lex, p.sol, (size_t)n * lex_src * sizeof(double), cudaMemcpyHostToDevice, s);
      dx0 = w.lex;
    }
    cudaMemsetAsync(w.flag, 0, sizeof(int), s);
    launch_finite(c, dx0, (size_t)n * lex_src, w.flag, s);
    cudaMemcpyAsync(&bad, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(c, e, "sq_solve initial guess");
    if (bad) return set_error(c, SQ_ERR_NONFINITE, "sq_solve: NaN or Inf in the initial guess");
    launch_pack(c, w.x64, dx0, 0, P64, n, s);
    c->launches += 2;
  } else {
    cudaMemsetAsync(w.x64.data, 0, field_bytes(c->Vh, P64, n), s);
  }
  cudaMemsetAsync(w.xs.data, 0, field_bytes(c->Vh, px_of(inner), n), s);
  p.target2.resize(n);
  p.enorm2.resize(n);
  for (int k = 0; k < n; k++) {
    p.enorm2[k] = eta2[k] + eta2[n + k];
    double t = p.tol * std::sqrt(p.enorm2[k]) / p.cs->a_bound;
    p.target2[k] = t * t;
  }
  if (prm.sites_per_block > 0 && prm.rhs_per_block > 0) {
    p.sh.sx = prm.sites_per_block;
    p.sh.ry = prm.rhs_per_block;
    p.sh.order = 0;
  } else {
    DslashCall tcall;
    memset(&tcall, 0, sizeof(tcall));
    tcall.prec = inner;
    tcall.recon = inner == P64 ? 18 : c->recon;
    tcall.cs = p.cs;
    tcall.clover = 1;
    tcall.out = w.to;
    tcall.in = w.p;
    tcall.p_out = 1;
    tcall.n = n;
    // defined input for the trial launches (p is overwritten before use)
    if (!dslash_tuned(c, tcall.prec, tcall.recon, n)) cudaMemsetAsync(w.p.data, 0, field_bytes(c->Vh, inner, n), s);
    p.sh = tune_dslash(c, tcall, s);
  }
  p.recon_in = inner == P64 ? 18 : c->recon;
  fns_for(inner, &p.iter, &p.upd);
  return SQ_OK;
}

// Solutions from the even-odd FP64 fields to the caller's lexicographic
// layout (through the staging buffer and one copy for host I/O), and the
// optional pion epilogue on the device solutions, all on stream s.
static void output_solutions(Prob& p, const sq_solve_params& prm, cudaStream_t s) {
  sq_ctx* c = p.c;
  Workspace& w = *p.w;
  double* dsol = prm.io == SQ_HOST ? w.lex : p.sol;
  launch_unpack(c, dsol, w.x64, 0, P64, p.n, s);
  launch_unpack(c, dsol, w.x64o, 1, P64, p.n, s);
  c->launches += 2;
  if (prm.pion) {
    double* dC = prm.io == SQ_HOST ? w.pion : prm.pion;
    const int* dt = prm.pion_tslice ? (prm.io == SQ_HOST ? w.tsl : prm.pion_tslice) : nullptr;
    launch_pion(c, dsol, p.n, dt, dC, s);
    c->launches += 1;
    if (prm.io == SQ_HOST)
      cudaMemcpyAsync(prm.pion, w.pion, (size_t)p.n * c->dims[3] * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  if (prm.io == SQ_HOST)
    cudaMemcpyAsync(p.sol, w.lex, (size_t)p.n * c->V * 24 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

// The iteration loop of all problems: each problem's `chunk` iterations are
// a branch of one captured CUDA graph (fork/join through events), so the
// problems advance concurrently from a single graph launch per chunk; the
// host reads one integer per problem (sources still active) per launch.
// Then per problem: reconstruction, FP64 full residual, solutions out.
static sq_status run_problems(std::vector<Prob>& P, const sq_solve_params& prm, cudaStream_t sb,
                              cudaGraphExec_t* graph, std::vector<unsigned long long>* gkey,
                              cudaGraphExec_t* graph2, std::vector<unsigned long long>* gkey2,
                              std::vector<cudaEvent_t>& evs, sq_status* result) {
  const int np = (int)P.size();
  const bool prof = prm.profile != 0 && np == 1;
  const unsigned pmask = profile_mask(prm.profile);
  // iterations per graph launch: fixed (prm.chunk), or, by default for one
  // problem, 24 in the first launch and 4 in each later one (graph2), so that
  // at most 3 iterations run after the last source has converged and no
  // graph is captured again when the iteration count changes
  const bool autoc = prm.chunk == 0 && np == 1 && graph2 != nullptr;
  const int tail = autoc ? 4 : (prm.chunk > 0 ? prm.chunk : 16);
  const int first = autoc ? 24 : tail;
  const int chunk = std::max(first, tail);  // the most iterations of one launch
  const double delta = prm.inner_prec == P64 ? 0.0 : prm.delta;
  sq_ctx* c0 = P[0].c;
  cudaError_t e = cudaSuccess;
  if (prof) {
    Workspace& w = *P[0].w;
    const size_t need = (size_t)chunk * (KC_N + 1);
    for (size_t i = w.pev.size(); i < need; i++) {
      cudaEvent_t ev;
      cudaEventCreate(&ev);
      w.pev.push_back(ev);
    }
    if (w.hist_chunk < chunk) {
      dev_free(w.mem, w.hist, 2 * (size_t)w.hist_chunk * sizeof(int));
      w.hist = nullptr;
      w.hist_chunk = 0;
      e = dev_alloc(w.mem, (void**)&w.hist, 2 * (size_t)chunk * sizeof(int));
      if (e != cudaSuccess) return cuda_check(c0, e, "profile buffers");
      w.hist_chunk = chunk;
    }
    for (int k = 0; k < KC_N; k++) c0->prof[k] = KStat();
    c0->prof_valid = 0;
    c0->prof_inner = prm.inner_prec;
  }
  while ((int)evs.size() < 2 * np + 2) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    evs.push_back(ev);
  }
  // pinned read-back buffer, kept in the first problem's workspace
  Workspace& w0 = *P[0].w;
  if (w0.h_pin_n < (size_t)(np + 2 * chunk)) {
    if (w0.h_pin) cudaFreeHost(w0.h_pin);
    w0.h_pin = nullptr;
    w0.h_pin_n = 0;
    e = cudaMallocHost((void**)&w0.h_pin, (np + 2 * chunk) * sizeof(int));
    if (e != cudaSuccess) {
      w0.h_pin = nullptr;
      return cuda_check(c0, e, "pinned read-back buffer");
    }
    w0.h_pin_n = np + 2 * chunk;
  }
  int* h_active = w0.h_pin;
  std::vector<int> tot_it(np, 0);
  for (int attempt = 0; attempt < 4; attempt++) {
    for (int i = 0; i < np; i++) {
      Prob& p = P[i];
      Workspace& w = *p.w;
      cudaMemcpyAsync(w.scal, p.target2.data(), p.n * sizeof(double), cudaMemcpyHostToDevice, p.s);
      // the iterated residual of FP16 fields can sit below the true one by
      // a few tens of percent, FP32 by much less: retire with a margin
      const double margin = prm.inner_prec == P16 ? 0.5 : prm.inner_prec == P32 ? 0.8 : 1.0;
      k_init<<<(p.n + 127) / 128, 128, 0, p.s>>>(w.st, w.ctl, w.update_list, w.scal, delta * delta,
                                                 margin * margin, prm.max_iter,
                                                 prm.outer == SQ_OUTER_DEFECT ? 1 : 0, w.refresh ? 1 : 0,
                                                 prm.breakdown_tol * prm.breakdown_tol, p.n);
      p.c->launches += 1;
      p.upd(p.c, w, *p.cs, p.kappa, p.s, attempt == 0 && !prm.use_x0);
      if (p.s != sb) {
        cudaEventRecord(evs[i], p.s);
        cudaStreamWaitEvent(sb, evs[i], 0);
      }
    }
    // the graph key holds everything baked into the captured kernels
    std::vector<unsigned long long> key = {(unsigned long long)np, (unsigned long long)prm.inner_prec,
                                           0ull, (unsigned long long)prof,
                                           (unsigned long long)prm.profile, (unsigned long long)prm.outer};
    for (auto& p : P) {
      unsigned long long kb;
      memcpy(&kb, &p.kappa, sizeof(kb));
      const unsigned long long v[] = {p.c->uid, (unsigned long long)p.n, (unsigned long long)p.sh.sx,
                                      (unsigned long long)p.sh.ry, (unsigned long long)p.sh.order,
                                      (unsigned long long)p.sh.kind,
                                      (unsigned long long)((p.sh.by << 24) ^ (p.sh.bz << 16) ^ (p.sh.bt << 8) ^
                                                           p.sh.nbuf),
                                      (unsigned long long)p.sh.sg, (unsigned long long)p.c->wait_cycles,
                                      (unsigned long long)p.c->wait_stall,
                                      (unsigned long long)p.c->recon, (unsigned long long)(uintptr_t)p.w->base,
                                      (unsigned long long)(uintptr_t)p.c->U64, (unsigned long long)(uintptr_t)p.c->U32,
                                      (unsigned long long)(uintptr_t)p.cs->Ainv64,
                                      (unsigned long long)(uintptr_t)p.cs->Ainv32,
                                      (unsigned long long)(uintptr_t)p.w->hist,
                                      (unsigned long long)(uintptr_t)(p.w->pev.empty() ? nullptr : p.w->pev[0]),
                                      (unsigned long long)(uintptr_t)p.s, kb};
      key.insert(key.end(), v, v + sizeof(v) / sizeof(v[0]));
    }
    const bool use_graph = prm.use_graph != 0;
    bool cond_ok = true;      // conditional update nodes may be used
    bool cond_failed = false;  // adding one failed during the capture
    int cur = first;  // iterations in the graph launched next
    auto launch_chunk = [&](bool capture) {
      for (int i = 0; i < np; i++) {
        Prob& p = P[i];
        cudaStream_t ps = np == 1 ? sb : p.s;
        if (ps != sb) {  // fork
          cudaEventRecord(evs[np + i], sb);
          cudaStreamWaitEvent(ps, evs[np + i], 0);
        }
        for (int it = 0; it < cur; it++) {
          Marks m;
          if (prof) {
            m.ev = &p.w->pev[(size_t)it * (KC_N + 1)];
            m.mask = pmask;
            m.capture = capture;
          }
          m.cond = capture && prm.profile != 1 && cond_ok;
          m.cond_failed = &cond_failed;
          p.iter(p.c, *p.w, *p.cs, p.kappa, p.sh, ps, m, it, cur);
        }
        if (ps != sb) {  // join
          cudaEventRecord(evs[i], ps);
          cudaStreamWaitEvent(sb, evs[i], 0);
        }
      }
    };
    // the graph of `cur` iterations (the first chunk's, or the tail's when
    // chunks are sized automatically), captured when its key changes
    auto ensure_graph = [&](cudaGraphExec_t* gx, std::vector<unsigned long long>* gk) -> cudaError_t {
      key[2] = (unsigned long long)cur;
      if (!use_graph || (*gx && key == *gk)) return cudaSuccess;
      if (*gx) {
        cudaGraphExecDestroy(*gx);
        *gx = nullptr;
      }
      cond_ok = true;
      cond_failed = false;
      cudaGraph_t g;
      cudaError_t ce = cudaStreamBeginCapture(sb, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        launch_chunk(true);
        ce = cudaStreamEndCapture(sb, &g);
      }
      if (ce == cudaSuccess && cond_failed) {
        // a conditional node could not be added: capture again with the
        // update paths as plain launches (they exit on an empty list)
        cudaGraphDestroy(g);
        cond_ok = false;
        ce = cudaStreamBeginCapture(sb, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
          launch_chunk(true);
          ce = cudaStreamEndCapture(sb, &g);
        }
      }
      if (ce == cudaSuccess) {
        ce = cudaGraphInstantiate(gx, g, 0);
        cudaGraphDestroy(g);
      }
      if (ce == cudaSuccess) *gk = key;
      return ce;
    };
    long long launched = 0;
    const long long cap = (long long)prm.max_iter + 4LL * chunk;
    cur = first;
    for (;;) {
      cudaGraphExec_t* gx = (autoc && cur == tail && cur != first) ? graph2 : graph;
      std::vector<unsigned long long>* gk = gx == graph ? gkey : gkey2;
      e = ensure_graph(gx, gk);
      if (e != cudaSuccess) return cuda_check(c0, e, "graph capture of the inner loop");
      if (use_graph) e = cudaGraphLaunch(*gx, sb);
      else {
        launch_chunk(false);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) break;
      // launches inside conditional nodes are counted on the device
      for (auto& p : P)
        p.c->launches += (long long)cur * (kChainLaunches + (use_graph && prm.profile != 1
                                                                    ? 0
                                                                    : kUpdateLaunches * (p.w->refresh ? 2 : 1)));
      launched += cur;
      for (int i = 0; i < np; i++)
        cudaMemcpyAsync(h_active + i, &P[i].w->ctl->n_active, sizeof(int), cudaMemcpyDeviceToHost, sb);
      if (prof) cudaMemcpyAsync(h_active + np, P[0].w->hist, 2 * cur * sizeof(int), cudaMemcpyDeviceToHost, sb);
      e = cudaStreamSynchronize(sb);
      if (e != cudaSuccess) break;
      if (prof) {
        Workspace& w = *P[0].w;
        for (int i = 0; i < cur; i++) {
          const double na = h_active[np + i], nu = h_active[np + cur + i];
          for (int kc = 0; kc < KC_N; kc++) {
            if (!((pmask >> kc) & 1u) || !((pmask >> (kc + 1)) & 1u)) continue;
            float ms = 0;
            cudaEventElapsedTime(&ms, w.pev[(size_t)i * (KC_N + 1) + kc], w.pev[(size_t)i * (KC_N + 1) + kc + 1]);
            Cost cost = class_cost(kc, prm.inner_prec, P[0].recon_in, (double)P[0].c->Vh, na, nu);
            KStat& ks = c0->prof[kc];
            ks.launches += 1;
            ks.ms += ms;
            ks.bytes += cost.bytes;
            ks.flops += cost.flops;
          }
        }
        c0->prof_valid = 1;
      }
      int active = 0;
      for (int i = 0; i < np; i++) active += h_active[i];
      if (prm.verbose) fprintf(stderr, "libstochq: %lld iterations, %d sources active\n", launched, active);
      if (active == 0 || launched > cap) break;
      cur = tail;
    }
    if (e != cudaSuccess) return cuda_check(c0, e, "inner loop");
    // per problem: x64 += xs, psi_o = A_oo^{-1} (eta_o + k D_oe psi_e), full
    // FP64 residual
    bool retry = false;
    for (int i = 0; i < np; i++) {
      Prob& p = P[i];
      sq_ctx* c = p.c;
      Workspace& w = *p.w;
      const int n = p.n;
      {
        VArgs f = vargs(c, w, false);
        f.f0 = w.x64;
        f.f1 = w.xs;
        const dim3 fg((c->Vh + 127) / 128, n);
        if (prm.inner_prec == P64) k_flush<P64><<<fg, 128, 0, sb>>>(f);
        else k_flush<P32><<<fg, 128, 0, sb>>>(f);
        c->launches += 1;
      }
      DslashCall d;
      memset(&d, 0, sizeof(d));
      d.prec = P64;
      d.recon = 18;
      d.cs = p.cs;
      d.n = n;
      d.shape = kBlasShape;
      d.ra = red_args(w);
      if (prm.inner_prec != P64) {
        // emulated FP64, one launch: t64o = eta_o + k D_oe psi_e, psi_o = A_oo^{-1} t64o
        d.emul = 1;
        d.clover = 1;
        d.xfirst = 1;
        d.out2 = w.t64o;
        d.out = w.x64o; d.in = w.x64; d.x = w.eta_o; d.p_out = 1; d.xpay = 1; d.a = p.kappa;
        launch_dslash(c, d, sb);
        c->launches += 1;
      } else {
        d.out = w.t64o; d.in = w.x64; d.x = w.eta_o; d.p_out = 1; d.xpay = 1; d.a = p.kappa;
        launch_dslash(c, d, sb);
        Field none = make_field(nullptr, c->Vh, P64, n);
        launch_clover64(c, *p.cs, w.x64o, none, w.t64o, 1, 0.0, 1.0, 1, n, sb);
        c->launches += 2;
      }
      // solutions out (and the pion epilogue) on the side stream while the
      // FP64 check runs; a failed check redoes them after the next pass
      cudaEventRecord(w.ev_rec, sb);
      cudaStreamWaitEvent(w.aux, w.ev_rec, 0);
      output_solutions(p, prm, w.aux);
      cudaEventRecord(w.ev_out, w.aux);
      launch_full_residual(c, w, *p.cs, p.kappa, sb);
      std::vector<double> res2(2 * n);
      cudaMemcpyAsync(res2.data(), w.scal, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, sb);
      std::vector<RhsState> hs(n);
      cudaMemcpyAsync(hs.data(), w.st, n * sizeof(RhsState), cudaMemcpyDeviceToHost, sb);
      Control hc;
      cudaMemcpyAsync(&hc, w.ctl, sizeof(Control), cudaMemcpyDeviceToHost, sb);
      e = cudaStreamSynchronize(sb);
      c->launches += hc.launched;
      if (e != cudaSuccess) return cuda_check(c0, e, "final residual");
      for (int k = 0; k < n; k++) {
        double rr = p.enorm2[k] > 0 ? std::sqrt((res2[k] + res2[n + k]) / p.enorm2[k]) : 0.0;
        int status = hs[k].status;
        if (status == SQ_OK && !(rr <= p.tol)) {
          if (attempt < 3) {
            retry = true;
            p.target2[k] *= 1.0 / 16.0;
          } else {
            status = SQ_ERR_NOCONV;
          }
        }
        if (p.stats) {
          sq_solve_stats& o = p.stats[k];
          if (attempt == 0) memset(&o, 0, sizeof(o));
          o.status = status;
          o.iterations += hs[k].iter;
          o.updates += hs[k].updates;
          o.restarts += hs[k].restarts;
          o.breakdowns += hs[k].breakdowns;
          o.true_residual = rr;
        }
        if (status != SQ_OK && *result == SQ_OK) *result = (sq_status)status;
      }
    }
    if (!retry) break;
    *result = SQ_OK;
    if (prm.verbose) fprintf(stderr, "libstochq: tightening the Schur target\n");
    // the next pass continues from the current x (even sites in x64); it
    // rewrites x64 / x64o, so it waits for the output copies of this one
    for (auto& p : P) cudaStreamWaitEvent(sb, p.w->ev_out, 0);
    for (auto& p : P)
      if (p.s != sb) {
        cudaEventRecord(evs[0], sb);
        cudaStreamWaitEvent(p.s, evs[0], 0);
      }
  }
  for (auto& p : P) {
    e = cudaStreamSynchronize(p.w->aux);
    if (e != cudaSuccess) break;
  }
  return cuda_check(c0, e, "solution copy");
}

// A bounded device wait of the solve's kernels (the staged-spinor ring of the
// tiled dslash) that ran out: the results are not to be trusted.
static sq_status check_timeouts(sq_ctx* c, const char* what) {
  int bits = 0;
  sq_status st = read_error_word(c, &bits);
  if (st != SQ_OK) return st;
  if (bits & ERRBIT_TIMEOUT) return set_error(c, SQ_ERR_TIMEOUT, "%s: a bounded device wait ran out", what);
  return SQ_OK;
}

// FP16 inner solves whose sources end with NOCONV or BREAKDOWN (the FP16
// recurrence stagnated) are solved again by the FP32 inner solver from their
// current iterate; their statistics add up and carry fallback = 1, and their
// rows of the fused pion epilogue are recomputed. Returns the final status.
static sq_status fp16_fallback(sq_ctx* c, double kappa, double csw, const double* src, double* sol, int n,
                               double tol, const sq_solve_params& prm, sq_solve_stats* st) {
  std::vector<int> bad;
  for (int k = 0; k < n; k++)
    if (st[k].status == SQ_ERR_NOCONV || st[k].status == SQ_ERR_BREAKDOWN) bad.push_back(k);
  const int m = (int)bad.size();
  if (m > 0) {
    const size_t per = (size_t)c->V * 24;  // doubles per source
    sq_solve_params p2 = prm;
    p2.inner_prec = P32;
    p2.outer = SQ_OUTER_RELIABLE;
    p2.delta = 0.0;
    p2.use_x0 = 1;
    p2.fallback = 0;
    p2.profile = 0;
    p2.pion = nullptr;
    p2.pion_tslice = nullptr;
    if (prm.fallback_max_iter > 0) p2.max_iter = prm.fallback_max_iter;
    std::vector<sq_solve_stats> st2(m);
    std::vector<double> hs, hx;
    double* dbuf = nullptr;
    const double *s2 = nullptr;
    double* x2 = nullptr;
    if (prm.io == SQ_HOST) {
      hs.resize(m * per);
      hx.resize(m * per);
      for (int i = 0; i < m; i++) {
        memcpy(hs.data() + i * per, src + bad[i] * per, per * sizeof(double));
        memcpy(hx.data() + i * per, sol + bad[i] * per, per * sizeof(double));
      }
      s2 = hs.data();
      x2 = hx.data();
    } else {
      cudaError_t e = cudaMallocAsync((void**)&dbuf, 2 * m * per * sizeof(double), c->stream);
      if (e != cudaSuccess) return cuda_check(c, e, "sq_solve fallback buffers");
      for (int i = 0; i < m; i++) {
        cudaMemcpyAsync(dbuf + i * per, src + bad[i] * per, per * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream);
        cudaMemcpyAsync(dbuf + (m + i) * per, sol + bad[i] * per, per * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream);
      }
      s2 = dbuf;
      x2 = dbuf + m * per;
    }
    sq_status r2 = solve_impl(c, kappa, csw, s2, x2, m, tol, &p2, st2.data());
    if (r2 != SQ_OK && r2 != SQ_ERR_NOCONV && r2 != SQ_ERR_BREAKDOWN) {
      if (dbuf) cudaFreeAsync(dbuf, c->stream);
      return r2;
    }
    const int T = c->dims[3];
    for (int i = 0; i < m; i++) {
      const int k = bad[i];
      if (prm.io == SQ_HOST) memcpy(sol + k * per, x2 + i * per, per * sizeof(double));
      else cudaMemcpyAsync(sol + k * per, x2 + i * per, per * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
      sq_solve_stats& o = st[k];
      o.status = st2[i].status;
      o.iterations += st2[i].iterations;
      o.updates += st2[i].updates;
      o.restarts += st2[i].restarts;
      o.breakdowns += st2[i].breakdowns;
      o.true_residual = st2[i].true_residual;
      o.fallback = 1;
    }
    if (prm.pion) {  // those sources' correlator rows, from the new solutions
      double* dC = nullptr;
      double* dx = nullptr;
      cudaError_t e = cudaMallocAsync((void**)&dC, (size_t)m * T * sizeof(double), c->stream);
      if (e == cudaSuccess && prm.io == SQ_HOST) {
        e = cudaMallocAsync((void**)&dx, m * per * sizeof(double), c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x2, m * per * sizeof(double), cudaMemcpyHostToDevice, c->stream);
      }
      std::vector<int> ts(m, 0);
      if (e == cudaSuccess && prm.pion_tslice) {
        for (int i = 0; i < m && e == cudaSuccess; i++)
          e = cudaMemcpyAsync(&ts[i], prm.pion_tslice + bad[i], sizeof(int),
                              prm.io == SQ_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      }
      int* dts = nullptr;
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&dts, m * sizeof(int), c->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dts, ts.data(), m * sizeof(int), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) {
        launch_pion(c, prm.io == SQ_HOST ? dx : x2, m, dts, dC, c->stream);
        c->launches += 1;
        for (int i = 0; i < m && e == cudaSuccess; i++)
          e = cudaMemcpyAsync(prm.pion + (size_t)bad[i] * T, dC + (size_t)i * T, T * sizeof(double),
                              prm.io == SQ_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      }
      if (dts) cudaFreeAsync(dts, c->stream);
      if (dx) cudaFreeAsync(dx, c->stream);
      if (dC) cudaFreeAsync(dC, c->stream);
      if (e != cudaSuccess) {
        if (dbuf) cudaFreeAsync(dbuf, c->stream);
        return cuda_check(c, e, "sq_solve fallback correlator");
      }
    }
    if (dbuf) cudaFreeAsync(dbuf, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "sq_solve fallback");
  }
  for (int k = 0; k < n; k++)
    if (st[k].status != SQ_OK) return (sq_status)st[k].status;
  return SQ_OK;
}

sq_status solve_impl(sq_ctx* c, double kappa, double csw, const double* src, double* sol, int n, double tol,
                     const sq_solve_params* prm_in, sq_solve_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  if (!c) return SQ_ERR_ARG;
  sq_solve_params prm;
  if (prm_in) prm = *prm_in;
  else sq_default_params(&prm);
  sq_status st = validate_params(c, prm);
  if (st != SQ_OK) return st;
  // per-source statistics are needed to choose the sources of an FP16 fallback
  std::vector<sq_solve_stats> local;
  const bool fb = prm.inner_prec == P16 && prm.fallback && n > 0;
  if (fb && !stats) {
    local.resize(n);
    stats = local.data();
  }
  std::vector<Prob> P(1);
  Prob& p = P[0];
  p.c = c;
  p.kappa = kappa;
  p.csw = csw;
  p.tol = tol;
  p.src = src;
  p.sol = sol;
  p.n = n;
  p.stats = stats;
  p.w = &c->ws;
  p.s = c->stream;
  st = setup_problem(p, prm);
  if (st != SQ_OK) return st;
  std::vector<cudaEvent_t> evs;
  sq_status result = SQ_OK;
  st = run_problems(P, prm, c->stream, &c->ws.graph, &c->ws.graph_key, &c->ws.graph2, &c->ws.graph_key2, evs,
                    &result);
  for (auto ev : evs) cudaEventDestroy(ev);
  if (st != SQ_OK) return st;
  st = check_timeouts(c, "sq_solve");
  if (st != SQ_OK) return st;
  if (fb && result != SQ_OK) {
    if (prm.verbose) fprintf(stderr, "libstochq: FP16 solve incomplete, FP32 fallback\n");
    result = fp16_fallback(c, kappa, csw, src, sol, n, tol, prm, stats);
    if (result == SQ_ERR_CUDA || result == SQ_ERR_OOM || result == SQ_ERR_TIMEOUT || result == SQ_ERR_ARG)
      return result;
  }
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int k = 0; k < n; k++) stats[k].seconds = secs;
  if (result != SQ_OK) set_error(c, result, "sq_solve: some sources did not converge (see stats)");
  return result;
}

sq_status solve_batch_impl(const sq_problem* probs, int np, const sq_solve_params* prm_in, sq_solve_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  if (!probs || np <= 0) return SQ_ERR_ARG;
  for (int i = 0; i < np; i++)
    if (!probs[i].ctx) return SQ_ERR_ARG;
  sq_ctx* c0 = probs[0].ctx;
  for (int i = 1; i < np; i++)
    if (probs[i].ctx->device != c0->device) return set_error(c0, SQ_ERR_ARG, "sq_solve_batch: mixed devices");
  sq_solve_params prm;
  if (prm_in) prm = *prm_in;
  else sq_default_params(&prm);
  sq_status st = validate_params(c0, prm);
  if (st != SQ_OK) return st;
  prm.pion = nullptr;  // the pion epilogue is a single-problem option
  prm.pion_tslice = nullptr;
  if (!c0->batch) c0->batch = new BatchCache();
  BatchCache& B = *c0->batch;
  while ((int)B.ws.size() < np) B.ws.push_back(new Workspace());
  while ((int)B.streams.size() < np) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_check(c0, e, "sq_solve_batch streams");
    B.streams.push_back(s);
  }
  // order every problem's stream after its context's stream
  std::vector<Prob> P(np);
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  size_t off = 0;
  for (int i = 0; i < np; i++) {
    Prob& p = P[i];
    p.c = probs[i].ctx;
    p.kappa = probs[i].kappa;
    p.csw = probs[i].c_sw;
    p.tol = probs[i].tol;
    p.src = probs[i].sources;
    p.sol = probs[i].solutions;
    p.n = probs[i].n_rhs;
    p.stats = stats ? stats + off : nullptr;
    off += p.n > 0 ? p.n : 0;
    p.w = B.ws[i];
    p.s = B.streams[i];
    cudaEventRecord(ev, p.c->stream);
    cudaStreamWaitEvent(p.s, ev, 0);
  }
  for (int i = 0; i < np; i++) {
    st = setup_problem(P[i], prm);
    if (st != SQ_OK) {
      cudaEventDestroy(ev);
      if (P[i].c != c0) set_error(c0, st, "sq_solve_batch: problem %d: %s", i, P[i].c->last_error.c_str());
      return st;
    }
  }
  // the batch stream (first context's) waits for every problem's set-up
  for (auto& p : P) {
    cudaEventRecord(ev, p.s);
    cudaStreamWaitEvent(c0->stream, ev, 0);
  }
  cudaEventDestroy(ev);
  sq_status result = SQ_OK;
  st = run_problems(P, prm, c0->stream, &B.graph, &B.key, nullptr, nullptr, B.events, &result);
  if (st != SQ_OK) return st;
  for (int i = 0; i < np; i++) {
    bool seen = false;
    for (int j = 0; j < i; j++) seen = seen || P[j].c == P[i].c;
    if (seen) continue;
    st = check_timeouts(P[i].c, "sq_solve_batch");
    if (st != SQ_OK) {
      if (P[i].c != c0) set_error(c0, st, "%s", P[i].c->last_error.c_str());
      return st;
    }
  }
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (size_t k = 0; k < off; k++) stats[k].seconds = secs;
  if (result != SQ_OK) set_error(c0, result, "sq_solve_batch: some sources did not converge (see stats)");
  return result;
}

}  // namespace sq

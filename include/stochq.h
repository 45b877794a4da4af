/*
 * stochq.h - C ABI of libstochq, a GB300 (sm_103a) solver for the clover
 * Wilson-Dirac system M psi = eta on many stochastic noise sources.
 *
 * The operation (Giedt & Howarth, "Stochastic propagators for multi-pion
 * correlation functions in lattice QCD with GPUs", Sec. "Stochastic
 * propagators", Eq. Sfill): the stochastic all-to-all propagator is built
 * from solution vectors X_i = M^{-1} eta_i of random sources eta_i, where
 * M is the lattice fermion matrix of clover fermions with c_SW = 1.0
 * (Sec. "Correlation function"). The paper does not write M out; this
 * library uses the kappa-normalised Sheikholeslami-Wohlert operator
 *
 *   M = A - kappa D
 *   D psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)
 *   A(x)     = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu Fhat_mu_nu(x)
 *   Fhat     = (Q_mu_nu - Q_mu_nu^+)/8, traceless; Q = sum of the four clover leaves
 *
 * with DeGrand-Rossi gamma matrices (gamma5 = diag(1,1,-1,-1)), periodic
 * space and a factor t_bc on the fermion hop across the time boundary.
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every call
 * ---------------------------------------------------------------------------
 * Lattice dims[4] = {X, Y, Z, T}, each even and >= 2; V = X*Y*Z*T, Vh = V/2.
 * Site x = (x,y,z,t) has lexicographic index i = x + X*(y + Y*(z + Z*t)) and
 * parity p = (x+y+z+t) mod 2. Its checkerboard index within its parity is
 * cb = i / 2 (integer division).
 *
 * Host ("lexicographic") layouts, all FP64, real and imaginary interleaved:
 *   gauge field  U[t][z][y][x][mu][a][b][re,im]   (mu = 0..3 is x,y,z,t;
 *                                                   a = row, b = column)
 *   spinors      S[k][t][z][y][x][spin][colour][re,im]   (k = source)
 *
 * Device ("even-odd") spinor layout, one parity, n sources. A site holds
 * 12 complex numbers, index j = 3*spin + colour, stored in 16-byte chunks;
 * chunk c of source k at checkerboard site cb is element (k*NC + c)*Vh + cb:
 *   SQ_F64: NC = 12 chunks of double2, chunk c = complex j = c
 *   SQ_F32: NC = 6 chunks of float4,  chunk c = complex 2c, 2c+1
 *   SQ_F16: NC = 3 chunks of 8 x IEEE binary16, chunk c = complex 4c..4c+3,
 *           each value stored as v / norm; after the n*3*Vh chunks follow
 *           n*Vh FP32 norms (norm of source k at site cb at k*Vh + cb),
 *           norm = max |re|,|im| over the site's 24 reals (0 for a zero site).
 * sq_field_bytes() gives the size of one such field.
 *
 * Ownership: the context owns the gauge field, clover terms, workspace and
 * its CUDA stream. Caller buffers are never retained past a call.
 * Streams: every call runs on the context's own stream, ordered after the
 * work already queued on the caller's stream given to sq_create (and the
 * caller's stream waits for the call's work before the call returns).
 * Calls that take host buffers return when the results are in them.
 * Errors: every call returns a status; none aborts or exits. The message
 * of the last failure is kept per context (sq_last_error). Arguments are
 * validated before any kernel is launched. One context per host thread.
 */
#ifndef STOCHQ_H
#define STOCHQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sq_ctx sq_ctx;

typedef enum {
  SQ_OK = 0,
  SQ_ERR_ARG = 1,        /* invalid argument (dims, parity, sizes, NULL, ...) */
  SQ_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  SQ_ERR_OOM = 3,        /* device memory could not be allocated */
  SQ_ERR_NONFINITE = 4,  /* NaN or Inf in links or sources */
  SQ_ERR_CLOVER = 5,     /* a 6x6 clover block is singular */
  SQ_ERR_NOCONV = 6,     /* max_iter reached before tol on some source */
  SQ_ERR_BREAKDOWN = 7,  /* BiCGStab broke down and restarts did not help */
  SQ_ERR_TIMEOUT = 8,    /* a bounded device-side wait ran out */
  SQ_ERR_STATE = 9       /* call made in the wrong state (e.g. no gauge) */
} sq_status;

typedef enum { SQ_F64 = 0, SQ_F32 = 1, SQ_F16 = 2 } sq_prec;

/* Where a caller buffer lives. */
enum { SQ_HOST = 0, SQ_DEVICE = 1 };

/* sq_dslash_eo flags */
enum {
  SQ_DS_CLOVER_INV = 1, /* apply A_pp^{-1} after the hopping term */
  SQ_DS_XPAY = 2,       /* out = x + a * (...) instead of out = (...) */
  SQ_DS_SYNC = 4,       /* wait for the result before returning */
  SQ_DS_F64_EMULATED = 8 /* SQ_F64 fields: FP64-accurate double-FP32 arithmetic
                            on the FP32 pipe (the solver's FP64 steps; about
                            46 correct bits) instead of FP64 instructions */
};

/* sq_solve_params.outer */
enum { SQ_OUTER_RELIABLE = 0, SQ_OUTER_DEFECT = 1 };

typedef struct sq_solve_params {
  int inner_prec;      /* SQ_F64: plain FP64 solver; SQ_F32 / SQ_F16: mixed */
  int outer;           /* SQ_OUTER_RELIABLE (keep the Krylov space) or
                          SQ_OUTER_DEFECT (restart at every FP64 update)    */
  double delta;        /* FP64 update when ||r|| < delta * max||r|| since the
                          last update (reliable) or < delta * ||r_start||
                          (defect correction); <= 0 picks the default for
                          the inner precision (FP32 3e-6, FP16 3e-3, FP16
                          with defect correction 1e-4);
                          ignored for SQ_F64. With SQ_F16 and reliable
                          updates, an update while ||r|| is more than 1e-6
                          of the first FP64 residual recomputes r with the
                          FP32 operator instead (a refresh; the Krylov
                          space is kept); below that level updates are FP64 */
  int max_iter;        /* inner iterations per source (default 20000)      */
  int recon;           /* unused: the FP32 links (which FP16 solves also
                          hop with) follow sq_load_gauge's recon          */
  int sites_per_block; /* dslash CTA shape; 0 = autotune                   */
  int rhs_per_block;   /* dslash sources per CTA; 0 = autotune             */
  int chunk;           /* iterations per CUDA-graph launch; 0 (default):
                          24 in a single-problem solve's first launch and
                          4 in each later one, 16 per launch in batches    */
  int use_graph;       /* 1 (default): capture the inner loop in graphs    */
  int io;              /* SQ_HOST (default) or SQ_DEVICE for sources and
                          solutions                                        */
  int use_x0;          /* 1: solutions hold an initial guess on entry      */
  int verbose;         /* 1: progress lines on stderr                      */
  int profile;         /* 1: time every kernel of the inner loop with CUDA
                          events on the context's stream (event nodes in
                          the captured graph); 2: time only the two clover
                          dslash launches per iteration (fewer event
                          nodes); read with sq_get_profile                 */
  double *pion;        /* optional fused epilogue (NULL: none): the pion
                          correlator of every solution, exactly as
                          sq_contract_pion computes it, written to
                          pion[n_rhs][T] in host or device memory per io.
                          On the device it runs from the solutions while
                          the final FP64 residual check is in flight.
                          Ignored by sq_solve_batch.                       */
  const int *pion_tslice; /* [n_rhs] source time slices for pion, same
                          memory kind as pion; NULL: all 0                  */
  double breakdown_tol; /* BiCGStab restarts a source when |rho'| <
                          breakdown_tol ||rhat|| ||r|| (a near breakdown of
                          the recurrence); more than 64 restarts end it with
                          SQ_ERR_BREAKDOWN. <= 0: 1e-14 (the default)       */
  int fallback;        /* SQ_F16 inner only, sq_solve only: sources the FP16
                          solve leaves with SQ_ERR_NOCONV or SQ_ERR_BREAKDOWN
                          (a stagnating FP16 recurrence) are solved again
                          with the FP32 inner solver from their current
                          iterate; 1 (default) or 0                         */
  int fallback_max_iter; /* inner iterations of that FP32 solve; 0: max_iter */
} sq_solve_params;

typedef struct sq_solve_stats {
  int status;            /* sq_status of this source                      */
  int iterations;        /* inner BiCGStab iterations                     */
  int updates;           /* FP64 residual recomputations (reliable updates
                            or defect-correction cycles)                  */
  int restarts;          /* BiCGStab restarts (breakdown or defect cycle) */
  double true_residual;  /* ||eta - M psi|| / ||eta||, FP64, full lattice */
  double seconds;        /* wall time of the whole sq_solve call          */
  int breakdowns;        /* near breakdowns of the recurrence (restarts)   */
  int fallback;          /* 1: solved again with the FP32 inner solver
                            after the FP16 solve did not converge          */
} sq_solve_stats;

/* Fill *p with the defaults (FP32 inner, reliable updates, automatic delta). */
void sq_default_params(sq_solve_params *p);

/* Create a context for one lattice. dims = {X,Y,Z,T}, all even, >= 2.
 * t_bc = -1 (antiperiodic in time) or +1 (periodic). cuda_stream is a
 * cudaStream_t to order against (NULL = legacy default stream).
 * Errors: SQ_ERR_ARG (bad dims/t_bc/NULL ctx), SQ_ERR_CUDA. */
sq_status sq_create(sq_ctx **ctx, const int dims[4], int t_bc, void *cuda_stream);

/* Caller-supplied device memory for the context's persistent buffers (gauge
 * copies and the staging of host links, clover terms and the clover build's
 * field-strength scratch, solver workspaces, contraction and profiling
 * scratch), e.g. a framework's caching allocator. alloc returns a device
 * pointer to at least `bytes` bytes, 256-byte aligned, or NULL (reported as
 * SQ_ERR_OOM / SQ_ERR_CUDA by the call that needed it); free releases a
 * pointer alloc returned, with the same size. `stream` is the context's
 * cudaStream_t, on which the buffer is used; the library synchronises that
 * stream before it frees a buffer, so free may reuse the memory at once.
 * `user` is passed through. Both NULL restores cudaMalloc / cudaFree (the
 * default). The other per-call staging buffers for host I/O stay on the
 * CUDA stream-ordered pool (cudaMallocAsync on the context's stream), and
 * the context's 16-byte device error word and clover bound are allocated by
 * sq_create.
 * Errors: SQ_ERR_ARG (only one of alloc/free given), SQ_ERR_STATE (the
 * context already holds persistent buffers: call it before sq_load_gauge). */
typedef void *(*sq_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*sq_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
sq_status sq_set_allocator(sq_ctx *ctx, sq_alloc_fn alloc, sq_free_fn free_fn, void *user);

/* Free everything the context owns. NULL is accepted. */
sq_status sq_destroy(sq_ctx *ctx);

/* Load the gauge field U (host or device, lexicographic FP64, see above).
 * Kept on the device as FP64 reconstruct-18 and FP32 reconstruct-`recon`
 * (used by the FP32 and the FP16 operator), per-parity site-blocked (the analogue of the
 * array reordering between the paper's host code and its GPU inverter,
 * Sec. "Stochastic propagators"). Drops cached clover terms. Host links go
 * through a staging buffer of the context's size that the context keeps.
 * Errors: SQ_ERR_ARG (recon not 12/18, NULL), SQ_ERR_NONFINITE,
 * SQ_ERR_ARG if recon = 12 and some link is not SU(3) to 1e-6. */
sq_status sq_load_gauge(sq_ctx *ctx, const double *U, int recon, int where);

/* Build the clover term A and its inverse for (kappa, c_sw) on the device
 * in FP64: clover-leaf Fhat (Sec. "Correlation function": c_SW = 1.0 is
 * the paper's tree-level value), A as two 6x6 Hermitian blocks per site in
 * the chiral basis, each inverted in FP64 (LDL^H; partial-pivot
 * Gauss-Jordan when a block is not safely positive definite);
 * an FP32 copy of A^{-1} feeds the FP32 and FP16 operators. Up to 8
 * (kappa, c_sw) pairs are cached; a cached pair is reused.
 * Errors: SQ_ERR_STATE (no gauge), SQ_ERR_ARG (non-finite kappa/c_sw),
 * SQ_ERR_CLOVER (a block is singular: |pivot| < 1e-12 * block scale). */
sq_status sq_build_clover(sq_ctx *ctx, double kappa, double c_sw);

/* Bytes of one device even-odd field (one parity) of n_rhs sources. */
sq_status sq_field_bytes(const sq_ctx *ctx, sq_prec prec, int n_rhs, size_t *bytes);

/* Convert the parity-`parity` sites of n_rhs lexicographic FP64 spinors
 * (host or device per `where`) into a device even-odd field of precision
 * prec. Errors: SQ_ERR_ARG. */
sq_status sq_pack_spinor(sq_ctx *ctx, void *eo_out, const double *lex_in,
                         int parity, sq_prec prec, int n_rhs, int where);

/* Write the parity-`parity` sites of a device even-odd field into n_rhs
 * lexicographic FP64 spinors (host or device per `where`); sites of the
 * other parity are left unchanged. Errors: SQ_ERR_ARG. */
sq_status sq_unpack_spinor(sq_ctx *ctx, double *lex_out, const void *eo_in,
                           int parity, sq_prec prec, int n_rhs, int where);

/* One even-odd hopping application on device even-odd fields of precision
 * prec, n_rhs sources:
 *   w   = D_{p,1-p} in                      (hop from parity 1-p onto p)
 *   w  <- A_pp^{-1} w                       if flags & SQ_DS_CLOVER_INV
 *   out = x + a * w   if flags & SQ_DS_XPAY, else out = w
 * in has parity 1 - out_parity; out and x have parity out_parity (x may
 * equal out; in must not alias out). D_eo / D_oe are the blocks of the
 * hopping term D above (the Schur operator of the solver is
 * 1 - kappa^2 A_ee^{-1} D_eo A_oo^{-1} D_oe). SQ_DS_CLOVER_INV uses the
 * clover term of the last sq_build_clover. Asynchronous unless
 * SQ_DS_SYNC. Errors: SQ_ERR_ARG, SQ_ERR_STATE (no gauge / no clover). */
sq_status sq_dslash_eo(sq_ctx *ctx, void *out, const void *in, const void *x,
                       int out_parity, sq_prec prec, int n_rhs, int flags, double a);

/* Per-source squared L2 norms of a device even-odd field (one parity,
 * n_rhs sources, precision prec, layout above): out[k] = sum over the
 * sites and 24 reals of source k of v^2 (FP16: the stored values times
 * their site norm), accumulated in FP64 by a fixed-order two-level
 * reduction (per-CTA partials, then the last CTA of each source sums them
 * in block order), so the result is bitwise reproducible. The reduction
 * scratch comes from the context stream's allocator. out: n_rhs doubles,
 * host or device per `where`. Errors: SQ_ERR_ARG, SQ_ERR_OOM. */
sq_status sq_norm2_eo(sq_ctx *ctx, const void *eo_field, sq_prec prec, int n_rhs, double *out,
                      int where);

/* Allocation-free variant of sq_norm2_eo (the paper has no counterpart;
 * this is a service for callers of this library). It gives the same
 * per-source squared norms (within FP64 rounding: the sum is taken in a
 * different fixed order) but allocates no device memory at all, for callers
 * that must not allocate at the point of the call: code that enqueues work
 * while another thread captures a CUDA graph in global capture mode (an
 * allocation there invalidates the capture), real-time loops that cannot
 * afford the device synchronisation cudaMalloc may imply, and frameworks
 * whose memory pool owns all device memory. The reduction scratch is a
 * fixed static device array of 259 KiB that every GPU which loads the
 * library keeps until the process exits; n_rhs is limited to 256 sources
 * (larger n_rhs: SQ_ERR_ARG). The first call on a device looks up the
 * array's device address for that device and loads this entry point's
 * kernels of all three precisions (one-time set-up, whatever prec that
 * first call has); make that first call before any stream capture
 * starts. Every call shares the
 * array, which keeps the last call's contents: calls that overlap on one
 * GPU (other streams, other contexts, other threads) race and must be
 * serialised by the caller. Inputs and outputs as sq_norm2_eo.
 * Errors: SQ_ERR_ARG, SQ_ERR_CUDA. */
sq_status sq_norm2_eo_noalloc(sq_ctx *ctx, const void *eo_field, sq_prec prec, int n_rhs,
                              double *out, int where);

/* Full-lattice FP64 operator: out = M in for n_rhs lexicographic FP64
 * spinors (host or device per `where`), with the clover term for
 * (kappa, c_sw) (built if not cached). Errors: SQ_ERR_ARG, SQ_ERR_STATE,
 * SQ_ERR_CLOVER. */
sq_status sq_apply_M(sq_ctx *ctx, double *out, const double *in, int n_rhs,
                     double kappa, double c_sw, int where);

/* Solve M psi_k = eta_k for n_rhs sources (Eq. Sfill's X_i = M^{-1} eta_i)
 * with even-odd preconditioned BiCGStab on
 *   Mhat = 1 - kappa^2 A_ee^{-1} D_eo A_oo^{-1} D_oe,
 *   bhat = A_ee^{-1} (eta_e + kappa D_eo A_oo^{-1} eta_o),
 *   psi_o = A_oo^{-1} (eta_o + kappa D_oe psi_e),
 * batched over all sources, mixed precision per params (FP64 updates of
 * the true residual). Stops when the FP64 full-lattice relative residual
 * ||eta_k - M psi_k|| / ||eta_k|| <= tol for every source (checked).
 * sources/solutions: lexicographic FP64, host or device per params->io.
 * params NULL = defaults; stats (n_rhs entries) may be NULL.
 * Errors: SQ_ERR_ARG, SQ_ERR_STATE (no gauge), SQ_ERR_NONFINITE (source),
 * SQ_ERR_CLOVER, SQ_ERR_NOCONV / SQ_ERR_BREAKDOWN (solutions then hold the
 * best iterate; stats give the per-source reason), SQ_ERR_OOM, SQ_ERR_CUDA.
 * A zero source gives a zero solution. */
sq_status sq_solve(sq_ctx *ctx, double kappa, double c_sw, const double *sources,
                   double *solutions, int n_rhs, double tol,
                   const sq_solve_params *params, sq_solve_stats *stats);

/* One problem of a heterogeneous batch. */
typedef struct sq_problem {
  sq_ctx *ctx;            /* lattice (each problem may use its own)       */
  double kappa, c_sw;
  const double *sources;  /* lexicographic FP64, per params->io           */
  double *solutions;
  int n_rhs;
  double tol;
} sq_problem;

/* Solve several problems (different lattices and/or kappa; several
 * problems may share a context) in one iteration loop: every chunk of
 * iterations of every problem is one branch of a single captured CUDA
 * graph, so all problems advance concurrently from one graph launch, and
 * converged sources retire from every kernel of their problem. Each
 * problem keeps its own workspace (cached in the first problem's context
 * between calls). All contexts must be on the same CUDA device; params
 * apply to every problem (params->profile is ignored). stats holds
 * sum(n_rhs) entries in problem order. Errors as sq_solve (the message is
 * kept in the first problem's context). */
sq_status sq_solve_batch(const sq_problem *probs, int n_probs,
                         const sq_solve_params *params, sq_solve_stats *stats);

/* Dilution schemes of sq_dilute (Sec. "Stochastic propagators": the
 * paper's time-spin-colour dilution). */
enum { SQ_DILUTE_TIME = 1, SQ_DILUTE_SPIN_COLOUR = 2, SQ_DILUTE_FULL = 3 };

/* Diluted sources from noise vectors: D = T (time), 12 (spin-colour) or 12*T
 * (full) sources per noise vector, source k*D + d keeping noise vector k on
 * timeslice t = d (time), spin-colour component a = d = 3*spin + colour
 * (spin-colour) or t = d / 12 and a = d % 12 (full), zero elsewhere. The
 * sources of one noise vector sum to it and have disjoint supports. A noise
 * vector equal to 1 on the twelve components of one site and 0 elsewhere
 * gives, with SQ_DILUTE_SPIN_COLOUR, the twelve point sources of the point
 * propagator at that site. noise: n_noise lexicographic FP64 fields; out:
 * n_noise * D fields, same layout; both host or both device memory per
 * `where`, owned by the caller. Host memory: returns when out is written;
 * device memory: ordered after the caller's stream, no wait.
 * Errors: SQ_ERR_ARG (NULL, n_noise <= 0, unknown scheme, bad where),
 * SQ_ERR_CUDA. */
sq_status sq_dilute(sq_ctx *ctx, const double *noise, int n_noise, int scheme,
                    double *out, int where);

/* Pion correlator of each solution vector (the zero-momentum contraction
 * sum_{x in t} sum_y tr S S^+ of Sec. "Stochastic propagators", estimated
 * per source):  C[k][dt] = sum over sites x on timeslice (t_k + dt) mod T
 * of sum_{spin,colour} |psi_k(x)|^2, t_k = src_tslice[k] (0 if NULL).
 * Accumulated in FP64 in a fixed order. solutions: lexicographic FP64,
 * host or device per `where`; C: host, n_rhs * T doubles. No 1/N or
 * volume factor. Errors: SQ_ERR_ARG. */
sq_status sq_contract_pion(sq_ctx *ctx, const double *solutions, int n_rhs,
                           const int *src_tslice, double *C, int where);

/* Stochastic operators of Eq. stoop (Sec. "Stochastic propagators"): for
 * n_rhs noise sources eta_i and their solution vectors X_j = M^-1 eta_j,
 *   O[t][i][j] = sum over sites y on timeslice t of eta_i(y)^+ gamma5 X_j(y)
 * (spin and colour contracted, DeGrand-Rossi gamma5 = diag(1,1,-1,-1)),
 * complex, stored as O[(t*n_rhs + i)*n_rhs + j] = (re, im), T*n_rhs^2
 * pairs. If C is not NULL it also gets the correlator built from the
 * operators, averaged over the source timeslice:
 *   C[dt] = 1/(n_rhs^2 T) sum_t0 sum_{i,j} O_ij((t0+dt) mod T) O_ji(t0),
 * complex, T pairs (the i = j terms are the biased same-noise products;
 * they are kept, as in the formula). eta, X: lexicographic FP64 fields of
 * n_rhs vectors as sq_solve takes them. eta, X, O and C are all host or
 * all device memory per `where`; the caller owns them. FP64 throughout,
 * summed in a fixed order (bitwise reproducible for the same inputs and
 * device). Host memory: returns when O and C are written. Device memory:
 * ordered after the caller's stream and returns without waiting. The
 * context keeps a partial-sum buffer of T * n_rhs^2 * 16 bytes times the
 * number of K-groups (at most 4 CTAs per SM) between calls.
 * Errors: SQ_ERR_ARG (NULL eta/X/O, n_rhs <= 0 or > 4080, bad where),
 * SQ_ERR_CUDA. */
sq_status sq_contract_stoch_op(sq_ctx *ctx, const double *eta, const double *X,
                               int n_rhs, double *O, double *C, int where);

/* The operators of sq_contract_stoch_op (same O and C, same layouts) on the
 * tensor cores, for sources whose real and imaginary components are all
 * 0 or +-1 (Z2 and Z4 noise, diluted or not). gamma5 X is cut per source,
 * timeslice and block of 4096 rows into a 55-bit fixed-point integer
 * relative to the block's largest component and split into five 11-bit
 * digits; each digit's products with the sources are summed on the tensor
 * cores in FP16 x FP16 -> FP32, exactly (every partial sum is an integer
 * below 2^24), and the digits are combined in FP64 with power-of-two
 * weights. The result differs from sq_contract_stoch_op by the truncation
 * of X below 2^-55 of each block's largest component and by FP64 rounding
 * order. Always synchronises the context's stream (it reports the source
 * check). The context keeps a workspace of the packed operands (up to
 * 8 GiB; larger problems run in timeslice batches). Worth it for n_rhs of
 * about 128 and more (the tensor tiles hold 128 x 16 sources).
 * Errors: SQ_ERR_ARG (as sq_contract_stoch_op, or a source component not
 * 0 or +-1), SQ_ERR_NONFINITE (X), SQ_ERR_TIMEOUT (a bounded wait of the
 * kernel ran out; nothing hangs), SQ_ERR_CUDA. */
sq_status sq_contract_stoch_op_z4(sq_ctx *ctx, const double *eta, const double *X,
                                  int n_rhs, double *O, double *C, int where);

/* Traces of filled stochastic propagators without the fill (Eq. Sfill and
 * the "sum_x sum_z tr S_s S_s^+" entry of Table Lcomp, Sec. "Stochastic
 * propagators"): with S_A(t,z; t0,x) = (1/n_rhs) sum_i XA_i(t,z) etaA_i(t0,x)^+
 * and S_B likewise from the second set (etaB, XB),
 *   C[t0][t] = sum over source sites x on timeslice t0 and sink sites z on
 *              timeslice t of tr[S_A(t,z; t0,x) S_B(t,z; t0,x)^+]
 * (spin-colour trace), complex, T*T pairs, C[(t0*T + t)] = (re, im).
 * Computed as (1/n_rhs^2) tr[P(t) Q(t0)] with the Gram matrices
 * P_ji(t) = sum_{z in t} XB_j(z)^+ XA_i(z) and Q_ij(t0) = sum_{x in t0}
 * etaA_i(x)^+ etaB_j(x), so S (12*12*T*V_3^2 entries per t0) is never
 * formed. etaB = XB = NULL uses one set for both propagators (the paper's
 * correlated option; the i = j terms are kept as the formula has them).
 * Fields: lexicographic FP64, n_rhs vectors each, as sq_solve takes them;
 * all inputs and C host or all device memory per `where`; the caller owns
 * them. FP64, fixed summation order. Host memory: returns when C is
 * written; device memory: ordered after the caller's stream, no wait. Uses
 * the context's contraction buffer (2 + K-groups) * T * n_rhs^2 * 16 bytes.
 * Errors: SQ_ERR_ARG (NULL etaA/XA/C, only one of etaB/XB given,
 * n_rhs <= 0 or > 4080, bad where), SQ_ERR_CUDA. */
sq_status sq_contract_prop_trace(sq_ctx *ctx, const double *etaA, const double *XA,
                                 const double *etaB, const double *XB, int n_rhs,
                                 double *C, int where);

/* Diagram contractions of the two-pion correlation function at zero
 * momentum for one gauge configuration (Sec. "Stochastic propagators":
 * Diagram 0; Sec. "Correlation function": Diagrams 1-3 and the sum
 * C = C0 + C1 - C2 - C3). Inputs are lexicographic FP64 fields, as sq_solve
 * takes them:
 *   Xp        12 solutions Xp[a] = M^{-1} e_a, e_a the unit source of
 *             spin-colour a = 3*spin + colour at the origin: the point
 *             propagator S(.;0,0) (sq_dilute's spin-colour dilution of a
 *             noise vector equal to 1 on the twelve components of site 0
 *             gives the twelve sources)
 *   etaA, XA  n_rhs noise sources and their solutions, used for every
 *             all-to-all S of Eq. Sfill, S(w;w') ~ (1/n_rhs) sum_i XA_i(w) etaA_i(w')^+
 *   etaB, XB  a second, independent set, used for every S^+ (both NULL:
 *             set A, the paper's one-set option, which correlates S and S^+)
 * Output out[7][T] complex (re, im), q = 0..6 at sink timeslice t:
 *   0 P(t)   = sum_y tr[S(t,y;0,0) S^+(t,y;0,0)]   (real; Table Lcomp's
 *              "sum_y tr S_p S_p^+")
 *   1 Q0(t)  = sum_x sum_z tr[S(t,z;0,x) S^+(t,z;0,x)]   (Table Lcomp's
 *              "sum_x sum_z tr S_s S_s^+")
 *   2 Qtt(t) = sum_y sum_z tr[S(t,z;t,y) S^+(t,z;t,y)]
 *   3 C0(t)  = P(t) Q0(t)   Diagram 0 before its vacuum term <P><Q0>
 *   4 C1(t)  = Qtt(t) P(0)  Diagram 1 before its vacuum terms
 *   5 C2(t)  = sum_{x,y,z} tr[S^+(0,x;0,0) S(0,x;t,z) S^+(t,y;t,z) S(t,y;0,0)]
 *   6 C3(t)  = conj C2(t)   Diagram 3
 * with x on timeslice 0, y and z on timeslice t and daggers on spin-colour
 * only. Diagram 0's printed second trace pairs S(t,z;0,0) with S^+(t,x;0,0);
 * the library takes the text around it (a source at (0,x), a sink at
 * (t,z), the all-to-all S(t,z;0,x)). S is never formed: C2(t) =
 * (1/n^2) sum_ij Q_ij(t) W_ji(t) with Q_ij(t) = sum_{z in t} etaA_i^+ etaB_j
 * and W_ji(t) = sum_a conj(GB(t)_aj) GA(0)_ai, G(t)_ai = sum_{y in t}
 * Xp_a^+ X_i; FP64 with a fixed summation order. All inputs and out host or
 * all device per `where`; host memory: returns when out is written; device
 * memory: ordered after the caller's stream, no wait. Uses the context's
 * contraction buffer. Errors: SQ_ERR_ARG (NULL Xp/etaA/XA/out, only one of
 * etaB/XB, n_rhs <= 0 or > 4080, bad where), SQ_ERR_OOM, SQ_ERR_CUDA. */
sq_status sq_contract_diagrams(sq_ctx *ctx, const double *Xp, const double *etaA, const double *XA,
                               const double *etaB, const double *XB, int n_rhs, double *out, int where);

/* Vacuum-subtracted averages over n_cfg gauge configurations of the records
 * of sq_contract_diagrams (rec[cfg][7][T] complex; the paper averages every
 * diagram over configurations, Sec. "Correlation function"): out[5][T] complex,
 *   0 <C0> - <P><Q0>                   (Diagram 0 with its vacuum term)
 *   1 <(Qtt - <Qtt>)(P(0) - <P(0)>)>   (Diagram 1)
 *   2 <C2>   3 <C3>
 *   4 C = C0 + C1 - C2 - C3            (the sum of the diagrams)
 * on the context's GPU, configurations summed in order. rec and out host or
 * device per `where`. Errors: SQ_ERR_ARG (NULL, n_cfg <= 0, bad where),
 * SQ_ERR_CUDA. */
sq_status sq_diagrams_ensemble(sq_ctx *ctx, const double *rec, int n_cfg, double *out, int where);

/* Per kernel class of the solver's inner loop (profiling). */
typedef struct sq_kernel_stat {
  char name[48];       /* kernel class, e.g. "dslash_clover"              */
  long long launches;  /* launches timed                                  */
  double ms;           /* summed device time between the class's events   */
  double bytes;        /* summed algorithmic bytes: each datum of a launch
                          counted once (links and clover blocks once per
                          launch, spinors once per active source)         */
  double flops;        /* summed algorithmic flops (1320 per site and
                          source for the hopping term, 504 for a clover
                          block pair, BLAS-1 by its arithmetic)           */
} sq_kernel_stat;

/* Totals of the last sq_solve that ran with params->profile = 1, one entry
 * per kernel class (13). out may be NULL to query *n only; otherwise up to
 * max entries are written. Errors: SQ_ERR_ARG, SQ_ERR_STATE (no profiled
 * solve yet). */
sq_status sq_get_profile(const sq_ctx *ctx, sq_kernel_stat *out, int max, int *n);

/* Number of kernels this context has launched so far (kernel nodes of
 * replayed CUDA graphs included). */
sq_status sq_kernel_launches(const sq_ctx *ctx, long long *n);

/* Launch shape of the even-odd dslash for fields of precision prec with
 * n_rhs sources on this context's lattice: the autotuner's choice (made by
 * the first sq_dslash_eo or sq_solve that needs it, timing the candidates on
 * that call's own fields) or one set here, e.g. a shape saved from an
 * earlier run, which then replaces tuning for later calls.
 *   kind 0: per-site kernel; shape = {sites per CTA (multiple of 32),
 *           sources per CTA, grid order 0/1, 0, 0}
 *   kind 1: halo-tiled kernel (SQ_F32 / SQ_F16 with reconstruct-12 links;
 *           section "dslash" of the hopping term above): every CTA owns all
 *           X/2 checkerboard sites of shape[0] x shape[1] x shape[2] rows in
 *           (y, z, t) (each dividing Y, Z, T; 32..256 sites, a multiple of
 *           32; SQ_F16 needs X a multiple of 8) for shape[3] source slots,
 *           staging every source's input spinors plus halo rows in a shared-
 *           memory ring of depth shape[4] (2 or 3)
 * Errors: SQ_ERR_ARG (unknown kind, a shape the lattice or the shared
 * memory does not admit, n_rhs <= 0), SQ_ERR_STATE (get: no shape chosen
 * for this (prec, n_rhs) yet). */
sq_status sq_set_dslash_shape(sq_ctx *ctx, sq_prec prec, int n_rhs, int kind, const int shape[5]);
sq_status sq_get_dslash_shape(const sq_ctx *ctx, sq_prec prec, int n_rhs, int *kind, int shape[5]);

/* Persisted launch shapes. sq_tune_save appends one text line per shape
 * this context holds (tuned or set), keyed by the GPU's name, the lattice
 * dims, the precision, the reconstruction and n_rhs, to the file `path`;
 * sq_tune_load reads the lines of such a file that match this context's GPU
 * and lattice (later lines win) and installs their shapes, so later calls
 * for those keys skip the tuner. Lines that do not parse, belong to another
 * GPU or lattice, or name a shape this lattice does not admit are skipped;
 * *n_loaded (may be NULL) counts the shapes installed.
 * Errors: SQ_ERR_ARG (NULL path), SQ_ERR_STATE (the file cannot be opened
 * or written). */
sq_status sq_tune_save(const sq_ctx *ctx, const char *path);
sq_status sq_tune_load(sq_ctx *ctx, const char *path, int *n_loaded);

/* Limit, in SM clock cycles, of every bounded device-side wait in this
 * context's kernels (the bulk-copy rings of the halo-tiled dslash and of the
 * tensor-core stochastic operators); 0 restores the default of 4e9 cycles
 * (about 2 s). A wait that runs out records a timeout, lets the copies it
 * issued drain and returns, and the call reports SQ_ERR_TIMEOUT (sq_solve,
 * sq_dslash_eo with SQ_DS_SYNC, sq_contract_stoch_op_z4); the context stays
 * usable. stall_test = 1 (a test of that path) makes those kernels first
 * wait, with this limit, on a barrier that nothing completes, so the wait
 * runs out and the call returns SQ_ERR_TIMEOUT; 0 is normal operation.
 * Errors: SQ_ERR_ARG (negative cycles, stall_test not 0/1). */
sq_status sq_set_wait_cycles(sq_ctx *ctx, long long cycles, int stall_test);

const char *sq_status_string(sq_status s);
const char *sq_last_error(const sq_ctx *ctx);

/* Precision, in bits, in which this build of the library accumulates the
 * fused sums of sq_solve's inner iteration over FP32 and FP16 fields (the
 * BiCGStab inner products and norms that give alpha, omega and beta in the
 * solve of Eq. Sfill's X_i = M^{-1} eta_i): 32 = FP32 per thread and per
 * warp, then FP64 across warps (the default build); 64 = FP64 from the thread
 * level up (the build with SQ_INNER_SUMS_FP64). Sums over FP64 fields and
 * every reliable-update and true-residual sum are FP64 in both. No
 * arguments, no errors. */
int sq_inner_sum_bits(void);

#ifdef __cplusplus
}
#endif

#endif /* STOCHQ_H */

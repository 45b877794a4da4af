// Host-side internals of libstochq: the context, the solver workspace and
// the kernel launchers that the translation units share.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <map>
#include <string>
#include <vector>

#include "../../include/stochq.h"
#include "sq_solver_dev.cuh"

namespace sq {

// A device error word bit set by kernels (sticky until read).
enum { ERRBIT_NONFINITE = 1, ERRBIT_CLOVER = 2, ERRBIT_NOT_SU3 = 4, ERRBIT_TIMEOUT = 8 };

struct CloverSet {
  double kappa = 0, csw = 0;
  double2* A64 = nullptr;     // [2][36][Vh] packed A (FP64)
  double2* Ainv64 = nullptr;  // [2][36][Vh] packed A^{-1} (FP64)
  float4* Ainv32 = nullptr;   // [2][18][Vh]
  float4* Adf = nullptr;      // [2][36][Vh] A split into float pairs (re.h, im.h, re.l, im.l)
  float4* Ainvdf = nullptr;   // [2][36][Vh] A^{-1} split likewise
  double a_bound = 1.0;       // max over sites of a Gershgorin bound on ||A||_2
  int valid = 0;              // built for the current gauge field
  unsigned long long tick = 0;
};

// Dslash launch shape. kind 0: the per-site kernel, sites per CTA (x) and
// sources per CTA (y). kind 1: the halo-tiled kernel (FP32 / FP16,
// reconstruct-12), tile rows by x bz x bt (x complete), sg source slots per
// CTA, an nbuf-deep ring of staged source buffers.
struct Shape {
  int sx = 64, ry = 2;
  int order = 0;  // 0: source blocks fastest in the flattened grid
  int kind = 0;
  int by = 0, bz = 0, bt = 0, sg = 0, nbuf = 2;
};

// Device memory for persistent buffers: the caller's callbacks or
// cudaMalloc / cudaFree. A buffer is freed through the allocator that made it.
struct Allocator {
  sq_alloc_fn alloc = nullptr;
  sq_free_fn free = nullptr;
  void* user = nullptr;
  cudaStream_t stream = nullptr;  // the owning context's stream
};
cudaError_t dev_alloc(const Allocator& a, void** p, size_t bytes);
void dev_free(const Allocator& a, void* p, size_t bytes);  // p may be NULL

struct Workspace {
  Allocator mem;  // allocator of base and hist
  size_t bytes = 0;
  void* base = nullptr;
  int n_rhs = 0;
  int inner = -1;
  int Vh = 0;
  // FP64 fields (even parity unless noted), n_rhs sources each
  Field b64, x64, r64, t64o, x64o;  // t64o, x64o: odd parity
  // inner-precision fields
  Field r, rh, p, v, s, t, to;  // to: odd parity
  Field xs;                     // FP32 (or FP64) accumulator
  // lexicographic staging (n_rhs * V * 24 doubles) and eo source halves
  double* lex = nullptr;
  Field eta_e, eta_o;           // FP64
  // reductions and control
  double* partial = nullptr;
  unsigned* counter = nullptr;
  RhsState* st = nullptr;
  Control* ctl = nullptr;
  int* active_list = nullptr;
  int* update_list = nullptr;
  int* refresh_list = nullptr;  // sources whose update is an FP32 refresh
  bool refresh = false;         // FP32 refreshes enabled for this solve
  double* scal = nullptr;       // n_rhs * 4 doubles of scratch results
  int nblk_stride = 0;
  // solution output: unpack, copy-out and pion epilogue run on `aux`,
  // overlapped with the FP64 residual check on the solve stream
  double* pion = nullptr;       // n_rhs * T correlator (device)
  int* tsl = nullptr;           // n_rhs source time slices (device)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_rec = nullptr, ev_out = nullptr;
  cudaEvent_t ev_in[4] = {nullptr, nullptr, nullptr, nullptr};  // source groups copied in
  int* flag = nullptr;          // non-finite input flag
  // cached graph of `chunk` iterations, keyed by everything baked into it
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned long long> graph_key;
  cudaGraphExec_t graph2 = nullptr;  // the tail chunk's graph (chunks sized automatically)
  std::vector<unsigned long long> graph_key2;
  // profiling: one event before each iteration and after each of its kernels
  std::vector<cudaEvent_t> pev;
  int* hist = nullptr;  // [2][chunk]: sources active / updated per iteration
  int hist_chunk = 0;
  int* h_pin = nullptr;  // pinned host read-back buffer of the iteration loop
  size_t h_pin_n = 0;    // ints it holds
};

// Workspaces, streams and the captured graph of sq_solve_batch, kept in the
// first problem's context between calls.
struct BatchCache {
  std::vector<Workspace*> ws;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned long long> key;
};

// Kernel classes of one solver iteration (profiling), in launch order.
enum KClass {
  KC_DSLASH_CLOVER = 0,    // tmp_o = A_oo^{-1} D_oe p   (and of s)
  KC_DSLASH_XPAY_ALPHA,    // v = p - k^2 A_ee^{-1} D_eo tmp_o ; <rhat, v>
  KC_S_UPDATE,             // s = r - alpha v
  KC_DSLASH_CLOVER_2,      // second tmp_o (same kernel as class 0)
  KC_DSLASH_XPAY_OMEGA,    // t = s - k^2 ... ; <t, s>, <t, t>
  KC_XR_UPDATE,            // x += alpha p + omega s ; r = s - omega t ; norms
  KC_P_UPDATE,             // p = r + beta (p - omega v)
  KC_PLAN,                 // update lists (grouped across sources)
  KC_REFRESH,              // FP32 refresh: r = bhat - Mhat x in FP32
  KC_REL_X,                // FP64 update: x64 += xs ; r64 = b - x64
  KC_REL_DSLASH1,          // FP64 tmp = A^{-1} D x64
  KC_REL_DSLASH2,          // FP64 r64 += k^2 A^{-1} D tmp ; ||r64||^2
  KC_REL_R,                // r = r64 ; <rhat, r>
  KC_CONTROL,              // active list
  KC_N
};

struct KStat {
  long long launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};

}  // namespace sq

struct sq_ctx {
  int dims[4] = {0, 0, 0, 0};
  int V = 0, Vh = 0;
  int t_bc = -1;
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  // gauge
  int have_gauge = 0;
  int recon = 12;
  int su3 = 0;  // links passed the SU(3) check (needed by reconstruct-12)
  double2* U64 = nullptr;  // [2][4][9][Vh]
  void* U32 = nullptr;     // recon 12: float4 [2][4][3][Vh]; 18: float2 [2][4][9][Vh]
  float4* Udf = nullptr;   // [2][4][9][Vh] U64 split into float pairs (emulated FP64)
  // clover cache
  std::vector<sq::CloverSet> clover;
  int cur_clover = -1;
  unsigned long long tick = 0;
  // device error word, and the clover build's norm bound (same allocation)
  int* d_err = nullptr;
  unsigned long long* d_bound = nullptr;
  double2* cloverF = nullptr;  // [6][9][V] field strengths: the clover build's scratch
  double* gstage = nullptr;    // [V][4][3][3] complex: staging of host links (sq_load_gauge)
  sq::Workspace ws;
  sq::BatchCache* batch = nullptr;
  unsigned long long uid = 0;  // unique per context (graph cache keys)
  std::map<long long, sq::Shape> tuned;
  std::map<long long, std::array<int, 3>> tuned_meta;  // (prec, recon, n) of each tuned key
  std::string last_error;
  long long launches = 0;          // kernels launched (graph nodes included)
  int prof_valid = 0;
  int prof_inner = 0;
  sq::KStat prof[sq::KC_N];        // per-class totals of the last profiled solve
  sq::Allocator mem;               // persistent device buffers
  void* stoch_part = nullptr;      // K-group partials of the stochastic operators
  size_t stoch_cap = 0;            // bytes held by stoch_part
  long long wait_cycles = 0;       // limit of the bounded device waits (0: about 2 s)
  int wait_stall = 0;              // test: wait first on a barrier nothing completes
};

namespace sq {

Geom geom_of(const sq_ctx* c);
sq_status set_error(sq_ctx* c, sq_status s, const char* fmt, ...);
sq_status cuda_check(sq_ctx* c, cudaError_t e, const char* what);
size_t field_bytes(int Vh, int prec, int n);
Field make_field(void* data, int Vh, int prec, int n);
sq_status enter_stream(sq_ctx* c);  // order ctx stream after the caller's
sq_status leave_stream(sq_ctx* c);  // order the caller's stream after ctx
sq_status read_error_word(sq_ctx* c, int* bits);

// ---- gauge / clover (sq_gauge.cu)
sq_status gauge_convert(sq_ctx* c, const double* dev_lex);
sq_status clover_build(sq_ctx* c, CloverSet& cs, double kappa, double csw);
size_t clover_scratch_bytes(const sq_ctx* c);
// sets *flag (device) to 1 if any of the n doubles is not finite; no sync
void launch_finite(const sq_ctx* c, const double* dev, size_t n, int* flag, cudaStream_t s);

// ---- spinor layout, BLAS, reductions (sq_blas.cu)
void launch_pack(const sq_ctx* c, Field out, const double* lex, int parity, int prec, int n, cudaStream_t s);
void launch_unpack(const sq_ctx* c, double* lex, Field in, int parity, int prec, int n, cudaStream_t s);
// out = c1 * x + c2 * (C in), C = A (which=0) or A^{-1} (which=1), FP64
void launch_clover64(const sq_ctx* c, const CloverSet& cs, Field out, Field x, Field in, int parity,
                     double c1, double c2, int which, int n, cudaStream_t s);
// per-source FP64 norms^2 of an eo field (any precision) -> out[k]
void launch_norm2(const sq_ctx* c, Field f, int prec, int n, double* out, RedArgs ra, cudaStream_t s);
void launch_pack_norm2(const sq_ctx* c, Field out, const double* lex, int parity, int n, double* norm, RedArgs ra,
                       cudaStream_t s);

// ---- dslash (sq_dslash.cu)
struct DslashCall {
  Field out, in, x;
  int p_out;
  int prec, recon;
  int clover;  // 0: none, 1: apply A^{-1}
  int xpay;
  double a;
  const CloverSet* cs;
  // sources: identity 0..n-1 when list == nullptr
  const int* list;
  const int* count;
  int n;
  int fin;  // FinKind for fused reductions
  Field r1; // extra operand of the reduction (rhat for FIN_ALPHA)
  RedArgs ra;
  Shape shape;
  // FP64 fields only: emul = 1 does the arithmetic in double-FP32 on the
  // FP32 pipe (sq_dslash_df.cu); xfirst = 1 applies A^-1 after the xpay
  // (out = A^-1 (x + a D in)), writing x + a D in to out2 if it is set
  int emul;
  int xfirst;
  Field out2;
};
void launch_dslash(const sq_ctx* c, const DslashCall& d, cudaStream_t s);
// emulated-FP64 kernels (sq_dslash_df.cu)
bool launch_dslash_df(const sq_ctx* c, const DslashCall& d, Field out2, int xfirst, cudaStream_t s, int* nparts);
void launch_clover_df(const sq_ctx* c, const CloverSet& cs, Field out, Field x, Field in, int parity, double c1,
                      double c2, int which, int n, cudaStream_t s,
                      const RedArgs* norm = nullptr);
// halo-tiled kernel (sq_dslash_tile.cu): false if d.shape does not apply
bool launch_dslash_tile(const sq_ctx* c, const DslashCall& d, cudaStream_t s, int* nparts);
bool tile_shape_ok(const sq_ctx* c, int prec, int recon, const Shape& sh);
int dslash_nblk(const sq_ctx* c, Shape sh);
Shape tune_dslash(sq_ctx* c, DslashCall d, cudaStream_t s);
bool dslash_tuned(const sq_ctx* c, int prec, int recon, int n);

// ---- solver (sq_solver.cu)
sq_status solve_impl(sq_ctx* c, double kappa, double csw, const double* src, double* sol, int n,
                     double tol, const sq_solve_params* prm, sq_solve_stats* stats);
sq_status solve_batch_impl(const sq_problem* probs, int n_probs, const sq_solve_params* prm,
                           sq_solve_stats* stats);

void release_workspace(sq_ctx* c);

// ---- dilution (sq_dilute.cu)
int dilution_count(const sq_ctx* c, int scheme);  // sources per noise vector, 0 if scheme is unknown
void launch_dilute(const sq_ctx* c, const double* noise, int n_noise, int scheme, double* out, cudaStream_t s);

// ---- contraction (sq_contract.cu)
void launch_pion(const sq_ctx* c, const double* lex, int n, const int* tsl, double* C, cudaStream_t s);
int stoch_groups(const sq_ctx* c, int n);
int stoch_groups2(const sq_ctx* c, int ni, int nj);  // rectangular ni x nj pairs
void launch_stoch_op(const sq_ctx* c, const double* eta, const double* X, int n, double* O, double* C, double* part,
                     int nkg, cudaStream_t s);
// Tensor-core stochastic operators (sq_stoch_tc.cu): tile counts and the
// packed-operand workspace of a batch of Tb timeslices.
struct TcPlan {
  int T = 0, Tb = 0, nkt = 0, nch = 0, nit = 0, njt = 0;
  long long K = 0;
  size_t a_per_t = 0, b_per_t = 0, e_per_t = 0, bytes = 0;
};
TcPlan tc_plan(const sq_ctx* c, int n, size_t cap_bytes);
cudaError_t launch_stoch_tc(const sq_ctx* c, const TcPlan& p, const double* eta, const double* X, int n, double* O,
                            void* ws, int* err, cudaStream_t s);
void launch_stoch_corr(const sq_ctx* c, const double* O, int n, double* C, double* part, cudaStream_t s);
size_t corr_scratch_bytes(const sq_ctx* c, int n);
void launch_prop_trace(const sq_ctx* c, const double* etaA, const double* XA, const double* etaB, const double* XB,
                       int n, double* P, double* Q, double* C, double* part, int nkg, cudaStream_t s);
// diagram contractions (sq_contract.cu): scratch bytes and the launches
size_t diagram_scratch_bytes(const sq_ctx* c, int n);
void launch_diagrams(const sq_ctx* c, const double* Xp, const double* etaA, const double* XA, const double* etaB,
                     const double* XB, int n, double* out, void* scratch, cudaStream_t s);
void launch_diag_ensemble(const double* rec, int ncfg, int T, double* out, cudaStream_t s);

}  // namespace sq

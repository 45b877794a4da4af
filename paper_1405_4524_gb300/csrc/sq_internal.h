// Host-side internals of libstochq: the context, the solver workspace and
// the kernel launchers that the translation units share.
#pragma once

#include <cuda_runtime.h>

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
  uint4* Ainv16 = nullptr;    // [2][9][Vh]
  double a_bound = 1.0;       // max over sites of a Gershgorin bound on ||A||_2
  unsigned long long tick = 0;
};

// Dslash launch shape: sites per CTA (x) and sources per CTA (y).
struct Shape {
  int sx = 64, ry = 2;
};

struct Workspace {
  size_t bytes = 0;
  void* base = nullptr;
  int n_rhs = 0;
  int inner = -1;
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
  double* scal = nullptr;       // n_rhs * 4 doubles of scratch results
  int nblk_stride = 0;
  // cached graph of `chunk` iterations
  cudaGraphExec_t graph = nullptr;
  int graph_chunk = 0;
  int graph_key[8] = {0};
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
  uint2* U16 = nullptr;    // [2][4][3][Vh]
  // clover cache
  std::vector<sq::CloverSet> clover;
  int cur_clover = -1;
  unsigned long long tick = 0;
  // device error word
  int* d_err = nullptr;
  sq::Workspace ws;
  std::map<long long, sq::Shape> tuned;
  std::string last_error;
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
sq_status check_finite(sq_ctx* c, const double* dev, size_t n, int* bad);

// ---- spinor layout, BLAS, reductions (sq_blas.cu)
void launch_pack(const sq_ctx* c, Field out, const double* lex, int parity, int prec, int n, cudaStream_t s);
void launch_unpack(const sq_ctx* c, double* lex, Field in, int parity, int prec, int n, cudaStream_t s);
// out = c1 * x + c2 * (C in), C = A (which=0) or A^{-1} (which=1), FP64
void launch_clover64(const sq_ctx* c, const CloverSet& cs, Field out, Field x, Field in, int parity,
                     double c1, double c2, int which, int n, cudaStream_t s);
// per-source FP64 norms^2 of an eo field (any precision) -> out[k]
void launch_norm2(const sq_ctx* c, Field f, int prec, int n, double* out, RedArgs ra, cudaStream_t s);

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
};
void launch_dslash(const sq_ctx* c, const DslashCall& d, cudaStream_t s);
int dslash_nblk(const sq_ctx* c, Shape sh);
Shape tune_dslash(sq_ctx* c, DslashCall d, cudaStream_t s);

// ---- solver (sq_solver.cu)
sq_status solve_impl(sq_ctx* c, double kappa, double csw, const double* src, double* sol, int n,
                     double tol, const sq_solve_params* prm, sq_solve_stats* stats);

// ---- contraction (sq_contract.cu)
void launch_pion(const sq_ctx* c, const double* lex, int n, const int* tsl, double* C, cudaStream_t s);

}  // namespace sq

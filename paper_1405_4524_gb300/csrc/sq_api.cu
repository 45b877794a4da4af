// The extern "C" boundary of libstochq (declared in include/stochq.h):
// argument validation, context and stream handling, host <-> device
// staging, and dispatch to the kernels of the other translation units.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sq_internal.h"

namespace sq {

Geom geom_of(const sq_ctx* c) {
  Geom g;
  g.X = c->dims[0];
  g.Y = c->dims[1];
  g.Z = c->dims[2];
  g.T = c->dims[3];
  g.X2 = g.X / 2;
  g.Vh = c->Vh;
  g.tbc = (double)c->t_bc;
  return g;
}

sq_status set_error(sq_ctx* c, sq_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->last_error = buf;
  }
  return s;
}

sq_status cuda_check(sq_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SQ_OK;
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return set_error(c, SQ_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(c, SQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t field_bytes(int Vh, int prec, int n) {
  if (prec == P64) return (size_t)n * Vh * 192;
  if (prec == P32) return (size_t)n * Vh * 96;
  return (size_t)n * Vh * 52;  // 48 B of halves + 4 B norm
}

Field make_field(void* data, int Vh, int prec, int n) {
  Field f;
  f.data = data;
  f.Vh = Vh;
  f.norm = (prec == P16 && data) ? (float*)((uint4*)data + (size_t)n * 3 * Vh) : nullptr;
  return f;
}

sq_status enter_stream(sq_ctx* c) {
  cudaError_t e = cudaEventRecord(c->ev, c->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev, 0);
  return cuda_check(c, e, "stream ordering");
}

sq_status leave_stream(sq_ctx* c) {
  cudaError_t e = cudaEventRecord(c->ev, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->user_stream, c->ev, 0);
  return cuda_check(c, e, "stream ordering");
}

sq_status read_error_word(sq_ctx* c, int* bits) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  *bits = h;
  return cuda_check(c, e, "device error word");
}

cudaError_t dev_alloc(const Allocator& a, void** p, size_t bytes) {
  if (!a.alloc) return cudaMalloc(p, bytes);
  *p = a.alloc(bytes, (void*)a.stream, a.user);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void dev_free(const Allocator& a, void* p, size_t bytes) {
  if (!p) return;
  if (!a.free) {
    cudaFree(p);
    return;
  }
  cudaStreamSynchronize(a.stream);  // cudaFree would have waited too
  a.free(p, bytes, (void*)a.stream, a.user);
}

static size_t gauge32_bytes(const sq_ctx* c, int recon) {
  return recon == 12 ? 2 * 4 * 3 * (size_t)c->Vh * sizeof(float4) : 2 * 4 * 9 * (size_t)c->Vh * sizeof(float2);
}

static void free_clover(sq_ctx* c, CloverSet& cs) {
  const size_t Vh = c->Vh;
  dev_free(c->mem, cs.A64, 2 * 36 * Vh * sizeof(double2));
  dev_free(c->mem, cs.Ainv64, 2 * 36 * Vh * sizeof(double2));
  dev_free(c->mem, cs.Ainv32, 2 * 18 * Vh * sizeof(float4));
  dev_free(c->mem, cs.Adf, 2 * 36 * Vh * sizeof(float4));
  dev_free(c->mem, cs.Ainvdf, 2 * 36 * Vh * sizeof(float4));
  cs = CloverSet();
}

// Cached clover term for (kappa, c_sw); builds it if needed (LRU of 8).
// Buffers are reused in place (stable device addresses for captured graphs).
sq_status find_clover(sq_ctx* c, double kappa, double csw, CloverSet** out) {
  for (auto& cs : c->clover)
    if (cs.valid && cs.kappa == kappa && cs.csw == csw) {
      cs.tick = ++c->tick;
      *out = &cs;
      return SQ_OK;
    }
  if (!c->have_gauge) return set_error(c, SQ_ERR_STATE, "clover: no gauge field loaded");
  int slot = -1;
  for (size_t i = 0; i < c->clover.size(); i++)
    if (!c->clover[i].valid) { slot = (int)i; break; }
  if (slot < 0 && c->clover.size() < 8) {
    c->clover.reserve(8);
    c->clover.resize(c->clover.size() + 1);
    slot = (int)c->clover.size() - 1;
  }
  if (slot < 0) {
    slot = 0;
    for (size_t i = 1; i < c->clover.size(); i++)
      if (c->clover[i].tick < c->clover[slot].tick) slot = (int)i;
  }
  CloverSet& cs = c->clover[slot];
  cs.valid = 0;
  const size_t Vh = c->Vh;
  cudaError_t e = cudaSuccess;
  if (!cs.A64) e = dev_alloc(c->mem, (void**)&cs.A64, 2 * 36 * Vh * sizeof(double2));
  if (e == cudaSuccess && !cs.Ainv64) e = dev_alloc(c->mem, (void**)&cs.Ainv64, 2 * 36 * Vh * sizeof(double2));
  if (e == cudaSuccess && !cs.Ainv32) e = dev_alloc(c->mem, (void**)&cs.Ainv32, 2 * 18 * Vh * sizeof(float4));
  if (e == cudaSuccess && !cs.Adf) e = dev_alloc(c->mem, (void**)&cs.Adf, 2 * 36 * Vh * sizeof(float4));
  if (e == cudaSuccess && !cs.Ainvdf) e = dev_alloc(c->mem, (void**)&cs.Ainvdf, 2 * 36 * Vh * sizeof(float4));
  if (e != cudaSuccess) {
    free_clover(c, cs);
    return cuda_check(c, e, "clover allocation");
  }
  sq_status s = clover_build(c, cs, kappa, csw);
  c->launches += 2;
  // one read-back for the norm bound and the error word
  int bits = 0;
  unsigned long long hb = 0;
  if (s == SQ_OK) {
    e = cudaMemcpyAsync(&hb, c->d_bound, sizeof(hb), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    s = cuda_check(c, e, "clover build");
  }
  if (s == SQ_OK) memcpy(&cs.a_bound, &hb, sizeof(double));
  if (s == SQ_OK && (bits & ERRBIT_CLOVER))
    return set_error(c, SQ_ERR_CLOVER, "clover: a 6x6 block is singular for kappa=%g c_sw=%g", kappa, csw);
  if (s != SQ_OK) return s;
  cs.valid = 1;
  cs.tick = ++c->tick;
  *out = &cs;
  return SQ_OK;
}

}  // namespace sq

using namespace sq;

extern "C" {

void sq_default_params(sq_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->inner_prec = SQ_F32;
  p->outer = SQ_OUTER_RELIABLE;
  p->delta = 0.0;  // automatic per inner precision
  p->max_iter = 20000;
  p->recon = 12;
  p->chunk = 0;
  p->use_graph = 1;
  p->io = SQ_HOST;
  p->breakdown_tol = 1e-14;
  p->fallback = 1;
}

int sq_inner_sum_bits(void) { return (int)(8 * sizeof(sq::SumOf<float>::T)); }

const char* sq_status_string(sq_status s) {
  switch (s) {
    case SQ_OK: return "SQ_OK";
    case SQ_ERR_ARG: return "SQ_ERR_ARG: invalid argument";
    case SQ_ERR_CUDA: return "SQ_ERR_CUDA: CUDA runtime error";
    case SQ_ERR_OOM: return "SQ_ERR_OOM: out of device memory";
    case SQ_ERR_NONFINITE: return "SQ_ERR_NONFINITE: NaN or Inf in the input";
    case SQ_ERR_CLOVER: return "SQ_ERR_CLOVER: singular clover block";
    case SQ_ERR_NOCONV: return "SQ_ERR_NOCONV: not converged within max_iter";
    case SQ_ERR_BREAKDOWN: return "SQ_ERR_BREAKDOWN: BiCGStab breakdown";
    case SQ_ERR_TIMEOUT: return "SQ_ERR_TIMEOUT: device-side wait timed out";
    case SQ_ERR_STATE: return "SQ_ERR_STATE: call made in the wrong state";
  }
  return "unknown status";
}

const char* sq_last_error(const sq_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

sq_status sq_create(sq_ctx** out, const int dims[4], int t_bc, void* cuda_stream) {
  if (!out || !dims) return SQ_ERR_ARG;
  *out = nullptr;
  long long V = 1;
  for (int i = 0; i < 4; i++) {
    if (dims[i] < 2 || (dims[i] & 1)) return SQ_ERR_ARG;
    V *= dims[i];
  }
  if (V / 2 > (1LL << 30) / 36) return SQ_ERR_ARG;  // 32-bit site indices in every kernel
  if (t_bc != 1 && t_bc != -1) return SQ_ERR_ARG;
  sq_ctx* c = new sq_ctx();
  for (int i = 0; i < 4; i++) c->dims[i] = dims[i];
  c->V = (int)V;
  c->Vh = (int)(V / 2);
  c->t_bc = t_bc;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_err, 16);  // error word at 0, clover bound at 8
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 16);
  c->d_bound = (unsigned long long*)((char*)c->d_err + 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->d_err) cudaFree(c->d_err);
    delete c;
    return e == cudaErrorMemoryAllocation ? SQ_ERR_OOM : SQ_ERR_CUDA;
  }
  c->user_stream = (cudaStream_t)cuda_stream;
  c->mem.stream = c->stream;
  static std::atomic<unsigned long long> next_uid{1};
  c->uid = next_uid++;
  *out = c;
  return SQ_OK;
}

sq_status sq_set_allocator(sq_ctx* c, sq_alloc_fn alloc, sq_free_fn free_fn, void* user) {
  if (!c) return SQ_ERR_ARG;
  if ((!alloc) != (!free_fn)) return set_error(c, SQ_ERR_ARG, "sq_set_allocator: give both callbacks or neither");
  bool held = c->U64 || c->U32 || c->stoch_part || c->ws.base || c->batch;
  for (auto& cs : c->clover) held = held || cs.A64 || cs.Ainv64 || cs.Ainv32 || cs.Adf || cs.Ainvdf;
  held = held || c->Udf || c->cloverF || c->gstage;
  if (held) return set_error(c, SQ_ERR_STATE, "sq_set_allocator: the context already holds device buffers");
  c->mem.alloc = alloc;
  c->mem.free = free_fn;
  c->mem.user = user;
  return SQ_OK;
}

sq_status sq_destroy(sq_ctx* c) {
  if (!c) return SQ_OK;
  cudaStreamSynchronize(c->stream);
  release_workspace(c);
  for (auto& cs : c->clover) free_clover(c, cs);
  dev_free(c->mem, c->U64, 2 * 4 * 9 * (size_t)c->Vh * sizeof(double2));
  dev_free(c->mem, c->Udf, 2 * 4 * 9 * (size_t)c->Vh * sizeof(float4));
  dev_free(c->mem, c->U32, gauge32_bytes(c, c->recon));
  dev_free(c->mem, c->cloverF, clover_scratch_bytes(c));
  dev_free(c->mem, c->gstage, (size_t)c->V * 4 * 18 * sizeof(double));
  cudaFree(c->d_err);
  dev_free(c->mem, c->stoch_part, c->stoch_cap);
  cudaEventDestroy(c->ev);
  cudaStreamDestroy(c->stream);
  delete c;
  return SQ_OK;
}

sq_status sq_load_gauge(sq_ctx* c, const double* U, int recon, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!U) return set_error(c, SQ_ERR_ARG, "sq_load_gauge: null U");
  if (recon != 12 && recon != 18) return set_error(c, SQ_ERR_ARG, "sq_load_gauge: recon must be 12 or 18");
  if (where != SQ_HOST && where != SQ_DEVICE) return set_error(c, SQ_ERR_ARG, "sq_load_gauge: bad where");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const size_t Vh = c->Vh;
  // keep the device buffers (stable addresses); cached clover terms go stale
  for (auto& cs : c->clover) cs.valid = 0;
  c->have_gauge = 0;
  cudaError_t e = cudaSuccess;
  if (c->U32 && recon != c->recon) {
    dev_free(c->mem, c->U32, gauge32_bytes(c, c->recon));
    c->U32 = nullptr;
  }
  c->recon = recon;
  if (!c->U64) e = dev_alloc(c->mem, (void**)&c->U64, 2 * 4 * 9 * Vh * sizeof(double2));
  if (e == cudaSuccess && !c->U32) e = dev_alloc(c->mem, &c->U32, gauge32_bytes(c, recon));
  if (e == cudaSuccess && !c->Udf) e = dev_alloc(c->mem, (void**)&c->Udf, 2 * 4 * 9 * Vh * sizeof(float4));
  if (e != cudaSuccess) return cuda_check(c, e, "gauge allocation");
  const size_t nd = (size_t)c->V * 4 * 18;
  const double* dU = U;
  double* stage = nullptr;
  if (where == SQ_HOST) {  // staging buffer kept by the context (no allocation per load)
    if (!c->gstage) {
      e = dev_alloc(c->mem, (void**)&c->gstage, nd * sizeof(double));
      if (e != cudaSuccess) {
        c->gstage = nullptr;
        return cuda_check(c, e, "gauge staging");
      }
    }
    stage = c->gstage;
    cudaMemcpyAsync(stage, U, nd * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    dU = stage;
  }
  s = gauge_convert(c, dU);
  c->launches += 1;
  int bits = 0;
  if (s == SQ_OK) s = read_error_word(c, &bits);
  if (s != SQ_OK) return s;
  if (bits & ERRBIT_NONFINITE) return set_error(c, SQ_ERR_NONFINITE, "sq_load_gauge: NaN or Inf in U");
  c->su3 = !(bits & ERRBIT_NOT_SU3);
  if (!c->su3 && recon == 12)
    return set_error(c, SQ_ERR_ARG, "sq_load_gauge: links are not SU(3); reconstruct-12 needs SU(3) (use 18)");
  c->have_gauge = 1;
  return leave_stream(c);
}

sq_status sq_build_clover(sq_ctx* c, double kappa, double csw) {
  if (!c) return SQ_ERR_ARG;
  if (!std::isfinite(kappa) || !std::isfinite(csw))
    return set_error(c, SQ_ERR_ARG, "sq_build_clover: non-finite kappa or c_sw");
  if (!c->have_gauge) return set_error(c, SQ_ERR_STATE, "sq_build_clover: no gauge field loaded");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  CloverSet* cs = nullptr;
  s = find_clover(c, kappa, csw, &cs);
  if (s != SQ_OK) return s;
  c->cur_clover = (int)(cs - c->clover.data());
  return leave_stream(c);
}

sq_status sq_field_bytes(const sq_ctx* c, sq_prec prec, int n, size_t* bytes) {
  if (!c || !bytes || n < 0 || prec < SQ_F64 || prec > SQ_F16) return SQ_ERR_ARG;
  *bytes = field_bytes(c->Vh, prec, n);
  return SQ_OK;
}

static sq_status stage_in(sq_ctx* c, const double* lex, int n, int where, const double** dev, double** tmp) {
  *tmp = nullptr;
  *dev = lex;
  if (where == SQ_DEVICE) return SQ_OK;
  const size_t b = (size_t)n * c->V * 24 * sizeof(double);
  cudaError_t e = cudaMallocAsync((void**)tmp, b, c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "staging buffer");
  e = cudaMemcpyAsync(*tmp, lex, b, cudaMemcpyHostToDevice, c->stream);
  *dev = *tmp;
  return cuda_check(c, e, "host to device copy");
}

sq_status sq_pack_spinor(sq_ctx* c, void* eo_out, const double* lex_in, int parity, sq_prec prec, int n,
                         int where) {
  if (!c) return SQ_ERR_ARG;
  if (!eo_out || !lex_in || n <= 0 || (parity != 0 && parity != 1) || prec < SQ_F64 || prec > SQ_F16 ||
      (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_pack_spinor: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const double* dev;
  double* tmp;
  s = stage_in(c, lex_in, n, where, &dev, &tmp);
  if (s != SQ_OK) return s;
  launch_pack(c, make_field(eo_out, c->Vh, prec, n), dev, parity, prec, n, c->stream);
  if (tmp) cudaFreeAsync(tmp, c->stream);
  cudaError_t e = where == SQ_HOST ? cudaStreamSynchronize(c->stream) : cudaGetLastError();
  s = cuda_check(c, e, "sq_pack_spinor");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_unpack_spinor(sq_ctx* c, double* lex_out, const void* eo_in, int parity, sq_prec prec, int n,
                           int where) {
  if (!c) return SQ_ERR_ARG;
  if (!eo_in || !lex_out || n <= 0 || (parity != 0 && parity != 1) || prec < SQ_F64 || prec > SQ_F16 ||
      (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_unpack_spinor: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const size_t b = (size_t)n * c->V * 24 * sizeof(double);
  double* dev = lex_out;
  if (where == SQ_HOST) {
    cudaError_t e = cudaMallocAsync((void**)&dev, b, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "staging buffer");
    // the other parity's sites must come back unchanged
    cudaMemcpyAsync(dev, lex_out, b, cudaMemcpyHostToDevice, c->stream);
  }
  launch_unpack(c, dev, make_field((void*)eo_in, c->Vh, prec, n), parity, prec, n, c->stream);
  cudaError_t e = cudaGetLastError();
  if (where == SQ_HOST) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(lex_out, dev, b, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(dev, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  s = cuda_check(c, e, "sq_unpack_spinor");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_dslash_eo(sq_ctx* c, void* out, const void* in, const void* x, int out_parity, sq_prec prec, int n,
                       int flags, double a) {
  if (!c) return SQ_ERR_ARG;
  if (!out || !in || n <= 0 || (out_parity != 0 && out_parity != 1) || prec < SQ_F64 || prec > SQ_F16)
    return set_error(c, SQ_ERR_ARG, "sq_dslash_eo: bad argument");
  if ((flags & SQ_DS_XPAY) && !x) return set_error(c, SQ_ERR_ARG, "sq_dslash_eo: XPAY needs x");
  if (out == in) return set_error(c, SQ_ERR_ARG, "sq_dslash_eo: in must not alias out");
  if (!c->have_gauge) return set_error(c, SQ_ERR_STATE, "sq_dslash_eo: no gauge field loaded");
  const CloverSet* cs = nullptr;
  if (flags & SQ_DS_CLOVER_INV) {
    if (c->cur_clover < 0 || c->cur_clover >= (int)c->clover.size() || !c->clover[c->cur_clover].valid)
      return set_error(c, SQ_ERR_STATE, "sq_dslash_eo: no clover term built");
    cs = &c->clover[c->cur_clover];
  }
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  DslashCall d;
  memset(&d, 0, sizeof(d));
  d.out = make_field(out, c->Vh, prec, n);
  d.in = make_field((void*)in, c->Vh, prec, n);
  d.x = make_field((void*)x, c->Vh, prec, n);
  d.p_out = out_parity;
  d.prec = prec;
  d.recon = prec == SQ_F64 ? 18 : c->recon;  // FP16 fields use the FP32 links
  d.clover = (flags & SQ_DS_CLOVER_INV) ? 1 : 0;
  d.xpay = (flags & SQ_DS_XPAY) ? 1 : 0;
  d.emul = (prec == SQ_F64 && (flags & SQ_DS_F64_EMULATED)) ? 1 : 0;
  d.a = a;
  d.cs = cs;
  d.n = n;
  d.fin = FIN_NONE;
  {
    // autotuned shape, tuned once per (precision, recon, n) into scratch
    // output so that an in-place xpay (x == out) is never applied twice
    void* scratch = nullptr;
    long long key = ((long long)d.prec << 56) ^ ((long long)d.recon << 48) ^ ((long long)c->Vh << 12) ^ n;
    if (!d.emul && c->tuned.find(key) == c->tuned.end()) {
      cudaError_t e = cudaMallocAsync(&scratch, field_bytes(c->Vh, prec, n), c->stream);
      if (e != cudaSuccess) return cuda_check(c, e, "sq_dslash_eo tuning buffer");
      DslashCall t = d;
      t.out = make_field(scratch, c->Vh, prec, n);
      tune_dslash(c, t, c->stream);
      cudaFreeAsync(scratch, c->stream);
    }
    if (!d.emul) d.shape = tune_dslash(c, d, c->stream);  // the emulated kernel has one shape
  }
  launch_dslash(c, d, c->stream);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && (flags & SQ_DS_SYNC)) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_dslash_eo");
  if (s != SQ_OK) return s;
  if (flags & SQ_DS_SYNC) {
    int bits = 0;
    s = read_error_word(c, &bits);
    if (s != SQ_OK) return s;
    if (bits & ERRBIT_TIMEOUT) {
      leave_stream(c);
      return set_error(c, SQ_ERR_TIMEOUT, "sq_dslash_eo: a bounded wait on the staged spinors ran out");
    }
  }
  return leave_stream(c);
}

static long long shape_key(const sq_ctx* c, int prec, int n) {
  const int recon = prec == SQ_F64 ? 18 : c->recon;
  return ((long long)prec << 56) ^ ((long long)recon << 48) ^ ((long long)c->Vh << 12) ^ n;
}

sq_status sq_set_dslash_shape(sq_ctx* c, sq_prec prec, int n, int kind, const int shape[5]) {
  if (!c) return SQ_ERR_ARG;
  if (!shape || n <= 0 || prec < SQ_F64 || prec > SQ_F16 || (kind != 0 && kind != 1))
    return set_error(c, SQ_ERR_ARG, "sq_set_dslash_shape: bad argument");
  Shape sh;
  sh.kind = kind;
  if (kind == 0) {
    if (shape[0] <= 0 || shape[0] % 32 || shape[1] <= 0 || shape[0] * shape[1] > 256 ||
        (shape[2] != 0 && shape[2] != 1))
      return set_error(c, SQ_ERR_ARG, "sq_set_dslash_shape: bad per-site CTA shape");
    sh.sx = shape[0];
    sh.ry = shape[1];
    sh.order = shape[2];
  } else {
    sh.by = shape[0];
    sh.bz = shape[1];
    sh.bt = shape[2];
    sh.sg = shape[3];
    sh.nbuf = shape[4];
    const int recon = prec == SQ_F64 ? 18 : c->recon;
    if (!tile_shape_ok(c, prec, recon, sh))
      return set_error(c, SQ_ERR_ARG, "sq_set_dslash_shape: the tiled shape does not apply to this lattice");
  }
  c->tuned[shape_key(c, prec, n)] = sh;
  c->tuned_meta[shape_key(c, prec, n)] = {(int)prec, prec == SQ_F64 ? 18 : c->recon, n};
  return SQ_OK;
}

static std::string gpu_name(const sq_ctx* c) {
  cudaDeviceProp pr;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&pr, c->device) == cudaSuccess) name = pr.name;
  for (auto& ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  return name;
}

sq_status sq_tune_save(const sq_ctx* c, const char* path) {
  if (!c) return SQ_ERR_ARG;
  sq_ctx* cm = const_cast<sq_ctx*>(c);
  if (!path) return set_error(cm, SQ_ERR_ARG, "sq_tune_save: null path");
  FILE* f = fopen(path, "a");
  if (!f) return set_error(cm, SQ_ERR_STATE, "sq_tune_save: cannot open %s", path);
  const std::string g = gpu_name(c);
  for (const auto& kv : c->tuned) {
    auto m = c->tuned_meta.find(kv.first);
    if (m == c->tuned_meta.end()) continue;
    const Shape& sh = kv.second;
    fprintf(f, "stochq-shape %s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", g.c_str(), c->dims[0], c->dims[1],
            c->dims[2], c->dims[3], m->second[0], m->second[1], m->second[2], sh.kind, sh.sx, sh.ry, sh.order, sh.by,
            sh.bz, sh.bt, sh.sg, sh.nbuf);
  }
  const bool ok = fclose(f) == 0;
  return ok ? SQ_OK : set_error(cm, SQ_ERR_STATE, "sq_tune_save: cannot write %s", path);
}

sq_status sq_tune_load(sq_ctx* c, const char* path, int* n_loaded) {
  if (!c) return SQ_ERR_ARG;
  if (!path) return set_error(c, SQ_ERR_ARG, "sq_tune_load: null path");
  if (n_loaded) *n_loaded = 0;
  FILE* f = fopen(path, "r");
  if (!f) return set_error(c, SQ_ERR_STATE, "sq_tune_load: cannot open %s", path);
  const std::string g = gpu_name(c);
  char line[512], name[256];
  int cnt = 0;
  while (fgets(line, sizeof(line), f)) {
    int d[4], prec, recon, n, kind, sx, ry, order, by, bz, bt, sg, nbuf;
    if (sscanf(line, "stochq-shape %255s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d", name, &d[0], &d[1], &d[2],
               &d[3], &prec, &recon, &n, &kind, &sx, &ry, &order, &by, &bz, &bt, &sg, &nbuf) != 17)
      continue;
    if (g != name || d[0] != c->dims[0] || d[1] != c->dims[1] || d[2] != c->dims[2] || d[3] != c->dims[3]) continue;
    if (prec < SQ_F64 || prec > SQ_F16 || n <= 0 || recon != (prec == SQ_F64 ? 18 : c->recon)) continue;
    Shape sh;
    sh.kind = kind;
    sh.sx = sx;
    sh.ry = ry;
    sh.order = order;
    sh.by = by;
    sh.bz = bz;
    sh.bt = bt;
    sh.sg = sg;
    sh.nbuf = nbuf;
    if (kind == 1 && !tile_shape_ok(c, prec, recon, sh)) continue;
    if (kind == 0 && (sx <= 0 || sx % 32 || ry <= 0 || sx * ry > 256 || (order != 0 && order != 1))) continue;
    if (kind != 0 && kind != 1) continue;
    const long long key = shape_key(c, prec, n);
    c->tuned[key] = sh;
    c->tuned_meta[key] = {prec, recon, n};
    cnt++;
  }
  fclose(f);
  if (n_loaded) *n_loaded = cnt;
  return SQ_OK;
}

sq_status sq_get_dslash_shape(const sq_ctx* c, sq_prec prec, int n, int* kind, int shape[5]) {
  if (!c) return SQ_ERR_ARG;
  if (!kind || !shape || n <= 0 || prec < SQ_F64 || prec > SQ_F16)
    return set_error(const_cast<sq_ctx*>(c), SQ_ERR_ARG, "sq_get_dslash_shape: bad argument");
  auto it = c->tuned.find(shape_key(c, prec, n));
  if (it == c->tuned.end())
    return set_error(const_cast<sq_ctx*>(c), SQ_ERR_STATE, "sq_get_dslash_shape: no shape chosen yet");
  const Shape& sh = it->second;
  *kind = sh.kind;
  if (sh.kind == 0) {
    const int v[5] = {sh.sx, sh.ry, sh.order, 0, 0};
    for (int i = 0; i < 5; i++) shape[i] = v[i];
  } else {
    const int v[5] = {sh.by, sh.bz, sh.bt, sh.sg, sh.nbuf};
    for (int i = 0; i < 5; i++) shape[i] = v[i];
  }
  return SQ_OK;
}

sq_status sq_set_wait_cycles(sq_ctx* c, long long cycles, int stall_test) {
  if (!c) return SQ_ERR_ARG;
  if (cycles < 0 || (stall_test != 0 && stall_test != 1))
    return set_error(c, SQ_ERR_ARG, "sq_set_wait_cycles: bad argument");
  c->wait_cycles = cycles;
  c->wait_stall = stall_test;
  return SQ_OK;
}

sq_status sq_norm2_eo(sq_ctx* c, const void* field, sq_prec prec, int n, double* out, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!field || !out || n <= 0 || prec < SQ_F64 || prec > SQ_F16 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_norm2_eo: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const int nblk = (c->Vh + 127) / 128;
  const size_t b_part = (size_t)n * nblk * sizeof(double), b_cnt = (size_t)n * sizeof(unsigned);
  const size_t b_out = (size_t)n * sizeof(double);
  char* scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&scratch, b_part + b_cnt + b_out + 512, c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "sq_norm2_eo scratch");
  RedArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.partial = (double*)scratch;
  ra.counter = (unsigned*)(scratch + ((b_part + 255) & ~(size_t)255));
  double* dout = (double*)(scratch + ((b_part + 255) & ~(size_t)255) + ((b_cnt + 255) & ~(size_t)255));
  ra.nblk_stride = nblk;
  cudaMemsetAsync(ra.counter, 0, b_cnt, c->stream);
  launch_norm2(c, make_field((void*)field, c->Vh, prec, n), prec, n, dout, ra, c->stream);
  c->launches += 1;
  e = cudaMemcpyAsync(out, dout, b_out, where == SQ_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                      c->stream);
  cudaFreeAsync(scratch, c->stream);
  if (e == cudaSuccess && where == SQ_HOST) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_norm2_eo");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_apply_M(sq_ctx* c, double* out, const double* in, int n, double kappa, double csw, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!out || !in || n <= 0 || (where != SQ_HOST && where != SQ_DEVICE) || !std::isfinite(kappa) ||
      !std::isfinite(csw))
    return set_error(c, SQ_ERR_ARG, "sq_apply_M: bad argument");
  if (!c->have_gauge) return set_error(c, SQ_ERR_STATE, "sq_apply_M: no gauge field loaded");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  CloverSet* cs = nullptr;
  s = find_clover(c, kappa, csw, &cs);
  if (s != SQ_OK) return s;
  const double* dev;
  double* tmp;
  s = stage_in(c, in, n, where, &dev, &tmp);
  if (s != SQ_OK) return s;
  const size_t fb = field_bytes(c->Vh, P64, n);
  char* f = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&f, 4 * fb, c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "sq_apply_M buffers");
  Field ie = make_field(f, c->Vh, P64, n), io = make_field(f + fb, c->Vh, P64, n);
  Field oe = make_field(f + 2 * fb, c->Vh, P64, n), oo = make_field(f + 3 * fb, c->Vh, P64, n);
  Field none = make_field(nullptr, c->Vh, P64, n);
  launch_pack(c, ie, dev, 0, P64, n, c->stream);
  launch_pack(c, io, dev, 1, P64, n, c->stream);
  // out_p = A_pp in_p - kappa D_{p,1-p} in_{1-p}
  launch_clover64(c, *cs, oe, none, ie, 0, 0.0, 1.0, 0, n, c->stream);
  launch_clover64(c, *cs, oo, none, io, 1, 0.0, 1.0, 0, n, c->stream);
  DslashCall d;
  memset(&d, 0, sizeof(d));
  d.prec = P64;
  d.recon = 18;
  d.xpay = 1;
  d.a = -kappa;
  d.n = n;
  d.shape.sx = 64;
  d.shape.ry = 1;
  d.out = oe; d.in = io; d.x = oe; d.p_out = 0;
  launch_dslash(c, d, c->stream);
  d.out = oo; d.in = ie; d.x = oo; d.p_out = 1;
  launch_dslash(c, d, c->stream);
  double* dout = out;
  double* otmp = nullptr;
  const size_t lb = (size_t)n * c->V * 24 * sizeof(double);
  if (where == SQ_HOST) {
    e = cudaMallocAsync((void**)&otmp, lb, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "sq_apply_M output staging");
    dout = otmp;
  }
  launch_unpack(c, dout, oe, 0, P64, n, c->stream);
  launch_unpack(c, dout, oo, 1, P64, n, c->stream);
  if (where == SQ_HOST) cudaMemcpyAsync(out, otmp, lb, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(f, c->stream);
  if (tmp) cudaFreeAsync(tmp, c->stream);
  if (otmp) cudaFreeAsync(otmp, c->stream);
  e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_apply_M");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_solve(sq_ctx* c, double kappa, double csw, const double* sources, double* solutions, int n,
                   double tol, const sq_solve_params* params, sq_solve_stats* stats) {
  if (!c) return SQ_ERR_ARG;
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  s = solve_impl(c, kappa, csw, sources, solutions, n, tol, params, stats);
  sq_status s2 = leave_stream(c);
  return s != SQ_OK ? s : s2;
}

sq_status sq_dilute(sq_ctx* c, const double* noise, int n_noise, int scheme, double* out, int where) {
  if (!c) return SQ_ERR_ARG;
  const int D = dilution_count(c, scheme);
  if (!noise || !out || n_noise <= 0 || D == 0 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_dilute: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const double* dev;
  double* tmp;
  s = stage_in(c, noise, n_noise, where, &dev, &tmp);
  if (s != SQ_OK) return s;
  const size_t ob = (size_t)n_noise * D * c->V * 24 * sizeof(double);
  double* dout = out;
  cudaError_t e = cudaSuccess;
  if (where == SQ_HOST) e = cudaMallocAsync((void**)&dout, ob, c->stream);
  if (e == cudaSuccess) {
    launch_dilute(c, dev, n_noise, scheme, dout, c->stream);
    c->launches += 1;
    e = cudaGetLastError();
  }
  if (where == SQ_HOST) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, ob, cudaMemcpyDeviceToHost, c->stream);
    if (dout && dout != out) cudaFreeAsync(dout, c->stream);
  }
  if (tmp) cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess && where == SQ_HOST) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_dilute");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_contract_pion(sq_ctx* c, const double* sol, int n, const int* tsl, double* C, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!sol || !C || n <= 0 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_contract_pion: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const double* dev;
  double* tmp;
  s = stage_in(c, sol, n, where, &dev, &tmp);
  if (s != SQ_OK) return s;
  const int T = c->dims[3];
  double* dC = nullptr;
  int* dt = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dC, (size_t)n * T * sizeof(double), c->stream);
  if (e == cudaSuccess && tsl) {
    e = cudaMallocAsync((void**)&dt, n * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tsl, n * sizeof(int), cudaMemcpyHostToDevice, c->stream);
  }
  if (e != cudaSuccess) return cuda_check(c, e, "sq_contract_pion buffers");
  launch_pion(c, dev, n, dt, dC, c->stream);
  c->launches += 1;
  e = cudaMemcpyAsync(C, dC, (size_t)n * T * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(dC, c->stream);
  if (dt) cudaFreeAsync(dt, c->stream);
  if (tmp) cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_contract_pion");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

// Scratch of the pair contractions (K-group partials and operator
// matrices), kept in the context between calls and grown on demand.
static sq_status grow_contract_scratch(sq_ctx* c, size_t bytes) {
  if (c->stoch_cap >= bytes) return SQ_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) {
    dev_free(c->mem, c->stoch_part, c->stoch_cap);
    c->stoch_part = nullptr;
    c->stoch_cap = 0;
    e = dev_alloc(c->mem, &c->stoch_part, bytes);
    if (e == cudaSuccess) c->stoch_cap = bytes;
  }
  return cuda_check(c, e, "contraction scratch");
}

sq_status sq_contract_stoch_op(sq_ctx* c, const double* eta, const double* X, int n, double* O, double* C,
                               int where) {
  if (!c) return SQ_ERR_ARG;
  if (!eta || !X || !O || n <= 0 || n > 4080 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_contract_stoch_op: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const int T = c->dims[3];
  const int nkg = stoch_groups(c, n);
  const size_t ob = (size_t)T * n * n * 2 * sizeof(double), cb = (size_t)T * 2 * sizeof(double);
  s = grow_contract_scratch(c, std::max(ob * nkg, corr_scratch_bytes(c, n)));
  if (s != SQ_OK) return s;
  cudaError_t e = cudaSuccess;
  const double *deta, *dX;
  double *teta, *tX = nullptr;
  s = stage_in(c, eta, n, where, &deta, &teta);
  if (s == SQ_OK) s = stage_in(c, X, n, where, &dX, &tX);
  if (s != SQ_OK) {
    if (teta) cudaFreeAsync(teta, c->stream);
    return s;
  }
  double *dO = O, *dC = C;
  if (where == SQ_HOST) {
    e = cudaMallocAsync((void**)&dO, ob, c->stream);
    if (e == cudaSuccess && C) e = cudaMallocAsync((void**)&dC, cb, c->stream);
  }
  if (e == cudaSuccess) {
    launch_stoch_op(c, deta, dX, n, dO, dC, (double*)c->stoch_part, nkg, c->stream);
    c->launches += C ? 4 : 2;
    e = cudaGetLastError();
  }
  if (where == SQ_HOST) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(O, dO, ob, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, dC, cb, cudaMemcpyDeviceToHost, c->stream);
    if (dO && dO != O) cudaFreeAsync(dO, c->stream);
    if (C && dC && dC != C) cudaFreeAsync(dC, c->stream);
    if (teta) cudaFreeAsync(teta, c->stream);
    if (tX) cudaFreeAsync(tX, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  s = cuda_check(c, e, "sq_contract_stoch_op");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_contract_stoch_op_z4(sq_ctx* c, const double* eta, const double* X, int n, double* O, double* C,
                                  int where) {
  if (!c) return SQ_ERR_ARG;
  if (!eta || !X || !O || n <= 0 || n > 4080 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_contract_stoch_op_z4: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const TcPlan p = tc_plan(c, n, (size_t)8 << 30);
  const int T = c->dims[3];
  s = grow_contract_scratch(c, p.bytes + corr_scratch_bytes(c, n));
  if (s != SQ_OK) return s;
  const size_t ob = (size_t)T * n * n * 2 * sizeof(double), cb = (size_t)T * 2 * sizeof(double);
  const double *deta, *dX;
  double *teta, *tX = nullptr;
  s = stage_in(c, eta, n, where, &deta, &teta);
  if (s == SQ_OK) s = stage_in(c, X, n, where, &dX, &tX);
  if (s != SQ_OK) {
    if (teta) cudaFreeAsync(teta, c->stream);
    return s;
  }
  double *dO = O, *dC = C;
  cudaError_t e = cudaSuccess;
  if (where == SQ_HOST) {
    e = cudaMallocAsync((void**)&dO, ob, c->stream);
    if (e == cudaSuccess && C) e = cudaMallocAsync((void**)&dC, cb, c->stream);
  }
  int* flag = reinterpret_cast<int*>(static_cast<char*>(c->stoch_part) + p.bytes - 256);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = launch_stoch_tc(c, p, deta, dX, n, dO, c->stoch_part, c->d_err, c->stream);
  if (e == cudaSuccess) {
    c->launches += 3LL * ((T + p.Tb - 1) / p.Tb);
    if (C) {
      launch_stoch_corr(c, dO, n, dC, reinterpret_cast<double*>(static_cast<char*>(c->stoch_part) + p.bytes),
                        c->stream);
      c->launches += 2;
      e = cudaGetLastError();
    }
  }
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (where == SQ_HOST) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(O, dO, ob, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, dC, cb, cudaMemcpyDeviceToHost, c->stream);
    if (dO && dO != O) cudaFreeAsync(dO, c->stream);
    if (C && dC && dC != C) cudaFreeAsync(dC, c->stream);
  }
  if (teta) cudaFreeAsync(teta, c->stream);
  if (tX) cudaFreeAsync(tX, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_contract_stoch_op_z4");
  if (s != SQ_OK) return s;
  int bits = 0;
  s = read_error_word(c, &bits);
  if (s != SQ_OK) return s;
  if (bits & ERRBIT_TIMEOUT) return set_error(c, SQ_ERR_TIMEOUT, "sq_contract_stoch_op_z4: a tensor-core wait timed out");
  if (hflag & 1) return set_error(c, SQ_ERR_ARG, "sq_contract_stoch_op_z4: a source component is not 0 or +-1");
  if (hflag & 2) return set_error(c, SQ_ERR_NONFINITE, "sq_contract_stoch_op_z4: X is not finite");
  return leave_stream(c);
}

sq_status sq_contract_prop_trace(sq_ctx* c, const double* etaA, const double* XA, const double* etaB,
                                 const double* XB, int n, double* C, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!etaA || !XA || !C || n <= 0 || n > 4080 || (!etaB) != (!XB) || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_contract_prop_trace: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const int T = c->dims[3];
  const int nkg = stoch_groups(c, n);
  const size_t ob = (size_t)T * n * n * 2 * sizeof(double), cb = (size_t)T * T * 2 * sizeof(double);
  s = grow_contract_scratch(c, ob * (nkg + 2));
  if (s != SQ_OK) return s;
  double* part = (double*)c->stoch_part;
  double* P = part + (size_t)T * n * n * 2 * nkg;
  double* Q = P + (size_t)T * n * n * 2;
  const double* in[4] = {etaA, XA, etaB ? etaB : etaA, XB ? XB : XA};
  const double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
  double* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  const int nin = etaB ? 4 : 2;
  for (int k = 0; k < nin && s == SQ_OK; k++) s = stage_in(c, in[k], n, where, &dev[k], &tmp[k]);
  if (nin == 2) {
    dev[2] = dev[0];
    dev[3] = dev[1];
  }
  cudaError_t e = cudaSuccess;
  double* dC = C;
  if (s == SQ_OK && where == SQ_HOST) e = cudaMallocAsync((void**)&dC, cb, c->stream);
  if (s == SQ_OK && e == cudaSuccess) {
    launch_prop_trace(c, dev[0], dev[1], dev[2], dev[3], n, P, Q, dC, part, nkg, c->stream);
    c->launches += 5;
    e = cudaGetLastError();
    if (e == cudaSuccess && where == SQ_HOST) e = cudaMemcpyAsync(C, dC, cb, cudaMemcpyDeviceToHost, c->stream);
  }
  if (where == SQ_HOST && dC && dC != C) cudaFreeAsync(dC, c->stream);
  for (int k = 0; k < 4; k++)
    if (tmp[k]) cudaFreeAsync(tmp[k], c->stream);
  if (s != SQ_OK) return s;
  if (e == cudaSuccess && where == SQ_HOST) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_contract_prop_trace");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_contract_diagrams(sq_ctx* c, const double* Xp, const double* etaA, const double* XA,
                               const double* etaB, const double* XB, int n, double* out, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!Xp || !etaA || !XA || !out || n <= 0 || n > 4080 || (!etaB) != (!XB) ||
      (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_contract_diagrams: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const int T = c->dims[3];
  s = grow_contract_scratch(c, diagram_scratch_bytes(c, n));
  if (s != SQ_OK) return s;
  const double* in[5] = {Xp, etaA, XA, etaB ? etaB : etaA, XB ? XB : XA};
  const int cnt[5] = {12, n, n, n, n};
  const double* dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const int nin = etaB ? 5 : 3;
  for (int k = 0; k < nin && s == SQ_OK; k++) s = stage_in(c, in[k], cnt[k], where, &dev[k], &tmp[k]);
  if (nin == 3) {
    dev[3] = dev[1];
    dev[4] = dev[2];
  }
  const size_t ob = (size_t)7 * T * 2 * sizeof(double);
  cudaError_t e = cudaSuccess;
  double* dout = out;
  if (s == SQ_OK && where == SQ_HOST) e = cudaMallocAsync((void**)&dout, ob, c->stream);
  if (s == SQ_OK && e == cudaSuccess) {
    launch_diagrams(c, dev[0], dev[1], dev[2], dev[3], dev[4], n, dout, c->stoch_part, c->stream);
    c->launches += 11;
    e = cudaGetLastError();
    if (e == cudaSuccess && where == SQ_HOST) e = cudaMemcpyAsync(out, dout, ob, cudaMemcpyDeviceToHost, c->stream);
  }
  if (where == SQ_HOST && dout && dout != out) cudaFreeAsync(dout, c->stream);
  for (int k = 0; k < 5; k++)
    if (tmp[k]) cudaFreeAsync(tmp[k], c->stream);
  if (s != SQ_OK) return s;
  if (e == cudaSuccess && where == SQ_HOST) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_contract_diagrams");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_diagrams_ensemble(sq_ctx* c, const double* rec, int ncfg, double* out, int where) {
  if (!c) return SQ_ERR_ARG;
  if (!rec || !out || ncfg <= 0 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_diagrams_ensemble: bad argument");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  const int T = c->dims[3];
  const size_t rb = (size_t)ncfg * 7 * T * 2 * sizeof(double), ob = (size_t)5 * T * 2 * sizeof(double);
  const double* drec = rec;
  double* dout = out;
  char* tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (where == SQ_HOST) {
    e = cudaMallocAsync((void**)&tmp, rb + ob + 256, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, rec, rb, cudaMemcpyHostToDevice, c->stream);
    drec = (const double*)tmp;
    dout = (double*)(tmp + ((rb + 255) & ~(size_t)255));
  }
  if (e == cudaSuccess) {
    launch_diag_ensemble(drec, ncfg, T, dout, c->stream);
    c->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && where == SQ_HOST) e = cudaMemcpyAsync(out, dout, ob, cudaMemcpyDeviceToHost, c->stream);
  if (tmp) cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess && where == SQ_HOST) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_diagrams_ensemble");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

sq_status sq_get_profile(const sq_ctx* c, sq_kernel_stat* out, int max, int* n) {
  static const char* names[KC_N] = {
      "dslash_clover",         "dslash_clover_xpay_alpha", "blas_s_update",
      "dslash_clover",         "dslash_clover_xpay_omega", "blas_xr_update_norms",
      "blas_p_update",         "plan_updates",             "fp32_refresh",
      "fp64_update_x",
      "fp64_dslash_clover",    "fp64_dslash_xpay_norm",    "fp64_update_r",
      "control"};
  if (!c || !n || max < 0) return SQ_ERR_ARG;
  if (!c->prof_valid) return SQ_ERR_STATE;
  *n = KC_N;
  if (!out) return SQ_OK;
  for (int k = 0; k < KC_N && k < max; k++) {
    memset(&out[k], 0, sizeof(out[k]));
    snprintf(out[k].name, sizeof(out[k].name), "%s", names[k]);
    out[k].launches = c->prof[k].launches;
    out[k].ms = c->prof[k].ms;
    out[k].bytes = c->prof[k].bytes;
    out[k].flops = c->prof[k].flops;
  }
  return SQ_OK;
}

sq_status sq_kernel_launches(const sq_ctx* c, long long* n) {
  if (!c || !n) return SQ_ERR_ARG;
  *n = c->launches;
  return SQ_OK;
}

sq_status sq_solve_batch(const sq_problem* probs, int n_probs, const sq_solve_params* params,
                         sq_solve_stats* stats) {
  if (!probs || n_probs <= 0) return SQ_ERR_ARG;
  std::vector<sq_ctx*> ctxs;
  for (int i = 0; i < n_probs; i++) {
    if (!probs[i].ctx) return SQ_ERR_ARG;
    bool seen = false;
    for (auto* c : ctxs) seen = seen || c == probs[i].ctx;
    if (!seen) ctxs.push_back(probs[i].ctx);
  }
  for (auto* c : ctxs) {
    sq_status s = enter_stream(c);
    if (s != SQ_OK) return s;
  }
  sq_status s = solve_batch_impl(probs, n_probs, params, stats);
  for (auto* c : ctxs) {
    sq_status s2 = leave_stream(c);
    if (s == SQ_OK) s = s2;
  }
  return s;
}

}  // extern "C"

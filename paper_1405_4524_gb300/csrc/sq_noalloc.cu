// sq_norm2_eo_noalloc: per-source squared norms of a device even-odd field
// without any device allocation, for callers that must not allocate device
// memory at the point of the call (see include/stochq.h).
//
// The reduction scratch (per-CTA partial sums, per-source arrival counters
// and the per-source results) lives in one file-scope __device__ array that
// every GPU which loads the library holds until the process exits. In host
// code the array's name is only a stand-in: its device address is fetched
// once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernel. Every call shares the array, so calls that overlap
// on one GPU race; the counters are cleared at the start of each call.
#include <cstring>
#include <mutex>

#include "sq_internal.h"

namespace sq {

namespace {

constexpr int kMaxRhs = 256;         // sources per call
constexpr int kBlocksPerSource = 128;  // CTAs per source (grid-stride over sites)
constexpr int kThreads = 128;

constexpr size_t kPartialBytes = (size_t)kMaxRhs * kBlocksPerSource * sizeof(double);  // 256 KiB
constexpr size_t kCounterBytes = (size_t)kMaxRhs * sizeof(unsigned);                    // 1 KiB
constexpr size_t kResultBytes = (size_t)kMaxRhs * sizeof(double);                       // 2 KiB
constexpr size_t kScratchBytes = kPartialBytes + kCounterBytes + kResultBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// The norm kernel of sq_norm2_eo with a fixed number of CTAs per source:
// each thread strides over the sites, then the same two-level reduction.
template <int P>
__global__ void __launch_bounds__(kThreads) k_norm2_fixed(int Vh, Field f, RedArgs ra);

// Device address of the scratch array on the current device (set up once).
// The one-time set-up also loads the kernels of all three precisions (CUDA
// loads modules lazily by default), so that no later call of any precision
// loads code, e.g. while another thread captures a graph.
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_norm2_fixed<P64>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_norm2_fixed<P32>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_norm2_fixed<P16>);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_norm2_fixed(int Vh, Field f, RedArgs ra) {
  typedef typename Real<P>::T R;
  const int k = blockIdx.y;
  double v[1] = {0.0};
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
    cx<R> a[12];
    SpinorIO<P>::load(f, k, cb, a);
    double t = 0;
#pragma unroll
    for (int j = 0; j < 12; j++) t += (double)a[j].re * a[j].re + (double)a[j].im * a[j].im;
    v[0] += t;
  }
  reduce_finalize<1, FIN_STORE>(ra, v, k, (int)gridDim.x, (int)blockIdx.x);
}

}  // namespace

}  // namespace sq

using namespace sq;

extern "C" sq_status sq_norm2_eo_noalloc(sq_ctx* c, const void* field, sq_prec prec, int n, double* out,
                                         int where) {
  if (!c) return SQ_ERR_ARG;
  if (!field || !out || n <= 0 || prec < SQ_F64 || prec > SQ_F16 || (where != SQ_HOST && where != SQ_DEVICE))
    return set_error(c, SQ_ERR_ARG, "sq_norm2_eo_noalloc: bad argument");
  if (n > kMaxRhs)
    return set_error(c, SQ_ERR_ARG, "sq_norm2_eo_noalloc: n_rhs = %d exceeds the maximum of %d sources", n,
                     kMaxRhs);
  // the context's device is made current for the call (and restored after)
  struct DeviceGuard {
    int prev = -1, want = -1;
    ~DeviceGuard() {
      if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
  } guard;
  cudaError_t e = cudaGetDevice(&guard.prev);
  guard.want = c->device;
  if (e == cudaSuccess && guard.prev != c->device) e = cudaSetDevice(c->device);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(c->device, &base);
  if (e != cudaSuccess) return cuda_check(c, e, "sq_norm2_eo_noalloc scratch address");
  sq_status s = enter_stream(c);
  if (s != SQ_OK) return s;
  char* b = (char*)base;
  RedArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.partial = (double*)b;
  ra.counter = (unsigned*)(b + kPartialBytes);
  double* results = (double*)(b + kPartialBytes + kCounterBytes);
  ra.out = results;
  ra.nblk_stride = kBlocksPerSource;
  // the array keeps the last call's contents: the counters must start at 0
  e = cudaMemsetAsync(ra.counter, 0, (size_t)n * sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "sq_norm2_eo_noalloc counters");
  const Field f = make_field((void*)field, c->Vh, prec, n);
  const dim3 grid(kBlocksPerSource, n);
  if (prec == SQ_F64) k_norm2_fixed<P64><<<grid, kThreads, 0, c->stream>>>(c->Vh, f, ra);
  else if (prec == SQ_F32) k_norm2_fixed<P32><<<grid, kThreads, 0, c->stream>>>(c->Vh, f, ra);
  else k_norm2_fixed<P16><<<grid, kThreads, 0, c->stream>>>(c->Vh, f, ra);
  e = cudaGetLastError();
  c->launches += 1;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, results, (size_t)n * sizeof(double),
                        where == SQ_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && where == SQ_HOST) e = cudaStreamSynchronize(c->stream);
  s = cuda_check(c, e, "sq_norm2_eo_noalloc");
  if (s != SQ_OK) return s;
  return leave_stream(c);
}

// G7: pion correlator of each solution vector,
//   C_k(dt) = sum_{x on timeslice (t_k + dt) mod T} sum_{spin,colour} |psi_k(x)|^2,
// the per-source stochastic estimate of sum_{x in t} sum_y tr S(x,y) S(x,y)^+
// (Sec. "Stochastic propagators": the zero-momentum pion correlator, and the
// "sum_y tr S_p S_p^+" row of Table Lcomp).
//
// One CTA per (source, timeslice): a timeslice of the lexicographic FP64
// field is one contiguous block of X*Y*Z*24 doubles, read with coalesced
// 16-byte loads and summed in FP64 in a fixed tree (bitwise reproducible).
#include "sq_internal.h"

namespace sq {

__global__ void __launch_bounds__(256) k_pion(const double2* lex, long long slice2, int T, const int* tsl,
                                              double* C) {
  const int t = blockIdx.x;
  const int k = blockIdx.y;
  const double2* p = lex + ((long long)k * T + t) * slice2;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < slice2; i += blockDim.x) {
    double2 v = p[i];
    acc = fma(v.x, v.x, acc);
    acc = fma(v.y, v.y, acc);
  }
  __shared__ double sm[8];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sm[w];
    const int t0 = tsl ? ((tsl[k] % T) + T) % T : 0;
    const int dt = ((t - t0) % T + T) % T;
    C[(size_t)k * T + dt] = s;
  }
}

void launch_pion(const sq_ctx* c, const double* lex, int n, const int* tsl, double* C, cudaStream_t s) {
  const int T = c->dims[3];
  const long long slice2 = (long long)c->dims[0] * c->dims[1] * c->dims[2] * 12;  // double2 per slice
  dim3 grid(T, n);
  k_pion<<<grid, 256, 0, s>>>((const double2*)lex, slice2, T, tsl, C);
}

}  // namespace sq

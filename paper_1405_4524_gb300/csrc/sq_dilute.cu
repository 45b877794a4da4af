// Dilution of noise vectors into sources (Sec. "Stochastic propagators":
// time-spin-colour dilution). Source d of noise vector k keeps the noise on
// its own part of the index space and is zero elsewhere:
//   time:        d = t            keeps timeslice t
//   spin-colour: d = 3*spin + c   keeps spin-colour component d
//   full:        d = 12*t + a     keeps both
// Summed over d the sources of one noise vector give the noise vector back,
// and their supports are disjoint. A noise vector that is 1 on the twelve
// components of one site and 0 elsewhere gives, with spin-colour dilution,
// the twelve point sources at that site.

#include "sq_internal.h"

namespace sq {

// one thread per output complex component; grid-stride; writes every output
__global__ void k_dilute(const double2* noise, int n_noise, int scheme, int T, long long V3, double2* out) {
  const int D = scheme == SQ_DILUTE_TIME ? T : (scheme == SQ_DILUTE_SPIN_COLOUR ? 12 : 12 * T);
  const long long per = (long long)T * V3 * 12;  // complex components per field
  const long long total = (long long)n_noise * D * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long src = e / per, off = e - src * per;
    const int k = (int)(src / D), d = (int)(src - (long long)k * D);
    const int a = (int)(off % 12);
    const int t = (int)(off / (V3 * 12));
    bool keep;
    if (scheme == SQ_DILUTE_TIME) keep = (t == d);
    else if (scheme == SQ_DILUTE_SPIN_COLOUR) keep = (a == d);
    else keep = (t == d / 12) && (a == d % 12);
    out[e] = keep ? noise[(long long)k * per + off] : make_double2(0.0, 0.0);
  }
}

int dilution_count(const sq_ctx* c, int scheme) {
  if (scheme == SQ_DILUTE_TIME) return c->dims[3];
  if (scheme == SQ_DILUTE_SPIN_COLOUR) return 12;
  if (scheme == SQ_DILUTE_FULL) return 12 * c->dims[3];
  return 0;
}

void launch_dilute(const sq_ctx* c, const double* noise, int n_noise, int scheme, double* out, cudaStream_t s) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const long long V3 = (long long)c->dims[0] * c->dims[1] * c->dims[2];
  const long long total = (long long)n_noise * dilution_count(c, scheme) * c->dims[3] * V3 * 12;
  long long blocks = (total + 255) / 256;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  if (blocks < 1) blocks = 1;
  k_dilute<<<(unsigned)blocks, 256, 0, s>>>((const double2*)noise, n_noise, scheme, c->dims[3], V3, (double2*)out);
}

}  // namespace sq

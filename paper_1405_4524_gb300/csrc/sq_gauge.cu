// G0 gauge-field layout conversion and G2 clover build + FP64 inversion.
//
// Clover term (Sheikholeslami-Wohlert, kappa-normalised; c_SW = 1.0 is the
// tree-level value of Sec. "Correlation function"):
//   A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu Fhat_mu_nu(x),
//   Fhat = (Q - Q^+)/8 minus trace/3, Q = the four clover leaves at x.
// In the DeGrand-Rossi basis g_mu = [[0, B_mu], [B_mu^+, 0]] with
// B_x = i s1, B_y = -i s2, B_z = i s3, B_t = 1 (s = Pauli matrices), so
// sigma_mu_nu = (i/2)[g_mu, g_nu] is block diagonal in chirality:
//   chirality 0 (spins 0,1): s01 = s3, s02 = s2, s03 = -s1, s12 = s1, s13 = s2,  s23 = -s3
//   chirality 1 (spins 2,3): s01 = s3, s02 = s2, s03 = s1,  s12 = s1, s13 = -s2, s23 = s3
// and each chiral block is 1 + i kappa c_sw (s1 (x) G1 + s2 (x) G2 + s3 (x) G3)
// with G = the matching signed sums of Fhat.
#include <cstring>

#include "sq_internal.h"

namespace sq {

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------
__global__ void k_gauge_convert(Geom g, const double* lex, double2* U64, void* U32, int recon,
                                uint2* U16, int* err) {
  const long long V = 2LL * g.Vh;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * 4) return;
  const int mu = (int)(tid & 3);
  const long long i = tid >> 2;
  const int x = (int)(i % g.X);
  long long r = i / g.X;
  const int y = (int)(r % g.Y);
  r /= g.Y;
  const int z = (int)(r % g.Z);
  const int t = (int)(r / g.Z);
  const int p = (x + y + z + t) & 1;
  const int cb = (int)(i >> 1);
  const double2* src = (const double2*)lex + (i * 4 + mu) * 9;
  double2 u[9];
  bool finite = true;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    u[e] = src[e];
    finite = finite && isfinite(u[e].x) && isfinite(u[e].y);
  }
  if (!finite) atomicOr(err, 1);
  // SU(3) check (needed by reconstruct-12): U^+ U = 1 and det U = 1
  double dev = 0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double re = 0, im = 0;
      for (int c = 0; c < 3; c++) {
        double2 ca = u[c * 3 + a], cb2 = u[c * 3 + b];
        re += ca.x * cb2.x + ca.y * cb2.y;
        im += ca.x * cb2.y - ca.y * cb2.x;
      }
      if (a == b) re -= 1.0;
      dev = fmax(dev, fabs(re) + fabs(im));
    }
  {
    cx<double> m[9];
    for (int e = 0; e < 9; e++) m[e] = mk(u[e].x, u[e].y);
    cx<double> det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                     m[2] * (m[3] * m[7] - m[4] * m[6]);
    dev = fmax(dev, fabs(det.re - 1.0) + fabs(det.im));
  }
  if (!(dev < 1e-6)) atomicOr(err, 4);
  const size_t base9 = (size_t)(p * 4 + mu) * 9;
  const size_t base3 = (size_t)(p * 4 + mu) * 3;
#pragma unroll
  for (int e = 0; e < 9; e++) U64[(base9 + e) * g.Vh + cb] = u[e];
  if (recon == 12) {
    float4* q = (float4*)U32;
#pragma unroll
    for (int c = 0; c < 3; c++)
      q[(base3 + c) * g.Vh + cb] =
          make_float4((float)u[2 * c].x, (float)u[2 * c].y, (float)u[2 * c + 1].x, (float)u[2 * c + 1].y);
  } else {
    float2* q = (float2*)U32;
#pragma unroll
    for (int e = 0; e < 9; e++) q[(base9 + e) * g.Vh + cb] = make_float2((float)u[e].x, (float)u[e].y);
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    uint2 h;
    h.x = f2h((float)u[2 * c].x, (float)u[2 * c].y);
    h.y = f2h((float)u[2 * c + 1].x, (float)u[2 * c + 1].y);
    U16[(base3 + c) * g.Vh + cb] = h;
  }
}

sq_status gauge_convert(sq_ctx* c, const double* dev_lex) {
  Geom g = geom_of(c);
  long long n = (long long)c->V * 4;
  k_gauge_convert<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(g, dev_lex, c->U64, c->U32, c->recon,
                                                                      c->U16, c->d_err);
  return cuda_check(c, cudaGetLastError(), "gauge conversion launch");
}

// ---------------------------------------------------------------------------
// 3x3 complex matrices (FP64)
// ---------------------------------------------------------------------------
struct M3 {
  cx<double> e[9];
};

__device__ __forceinline__ M3 load_link(const Geom& g, const double2* U64, int mu, Coord c) {
  M3 m;
  const int p = (c.x + c.y + c.z + c.t) & 1;
  const int cb = cb_of(g, c.x, c.y, c.z, c.t);
  const double2* q = U64 + ((size_t)(p * 4 + mu) * 9) * g.Vh + cb;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    double2 v = q[(size_t)e * g.Vh];
    m.e[e] = mk(v.x, v.y);
  }
  return m;
}

// op: 0 = A B, 1 = A B^+, 2 = A^+ B
template <int OP>
__device__ __forceinline__ M3 mm(const M3& A, const M3& B) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cx<double> s = zero<double>();
#pragma unroll
      for (int k = 0; k < 3; k++) {
        if (OP == 0) s = cfma(A.e[i * 3 + k], B.e[k * 3 + j], s);
        if (OP == 1) s = s + A.e[i * 3 + k] * conj(B.e[j * 3 + k]);
        if (OP == 2) s = cjfma(A.e[k * 3 + i], B.e[k * 3 + j], s);
      }
      C.e[i * 3 + j] = s;
    }
  return C;
}

__device__ __forceinline__ M3 dag(const M3& A) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) C.e[i * 3 + j] = conj(A.e[j * 3 + i]);
  return C;
}

// Fhat_mu_nu(x): clover leaves, all in the (mu, then nu) orientation
__device__ M3 fhat(const Geom& g, const double2* U64, Coord x, int mu, int nu) {
  Coord xpm = step(g, x, mu, +1), xpn = step(g, x, nu, +1);
  Coord xmm = step(g, x, mu, -1), xmn = step(g, x, nu, -1);
  Coord xmmpn = step(g, xmm, nu, +1), xmmmn = step(g, xmm, nu, -1), xmnpm = step(g, xmn, mu, +1);
  M3 Um_x = load_link(g, U64, mu, x), Un_x = load_link(g, U64, nu, x);
  M3 Q;
  // x -> x+mu -> x+mu+nu -> x+nu -> x
  M3 l = mm<0>(Um_x, load_link(g, U64, nu, xpm));
  l = mm<1>(l, load_link(g, U64, mu, xpn));
  l = mm<1>(l, Un_x);
  Q = l;
  // x -> x+nu -> x-mu+nu -> x-mu -> x
  M3 Um_xmm = load_link(g, U64, mu, xmm);
  l = mm<1>(Un_x, load_link(g, U64, mu, xmmpn));
  l = mm<1>(l, load_link(g, U64, nu, xmm));
  l = mm<0>(l, Um_xmm);
#pragma unroll
  for (int e = 0; e < 9; e++) Q.e[e] = Q.e[e] + l.e[e];
  // x -> x-mu -> x-mu-nu -> x-nu -> x
  M3 Un_xmn = load_link(g, U64, nu, xmn);
  l = mm<2>(Um_xmm, dag(load_link(g, U64, nu, xmmmn)));
  l = mm<0>(l, load_link(g, U64, mu, xmmmn));
  l = mm<0>(l, Un_xmn);
#pragma unroll
  for (int e = 0; e < 9; e++) Q.e[e] = Q.e[e] + l.e[e];
  // x -> x-nu -> x-nu+mu -> x+mu -> x
  l = mm<2>(Un_xmn, load_link(g, U64, mu, xmn));
  l = mm<0>(l, load_link(g, U64, nu, xmnpm));
  l = mm<1>(l, Um_x);
#pragma unroll
  for (int e = 0; e < 9; e++) Q.e[e] = Q.e[e] + l.e[e];
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cx<double> a = Q.e[i * 3 + j], b = conj(Q.e[j * 3 + i]);
      F.e[i * 3 + j] = 0.125 * (a - b);
    }
  cx<double> tr3 = (1.0 / 3.0) * (F.e[0] + F.e[4] + F.e[8]);
  F.e[0] = F.e[0] - tr3;
  F.e[4] = F.e[4] - tr3;
  F.e[8] = F.e[8] - tr3;
  return F;
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting.
// Returns false if some pivot is below tol_rel * max|a_ij|.
__device__ bool inv6(cx<double> a[36], cx<double> b[36]) {
  double scale = 0;
  for (int i = 0; i < 36; i++) scale = fmax(scale, fabs(a[i].re) + fabs(a[i].im));
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) b[i * 6 + j] = mk(i == j ? 1.0 : 0.0, 0.0);
  bool ok = scale > 0;
  for (int col = 0; col < 6; col++) {
    int piv = col;
    double best = 0;
    for (int r = col; r < 6; r++) {
      double m = a[r * 6 + col].re * a[r * 6 + col].re + a[r * 6 + col].im * a[r * 6 + col].im;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (!(sqrt(best) > 1e-12 * scale)) {
      ok = false;
      break;
    }
    if (piv != col)
      for (int j = 0; j < 6; j++) {
        cx<double> t = a[col * 6 + j];
        a[col * 6 + j] = a[piv * 6 + j];
        a[piv * 6 + j] = t;
        t = b[col * 6 + j];
        b[col * 6 + j] = b[piv * 6 + j];
        b[piv * 6 + j] = t;
      }
    cx<double> d = a[col * 6 + col];
    double dn = d.re * d.re + d.im * d.im;
    cx<double> inv = mk(d.re / dn, -d.im / dn);
    for (int j = 0; j < 6; j++) {
      a[col * 6 + j] = a[col * 6 + j] * inv;
      b[col * 6 + j] = b[col * 6 + j] * inv;
    }
    for (int r = 0; r < 6; r++) {
      if (r == col) continue;
      cx<double> f = a[r * 6 + col];
      for (int j = 0; j < 6; j++) {
        a[r * 6 + j] = a[r * 6 + j] - f * a[col * 6 + j];
        b[r * 6 + j] = b[r * 6 + j] - f * b[col * 6 + j];
      }
    }
  }
  return ok;
}

// pack a Hermitian 6x6 (Hermitian part of m) into 36 reals
__device__ void pack_herm(const cx<double> m[36], double o[36]) {
  for (int i = 0; i < 6; i++) o[i] = m[i * 6 + i].re;
  for (int i = 1; i < 6; i++)
    for (int j = 0; j < i; j++) {
      cx<double> l = 0.5 * (m[i * 6 + j] + conj(m[j * 6 + i]));
      o[6 + 2 * tri(i, j)] = l.re;
      o[6 + 2 * tri(i, j) + 1] = l.im;
    }
}

__global__ void k_clover(Geom g, const double2* U64, double kappa, double csw, double2* A64, double2* Ainv64,
                         float4* Ainv32, uint4* Ainv16, unsigned long long* abound, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  Coord x;
  x.x = i % g.X;
  int r = i / g.X;
  x.y = r % g.Y;
  r /= g.Y;
  x.z = r % g.Z;
  x.t = r / g.Z;
  const int p = (x.x + x.y + x.z + x.t) & 1;
  const int cb = i >> 1;
  // planes: 01 02 03 12 13 23
  M3 F01 = fhat(g, U64, x, 0, 1), F02 = fhat(g, U64, x, 0, 2), F03 = fhat(g, U64, x, 0, 3);
  M3 F12 = fhat(g, U64, x, 1, 2), F13 = fhat(g, U64, x, 1, 3), F23 = fhat(g, U64, x, 2, 3);
  const double kc = kappa * csw;
  double packA[72], packI[72];
  bool ok = true;
  double bound = 0;
  for (int ch = 0; ch < 2; ch++) {
    const double sg = ch == 0 ? -1.0 : 1.0;
    // G1 (s1), G2 (s2), G3 (s3) for this chirality
    M3 G1, G2, G3;
    for (int e = 0; e < 9; e++) {
      G1.e[e] = F12.e[e] + sg * F03.e[e];
      G2.e[e] = F02.e[e] - sg * F13.e[e];
      G3.e[e] = F01.e[e] + sg * F23.e[e];
    }
    // A = 1 + i kc [[G3, G1 - i G2], [G1 + i G2, -G3]]  (spin-major 6x6)
    cx<double> A[36], Ai[36];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        cx<double> g1 = G1.e[a * 3 + b], g2 = G2.e[a * 3 + b], g3 = G3.e[a * 3 + b];
        cx<double> d00 = g3, d01 = g1 - itimes(g2), d10 = g1 + itimes(g2), d11 = mk(-g3.re, -g3.im);
        A[(0 + a) * 6 + (0 + b)] = kc * itimes(d00);
        A[(0 + a) * 6 + (3 + b)] = kc * itimes(d01);
        A[(3 + a) * 6 + (0 + b)] = kc * itimes(d10);
        A[(3 + a) * 6 + (3 + b)] = kc * itimes(d11);
      }
    for (int d = 0; d < 6; d++) A[d * 6 + d].re += 1.0;
    for (int a = 0; a < 6; a++) {
      double rs = 0;
      for (int b = 0; b < 6; b++) rs += sqrt(A[a * 6 + b].re * A[a * 6 + b].re + A[a * 6 + b].im * A[a * 6 + b].im);
      bound = fmax(bound, rs);
    }
    pack_herm(A, packA + 36 * ch);
    cx<double> work[36];
    for (int e = 0; e < 36; e++) work[e] = A[e];
    ok = inv6(work, Ai) && ok;
    pack_herm(Ai, packI + 36 * ch);
  }
  if (!ok) atomicOr(err, 2);
  atomicMax(abound, (unsigned long long)__double_as_longlong(bound));
  for (int j = 0; j < 36; j++) {
    A64[((size_t)p * 36 + j) * g.Vh + cb] = make_double2(packA[2 * j], packA[2 * j + 1]);
    Ainv64[((size_t)p * 36 + j) * g.Vh + cb] = make_double2(packI[2 * j], packI[2 * j + 1]);
  }
  for (int j = 0; j < 18; j++)
    Ainv32[((size_t)p * 18 + j) * g.Vh + cb] = make_float4((float)packI[4 * j], (float)packI[4 * j + 1],
                                                           (float)packI[4 * j + 2], (float)packI[4 * j + 3]);
  for (int j = 0; j < 9; j++) {
    uint4 h;
    h.x = f2h((float)packI[8 * j + 0], (float)packI[8 * j + 1]);
    h.y = f2h((float)packI[8 * j + 2], (float)packI[8 * j + 3]);
    h.z = f2h((float)packI[8 * j + 4], (float)packI[8 * j + 5]);
    h.w = f2h((float)packI[8 * j + 6], (float)packI[8 * j + 7]);
    Ainv16[((size_t)p * 9 + j) * g.Vh + cb] = h;
  }
}

sq_status clover_build(sq_ctx* c, CloverSet& cs, double kappa, double csw) {
  Geom g = geom_of(c);
  unsigned long long* d_bound = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d_bound, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "clover bound alloc");
  cudaMemsetAsync(d_bound, 0, sizeof(unsigned long long), c->stream);
  k_clover<<<(2 * c->Vh + 127) / 128, 128, 0, c->stream>>>(g, c->U64, kappa, csw, cs.A64, cs.Ainv64, cs.Ainv32,
                                                          cs.Ainv16, d_bound, c->d_err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "clover launch");
  unsigned long long hb = 0;
  cudaMemcpyAsync(&hb, d_bound, sizeof(hb), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d_bound, c->stream);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "clover build");
  double b;
  memcpy(&b, &hb, sizeof(b));
  cs.a_bound = b;
  cs.kappa = kappa;
  cs.csw = csw;
  return SQ_OK;
}

// ---------------------------------------------------------------------------
// finiteness check of a device FP64 array
// ---------------------------------------------------------------------------
__global__ void k_finite(const double* a, size_t n, int* bad) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  int b = 0;
  for (; i < n; i += stride) b |= !isfinite(a[i]);
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}

sq_status check_finite(sq_ctx* c, const double* dev, size_t n, int* bad) {
  int* d_bad = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d_bad, sizeof(int), c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "finite check alloc");
  cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  size_t want = (n + 255) / 256;
  unsigned grid = (unsigned)(want < (size_t)sms * 8 ? (want > 0 ? want : 1) : (size_t)sms * 8);
  k_finite<<<grid, 256, 0, c->stream>>>(dev, n, d_bad);
  int h = 0;
  cudaMemcpyAsync(&h, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d_bad, c->stream);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "finite check");
  *bad = h;
  return SQ_OK;
}

}  // namespace sq

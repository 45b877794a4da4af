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

#include "sq_df32.cuh"
#include "sq_internal.h"

namespace sq {

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------
// lex -> U64 (FP64), U32 (reconstruct-12 or -18 FP32) and Udf (each FP64
// element as a rounded float pair for the emulated-FP64 operator), with the
// finiteness and SU(3) checks
__global__ void k_gauge_convert(Geom g, const double* lex, double2* U64, void* U32, float4* Udf, int recon, int* err) {
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
  for (int e = 0; e < 9; e++) {
    U64[(base9 + e) * g.Vh + cb] = u[e];
    const float hr = __double2float_rn(u[e].x), hi = __double2float_rn(u[e].y);
    Udf[(base9 + e) * g.Vh + cb] =
        make_float4(hr, hi, __double2float_rn(u[e].x - (double)hr), __double2float_rn(u[e].y - (double)hi));
  }
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
}

sq_status gauge_convert(sq_ctx* c, const double* dev_lex) {
  Geom g = geom_of(c);
  long long n = (long long)c->V * 4;
  k_gauge_convert<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(g, dev_lex, c->U64, c->U32, c->Udf, c->recon,
                                                                      c->d_err);
  return cuda_check(c, cudaGetLastError(), "gauge conversion launch");
}

// ---------------------------------------------------------------------------
// 3x3 complex matrices (FP64)
// ---------------------------------------------------------------------------
struct M3 {
  cx<double> e[9];
};

// ---------------------------------------------------------------------------
// clover leaves in double-FP32 (sq_df32.cuh) on the FP32 pipe
// ---------------------------------------------------------------------------
struct M3d {
  cdf e[9];
};

// U_mu(y), or U_mu(y)^+ when dag, from the pre-split link copy
__device__ __forceinline__ M3d load_link_df3(const Geom& g, const float4* Udf, int mu, Coord y, bool dag) {
  const int p = (y.x + y.y + y.z + y.t) & 1;
  const float4* q = Udf + ((size_t)(p * 4 + mu) * 9) * g.Vh + cb_of(g, y.x, y.y, y.z, y.t);
  const float si = dag ? -1.f : 1.f;
  M3d m;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const cdf v = cdf_of(__ldg(q + (size_t)(dag ? j * 3 + i : i * 3 + j) * g.Vh));
      m.e[i * 3 + j] = cdf{v.re, df{si * v.im.h, si * v.im.l}};
    }
  return m;
}

__device__ __forceinline__ M3d mm_df3(const M3d& A, const M3d& B) {
  const cdf z{df{0.f, 0.f}, df{0.f, 0.f}};
  M3d C;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cdf r = cfma_df(A.e[i * 3], B.e[j], z);
      r = cfma_df(A.e[i * 3 + 1], B.e[3 + j], r);
      C.e[i * 3 + j] = cfma_df(A.e[i * 3 + 2], B.e[6 + j], r);
    }
  return C;
}

// The four clover leaves of the (mu, nu) plane at x, each the product of
// the four links around a plaquette with a corner at x, walked from x:
//   x, x+mu, x+mu+nu, x+nu;   x, x+nu, x-mu+nu, x-mu;
//   x, x-mu, x-mu-nu, x-nu;   x, x-nu, x-nu+mu, x+mu.
// Factor f of leaf l is U_d(x + a_mu mu + a_nu nu), daggered when the walk
// goes against d: {d (0 = mu, 1 = nu), a_mu, a_nu, dagger}.
__constant__ signed char kLeaf[4][4][4] = {
    {{0, 0, 0, 0}, {1, 1, 0, 0}, {0, 0, 1, 1}, {1, 0, 0, 1}},
    {{1, 0, 0, 0}, {0, -1, 1, 1}, {1, -1, 0, 1}, {0, -1, 0, 0}},
    {{0, -1, 0, 1}, {1, -1, -1, 1}, {0, -1, -1, 0}, {1, 0, -1, 0}},
    {{1, 0, -1, 1}, {0, 0, -1, 0}, {1, 1, -1, 0}, {0, 0, 0, 1}}};

// Q = the sum of the four leaves (double-FP32 products: every product of
// leading parts exact, trailing parts and cross terms in FP32; about 2^-44
// of the O(1) link products per entry), rounded to FP64
__device__ void clover_leaves(const Geom& g, const float4* Udf, Coord x, int mu, int nu, cx<double> Q[9]) {
#pragma unroll
  for (int e = 0; e < 9; e++) Q[e] = zero<double>();
#pragma unroll 1
  for (int l = 0; l < 4; l++) {
    M3d acc;
#pragma unroll 1
    for (int f = 0; f < 4; f++) {
      const signed char* t = kLeaf[l][f];
      Coord y = x;
      if (t[1]) y = step(g, y, mu, t[1]);
      if (t[2]) y = step(g, y, nu, t[2]);
      const M3d W = load_link_df3(g, Udf, t[0] ? nu : mu, y, t[3] != 0);
      if (f == 0) acc = W;
      else acc = mm_df3(acc, W);
    }
#pragma unroll
    for (int e = 0; e < 9; e++) {
      const double2 v = double2_of(acc.e[e]);
      Q[e] = Q[e] + mk(v.x, v.y);
    }
  }
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

// Inverse of a packed Hermitian 6x6 block by A = L D L^+ (unit lower L,
// real D) with fully static indexing, so everything stays in registers:
// A^{-1}_ij = sum_{k >= max(i,j)} conj(M_ki) M_kj / d_k with M = L^{-1}.
// Returns false when a pivot is below 5% of the largest diagonal (the block
// is then not safely positive definite; the caller uses pivoted
// Gauss-Jordan instead).
__device__ bool herm6_inverse_ldl(const double a[36], double out[36]) {
  double d[6], id[6], lr[15], li[15], mr[15], mi[15];
  double scale = 0;
#pragma unroll
  for (int i = 0; i < 6; i++) scale = fmax(scale, fabs(a[i]));
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; j++) {
    double dj = a[j];
#pragma unroll
    for (int k = 0; k < j; k++) dj -= (lr[tri(j, k)] * lr[tri(j, k)] + li[tri(j, k)] * li[tri(j, k)]) * d[k];
    ok = ok && (dj > 0.05 * scale);
    d[j] = dj;
    id[j] = 1.0 / dj;
#pragma unroll
    for (int i = j + 1; i < 6; i++) {
      double sr = a[6 + 2 * tri(i, j)], si = a[6 + 2 * tri(i, j) + 1];
#pragma unroll
      for (int k = 0; k < j; k++) {  // - L_ik conj(L_jk) d_k
        const double xr = lr[tri(i, k)], xi = li[tri(i, k)], yr = lr[tri(j, k)], yi = li[tri(j, k)];
        sr -= (xr * yr + xi * yi) * d[k];
        si -= (xi * yr - xr * yi) * d[k];
      }
      lr[tri(i, j)] = sr * id[j];
      li[tri(i, j)] = si * id[j];
    }
  }
  if (!ok) return false;
#pragma unroll
  for (int j = 0; j < 6; j++)
#pragma unroll
    for (int i = j + 1; i < 6; i++) {  // M_ij = -(L_ij + sum_{j<k<i} L_ik M_kj)
      double sr = lr[tri(i, j)], si = li[tri(i, j)];
#pragma unroll
      for (int k = j + 1; k < i; k++) {
        sr += lr[tri(i, k)] * mr[tri(k, j)] - li[tri(i, k)] * mi[tri(k, j)];
        si += lr[tri(i, k)] * mi[tri(k, j)] + li[tri(i, k)] * mr[tri(k, j)];
      }
      mr[tri(i, j)] = -sr;
      mi[tri(i, j)] = -si;
    }
#pragma unroll
  for (int i = 0; i < 6; i++) {
    double s = id[i];
#pragma unroll
    for (int k = i + 1; k < 6; k++) s += (mr[tri(k, i)] * mr[tri(k, i)] + mi[tri(k, i)] * mi[tri(k, i)]) * id[k];
    out[i] = s;
  }
#pragma unroll
  for (int i = 1; i < 6; i++)
#pragma unroll
    for (int j = 0; j < i; j++) {
      double sr = mr[tri(i, j)] * id[i], si = mi[tri(i, j)] * id[i];
#pragma unroll
      for (int k = i + 1; k < 6; k++) {  // conj(M_ki) M_kj / d_k
        const double ar = mr[tri(k, i)], ai = mi[tri(k, i)], br = mr[tri(k, j)], bi = mi[tri(k, j)];
        sr += (ar * br + ai * bi) * id[k];
        si += (ar * bi - ai * br) * id[k];
      }
      out[6 + 2 * tri(i, j)] = sr;
      out[6 + 2 * tri(i, j) + 1] = si;
    }
  return true;
}

// Clover build in two kernels.
// k_clover_F, one thread per site and plane (blockIdx.y = plane 01, 02, 03,
// 12, 13, 23): Fhat = (Q - Q^+)/8 minus its trace/3 in FP64 from the leaves,
// to F[plane][9][V] (lexicographic site index).
// k_clover, two threads per site (chiral block ch): the G combinations of
// the six planes into shared memory, then
// A = 1 + i kc [[G3, G1 - i G2], [G1 + i G2, -G3]] packed, its norm bound,
// its inverse, and A, A^{-1} (FP64) and the FP32 A^{-1} copy written.
constexpr int kCloverSites = 32;

__global__ void __launch_bounds__(128, 4) k_clover_F(Geom g, const float4* Udf, double2* F) {
  const int V = 2 * g.Vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int pl = blockIdx.y;
  if (i >= V) return;
  const int mu = pl < 3 ? 0 : pl < 5 ? 1 : 2;
  const int nu = pl < 3 ? pl + 1 : pl < 5 ? pl - 1 : 3;
  Coord x;
  x.x = i % g.X;
  int r = i / g.X;
  x.y = r % g.Y;
  r /= g.Y;
  x.z = r % g.Z;
  x.t = r / g.Z;
  cx<double> Q[9];
  clover_leaves(g, Udf, x, mu, nu, Q);
  cx<double> Fm[9];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) Fm[a * 3 + b] = 0.125 * (Q[a * 3 + b] - conj(Q[b * 3 + a]));
  const cx<double> tr3 = (1.0 / 3.0) * (Fm[0] + Fm[4] + Fm[8]);
  Fm[0] = Fm[0] - tr3;
  Fm[4] = Fm[4] - tr3;
  Fm[8] = Fm[8] - tr3;
#pragma unroll
  for (int e = 0; e < 9; e++) F[((size_t)pl * 9 + e) * V + i] = make_double2(Fm[e].re, Fm[e].im);
}

// a double pair as rounded float pairs (re.h, im.h, re.l, im.l)
__device__ __forceinline__ float4 split_pair(double a, double b) {
  const float ha = __double2float_rn(a), hb = __double2float_rn(b);
  return make_float4(ha, hb, __double2float_rn(a - (double)ha), __double2float_rn(b - (double)hb));
}

__global__ void __launch_bounds__(2 * kCloverSites) k_clover(Geom g, const double2* F, double kappa, double csw,
                                                             double2* A64, double2* Ainv64, float4* Ainv32,
                                                             float4* Adf, float4* Ainvdf,
                                                             unsigned long long* abound, int* err) {
  __shared__ M3 sG[kCloverSites][2][3];
  const int t = threadIdx.x;
  const int V = 2 * g.Vh;
  {
    // chirality 0 / 1: G3 = F01 -+ F23, G2 = F02 +- F13, G1 = F12 -+ F03
    const int s = t >> 1, ch = t & 1;
    const int i = blockIdx.x * kCloverSites + s;
    if (i < V) {
      const double sgn = ch ? 1.0 : -1.0;
#pragma unroll
      for (int e = 0; e < 9; e++) {
        const double2 f01 = F[(size_t)(0 * 9 + e) * V + i], f02 = F[(size_t)(1 * 9 + e) * V + i];
        const double2 f03 = F[(size_t)(2 * 9 + e) * V + i], f12 = F[(size_t)(3 * 9 + e) * V + i];
        const double2 f13 = F[(size_t)(4 * 9 + e) * V + i], f23 = F[(size_t)(5 * 9 + e) * V + i];
        sG[s][ch][0].e[e] = mk(f01.x + sgn * f23.x, f01.y + sgn * f23.y);
        sG[s][ch][1].e[e] = mk(f02.x - sgn * f13.x, f02.y - sgn * f13.y);
        sG[s][ch][2].e[e] = mk(f12.x + sgn * f03.x, f12.y + sgn * f03.y);
      }
    }
  }
  __syncthreads();
  const int s = t >> 1, ch = t & 1;
  const int i = blockIdx.x * kCloverSites + s;
  if (i >= V) return;
  int xi = i % g.X, r = i / g.X, yi = r % g.Y;
  r /= g.Y;
  const int zi = r % g.Z, ti = r / g.Z;
  const int p = (xi + yi + zi + ti) & 1;
  const int cb = i >> 1;
  const double kc = kappa * csw;
  const M3& G1 = sG[s][ch][2];
  const M3& G2 = sG[s][ch][1];
  const M3& G3 = sG[s][ch][0];
  // element (row, col) of i kc [[G3, G1 - iG2], [G1 + iG2, -G3]]
  auto elem = [&](int row, int col) -> cx<double> {
    const int sr = row / 3, a = row % 3, sc = col / 3, b = col % 3;
    const cx<double> g1 = G1.e[a * 3 + b], g2 = G2.e[a * 3 + b], g3 = G3.e[a * 3 + b];
    cx<double> d;
    if (sr == 0 && sc == 0) d = g3;
    else if (sr == 0) d = g1 - itimes(g2);
    else if (sc == 0) d = g1 + itimes(g2);
    else d = mk(-g3.re, -g3.im);
    return kc * itimes(d);
  };
  double pa[36], pi[36];
#pragma unroll
  for (int k = 0; k < 6; k++) pa[k] = 1.0 + elem(k, k).re;
#pragma unroll
  for (int row = 1; row < 6; row++)
#pragma unroll
    for (int col = 0; col < row; col++) {
      const cx<double> v = elem(row, col);
      pa[6 + 2 * tri(row, col)] = v.re;
      pa[6 + 2 * tri(row, col) + 1] = v.im;
    }
  // Gershgorin bound on ||A||_2 from the packed Hermitian rows
  double bound = 0;
#pragma unroll
  for (int row = 0; row < 6; row++) {
    double rs = fabs(pa[row]);
#pragma unroll
    for (int col = 0; col < 6; col++) {
      if (col == row) continue;
      const int hi = row > col ? row : col, lo = row > col ? col : row;
      rs += sqrt(pa[6 + 2 * tri(hi, lo)] * pa[6 + 2 * tri(hi, lo)] +
                 pa[6 + 2 * tri(hi, lo) + 1] * pa[6 + 2 * tri(hi, lo) + 1]);
    }
    bound = fmax(bound, rs);
  }
  atomicMax(abound, (unsigned long long)__double_as_longlong(bound));
#pragma unroll
  for (int m = 0; m < 18; m++) {
    A64[((size_t)p * 36 + 18 * ch + m) * g.Vh + cb] = make_double2(pa[2 * m], pa[2 * m + 1]);
    Adf[((size_t)p * 36 + 18 * ch + m) * g.Vh + cb] = split_pair(pa[2 * m], pa[2 * m + 1]);
  }
  if (!herm6_inverse_ldl(pa, pi)) {
    cx<double> A[36], Ai[36];
    for (int row = 0; row < 6; row++)
      for (int col = 0; col < 6; col++) {
        cx<double> v = elem(row, col);
        if (row == col) v.re += 1.0;
        A[row * 6 + col] = v;
      }
    if (!inv6(A, Ai)) atomicOr(err, 2);
    pack_herm(Ai, pi);
  }
#pragma unroll
  for (int m = 0; m < 18; m++) {
    Ainv64[((size_t)p * 36 + 18 * ch + m) * g.Vh + cb] = make_double2(pi[2 * m], pi[2 * m + 1]);
    Ainvdf[((size_t)p * 36 + 18 * ch + m) * g.Vh + cb] = split_pair(pi[2 * m], pi[2 * m + 1]);
  }
#pragma unroll
  for (int m = 0; m < 9; m++)
    Ainv32[((size_t)p * 18 + 9 * ch + m) * g.Vh + cb] =
        make_float4((float)pi[4 * m], (float)pi[4 * m + 1], (float)pi[4 * m + 2], (float)pi[4 * m + 3]);
}

size_t clover_scratch_bytes(const sq_ctx* c) { return 6 * 9 * 2 * (size_t)c->Vh * sizeof(double2); }

// Launches the build of cs (no host synchronisation): A, A^{-1} (FP64, and
// as float pairs for the emulated-FP64 operator), the FP32 A^{-1}, the norm bound into c->d_bound (read back by the caller with
// the error word) and ERRBIT_CLOVER for a singular block.
sq_status clover_build(sq_ctx* c, CloverSet& cs, double kappa, double csw) {
  Geom g = geom_of(c);
  if (!c->cloverF) {
    cudaError_t e = dev_alloc(c->mem, (void**)&c->cloverF, clover_scratch_bytes(c));
    if (e != cudaSuccess) {
      c->cloverF = nullptr;
      return cuda_check(c, e, "clover field-strength scratch");
    }
  }
  const size_t V = 2 * (size_t)c->Vh;
  cudaMemsetAsync(c->d_bound, 0, sizeof(unsigned long long), c->stream);
  k_clover_F<<<dim3((unsigned)((V + 127) / 128), 6), 128, 0, c->stream>>>(g, (const float4*)c->Udf, c->cloverF);
  k_clover<<<(unsigned)((V + kCloverSites - 1) / kCloverSites), 2 * kCloverSites, 0, c->stream>>>(
      g, c->cloverF, kappa, csw, cs.A64, cs.Ainv64, cs.Ainv32, cs.Adf, cs.Ainvdf, c->d_bound, c->d_err);
  cs.kappa = kappa;
  cs.csw = csw;
  return cuda_check(c, cudaGetLastError(), "clover launch");
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

void launch_finite(const sq_ctx* c, const double* dev, size_t n, int* flag, cudaStream_t s) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  size_t want = (n + 255) / 256;
  unsigned grid = (unsigned)(want < (size_t)sms * 8 ? (want > 0 ? want : 1) : (size_t)sms * 8);
  k_finite<<<grid, 256, 0, s>>>(dev, n, flag);
}

}  // namespace sq

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

// ---------------------------------------------------------------------------
// Stochastic-operator contraction (Eq. stoop): per timeslice t the complex
// n x n matrix O(t) = H(t)^+ G(t), H = [eta_1 .. eta_n], G = gamma5 [X_1 ..
// X_n], K = X*Y*Z*12 rows (the sites of the slice times spin-colour). With
// a = eta_i(y), b = (gamma5 X_j)(y), every term conj(a) b is formed from three
// real products (the three-multiplication form of a complex product):
//   P1 += ar br,  P2 += ai bi,  P3 += (ar - ai)(br + bi),
//   Re O = P1 + P2,  Im O = P3 - P1 + P2,
// so the contraction costs 3 FP64 FMAs per term instead of 4; the sums
// ar - ai and br + bi are formed once per row element when it is staged,
// shared by the 16 pairs of a tile row. GB300's FP64 rate bounds it.
//
// The same kernel without gamma5 gives the Gram matrices Sum_y F_k(y)^+ G_l(y)
// of two fields per timeslice (G5 = false), from which the traces of
// products of filled stochastic propagators follow (Eq. Sfill).
//
// k_pair_partial: CTA (t, kg, tile) sums the rows of its K-range for a
// 16 x 16 tile of (i, j) pairs, one pair per thread. The K-range is walked
// in chunks of kStochChunk rows (whole sites, so the gamma5 sign of a row
// position is fixed: spins 0, 1 are rows 0..5 of a site, spins 2, 3 rows
// 6..11; the sign is applied to b when it is staged). The K-group partials
// are added in a fixed order by k_stoch_sum (bitwise reproducible).
// ---------------------------------------------------------------------------
constexpr int kStochTile = 16;
constexpr int kStochChunk = 48;            // rows per chunk: 4 sites x 12
constexpr int kStochPitch = kStochChunk + 1;  // odd pitch: the 16 rows of a tile fall in 16 banks

__device__ __forceinline__ double flip_sign(double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
}

// The 2 x 16 x 48 elements of a chunk's tile rows, 6 per thread: element
// k < 3 is an eta row entry, k >= 3 the X row entry at the same tile
// position. ea / xa point at the tile's first row in chunk r0 = 0, stride is
// the distance between sources, ne / nx the number of rows of the tiles
// that exist. A slice holds X*Y*Z*12 rows, a multiple of 96 for even
// extents, so a chunk never runs past its slice.
__device__ __forceinline__ void stoch_fetch(double2 (&v)[6], const double2* ea, const double2* xa, long long stride,
                                            int ne, int nx, long long r0) {
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int rem = (int)threadIdx.x + 256 * k;
    const int row = rem / kStochChunk, q = rem - row * kStochChunk;
    const long long o = row * stride + r0 + q;
    v[k] = row < ne ? ea[o] : make_double2(0.0, 0.0);
    v[k + 3] = row < nx ? xa[o] : make_double2(0.0, 0.0);
  }
}

template <bool G5>
__global__ void __launch_bounds__(256, 4) k_pair_partial(const double2* eta, const double2* X, int n, int T,
                                                         long long slice2, int nkg, double2* part) {
  __shared__ double a_r[kStochTile][kStochPitch], a_i[kStochTile][kStochPitch], a_d[kStochTile][kStochPitch];
  __shared__ double b_r[kStochTile][kStochPitch], b_i[kStochTile][kStochPitch], b_s[kStochTile][kStochPitch];
  const int t = blockIdx.x, kg = blockIdx.y;
  const int ntile = (n + kStochTile - 1) / kStochTile;
  const int ti = blockIdx.z / ntile, tj = blockIdx.z - ti * ntile;
  const int li = threadIdx.x / kStochTile, lj = threadIdx.x - li * kStochTile;
  const int i = ti * kStochTile + li, j = tj * kStochTile + lj;
  const long long nchunk = (slice2 + kStochChunk - 1) / kStochChunk;
  const long long c0 = nchunk * kg / nkg, c1 = nchunk * (kg + 1) / nkg;
  double P1 = 0, P2 = 0, P3 = 0;
  const long long stride = (long long)T * slice2;
  const double2* ea = eta + (long long)ti * kStochTile * stride + (long long)t * slice2;
  const double2* xa = X + (long long)tj * kStochTile * stride + (long long)t * slice2;
  const int ne = min(kStochTile, n - ti * kStochTile), nx = min(kStochTile, n - tj * kStochTile);
  double2 v[6];
  if (c0 < c1) stoch_fetch(v, ea, xa, stride, ne, nx, c0 * kStochChunk);
  for (long long c = c0; c < c1; c++) {
    __syncthreads();  // the previous chunk's products are done
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const int rem = (int)threadIdx.x + 256 * (k % 3);
      const int row = rem / kStochChunk, q = rem - row * kStochChunk;
      if (k < 3) {
        a_r[row][q] = v[k].x;
        a_i[row][q] = v[k].y;
        a_d[row][q] = v[k].x - v[k].y;
      } else {
        const double sum = v[k].x + v[k].y;
        const bool lower = G5 && (q % 12) >= 6;  // gamma5 = -1 on spins 2, 3
        b_r[row][q] = lower ? flip_sign(v[k].x) : v[k].x;
        b_i[row][q] = lower ? flip_sign(v[k].y) : v[k].y;
        b_s[row][q] = lower ? flip_sign(sum) : sum;
      }
    }
    __syncthreads();
    // the next chunk's loads are in flight during this chunk's products
    if (c + 1 < c1) stoch_fetch(v, ea, xa, stride, ne, nx, (c + 1) * kStochChunk);
#pragma unroll 8
    for (int q = 0; q < kStochChunk; q++) {
      P1 = fma(a_r[li][q], b_r[lj][q], P1);
      P2 = fma(a_i[li][q], b_i[lj][q], P2);
      P3 = fma(a_d[li][q], b_s[lj][q], P3);
    }
  }
  if (i < n && j < n) part[(((long long)t * nkg + kg) * n + i) * n + j] = make_double2(P1 + P2, P3 - P1 + P2);
}

// O[t][i][j] = sum over K-groups in order
__global__ void k_stoch_sum(const double2* part, int n, int T, int nkg, double2* O) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)T * n * n;
  if (idx >= total) return;
  const long long t = idx / ((long long)n * n), ij = idx - t * n * n;
  double re = 0, im = 0;
  for (int kg = 0; kg < nkg; kg++) {
    const double2 v = part[(t * nkg + kg) * n * n + ij];
    re += v.x;
    im += v.y;
  }
  O[idx] = make_double2(re, im);
}

// C[dt] = 1/(n^2 T) sum_t0 S((t0 + dt) mod T, t0), S(ta, tb) = sum_ij
// O_ij(ta) O_ji(tb). S is symmetric (swap i and j), so only ta >= tb is
// formed: k_stoch_corr_pairs, grid (pair, group), walks 32 x 32 tiles of
// O(ta) and the transposed tiles of O(tb) through shared memory (both read
// along rows), one partial per (pair, group); k_stoch_corr_sum adds the
// groups and then the timeslices in a fixed order.
__global__ void __launch_bounds__(256) k_stoch_corr_pairs(const double2* O, int n, int T, int G, double2* part) {
  const int p = blockIdx.x, g = blockIdx.y;
  int ta = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (ta * (ta + 1) / 2 > p) ta--;
  while ((ta + 1) * (ta + 2) / 2 <= p) ta++;
  const int tb = p - ta * (ta + 1) / 2;
  __shared__ double2 sa[32][33], sb[32][33];
  const long long nn = (long long)n * n;
  const int nt = (n + 31) / 32;
  double re = 0, im = 0;
  for (int tile = g; tile < nt * nt; tile += G) {
    const int I = tile / nt, J = tile - (tile / nt) * nt;
    __syncthreads();
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      const int r = e >> 5, c = e & 31;
      const int ia = I * 32 + r, ja = J * 32 + c;  // O(ta)[ia][ja]
      const int jb = J * 32 + r, ib = I * 32 + c;  // O(tb)[jb][ib]
      sa[r][c] = (ia < n && ja < n) ? O[ta * nn + (long long)ia * n + ja] : make_double2(0.0, 0.0);
      sb[r][c] = (jb < n && ib < n) ? O[tb * nn + (long long)jb * n + ib] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      const int r = e >> 5, c = e & 31;  // i = I*32 + r, j = J*32 + c
      const double2 a = sa[r][c], b = sb[c][r];
      re = fma(a.x, b.x, re);
      re = fma(-a.y, b.y, re);
      im = fma(a.x, b.y, im);
      im = fma(a.y, b.x, im);
    }
  }
  __shared__ double sr[8], si[8];
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      a += sr[w];
      b += si[w];
    }
    part[(long long)p * G + g] = make_double2(a, b);
  }
}

__global__ void k_stoch_corr_sum(const double2* part, int n, int T, int G, double2* C) {
  const int dt = blockIdx.x * blockDim.x + threadIdx.x;
  if (dt >= T) return;
  double a = 0, b = 0;
  for (int t0 = 0; t0 < T; t0++) {
    const int t1 = (t0 + dt) % T;
    const int ta = max(t0, t1), tb = min(t0, t1);
    const long long p = (long long)ta * (ta + 1) / 2 + tb;
    double pa = 0, pb = 0;
    for (int g = 0; g < G; g++) {
      pa += part[p * G + g].x;
      pb += part[p * G + g].y;
    }
    a += pa;
    b += pb;
  }
  const double f = 1.0 / ((double)n * n * T);
  C[dt] = make_double2(a * f, b * f);
}

// groups per timeslice pair of the correlator: about 4 CTAs per SM in all
int corr_groups(const sq_ctx* c, int n) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const long long T = c->dims[3], pairs = T * (T + 1) / 2;
  const long long nt = (n + 31) / 32;
  long long g = (4LL * sms + pairs - 1) / pairs;
  if (g > nt * nt) g = nt * nt;
  if (g < 1) g = 1;
  return (int)g;
}

size_t corr_scratch_bytes(const sq_ctx* c, int n) {
  const long long T = c->dims[3];
  return (size_t)(T * (T + 1) / 2) * corr_groups(c, n) * 2 * sizeof(double);
}

// C[t0][t] = 1/n^2 sum_ij P_ji(t) Q_ij(t0) = tr[P(t) Q(t0)] / n^2; one CTA per
// (t0, t), fixed-order tree
__global__ void __launch_bounds__(256) k_prop_trace(const double2* P, const double2* Q, int n, int T, double2* C) {
  const int t0 = blockIdx.x / T, t = blockIdx.x - t0 * T;
  const long long nn = (long long)n * n;
  double re = 0, im = 0;
  for (long long ij = threadIdx.x; ij < nn; ij += blockDim.x) {
    const int i = (int)(ij / n), j = (int)(ij - (long long)i * n);
    const double2 a = P[t * nn + (long long)j * n + i];
    const double2 b = Q[t0 * nn + ij];
    re += a.x * b.x - a.y * b.y;
    im += a.x * b.y + a.y * b.x;
  }
  __shared__ double sr[8], si[8];
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      a += sr[w];
      b += si[w];
    }
    const double f = 1.0 / ((double)n * n);
    C[blockIdx.x] = make_double2(a * f, b * f);
  }
}

// K-groups per timeslice: about four CTAs per SM in one wave
int stoch_groups(const sq_ctx* c, int n) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int T = c->dims[3];
  const int ntile = (n + kStochTile - 1) / kStochTile;
  const long long slice2 = (long long)c->dims[0] * c->dims[1] * c->dims[2] * 12;
  const long long nchunk = (slice2 + kStochChunk - 1) / kStochChunk;
  long long g = 4LL * sms / ((long long)T * ntile * ntile);
  if (g < 1) g = 1;
  if (g > nchunk) g = nchunk;
  return (int)g;
}

// out[t][k][l] = sum over timeslice t of F_k^+ (gamma5) G_l
static void launch_pairs(const sq_ctx* c, bool g5, const double* F, const double* G, int n, double* out, double* part,
                         int nkg, cudaStream_t s) {
  const int T = c->dims[3];
  const long long slice2 = (long long)c->dims[0] * c->dims[1] * c->dims[2] * 12;
  const int ntile = (n + kStochTile - 1) / kStochTile;
  const dim3 grid(T, nkg, ntile * ntile);
  if (g5)
    k_pair_partial<true><<<grid, 256, 0, s>>>((const double2*)F, (const double2*)G, n, T, slice2, nkg, (double2*)part);
  else
    k_pair_partial<false><<<grid, 256, 0, s>>>((const double2*)F, (const double2*)G, n, T, slice2, nkg, (double2*)part);
  const long long total = (long long)T * n * n;
  k_stoch_sum<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const double2*)part, n, T, nkg, (double2*)out);
}

void launch_stoch_op(const sq_ctx* c, const double* eta, const double* X, int n, double* O, double* C, double* part,
                     int nkg, cudaStream_t s) {
  launch_pairs(c, true, eta, X, n, O, part, nkg, s);
  if (C) launch_stoch_corr(c, O, n, C, part, s);
}

void launch_stoch_corr(const sq_ctx* c, const double* O, int n, double* C, double* part, cudaStream_t s) {
  const int T = c->dims[3], G = corr_groups(c, n);
  k_stoch_corr_pairs<<<dim3(T * (T + 1) / 2, G), 256, 0, s>>>((const double2*)O, n, T, G, (double2*)part);
  k_stoch_corr_sum<<<(T + 127) / 128, 128, 0, s>>>((const double2*)part, n, T, G, (double2*)C);
}

void launch_prop_trace(const sq_ctx* c, const double* etaA, const double* XA, const double* etaB, const double* XB,
                       int n, double* P, double* Q, double* C, double* part, int nkg, cudaStream_t s) {
  const int T = c->dims[3];
  launch_pairs(c, false, XB, XA, n, P, part, nkg, s);     // P_ji(t) = sum_z XB_j^+ XA_i
  launch_pairs(c, false, etaA, etaB, n, Q, part, nkg, s);  // Q_ij(t0) = sum_x etaA_i^+ etaB_j
  k_prop_trace<<<T * T, 256, 0, s>>>((const double2*)P, (const double2*)Q, n, T, (double2*)C);
}

}  // namespace sq

// G7: pion correlator of each solution vector,
//   C_k(dt) = sum_{x on timeslice (t_k + dt) mod T} sum_{spin,colour} |psi_k(x)|^2,
// the per-source stochastic estimate of sum_{x in t} sum_y tr S(x,y) S(x,y)^+
// (Sec. "Stochastic propagators": the zero-momentum pion correlator, and the
// "sum_y tr S_p S_p^+" row of Table Lcomp).
//
// One CTA per (source, timeslice): a timeslice of the lexicographic FP64
// field is one contiguous block of X*Y*Z*24 doubles, read with coalesced
// 16-byte loads and summed in FP64 in a fixed tree (bitwise reproducible).
#include <algorithm>

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
__global__ void __launch_bounds__(256, 4) k_pair_partial(const double2* eta, const double2* X, int ni, int nj,
                                                         int T, long long slice2, int nkg, double2* part) {
  __shared__ double a_r[kStochTile][kStochPitch], a_i[kStochTile][kStochPitch], a_d[kStochTile][kStochPitch];
  __shared__ double b_r[kStochTile][kStochPitch], b_i[kStochTile][kStochPitch], b_s[kStochTile][kStochPitch];
  const int t = blockIdx.x, kg = blockIdx.y;
  const int ntj = (nj + kStochTile - 1) / kStochTile;
  const int ti = blockIdx.z / ntj, tj = blockIdx.z - ti * ntj;
  const int li = threadIdx.x / kStochTile, lj = threadIdx.x - li * kStochTile;
  const int i = ti * kStochTile + li, j = tj * kStochTile + lj;
  const long long nchunk = (slice2 + kStochChunk - 1) / kStochChunk;
  const long long c0 = nchunk * kg / nkg, c1 = nchunk * (kg + 1) / nkg;
  double P1 = 0, P2 = 0, P3 = 0;
  const long long stride = (long long)T * slice2;
  const double2* ea = eta + (long long)ti * kStochTile * stride + (long long)t * slice2;
  const double2* xa = X + (long long)tj * kStochTile * stride + (long long)t * slice2;
  const int ne = min(kStochTile, ni - ti * kStochTile), nx = min(kStochTile, nj - tj * kStochTile);
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
  if (i < ni && j < nj) part[(((long long)t * nkg + kg) * ni + i) * nj + j] = make_double2(P1 + P2, P3 - P1 + P2);
}

// O[t][i][j] = sum over K-groups in order (ni x nj pairs per timeslice)
__global__ void k_stoch_sum(const double2* part, int ni, int nj, int T, int nkg, double2* O) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nn = (long long)ni * nj;
  const long long total = (long long)T * nn;
  if (idx >= total) return;
  const long long t = idx / nn, ij = idx - t * nn;
  double re = 0, im = 0;
  for (int kg = 0; kg < nkg; kg++) {
    const double2 v = part[(t * nkg + kg) * nn + ij];
    re += v.x;
    im += v.y;
  }
  O[idx] = make_double2(re, im);
}

// C[dt] = 1/(n^2 T) sum_t0 S((t0 + dt) mod T, t0), S(ta, tb) = sum_ij
// O_ij(ta) O_ji(tb). S is symmetric (swap i and j), so only blocks of
// 4 x 4 timeslices (ta block >= tb block) are formed. k_stoch_corr_blocks,
// grid (block pair, group): the CTA walks 16 x 16 tiles (I, J) of the pair
// index, stages O(ta)[I, J] for its four ta and O(tb)[J, I] for its four tb in
// shared memory (both read along rows), and every thread forms the 16
// products of its (i, j) for all (ta, tb) of the block pair (the 10 with
// ta >= tb in a diagonal block), so each staged value feeds up to four
// complex FMAs. One partial per (block pair, group, ta, tb);
// k_stoch_corr_sum adds the groups, then the timeslices, in a fixed order.
constexpr int kCorrTB = 4;   // timeslices per block
constexpr int kCorrTile = 16;

__global__ void __launch_bounds__(256) k_stoch_corr_blocks(const double2* O, int n, int T, int G, double2* part) {
  const int bp = blockIdx.x, g = blockIdx.y;
  int ba = (int)((sqrt(8.0 * bp + 1.0) - 1.0) * 0.5);
  while (ba * (ba + 1) / 2 > bp) ba--;
  while ((ba + 1) * (ba + 2) / 2 <= bp) ba++;
  const int bb = bp - ba * (ba + 1) / 2;
  __shared__ double2 sa[kCorrTB][kCorrTile][kCorrTile + 1], sb[kCorrTB][kCorrTile][kCorrTile + 1];
  const long long nn = (long long)n * n;
  const int nt = (n + kCorrTile - 1) / kCorrTile;
  const int r = threadIdx.x / kCorrTile, c = threadIdx.x - r * kCorrTile;
  double re[kCorrTB][kCorrTB], im[kCorrTB][kCorrTB];
#pragma unroll
  for (int q = 0; q < kCorrTB; q++)
#pragma unroll
    for (int p = 0; p < kCorrTB; p++) re[q][p] = im[q][p] = 0.0;
  for (int tile = g; tile < nt * nt; tile += G) {
    const int I = tile / nt, J = tile - (tile / nt) * nt;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kCorrTB; q++) {
      const int ta = ba * kCorrTB + q, tb = bb * kCorrTB + q;
      const int ia = I * kCorrTile + r, ja = J * kCorrTile + c;  // O(ta)[ia][ja]
      const int jb = J * kCorrTile + r, ib = I * kCorrTile + c;  // O(tb)[jb][ib]
      sa[q][r][c] = (ta < T && ia < n && ja < n) ? O[ta * nn + (long long)ia * n + ja] : make_double2(0.0, 0.0);
      sb[q][r][c] = (tb < T && jb < n && ib < n) ? O[tb * nn + (long long)jb * n + ib] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double2 a[kCorrTB], b[kCorrTB];
#pragma unroll
    for (int q = 0; q < kCorrTB; q++) {
      a[q] = sa[q][r][c];  // O(ta)[i][j], i = I*16 + r, j = J*16 + c
      b[q] = sb[q][c][r];  // O(tb)[j][i]
    }
    if (ba != bb) {
#pragma unroll
      for (int q = 0; q < kCorrTB; q++)
#pragma unroll
        for (int p = 0; p < kCorrTB; p++) {
          re[q][p] = fma(a[q].x, b[p].x, re[q][p]);
          re[q][p] = fma(-a[q].y, b[p].y, re[q][p]);
          im[q][p] = fma(a[q].x, b[p].y, im[q][p]);
          im[q][p] = fma(a[q].y, b[p].x, im[q][p]);
        }
    } else {  // diagonal block: the sum reads ta >= tb (q >= p) only
#pragma unroll
      for (int q = 0; q < kCorrTB; q++)
#pragma unroll
        for (int p = 0; p <= q; p++) {
          re[q][p] = fma(a[q].x, b[p].x, re[q][p]);
          re[q][p] = fma(-a[q].y, b[p].y, re[q][p]);
          im[q][p] = fma(a[q].x, b[p].y, im[q][p]);
          im[q][p] = fma(a[q].y, b[p].x, im[q][p]);
        }
    }
  }
  // fixed-order block reduction of the 16 complex sums
  __shared__ double red[8][kCorrTB * kCorrTB][2];
#pragma unroll
  for (int q = 0; q < kCorrTB; q++)
#pragma unroll
    for (int p = 0; p < kCorrTB; p++) {
      const double x = warp_sum(re[q][p]), y = warp_sum(im[q][p]);
      if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][q * kCorrTB + p][0] = x;
        red[threadIdx.x >> 5][q * kCorrTB + p][1] = y;
      }
    }
  __syncthreads();
  if (threadIdx.x < kCorrTB * kCorrTB) {
    double x = 0, y = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      x += red[w][threadIdx.x][0];
      y += red[w][threadIdx.x][1];
    }
    part[((long long)bp * G + g) * (kCorrTB * kCorrTB) + threadIdx.x] = make_double2(x, y);
  }
}

// one warp per dt: lane l adds the terms l, l + 32, ... of the (t0, group)
// sequence in order, then a fixed butterfly (deterministic)
__global__ void k_stoch_corr_sum(const double2* part, int n, int T, int G, double2* C) {
  const int dt = blockIdx.x, lane = threadIdx.x;
  double a = 0, b = 0;
  for (int e = lane; e < T * G; e += 32) {
    const int t0 = e / G, g = e - t0 * G;
    const int t1 = (t0 + dt) % T;
    const int ta = max(t0, t1), tb = min(t0, t1);
    const int ba = ta / kCorrTB, bb = tb / kCorrTB;
    const long long bp = (long long)ba * (ba + 1) / 2 + bb;
    const double2 v = part[(bp * G + g) * (kCorrTB * kCorrTB) + (ta % kCorrTB) * kCorrTB + (tb % kCorrTB)];
    a += v.x;
    b += v.y;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    const double f = 1.0 / ((double)n * n * T);
    C[dt] = make_double2(a * f, b * f);
  }
}

static long long corr_block_pairs(const sq_ctx* c) {
  const long long nb = (c->dims[3] + kCorrTB - 1) / kCorrTB;
  return nb * (nb + 1) / 2;
}

// groups per block pair of the correlator: about 4 CTAs per SM in all
int corr_groups(const sq_ctx* c, int n) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const long long pairs = corr_block_pairs(c);
  const long long nt = (n + kCorrTile - 1) / kCorrTile;
  long long g = (4LL * sms + pairs - 1) / pairs;
  if (g > nt * nt) g = nt * nt;
  if (g < 1) g = 1;
  return (int)g;
}

size_t corr_scratch_bytes(const sq_ctx* c, int n) {
  return (size_t)corr_block_pairs(c) * corr_groups(c, n) * kCorrTB * kCorrTB * 2 * sizeof(double);
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
int stoch_groups(const sq_ctx* c, int n) { return stoch_groups2(c, n, n); }

int stoch_groups2(const sq_ctx* c, int ni, int nj) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int T = c->dims[3];
  const long long nti = (ni + kStochTile - 1) / kStochTile, ntj = (nj + kStochTile - 1) / kStochTile;
  const long long slice2 = (long long)c->dims[0] * c->dims[1] * c->dims[2] * 12;
  const long long nchunk = (slice2 + kStochChunk - 1) / kStochChunk;
  long long g = 4LL * sms / ((long long)T * nti * ntj);
  if (g < 1) g = 1;
  if (g > nchunk) g = nchunk;
  return (int)g;
}

// out[t][k][l] = sum over timeslice t of F_k^+ (gamma5) G_l, k < ni, l < nj
static void launch_pairs(const sq_ctx* c, bool g5, const double* F, const double* G, int ni, int nj, double* out,
                         double* part, int nkg, cudaStream_t s) {
  const int T = c->dims[3];
  const long long slice2 = (long long)c->dims[0] * c->dims[1] * c->dims[2] * 12;
  const int nti = (ni + kStochTile - 1) / kStochTile, ntj = (nj + kStochTile - 1) / kStochTile;
  const dim3 grid(T, nkg, nti * ntj);
  if (g5)
    k_pair_partial<true><<<grid, 256, 0, s>>>((const double2*)F, (const double2*)G, ni, nj, T, slice2, nkg,
                                              (double2*)part);
  else
    k_pair_partial<false><<<grid, 256, 0, s>>>((const double2*)F, (const double2*)G, ni, nj, T, slice2, nkg,
                                               (double2*)part);
  const long long total = (long long)T * ni * nj;
  k_stoch_sum<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const double2*)part, ni, nj, T, nkg, (double2*)out);
}

void launch_stoch_op(const sq_ctx* c, const double* eta, const double* X, int n, double* O, double* C, double* part,
                     int nkg, cudaStream_t s) {
  launch_pairs(c, true, eta, X, n, n, O, part, nkg, s);
  if (C) launch_stoch_corr(c, O, n, C, part, s);
}

void launch_stoch_corr(const sq_ctx* c, const double* O, int n, double* C, double* part, cudaStream_t s) {
  const int T = c->dims[3], G = corr_groups(c, n);
  k_stoch_corr_blocks<<<dim3((unsigned)corr_block_pairs(c), G), 256, 0, s>>>((const double2*)O, n, T, G,
                                                                              (double2*)part);
  k_stoch_corr_sum<<<T, 32, 0, s>>>((const double2*)part, n, T, G, (double2*)C);
}

void launch_prop_trace(const sq_ctx* c, const double* etaA, const double* XA, const double* etaB, const double* XB,
                       int n, double* P, double* Q, double* C, double* part, int nkg, cudaStream_t s) {
  const int T = c->dims[3];
  launch_pairs(c, false, XB, XA, n, n, P, part, nkg, s);     // P_ji(t) = sum_z XB_j^+ XA_i
  launch_pairs(c, false, etaA, etaB, n, n, Q, part, nkg, s);  // Q_ij(t0) = sum_x etaA_i^+ etaB_j
  k_prop_trace<<<T * T, 256, 0, s>>>((const double2*)P, (const double2*)Q, n, T, (double2*)C);
}

// ---------------------------------------------------------------------------
// Diagram contractions of the two-pion correlation function at zero momentum
// (Sec. "Stochastic propagators": Diagram 0; Sec. "Correlation function":
// Diagrams 1-3), per gauge configuration. With the twelve point solutions
// Xp[a] = M^{-1} e_a (unit source at the origin) and two sets of noise
// sources / solutions (A for every S, B for every S^+ of Eq. Sfill):
//   P(t)   = sum_a sum_{y in t} |Xp[a](y)|^2            (k_pion, summed over a)
//   Q0(t)  = Ctr[0][t],  Qtt(t) = Ctr[t][t]             (k_prop_trace)
//   C0(t)  = P(t) Q0(t),  C1(t) = Qtt(t) P(0)
//   C2(t)  = (1/n^2) sum_ij Q_ij(t) W_ji(t),  W_ji(t) = sum_a conj(GB(t)_aj) GA(0)_ai
//            with Q_ij(t) = sum_{z in t} etaA_i^+ etaB_j and the Gram matrices
//            G(t)_ai = sum_{y in t} Xp[a]^+ X_i of the point and noise solutions
//   C3(t)  = conj C2(t)
// ---------------------------------------------------------------------------

// one CTA per sink timeslice t; fixed-order tree (bitwise reproducible)
__global__ void __launch_bounds__(256) k_diag_c2(const double2* Q, const double2* GA, const double2* GB, int n,
                                                 double2* C2) {
  const int t = blockIdx.x;
  const long long nn = (long long)n * n;
  const double2* q = Q + t * nn;
  const double2* ga = GA;                    // timeslice 0: [a][i]
  const double2* gb = GB + (long long)t * 12 * n;  // timeslice t: [a][j]
  double re = 0, im = 0;
  for (long long ij = threadIdx.x; ij < nn; ij += blockDim.x) {
    const int i = (int)(ij / n), j = (int)(ij - (long long)i * n);
    double wr = 0, wi = 0;  // W_ji = sum_a conj(gb[a][j]) ga[a][i]
#pragma unroll
    for (int a = 0; a < 12; a++) {
      const double2 x = gb[(long long)a * n + j], y = ga[(long long)a * n + i];
      wr = fma(x.x, y.x, wr);
      wr = fma(x.y, y.y, wr);
      wi = fma(x.x, y.y, wi);
      wi = fma(-x.y, y.x, wi);
    }
    const double2 v = q[ij];
    re = fma(v.x, wr, re);
    re = fma(-v.y, wi, re);
    im = fma(v.x, wi, im);
    im = fma(v.y, wr, im);
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
    C2[t] = make_double2(a * f, b * f);
  }
}

// out[q][t], q = P, Q0, Qtt, C0, C1, C2, C3 (complex; P real)
__global__ void k_diag_final(const double* Cp, const double2* Ctr, const double2* C2, int T, double2* out) {
  const int t = threadIdx.x;
  if (t >= T) return;
  double P = 0, P0 = 0;
  for (int a = 0; a < 12; a++) {
    P += Cp[(long long)a * T + t];
    P0 += Cp[(long long)a * T];
  }
  const double2 q0 = Ctr[t], qtt = Ctr[(long long)t * T + t], c2 = C2[t];
  out[0 * T + t] = make_double2(P, 0.0);
  out[1 * T + t] = q0;
  out[2 * T + t] = qtt;
  out[3 * T + t] = make_double2(P * q0.x, P * q0.y);
  out[4 * T + t] = make_double2(qtt.x * P0, qtt.y * P0);
  out[5 * T + t] = c2;
  out[6 * T + t] = make_double2(c2.x, -c2.y);
}

size_t diagram_scratch_bytes(const sq_ctx* c, int n) {
  const size_t T = c->dims[3];
  const size_t nkg = stoch_groups(c, n), nkg2 = stoch_groups2(c, 12, n);
  const size_t part = std::max(nkg * T * n * n, nkg2 * T * 12 * n) * 16;
  return part + 2 * T * n * n * 16 + 2 * T * 12 * n * 16 + 12 * T * 8 + T * T * 16 + T * 16 + 8 * 256;
}

void launch_diagrams(const sq_ctx* c, const double* Xp, const double* etaA, const double* XA, const double* etaB,
                     const double* XB, int n, double* out, void* scratch, cudaStream_t s) {
  const int T = c->dims[3];
  const int nkg = stoch_groups(c, n), nkg2 = stoch_groups2(c, 12, n);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* b = (char*)scratch;
  double* part = (double*)b;
  b += al(std::max((size_t)nkg * T * n * n, (size_t)nkg2 * T * 12 * n) * 16);
  double* P = (double*)b;
  b += al((size_t)T * n * n * 16);
  double* Q = (double*)b;
  b += al((size_t)T * n * n * 16);
  double* GA = (double*)b;
  b += al((size_t)T * 12 * n * 16);
  double* GB = (double*)b;
  b += al((size_t)T * 12 * n * 16);
  double* Cp = (double*)b;
  b += al((size_t)12 * T * 8);
  double* Ctr = (double*)b;
  b += al((size_t)T * T * 16);
  double* C2 = (double*)b;
  launch_pion(c, Xp, 12, nullptr, Cp, s);
  launch_prop_trace(c, etaA, XA, etaB, XB, n, P, Q, Ctr, part, nkg, s);
  launch_pairs(c, false, Xp, XA, 12, n, GA, part, nkg2, s);  // GA(t)_ai = sum Xp_a^+ XA_i
  launch_pairs(c, false, Xp, XB, 12, n, GB, part, nkg2, s);  // GB(t)_aj = sum Xp_a^+ XB_j
  k_diag_c2<<<T, 256, 0, s>>>((const double2*)Q, (const double2*)GA, (const double2*)GB, n, (double2*)C2);
  k_diag_final<<<1, ((T + 31) / 32) * 32, 0, s>>>(Cp, (const double2*)Ctr, (const double2*)C2, T, (double2*)out);
}

// Vacuum-subtracted averages over configurations (the paper's ensemble
// average, Sec. "Correlation function"): from records rec[cfg][q][t]
// (q as k_diag_final writes them) out[r][t], r = C0 - <P><Q0>,
// <(Qtt - <Qtt>)(P(0) - <P(0)>)>, <C2>, <C3>, C = C0 + C1 - C2 - C3.
// One thread per t; the configurations are summed in order.
__global__ void k_diag_ensemble(const double2* rec, int ncfg, int T, double2* out) {
  const int t = threadIdx.x;
  if (t >= T) return;
  double2 m[7], p0 = make_double2(0, 0);
  for (int q = 0; q < 7; q++) m[q] = make_double2(0, 0);
  for (int k = 0; k < ncfg; k++) {
    for (int q = 0; q < 7; q++) {
      const double2 v = rec[((long long)k * 7 + q) * T + t];
      m[q].x += v.x;
      m[q].y += v.y;
    }
    const double2 v0 = rec[(long long)k * 7 * T];  // P(0)
    p0.x += v0.x;
    p0.y += v0.y;
  }
  const double f = 1.0 / ncfg;
  for (int q = 0; q < 7; q++) m[q] = make_double2(m[q].x * f, m[q].y * f);
  p0 = make_double2(p0.x * f, p0.y * f);
  // complex products <P><Q0>, <Qtt><P(0)>
  const double2 pq = make_double2(m[0].x * m[1].x - m[0].y * m[1].y, m[0].x * m[1].y + m[0].y * m[1].x);
  const double2 qp = make_double2(m[2].x * p0.x - m[2].y * p0.y, m[2].x * p0.y + m[2].y * p0.x);
  const double2 c0 = make_double2(m[3].x - pq.x, m[3].y - pq.y);
  const double2 c1 = make_double2(m[4].x - qp.x, m[4].y - qp.y);
  out[0 * T + t] = c0;
  out[1 * T + t] = c1;
  out[2 * T + t] = m[5];
  out[3 * T + t] = m[6];
  out[4 * T + t] = make_double2(c0.x + c1.x - m[5].x - m[6].x, c0.y + c1.y - m[5].y - m[6].y);
}

void launch_diag_ensemble(const double* rec, int ncfg, int T, double* out, cudaStream_t s) {
  k_diag_ensemble<<<1, ((T + 31) / 32) * 32, 0, s>>>((const double2*)rec, ncfg, T, (double2*)out);
}

}  // namespace sq

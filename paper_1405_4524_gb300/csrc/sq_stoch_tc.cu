// Stochastic operators O_ij(t) (Eq. stoop) on the fifth-generation tensor
// cores, for sources whose real and imaginary components are all 0 or +-1
// (Z2 and Z4 noise and their dilutions).
//
// Exactness. With such sources O_ij(t) is a sum of signed components of
// gamma5 X_j. Every component x of gamma5 X_j is cut, per source, timeslice
// and chunk of 4096 complex rows, into a 55-bit fixed-point integer relative
// to the chunk's largest component (|x| < 2^e):  m = trunc(x 2^(55-e)),
// split into five signed 11-bit digits d_s (m = sum_s d_s 2^(11(4-s))), each
// exact in FP16. One FP16 x FP16 -> FP32 tensor-core product per digit then
// sums at most 8192 terms of magnitude <= 2047, so every partial sum is an
// integer below 2^24 and exact in FP32, whatever order the hardware adds in.
// The digits are combined in FP64 with exact power-of-two weights
// 2^(e - 55 + 11(4-s)), chunk by chunk in a fixed order. The only
// approximation is the truncation of x below 2^(e-55) (relative 2^-55 of the
// chunk's largest component) and the FP64 roundings of that combination.
//
// Real form. K' = 2K columns per timeslice (K = 12 * X*Y*Z complex rows;
// column 2k is the real part of row k, 2k+1 the imaginary part):
//   A (M side, 128 sources i per tile):  a(i, 2k) = Re eta_i(k), a(i, 2k+1) = Im eta_i(k)
//   B (N side, 16 sources j per tile, 10 rows each, row (s*2 + c)*16 + j):
//     c = 0:  b(2k) = d_s(Re y_j(k)),  b(2k+1) = d_s(Im y_j(k))     -> Re O_ij
//     c = 1:  b(2k) = d_s(Im y_j(k)),  b(2k+1) = -d_s(Re y_j(k))    -> Im O_ij
//   with y = gamma5 X. D = A B^T accumulates in tensor memory (128 lanes =
// sources i, 160 columns = (digit, part, j)).
//
// Layout. Operand tiles of 64 columns are stored in global memory already
// in the tensor core's K-major no-swizzle shared-memory layout: 8-row x
// 16-byte core matrices, the core matrix of row group g and column group q
// at byte ((q * R/8) + g) * 128 (R = 128 rows for A, 160 for B), so that one
// bulk copy moves a tile and the matrix descriptors use a leading (column
// group) stride of R*16 bytes and a stride (row group) of 128 bytes.
//
// Kernel. One CTA per (16-source j tile, 128-source i tile, timeslice), two
// CTAs per SM: warp 4 streams the tiles through a 3-stage shared-memory ring
// with cp.async.bulk, warp 5 issues tcgen05.mma (4 per tile, K = 16 each)
// into a tensor-memory accumulator of 160 columns (one chunk of 128 tiles at
// a time), warps 0-3 read the accumulator with tcgen05.ld (warp w owns lanes
// 32w..32w+31) and add the digits into FP64 registers; while one CTA runs
// that epilogue the other CTA on the SM keeps the tensor pipe busy. Every
// wait is bounded; on a timeout the CTA records ERRBIT_TIMEOUT, lets its
// copies and products drain, frees its tensor memory and returns, and the
// CTAs that start later see the error word and do no work.

#include <cuda_fp16.h>
#include <stdint.h>

#include "sq_async.cuh"
#include "sq_internal.h"

namespace sq {

constexpr int kTcM = 128;                  // i rows per tile
constexpr int kTcJ = 16;                   // j sources per tile
constexpr int kTcN = 10 * kTcJ;            // B rows per tile
constexpr int kTcK = 64;                   // K' columns per tile (32 complex rows)
constexpr int kTcStages = 3;
constexpr int kTcChunkTiles = 128;         // tiles per exact chunk (8192 columns)
constexpr int kTcChunkRows = kTcChunkTiles * kTcK / 2;  // complex rows per chunk
constexpr int kTcABytes = kTcM * kTcK * 2;  // 16384
constexpr int kTcBBytes = kTcN * kTcK * 2;  // 20480
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;
constexpr int kTcTmemCols = 256;           // one accumulator of 160 columns
constexpr int kTcThreads = 192;
// dynamic shared memory: the ring, then the barriers; two CTAs per SM
constexpr int kTcBarOffset = kTcStages * kTcStageBytes;  // 110592
constexpr int kTcSmemBytes = kTcBarOffset + 256;
constexpr long long kTcWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

// ---- PTX wrappers (mbarriers and bulk copies: sq_async.cuh) ----------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle: start address,
// leading byte offset (between column groups), stride byte offset (between
// 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N = kTcN, M = kTcM.
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

// Wait, as a whole warp (uniform result), for the phase of parity `parity`
// of barrier `bar`; false after `limit` cycles (ERRBIT_TIMEOUT, abort set)
// or, if watch_abort, when another role has aborted. The waits that drain
// issued copies and products before the CTA leaves use the default limit.
__device__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* err, bool watch_abort,
                        long long limit) {
  const long long t0 = clock64();
  while (true) {
    const bool ready = mbar_try(bar, parity);
    if (__all_sync(0xffffffffu, ready)) return true;
    const bool timed_out = clock64() - t0 > limit;
    const bool stop = timed_out || (watch_abort && *abort);
    if (__any_sync(0xffffffffu, stop)) {
      if (__any_sync(0xffffffffu, timed_out) && (threadIdx.x & 31) == 0) {
        *abort = 1;
        atomicOr(err, ERRBIT_TIMEOUT);
      }
      return false;
    }
  }
}

// ---- operand packing -------------------------------------------------------
// byte offset of element (row r, column k) inside a tile of R rows
__host__ __device__ constexpr int tile_offset(int R, int r, int k) {
  return (((k >> 3) * (R >> 3)) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  uint4 u;
  __half2 h;
  h = __floats2half2_rn(f[0], f[1]);
  u.x = *reinterpret_cast<uint32_t*>(&h);
  h = __floats2half2_rn(f[2], f[3]);
  u.y = *reinterpret_cast<uint32_t*>(&h);
  h = __floats2half2_rn(f[4], f[5]);
  u.z = *reinterpret_cast<uint32_t*>(&h);
  h = __floats2half2_rn(f[6], f[7]);
  u.w = *reinterpret_cast<uint32_t*>(&h);
  return u;
}

// FP16 bits of v in {0, +1, -1} from its FP64 bits (integer pipe only);
// clears ok for any other value (NaN included)
__device__ __forceinline__ uint32_t ternary_half(double v, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFULL;
  ok = ok && (mag == 0 || mag == 0x3FF0000000000000ULL);
  const uint32_t sign = (uint32_t)(b >> 63) << 15;
  return mag == 0 ? 0u : (sign | 0x3C00u);
}

// A tiles of timeslices t0 .. t0 + Tb - 1: grid (nkt, n_itiles, Tb), 256 threads.
// The tile is assembled in shared memory from row-contiguous reads (eight
// threads per source row, 512 bytes) and written out as one contiguous
// 16 KB block. Sets bit 1 of *flag if a component is not 0 or +-1.
__global__ void __launch_bounds__(256) k_tc_pack_eta(const double2* eta, int n, int T, int t0, long long K,
                                                     int nkt, int nit, uint4* A, int* flag) {
  __shared__ __align__(16) unsigned char tile[kTcABytes];
  const int kt = blockIdx.x, it = blockIdx.y, tb = blockIdx.z;
  bool ok = true;
  for (int v = threadIdx.x; v < kTcM * 8; v += blockDim.x) {
    const int q = v & 7, r = v >> 3;  // group of 8 columns (4 complex rows) fastest
    const int i = it * kTcM + r;
    uint32_t h[4] = {0, 0, 0, 0};
    if (i < n) {
      const double2* src = eta + ((long long)i * T + t0 + tb) * K + (long long)kt * (kTcK / 2) + q * 4;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const double2 d = src[c];
        const uint32_t lo = ternary_half(d.x, ok), hi = ternary_half(d.y, ok);
        h[c] = lo | (hi << 16);
      }
    }
    *reinterpret_cast<uint4*>(tile + tile_offset(kTcM, r, q * 8)) = make_uint4(h[0], h[1], h[2], h[3]);
  }
  if (!ok) atomicOr(flag, 1);
  __syncthreads();
  uint4* blk = A + (((long long)tb * nit + it) * nkt + kt) * (kTcABytes / 16);
  for (int v = threadIdx.x; v < kTcABytes / 16; v += blockDim.x) blk[v] = reinterpret_cast<const uint4*>(tile)[v];
}

// trunc(x 2^(55-e)) for |x| < 2^e, from the bits of x (integer pipe only)
__device__ __forceinline__ long long fixed55(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return 0;  // zero or subnormal
  const long long mant = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int sh = E - 1075 + 55 - e;
  const long long m = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0LL);
  return b < 0 ? -m : m;
}

// digit s (0 = most significant) of |m| as a float with the sign of m:
// 0 <= d < 2^11 placed in the mantissa of 2^23 and 2^23 taken away again
// (exact, no integer-to-float conversion), the sign bit set directly
__device__ __forceinline__ float digit(unsigned long long a, unsigned sign, int s) {
  const unsigned d = (unsigned)(a >> (11 * (4 - s))) & 2047u;
  const float v = __uint_as_float(0x4B000000u | d) - 8388608.0f;
  return __uint_as_float(__float_as_uint(v) | sign);
}

// B tiles and chunk exponents of timeslices t0 .. t0 + Tb - 1: grid (nch,
// njt, Tb), 256 threads; a CTA handles the 16 sources of a j tile so that
// 16 consecutive threads fill two adjacent core matrices. Sets bit 2 of
// *flag on a non-finite x.
__global__ void __launch_bounds__(256) k_tc_pack_x(const double2* X, int n, int T, int t0, long long K, int nkt,
                                                   int njt, int nch, uint4* B, int* exps, int* flag) {
  const int ch = blockIdx.x, jt = blockIdx.y, tb = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)ch * kTcChunkRows;
  const long long r1 = min(K, r0 + kTcChunkRows);
  __shared__ int se[kTcJ];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // largest |component| of the chunk per source (bits order |x| for x >= 0)
  for (int jl = warp; jl < kTcJ; jl += blockDim.x >> 5) {
    const int j = jt * kTcJ + jl;
    unsigned long long mx = 0;
    if (j < n) {
      const double2* src = X + ((long long)j * T + t0 + tb) * K;
      for (long long r = r0 + lane; r < r1; r += 32) {
        const double2 d = src[r];
        mx = max(mx, (unsigned long long)__double_as_longlong(d.x) & 0x7FFFFFFFFFFFFFFFULL);
        mx = max(mx, (unsigned long long)__double_as_longlong(d.y) & 0x7FFFFFFFFFFFFFFFULL);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      const int Eb = (int)(mx >> 52);
      if (Eb == 0x7ff) bad = 1;
      const int e = mx == 0 ? 0 : Eb - 1023 + 1;  // |x| < 2^e
      se[jl] = e;
      exps[((long long)tb * njt * kTcJ + jt * kTcJ + jl) * nch + ch] = e;
    }
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicOr(flag, 2);
    return;
  }
  const int kt0 = ch * kTcChunkTiles, kt1 = min(nkt, kt0 + kTcChunkTiles);
  for (int v = threadIdx.x; v < (kt1 - kt0) * 8 * kTcJ; v += blockDim.x) {
    const int jl = v & (kTcJ - 1), q = (v >> 4) & 7, kt = kt0 + (v >> 7);
    const int j = jt * kTcJ + jl, e = se[jl];
    const long long row = (long long)kt * (kTcK / 2) + q * 4;
    // the 4 rows start at a multiple of 4: spin rows 6..11 (gamma5 = -1 on
    // spins 2, 3) are all four (row % 12 == 8) or the last two (== 4)
    const int g = (int)(row % 12);
    unsigned long long ar[4], ai[4];
    unsigned sr[4], si[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      double2 d = make_double2(0.0, 0.0);
      if (j < n) d = X[((long long)j * T + t0 + tb) * K + row + c];
      long long mr = fixed55(d.x, e), mi = fixed55(d.y, e);
      if (g == 8 || (g == 4 && c >= 2)) {
        mr = -mr;
        mi = -mi;
      }
      ar[c] = (unsigned long long)(mr < 0 ? -mr : mr);
      ai[c] = (unsigned long long)(mi < 0 ? -mi : mi);
      sr[c] = mr < 0 ? 0x80000000u : 0u;
      si[c] = mi < 0 ? 0x80000000u : 0u;
    }
    char* blk = reinterpret_cast<char*>(B) + (((long long)tb * njt + jt) * nkt + kt) * kTcBBytes;
#pragma unroll
    for (int s = 0; s < 5; s++) {
      float fr[8], fi[8];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const float dr = digit(ar[c], sr[c], s), di = digit(ai[c], si[c], s);
        fr[2 * c] = dr;
        fr[2 * c + 1] = di;
        fi[2 * c] = di;
        fi[2 * c + 1] = -dr;
      }
      *reinterpret_cast<uint4*>(blk + tile_offset(kTcN, (s * 2 + 0) * kTcJ + jl, q * 8)) = pack8(fr);
      *reinterpret_cast<uint4*>(blk + tile_offset(kTcN, (s * 2 + 1) * kTcJ + jl, q * 8)) = pack8(fi);
    }
  }
}

// ---- the product -----------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 2)
    k_stoch_tc(const uint4* A, const uint4* B, const int* exps, int n, int t0, int nkt, int nit, int njt, int nch,
               double2* O, int* err, long long wait, int stall) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int jt = blockIdx.x, it = blockIdx.y, tb = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kTcBarOffset);
  // bars: full[stages], empty[stages], accf, acce, done
  const uint32_t full0 = smem_addr(bars), empty0 = full0 + 8 * kTcStages;
  const uint32_t accf = empty0 + 8 * kTcStages, acce = accf + 8, done = acce + 8;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTcBarOffset + 8 * (2 * kTcStages + 3));
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const uint32_t never = smem_addr(bars) + 8 * (2 * kTcStages + 3) + 8;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; s++) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 128);
    mbar_init(done, 1);
    mbar_init(never, 1);  // nothing arrives on it (the stall test)
    // a timeout anywhere in this launch: the CTAs that start later do no work
    *abort = *(volatile int*)err & ERRBIT_TIMEOUT;
    mbar_init_fence();
  }
  __syncthreads();
  const bool skip = *abort != 0;
  if (warp == 0 && !skip) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const char* Ablk = reinterpret_cast<const char*>(A) + ((long long)tb * nit + it) * nkt * (long long)kTcABytes;
  const char* Bblk = reinterpret_cast<const char*>(B) + ((long long)tb * njt + jt) * nkt * (long long)kTcBBytes;
  const uint32_t ring = smem_addr(smem);

  if (skip) {
    // nothing to do; fall through to the common exit
  } else   if (warp == 4) {
    // producer: tile kt into stage kt % stages once the products of the
    // tile before it in that stage are done (the whole warp waits, lane 0
    // issues)
    int kt = 0;
    for (; kt < nkt; kt++) {
      const int s = kt % kTcStages;
      if (kt >= kTcStages && !tc_wait(empty0 + 8 * s, ((kt / kTcStages) - 1) & 1, abort, err, true, wait)) break;
      if (lane == 0) {
        mbar_expect_tx(full0 + 8 * s, kTcStageBytes);
        bulk_load(ring + s * kTcStageBytes, Ablk + (long long)kt * kTcABytes, kTcABytes, full0 + 8 * s);
        bulk_load(ring + s * kTcStageBytes + kTcABytes, Bblk + (long long)kt * kTcBBytes, kTcBBytes, full0 + 8 * s);
      }
      __syncwarp();
    }
    // every copy issued has landed before the CTA can leave
    for (int k = max(0, kt - kTcStages); k < kt; k++)
      tc_wait(full0 + 8 * (k % kTcStages), (k / kTcStages) & 1, abort, err, false, kTcWaitCycles);
  } else if (warp == 5) {
    // products (the whole warp waits, lane 0 issues); chunk c starts once
    // the epilogue has read chunk c - 1
    const bool stalled = stall && !tc_wait(never, 0, abort, err, true, wait);
    for (int kt = 0; kt < nkt && !stalled; kt++) {
      const int s = kt % kTcStages, c = kt / kTcChunkTiles;
      const bool first = (kt % kTcChunkTiles) == 0;
      if (first && c >= 1 && !tc_wait(acce, (c - 1) & 1, abort, err, true, wait)) break;
      if (!tc_wait(full0 + 8 * s, (kt / kTcStages) & 1, abort, err, true, wait)) break;
      tc_fence_after();
      if (lane == 0) {
        const uint32_t a0 = ring + s * kTcStageBytes, b0 = a0 + kTcABytes;
#pragma unroll
        for (int ks = 0; ks < kTcK / 16; ks++) {
          const uint64_t ad = smem_desc(a0 + ks * 2 * (kTcM * 16), kTcM * 16, 128);
          const uint64_t bd = smem_desc(b0 + ks * 2 * (kTcN * 16), kTcN * 16, 128);
          tc_mma(tmem, ad, bd, kTcIdesc, (first && ks == 0) ? 0u : 1u);
        }
        tc_commit(empty0 + 8 * s);
        if ((kt % kTcChunkTiles) == kTcChunkTiles - 1 || kt == nkt - 1) tc_commit(accf);
      }
      __syncwarp();
    }
    // all products issued by lane 0 have finished
    if (lane == 0) tc_commit(done);
    __syncwarp();
    tc_wait(done, 0, abort, err, false, kTcWaitCycles);
  } else if (warp < 4) {
    double re[kTcJ], im[kTcJ];
#pragma unroll
    for (int q = 0; q < kTcJ; q++) re[q] = im[q] = 0.0;
    const int* ex = exps + ((long long)tb * njt * kTcJ + jt * kTcJ) * nch;
    for (int c = 0; c < nch; c++) {
      if (!tc_wait(accf, c & 1, abort, err, true, wait)) break;
      tc_fence_after();
      int e[kTcJ];
#pragma unroll
      for (int q = 0; q < kTcJ; q++) e[q] = ex[q * nch + c];
      const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int s = 0; s < 5; s++) {
        uint32_t vr[16], vi[16];
        tc_ld16(tbase + (s * 2 + 0) * kTcJ, vr);
        tc_ld16(tbase + (s * 2 + 1) * kTcJ, vi);
        tc_wait_ld();
#pragma unroll
        for (int q = 0; q < kTcJ; q++) {
          // exact power of two 2^E, from its bits in the normal range (E <
          // 1025 always); subnormal or zero weights, for chunks whose largest
          // component is near the bottom of the FP64 range, through scalbn
          const int E = e[q] - 55 + 11 * (4 - s);
          const double w = E >= -1022 ? __longlong_as_double((long long)(1023 + E) << 52) : scalbn(1.0, E);
          re[q] = fma((double)__uint_as_float(vr[q]), w, re[q]);
          im[q] = fma((double)__uint_as_float(vi[q]), w, im[q]);
        }
      }
      tc_fence_before();
      mbar_arrive(acce);
    }
    const int i = it * kTcM + warp * 32 + lane;
    if (i < n && !*abort) {
      double2* o = O + ((long long)(t0 + tb) * n + i) * n + jt * kTcJ;
#pragma unroll
      for (int q = 0; q < kTcJ; q++)
        if (jt * kTcJ + q < n) o[q] = make_double2(re[q], im[q]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && !skip) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
}

// ---- host side -------------------------------------------------------------
TcPlan tc_plan(const sq_ctx* c, int n, size_t cap_bytes) {
  TcPlan p;
  const long long K = (long long)c->dims[0] * c->dims[1] * c->dims[2] * 12;
  p.T = c->dims[3];
  p.K = K;
  p.nkt = (int)(2 * K / kTcK);
  p.nch = (p.nkt + kTcChunkTiles - 1) / kTcChunkTiles;
  p.nit = (n + kTcM - 1) / kTcM;
  p.njt = (n + kTcJ - 1) / kTcJ;
  p.a_per_t = (size_t)p.nit * p.nkt * kTcABytes;
  p.b_per_t = (size_t)p.njt * p.nkt * kTcBBytes;
  p.e_per_t = (size_t)p.njt * kTcJ * p.nch * sizeof(int);
  const size_t per_t = p.a_per_t + p.b_per_t + ((p.e_per_t + 255) & ~(size_t)255);
  long long tb = (long long)(cap_bytes / per_t);
  if (tb < 1) tb = 1;
  if (tb > p.T) tb = p.T;
  // equal batches (no short tail batch that leaves most SMs idle)
  const long long nbatch = (p.T + tb - 1) / tb;
  p.Tb = (int)((p.T + nbatch - 1) / nbatch);
  p.bytes = per_t * p.Tb + 256;
  return p;
}

// The packed tiles, the exponents and the flag live in ws (p.bytes); the
// flag word (bits 1: eta not 0/+-1, 2: X not finite) is at the end.
cudaError_t launch_stoch_tc(const sq_ctx* c, const TcPlan& p, const double* eta, const double* X, int n, double* O,
                            void* ws, int* err, cudaStream_t s) {
  // per call: the attribute belongs to the current device, and contexts of
  // one process may sit on different devices
  cudaError_t e0 = cudaFuncSetAttribute(k_stoch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
  if (e0 != cudaSuccess) return e0;
  char* base = static_cast<char*>(ws);
  uint4* A = reinterpret_cast<uint4*>(base);
  uint4* B = reinterpret_cast<uint4*>(base + p.a_per_t * p.Tb);
  int* exps = reinterpret_cast<int*>(base + (p.a_per_t + p.b_per_t) * p.Tb);
  int* flag = reinterpret_cast<int*>(base + p.bytes - 256);
  for (int t0 = 0; t0 < p.T; t0 += p.Tb) {
    const int tb = min(p.Tb, p.T - t0);
    k_tc_pack_eta<<<dim3(p.nkt, p.nit, tb), 256, 0, s>>>((const double2*)eta, n, p.T, t0, p.K, p.nkt, p.nit, A,
                                                          flag);
    k_tc_pack_x<<<dim3(p.nch, p.njt, tb), 256, 0, s>>>((const double2*)X, n, p.T, t0, p.K, p.nkt, p.njt,
                                                               p.nch, B, exps, flag);
    k_stoch_tc<<<dim3(p.njt, p.nit, tb), kTcThreads, kTcSmemBytes, s>>>(A, B, exps, n, t0, p.nkt, p.nit, p.njt,
                                                                         p.nch, (double2*)O, err,
                                                                         c->wait_cycles > 0 ? c->wait_cycles
                                                                                            : kTcWaitCycles,
                                                                         c->wait_stall);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace sq

// Device-side building blocks shared by the libstochq kernels: complex
// arithmetic, precision traits, the even-odd field layouts, link and clover
// loaders, neighbour geometry and deterministic block reductions.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sq {

enum { P64 = 0, P32 = 1, P16 = 2 };

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return mk(a.re, -a.im); }
// conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// i * a
template <typename R>
__device__ __forceinline__ cx<R> itimes(cx<R> a) { return mk(-a.im, a.re); }
template <typename R>
__device__ __forceinline__ cx<R> zero() { return mk(R(0), R(0)); }
// a + b * c  (complex fused)
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> b, cx<R> c, cx<R> a) {
  a.re = fma(b.re, c.re, a.re);
  a.re = fma(-b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im);
  a.im = fma(b.im, c.re, a.im);
  return a;
}
// a + conj(b) * c
template <typename R>
__device__ __forceinline__ cx<R> cjfma(cx<R> b, cx<R> c, cx<R> a) {
  a.re = fma(b.re, c.re, a.re);
  a.re = fma(b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im);
  a.im = fma(-b.im, c.re, a.im);
  return a;
}

template <int P>
struct Real {
  typedef float T;
};
template <>
struct Real<P64> {
  typedef double T;
};

// Storage precision of BiCGStab's shadow residual r-hat for inner fields of
// precision P: FP16 (with its per-site norm) under FP32 and FP16 fields.
// r-hat is any fixed vector with <r-hat, r0> != 0 and is only read in inner
// products, so storing it rounded changes which fixed vector it is, not the
// method; FP64 fields keep it in FP64.
template <int P>
struct ShadowPrec {
  static constexpr int value = P == P64 ? P64 : P16;
};

// Accumulator of the inner iteration's fused sums (the BiCGStab inner
// products and norms reduced in the operator and update kernels) for fields
// of real type R. FP64 fields sum in FP64. FP32 and FP16 fields sum in FP32
// per thread and per warp and in FP64 across warps; a build with
// -DSQ_INNER_SUMS_FP64 sums them in FP64 from the thread level up.
template <typename R>
struct SumOf {
  typedef R T;
};
#ifdef SQ_INNER_SUMS_FP64
template <>
struct SumOf<float> {
  typedef double T;
};
#endif

// ---------------------------------------------------------------------------
// lattice geometry
// ---------------------------------------------------------------------------
struct Geom {
  int X, Y, Z, T;
  int X2;      // X / 2
  int Vh;      // sites per parity
  double tbc;  // factor on the fermion hop across the time boundary
};

struct Coord {
  int x, y, z, t;
};

__device__ __forceinline__ Coord cb_coords(const Geom& g, int cb, int parity) {
  Coord c;
  int xh = cb % g.X2;
  int r = cb / g.X2;
  c.y = r % g.Y;
  r /= g.Y;
  c.z = r % g.Z;
  c.t = r / g.Z;
  c.x = 2 * xh + ((c.y + c.z + c.t + parity) & 1);
  return c;
}

__device__ __forceinline__ int cb_of(const Geom& g, int x, int y, int z, int t) {
  return (x + g.X * (y + g.Y * (z + g.Z * t))) >> 1;
}

// neighbour of c one step in direction mu (dir = +1 or -1), with wrap
__device__ __forceinline__ Coord step(const Geom& g, Coord c, int mu, int dir) {
  if (mu == 0) {
    c.x += dir;
    c.x = c.x < 0 ? g.X - 1 : (c.x >= g.X ? 0 : c.x);
  } else if (mu == 1) {
    c.y += dir;
    c.y = c.y < 0 ? g.Y - 1 : (c.y >= g.Y ? 0 : c.y);
  } else if (mu == 2) {
    c.z += dir;
    c.z = c.z < 0 ? g.Z - 1 : (c.z >= g.Z ? 0 : c.z);
  } else {
    c.t += dir;
    c.t = c.t < 0 ? g.T - 1 : (c.t >= g.T ? 0 : c.t);
  }
  return c;
}

// ---------------------------------------------------------------------------
// even-odd spinor fields (layout documented in include/stochq.h)
// ---------------------------------------------------------------------------
struct Field {
  void* data;   // chunk array
  float* norm;  // FP16 only: per (source, site) scale
  int Vh;
};

template <int P>
struct SpinorIO;

template <>
struct SpinorIO<P64> {
  static constexpr int NC = 12;
  static __device__ __forceinline__ void round_trip(cx<double>*) {}  // stored exactly
  static __device__ __forceinline__ void load(const Field& f, int k, int cb, cx<double> v[12]) {
    const double2* p = (const double2*)f.data + (size_t)k * 12 * f.Vh + cb;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      double2 q = __ldg(p + (size_t)c * f.Vh);
      v[c] = mk(q.x, q.y);
    }
  }
  static __device__ __forceinline__ void store(const Field& f, int k, int cb, const cx<double> v[12]) {
    double2* p = (double2*)f.data + (size_t)k * 12 * f.Vh + cb;
#pragma unroll
    for (int c = 0; c < 12; c++) p[(size_t)c * f.Vh] = make_double2(v[c].re, v[c].im);
  }
};

template <>
struct SpinorIO<P32> {
  static constexpr int NC = 6;
  static __device__ __forceinline__ void load(const Field& f, int k, int cb, cx<float> v[12]) {
    const float4* p = (const float4*)f.data + (size_t)k * 6 * f.Vh + cb;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      float4 q = __ldg(p + (size_t)c * f.Vh);
      v[2 * c] = mk(q.x, q.y);
      v[2 * c + 1] = mk(q.z, q.w);
    }
  }
  static __device__ __forceinline__ void store(const Field& f, int k, int cb, const cx<float> v[12]) {
    float4* p = (float4*)f.data + (size_t)k * 6 * f.Vh + cb;
#pragma unroll
    for (int c = 0; c < 6; c++)
      p[(size_t)c * f.Vh] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
  }
};

__device__ __forceinline__ float2 h2f(uint32_t u) {
  __half2 h = *reinterpret_cast<__half2*>(&u);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

template <>
struct SpinorIO<P16> {
  static constexpr int NC = 3;
  static __device__ __forceinline__ void load(const Field& f, int k, int cb, cx<float> v[12]) {
    const uint4* p = (const uint4*)f.data + (size_t)k * 3 * f.Vh + cb;
    float s = __ldg(f.norm + (size_t)k * f.Vh + cb);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 q = __ldg(p + (size_t)c * f.Vh);
      float2 a = h2f(q.x), b = h2f(q.y), d = h2f(q.z), e = h2f(q.w);
      v[4 * c + 0] = mk(a.x * s, a.y * s);
      v[4 * c + 1] = mk(b.x * s, b.y * s);
      v[4 * c + 2] = mk(d.x * s, d.y * s);
      v[4 * c + 3] = mk(e.x * s, e.y * s);
    }
  }
  // values as stored (no norm applied); returns the site's norm: a linear
  // stencil applies it once to its result instead of to all 24 inputs
  static __device__ __forceinline__ float load_raw(const Field& f, int k, int cb, cx<float> v[12]) {
    const uint4* p = (const uint4*)f.data + (size_t)k * 3 * f.Vh + cb;
    const float s = __ldg(f.norm + (size_t)k * f.Vh + cb);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 q = __ldg(p + (size_t)c * f.Vh);
      float2 a = h2f(q.x), b = h2f(q.y), d = h2f(q.z), e = h2f(q.w);
      v[4 * c + 0] = mk(a.x, a.y);
      v[4 * c + 1] = mk(b.x, b.y);
      v[4 * c + 2] = mk(d.x, d.y);
      v[4 * c + 3] = mk(e.x, e.y);
    }
    return s;
  }
  static __device__ __forceinline__ void store(const Field& f, int k, int cb, const cx<float> v[12]) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 12; j++) m = fmaxf(m, fmaxf(fabsf(v[j].re), fabsf(v[j].im)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* p = (uint4*)f.data + (size_t)k * 3 * f.Vh + cb;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 q;
      q.x = f2h(v[4 * c + 0].re * inv, v[4 * c + 0].im * inv);
      q.y = f2h(v[4 * c + 1].re * inv, v[4 * c + 1].im * inv);
      q.z = f2h(v[4 * c + 2].re * inv, v[4 * c + 2].im * inv);
      q.w = f2h(v[4 * c + 3].re * inv, v[4 * c + 3].im * inv);
      p[(size_t)c * f.Vh] = q;
    }
    f.norm[(size_t)k * f.Vh + cb] = m;
  }
  // the values that a store followed by a load gives back, without memory
  static __device__ __forceinline__ void round_trip(cx<float> v[12]) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 12; j++) m = fmaxf(m, fmaxf(fabsf(v[j].re), fabsf(v[j].im)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
    for (int j = 0; j < 12; j++) {
      const float2 a = h2f(f2h(v[j].re * inv, v[j].im * inv));
      v[j] = mk(a.x * m, a.y * m);
    }
  }
};

// ---------------------------------------------------------------------------
// gauge links, per parity p of the site the link leaves from, direction mu
//   FP64 recon-18: double2 [p][mu][9][Vh]
//   FP32 recon-12: float4  [p][mu][3][Vh]  (complex 2c, 2c+1 of rows 0,1)
//   FP32 recon-18: float2  [p][mu][9][Vh]
// (FP16 fields are hopped with the FP32 links.)
// Row-major complex index a*3+b. Reconstruct-12 keeps rows 0 and 1 and
// rebuilds row 2 = conj(row0 x row1), exact for SU(3).
// ---------------------------------------------------------------------------
template <typename R>
struct Link {
  cx<R> e[9];
};

template <typename R>
__device__ __forceinline__ void reconstruct_row2(Link<R>& u) {
  u.e[6] = conj(u.e[1] * u.e[5] - u.e[2] * u.e[4]);
  u.e[7] = conj(u.e[2] * u.e[3] - u.e[0] * u.e[5]);
  u.e[8] = conj(u.e[0] * u.e[4] - u.e[1] * u.e[3]);
}

template <int P, int RECON>
struct LinkIO;

template <>
struct LinkIO<P64, 18> {
  static __device__ __forceinline__ void load(const void* base, int Vh, int p, int mu, int cb, Link<double>& u) {
    const double2* q = (const double2*)base + ((size_t)(p * 4 + mu) * 9) * Vh + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      double2 a = __ldg(q + (size_t)c * Vh);
      u.e[c] = mk(a.x, a.y);
    }
  }
};

template <>
struct LinkIO<P32, 12> {
  static __device__ __forceinline__ void load(const void* base, int Vh, int p, int mu, int cb, Link<float>& u) {
    const float4* q = (const float4*)base + ((size_t)(p * 4 + mu) * 3) * Vh + cb;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float4 a = __ldg(q + (size_t)c * Vh);
      u.e[2 * c] = mk(a.x, a.y);
      u.e[2 * c + 1] = mk(a.z, a.w);
    }
    reconstruct_row2(u);
  }
};

template <>
struct LinkIO<P32, 18> {
  static __device__ __forceinline__ void load(const void* base, int Vh, int p, int mu, int cb, Link<float>& u) {
    const float2* q = (const float2*)base + ((size_t)(p * 4 + mu) * 9) * Vh + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      float2 a = __ldg(q + (size_t)c * Vh);
      u.e[c] = mk(a.x, a.y);
    }
  }
};


// ---------------------------------------------------------------------------
// clover blocks: per site two 6x6 Hermitian blocks (chirality 0: spins 0,1;
// chirality 1: spins 2,3), row index 3*(spin mod 2) + colour. Packed as 36
// reals per block: 6 real diagonals, then the 15 strictly-lower entries
// (i>j, row by row: 10,20,21,30,31,32,40,...,54) as (re, im). 72 reals/site:
//   FP64: double2 [p][36][Vh]   FP32: float4 [p][18][Vh]
// (FP16 fields use the FP32 blocks.)
// ---------------------------------------------------------------------------
template <int P>
struct CloverIO;

template <>
struct CloverIO<P64> {
  template <int CH>
  static __device__ __forceinline__ void load_block(const void* base, int Vh, int p, int cb, double a[36]) {
    const double2* q = (const double2*)base + ((size_t)p * 36 + CH * 18) * Vh + cb;
#pragma unroll
    for (int c = 0; c < 18; c++) {
      double2 v = __ldg(q + (size_t)c * Vh);
      a[2 * c] = v.x;
      a[2 * c + 1] = v.y;
    }
  }
};

template <>
struct CloverIO<P32> {
  template <int CH>
  static __device__ __forceinline__ void load_block(const void* base, int Vh, int p, int cb, float a[36]) {
    const float4* q = (const float4*)base + ((size_t)p * 18 + CH * 9) * Vh + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      float4 v = __ldg(q + (size_t)c * Vh);
      a[4 * c] = v.x;
      a[4 * c + 1] = v.y;
      a[4 * c + 2] = v.z;
      a[4 * c + 3] = v.w;
    }
  }
};


// off-diagonal packed index of (i, j), i > j
__host__ __device__ constexpr int tri(int i, int j) { return i * (i - 1) / 2 + j; }

// w = B v for one packed Hermitian 6x6 block
template <typename R>
__device__ __forceinline__ void herm6_apply(const R a[36], const cx<R> v[6], cx<R> w[6]) {
#pragma unroll
  for (int i = 0; i < 6; i++) w[i] = a[i] * v[i];
#pragma unroll
  for (int i = 1; i < 6; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      cx<R> l = mk(a[6 + 2 * tri(i, j)], a[6 + 2 * tri(i, j) + 1]);
      w[i] = cfma(l, v[j], w[i]);   // L_ij v_j
      w[j] = cjfma(l, v[i], w[j]);  // conj(L_ij) v_i
    }
  }
}

// ---------------------------------------------------------------------------
// deterministic reductions (fixed tree for a fixed block shape)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sq

// G0 spinor layout conversion, G3 precision conversion, G4 fused BiCGStab
// vector updates and G5 deterministic per-source reductions.
//
// Every kernel here is a streaming pass over even-odd fields: one thread per
// (checkerboard site, source slot), 16-byte chunk loads and stores that are
// contiguous across a warp, and the source slots taken from the solver's
// active / update lists so that retired sources cost nothing.
#include "sq_internal.h"

namespace sq {

// ---------------------------------------------------------------------------
// lexicographic FP64 <-> even-odd field of any precision
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_pack(Geom g, Field out, const double* lex, int parity, int n) {
  typedef typename Real<P>::T R;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (cb >= g.Vh || k >= n) return;
  Coord c = cb_coords(g, cb, parity);
  size_t site = (size_t)c.x + (size_t)g.X * (c.y + (size_t)g.Y * (c.z + (size_t)g.Z * c.t));
  const double2* src = (const double2*)lex + ((size_t)k * 2 * g.Vh + site) * 12;
  cx<R> v[12];
#pragma unroll
  for (int j = 0; j < 12; j++) {
    double2 q = src[j];
    v[j] = mk((R)q.x, (R)q.y);
  }
  SpinorIO<P>::store(out, k, cb, v);
}

template <int P>
__global__ void k_unpack(Geom g, double* lex, Field in, int parity, int n) {
  typedef typename Real<P>::T R;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (cb >= g.Vh || k >= n) return;
  Coord c = cb_coords(g, cb, parity);
  size_t site = (size_t)c.x + (size_t)g.X * (c.y + (size_t)g.Y * (c.z + (size_t)g.Z * c.t));
  double2* dst = (double2*)lex + ((size_t)k * 2 * g.Vh + site) * 12;
  cx<R> v[12];
  SpinorIO<P>::load(in, k, cb, v);
#pragma unroll
  for (int j = 0; j < 12; j++) dst[j] = make_double2((double)v[j].re, (double)v[j].im);
}

// FP64 packing with the per-source squared norm of the packed field, in the
// grid and reduction order of k_norm2<P64> (bitwise the same sums)
__global__ void __launch_bounds__(128) k_pack_norm2(Geom g, Field out, const double* lex, int parity, int n,
                                                   RedArgs ra) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y < n ? (int)blockIdx.y : -1;
  double v[1] = {0.0};
  if (k >= 0 && cb < g.Vh) {
    Coord c = cb_coords(g, cb, parity);
    size_t site = (size_t)c.x + (size_t)g.X * (c.y + (size_t)g.Y * (c.z + (size_t)g.Z * c.t));
    const double2* src = (const double2*)lex + ((size_t)k * 2 * g.Vh + site) * 12;
    cx<double> a[12];
#pragma unroll
    for (int j = 0; j < 12; j++) {
      const double2 q = src[j];
      a[j] = mk(q.x, q.y);
    }
    SpinorIO<P64>::store(out, k, cb, a);
    double t = 0;
#pragma unroll
    for (int j = 0; j < 12; j++) t += (double)a[j].re * a[j].re + (double)a[j].im * a[j].im;
    v[0] = t;
  }
  reduce_finalize<1, FIN_STORE>(ra, v, k, (int)gridDim.x, (int)blockIdx.x);
}

void launch_pack_norm2(const sq_ctx* c, Field out, const double* lex, int parity, int n, double* norm, RedArgs ra,
                       cudaStream_t s) {
  ra.out = norm;
  dim3 grid((c->Vh + 127) / 128, n);
  k_pack_norm2<<<grid, 128, 0, s>>>(geom_of(c), out, lex, parity, n, ra);
}

void launch_pack(const sq_ctx* c, Field out, const double* lex, int parity, int prec, int n, cudaStream_t s) {
  Geom g = geom_of(c);
  dim3 grid((c->Vh + 127) / 128, n);
  if (prec == P64) k_pack<P64><<<grid, 128, 0, s>>>(g, out, lex, parity, n);
  else if (prec == P32) k_pack<P32><<<grid, 128, 0, s>>>(g, out, lex, parity, n);
  else k_pack<P16><<<grid, 128, 0, s>>>(g, out, lex, parity, n);
}

void launch_unpack(const sq_ctx* c, double* lex, Field in, int parity, int prec, int n, cudaStream_t s) {
  Geom g = geom_of(c);
  dim3 grid((c->Vh + 127) / 128, n);
  if (prec == P64) k_unpack<P64><<<grid, 128, 0, s>>>(g, lex, in, parity, n);
  else if (prec == P32) k_unpack<P32><<<grid, 128, 0, s>>>(g, lex, in, parity, n);
  else k_unpack<P16><<<grid, 128, 0, s>>>(g, lex, in, parity, n);
}

// ---------------------------------------------------------------------------
// FP64 site-local clover: out = c1 x + c2 (C in), C = A or A^{-1}
// ---------------------------------------------------------------------------
__global__ void k_clover64(int Vh, Field out, Field x, Field in, const double2* C, int parity,
                           double c1, double c2, int n) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (cb >= Vh || k >= n) return;
  cx<double> v[12], w[12];
  SpinorIO<P64>::load(in, k, cb, v);
  double blk[36];
  CloverIO<P64>::load_block<0>(C, Vh, parity, cb, blk);
  herm6_apply(blk, v, w);
  CloverIO<P64>::load_block<1>(C, Vh, parity, cb, blk);
  herm6_apply(blk, v + 6, w + 6);
  if (x.data) {
    cx<double> xv[12];
    SpinorIO<P64>::load(x, k, cb, xv);
#pragma unroll
    for (int j = 0; j < 12; j++) w[j] = mk(c1 * xv[j].re + c2 * w[j].re, c1 * xv[j].im + c2 * w[j].im);
  } else {
#pragma unroll
    for (int j = 0; j < 12; j++) w[j] = c2 * w[j];
  }
  SpinorIO<P64>::store(out, k, cb, w);
}

void launch_clover64(const sq_ctx* c, const CloverSet& cs, Field out, Field x, Field in, int parity,
                     double c1, double c2, int which, int n, cudaStream_t s) {
  dim3 grid((c->Vh + 127) / 128, n);
  k_clover64<<<grid, 128, 0, s>>>(c->Vh, out, x, in, which ? cs.Ainv64 : cs.A64, parity, c1, c2, n);
}

// ---------------------------------------------------------------------------
// per-source squared norms
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) k_norm2(int Vh, Field f, int n, RedArgs ra) {
  typedef typename Real<P>::T R;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int ky = (int)(blockIdx.y * blockDim.y + threadIdx.y);
  const int k = ky < n ? ky : -1;
  double v[1] = {0.0};
  if (k >= 0 && cb < Vh) {
    cx<R> a[12];
    SpinorIO<P>::load(f, k, cb, a);
    double t = 0;
#pragma unroll
    for (int j = 0; j < 12; j++) t += (double)a[j].re * a[j].re + (double)a[j].im * a[j].im;
    v[0] = t;
  }
  reduce_finalize<1, FIN_STORE>(ra, v, k, (int)gridDim.x, (int)blockIdx.x);
}

void launch_norm2(const sq_ctx* c, Field f, int prec, int n, double* out, RedArgs ra, cudaStream_t s) {
  ra.out = out;
  dim3 grid((c->Vh + 127) / 128, n);
  if (prec == P64) k_norm2<P64><<<grid, 128, 0, s>>>(c->Vh, f, n, ra);
  else if (prec == P32) k_norm2<P32><<<grid, 128, 0, s>>>(c->Vh, f, n, ra);
  else k_norm2<P16><<<grid, 128, 0, s>>>(c->Vh, f, n, ra);
}

}  // namespace sq

// Vector kernels of the non-domain-decomposed comparison solver: BiCGstab in FP64, or in
// FP32 inside an FP64 Richardson iteration (the standard solvers the paper's domain
// decomposition is measured against, Sec. IV-C, Table III).
//
// Fields are in the internal layout; a 16-byte unit is a float4 (two complex numbers) in
// FP32 and a double2 (one complex number) in FP64.  The scalars of the recurrence live in
// device memory (FP64 complex), so an iteration needs no host round trip until its
// residual norm is read.  Inner products: per-thread sums in the unit's precision, block
// and grid sums in FP64, in a fixed order.
#include <type_traits>

#include "dd_kernels.hpp"

namespace dd {

namespace {
constexpr int KT = 256;

__device__ inline double2 cdot_acc(double2 s, double2 a, double2 b) {   // s + conj(a) b
  return make_double2(s.x + a.x * b.x + a.y * b.y, s.y + a.x * b.y - a.y * b.x);
}
__device__ inline double2 cdot_acc(double2 s, float4 a, float4 b) {
  const float re = a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
  const float im = a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
  return make_double2(s.x + re, s.y + im);
}

// y + c x for one unit, c complex
__device__ inline double2 caxpy(double2 y, zd c, double2 x) {
  return make_double2(y.x + c.re * x.x - c.im * x.y, y.y + c.re * x.y + c.im * x.x);
}
__device__ inline float4 caxpy(float4 y, zd cd, float4 x) {
  const float cr = (float)cd.re, ci = (float)cd.im;
  return make_float4(y.x + cr * x.x - ci * x.y, y.y + cr * x.y + ci * x.x, y.z + cr * x.z - ci * x.w,
                     y.w + cr * x.w + ci * x.z);
}
__device__ inline double norm2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline double norm2(float4 a) { return (double)(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w); }

__device__ inline void block_sum2(double2& a, double2& b, double2* out) {
  __shared__ double2 sh[KT / 32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
    b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
  }
  if (lane == 0) { sh[w][0] = a; sh[w][1] = b; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double2 t = make_double2(0, 0);
    for (int k = 0; k < KT / 32; ++k) { t.x += sh[k][threadIdx.x].x; t.y += sh[k][threadIdx.x].y; }
    out[threadIdx.x] = t;
  }
}
}  // namespace

// partial[blk][0] = sum conj(a) b, partial[blk][1] = sum conj(c) d (c, d may be null).
template <typename U>
__global__ void __launch_bounds__(KT) bicg_dot2_kernel(const U* a, const U* b, const U* c, const U* d, long long n,
                                                       double2* partial) {
  double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
  for (long long q = blockIdx.x * (long long)KT + threadIdx.x; q < n; q += (long long)gridDim.x * KT) {
    s0 = cdot_acc(s0, a[q], b[q]);
    if (c) s1 = cdot_acc(s1, c[q], d[q]);
  }
  __shared__ double2 out[2];
  block_sum2(s0, s1, out);
  if (threadIdx.x == 0) {
    partial[2 * (long long)blockIdx.x] = out[0];
    partial[2 * (long long)blockIdx.x + 1] = out[1];
  }
}

// Scalars of one BiCGstab recurrence, sc[]: 0 rho, 1 alpha, 2 omega, 3 beta, 4 <rhat, r>,
// 5 <rhat, v>, 6 <t, s>, 7 <t, t>, 8 |r|^2 (re), 9 restart flag (re).
//   stage 0: beta = (<rhat, r> / rho) (alpha / omega), rho = <rhat, r>
//   stage 1: alpha = rho / <rhat, v>
//   stage 2: omega = <t, s> / <t, t>
// A vanishing or non-finite denominator sets the restart flag (the host then restarts the
// recurrence with rhat = r).
__global__ void bicg_scalars_kernel(zd* sc, int stage) {
  auto bad = [](zd z) { return !(abs2(z) > 0.0) || !isfinite(z.re) || !isfinite(z.im); };
  if (stage == 0) {
    if (bad(sc[0]) || bad(sc[2]) || bad(sc[4])) { sc[9] = Z(1.0); sc[3] = Z(0.0); return; }
    sc[3] = zdiv(sc[4], sc[0]) * zdiv(sc[1], sc[2]);
    sc[0] = sc[4];
  } else if (stage == 1) {
    if (bad(sc[5])) { sc[9] = Z(1.0); sc[1] = Z(0.0); return; }
    sc[1] = zdiv(sc[0], sc[5]);
  } else {
    if (bad(sc[7])) { sc[9] = Z(1.0); sc[2] = Z(0.0); return; }
    sc[2] = zdiv(sc[6], sc[7]);
  }
}

// rho = alpha = omega = 1, flag = 0
__global__ void bicg_reset_kernel(zd* sc) {
  sc[0] = sc[1] = sc[2] = Z(1.0);
  sc[3] = Z(0.0);
  sc[9] = Z(0.0);
}

// p = r + beta (p - omega v)
template <typename U>
__global__ void __launch_bounds__(KT) bicg_p_kernel(U* p, const U* r, const U* v, const zd* sc, long long n) {
  const zd beta = sc[3], bw = Z(0.0) - sc[3] * sc[2];
  for (long long q = blockIdx.x * (long long)KT + threadIdx.x; q < n; q += (long long)gridDim.x * KT) {
    U t = caxpy(r[q], beta, p[q]);
    p[q] = caxpy(t, bw, v[q]);
  }
}

// s = r - alpha v
template <typename U>
__global__ void __launch_bounds__(KT) bicg_s_kernel(U* s, const U* r, const U* v, const zd* sc, long long n) {
  const zd ma = Z(0.0) - sc[1];
  for (long long q = blockIdx.x * (long long)KT + threadIdx.x; q < n; q += (long long)gridDim.x * KT)
    s[q] = caxpy(r[q], ma, v[q]);
}

// x += alpha p + omega s; r = s - omega t; partial[blk] = |r|^2 over the block's share
template <typename U>
__global__ void __launch_bounds__(KT) bicg_xr_kernel(U* x, U* r, const U* p, const U* s, const U* t, const zd* sc,
                                                    long long n, double2* partial) {
  const zd al = sc[1], om = sc[2], mom = Z(0.0) - sc[2];
  double2 n2 = make_double2(0, 0), dummy = make_double2(0, 0);
  for (long long q = blockIdx.x * (long long)KT + threadIdx.x; q < n; q += (long long)gridDim.x * KT) {
    const U sq = s[q];
    x[q] = caxpy(caxpy(x[q], al, p[q]), om, sq);
    const U rq = caxpy(sq, mom, t[q]);
    r[q] = rq;
    n2.x += norm2(rq);
  }
  __shared__ double2 out[2];
  block_sum2(n2, dummy, out);
  if (threadIdx.x == 0) {
    partial[2 * (long long)blockIdx.x] = out[0];
    partial[2 * (long long)blockIdx.x + 1] = make_double2(0, 0);
  }
}

// dst = src (units), and zero-fill when src is null
template <typename U>
__global__ void __launch_bounds__(KT) bicg_copy_kernel(U* dst, const U* src, long long n) {
  for (long long q = blockIdx.x * (long long)KT + threadIdx.x; q < n; q += (long long)gridDim.x * KT) {
    U z;
    memset(&z, 0, sizeof(U));
    dst[q] = src ? src[q] : z;
  }
}

// sc[slot] = sum over blocks of partial[blk][0] (and sc[slot + 1] of [1] when two).
__global__ void bicg_reduce_kernel(const double2* partial, int nb, zd* sc, int slot, int two) {
  __shared__ double sh[4][256];
  double a = 0, b = 0, c = 0, d = 0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    a += partial[2 * k].x;
    b += partial[2 * k].y;
    c += partial[2 * k + 1].x;
    d += partial[2 * k + 1].y;
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  sh[3][threadIdx.x] = d;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int e = 0; e < 4; ++e) sh[e][threadIdx.x] += sh[e][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc[slot] = Z(sh[0][0], sh[1][0]);
    if (two) sc[slot + 1] = Z(sh[2][0], sh[3][0]);
  }
}

// ---------------------------------------------------------------- launchers
template <typename U>
static long long units(const Geom& g) {
  return std::is_same<U, float4>::value ? g.V * 6 : g.V * 12;
}

template <typename U>
void BicgKernels<U>::dot(const Geom& g, const U* a, const U* b, const U* c, const U* d, double2* partial, zd* sc,
                         int slot, cudaStream_t st) {
  const int nb = blas_partials_blocks();
  bicg_dot2_kernel<U><<<nb, KT, 0, st>>>(a, b, c, d, units<U>(g), partial);
  bicg_reduce_kernel<<<1, 256, 0, st>>>(partial, nb, sc, slot, c ? 1 : 0);
}
template <typename U>
void BicgKernels<U>::p_update(const Geom& g, U* p, const U* r, const U* v, const zd* sc, cudaStream_t st) {
  bicg_p_kernel<U><<<blas_partials_blocks(), KT, 0, st>>>(p, r, v, sc, units<U>(g));
}
template <typename U>
void BicgKernels<U>::s_update(const Geom& g, U* s, const U* r, const U* v, const zd* sc, cudaStream_t st) {
  bicg_s_kernel<U><<<blas_partials_blocks(), KT, 0, st>>>(s, r, v, sc, units<U>(g));
}
template <typename U>
void BicgKernels<U>::xr_update(const Geom& g, U* x, U* r, const U* p, const U* s, const U* t, zd* sc, double2* partial,
                               cudaStream_t st) {
  const int nb = blas_partials_blocks();
  bicg_xr_kernel<U><<<nb, KT, 0, st>>>(x, r, p, s, t, sc, units<U>(g), partial);
  bicg_reduce_kernel<<<1, 256, 0, st>>>(partial, nb, sc, 8, 0);
}
template <typename U>
void BicgKernels<U>::copy(const Geom& g, U* dst, const U* src, cudaStream_t st) {
  bicg_copy_kernel<U><<<blas_partials_blocks(), KT, 0, st>>>(dst, src, units<U>(g));
}

template struct BicgKernels<float4>;
template struct BicgKernels<double2>;

void launch_bicg_scalars(zd* sc, int stage, cudaStream_t st) { bicg_scalars_kernel<<<1, 1, 0, st>>>(sc, stage); }
void launch_bicg_reset(zd* sc, cudaStream_t st) { bicg_reset_kernel<<<1, 1, 0, st>>>(sc); }

}  // namespace dd

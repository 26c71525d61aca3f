// Vector kernels of the outer solver on FP32 (float4 = two complex numbers) and FP64
// (double2 = one complex number) fields in the internal layout.
//
// Inner products: every thread sums its share of the products in FP32 (a few hundred
// terms at most), converts once, and the block and grid reductions run in FP64.  The
// grid is a fixed multiple of the SM count, so the order of the final FP64 sum is
// fixed and the result is reproducible run to run.
#include "dd_kernels.hpp"

namespace dd {

constexpr int BT = 256;           // threads per block
constexpr int NCHUNK = 8;         // vectors per pass of the multi-dot
static int g_blocks = 0;

int blas_partials_blocks() {
  if (!g_blocks) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_blocks = 4 * (sms > 0 ? sms : 1);
  }
  return g_blocks;
}

__device__ inline cx<float> dot4(float4 v, float4 w) {  // conj(v) . w over two complex numbers
  return mk(v.x * w.x + v.y * w.y + v.z * w.z + v.w * w.w, v.x * w.y - v.y * w.x + v.z * w.w - v.w * w.z);
}

// Basis vectors in FP32 (float4: two complex numbers) or FP16 (uint2: the same two complex
// numbers as two half2); every kernel that reads or writes a basis does its arithmetic in
// FP32 on float4 values.
__device__ inline float4 ldv(const float4* p, long long q) { return p[q]; }
__device__ inline float4 ldv(const uint2* p, long long q) {
  const uint2 u = p[q];
  const float2 a = h2f(u.x), b = h2f(u.y);
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ inline void stv(float4* p, long long q, float4 v, float s) {
  p[q] = make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
}
__device__ inline void stv(uint2* p, long long q, float4 v, float s) {
  p[q] = make_uint2(f2h(v.x * s, v.y * s), f2h(v.z * s, v.w * s));
}

// Block reduction of NV complex doubles; thread 0 of the block ends with the sums in s[].
template <int NV>
__device__ inline void block_reduce(double2 (&v)[NV], double2* s_out) {
  __shared__ double2 sh[BT / 32][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v[i].x += __shfl_xor_sync(0xffffffffu, v[i].x, o);
      v[i].y += __shfl_xor_sync(0xffffffffu, v[i].y, o);
    }
    if (lane == 0) sh[w][i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double2 t = make_double2(0, 0);
    for (int k = 0; k < BT / 32; ++k) { t.x += sh[k][threadIdx.x].x; t.y += sh[k][threadIdx.x].y; }
    s_out[threadIdx.x] = t;
  }
  __syncthreads();
}

// partial[blockIdx][v0 + i] = sum over this block's share of conj(V_{v0+i}) . w
template <int NV>
__global__ void __launch_bounds__(BT) multi_dot_kernel(const float4* V, int v0, int nv, long long n4, const float4* w,
                                                       double2* partial, int ldp) {
  float re[NV], im[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) re[i] = im[i] = 0.f;
  for (long long q = blockIdx.x * (long long)BT + threadIdx.x; q < n4; q += (long long)gridDim.x * BT) {
    float4 wq = w[q];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (v0 + i < nv) {
        cx<float> d = dot4(V[(long long)(v0 + i) * n4 + q], wq);
        re[i] += d.re;
        im[i] += d.im;
      }
    }
  }
  double2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = make_double2(re[i], im[i]);
  __shared__ double2 out[NV];
  block_reduce<NV>(acc, out);
  if (threadIdx.x < NV && v0 + (int)threadIdx.x < nv) partial[(long long)blockIdx.x * ldp + v0 + threadIdx.x] = out[threadIdx.x];
}

int launch_multi_dot(const float4* V, int nv, long long n4, const float4* w, double2* partial, cudaStream_t st) {
  int nb = blas_partials_blocks(), n = 0;
  for (int v0 = 0; v0 < nv; v0 += NCHUNK, ++n) multi_dot_kernel<NCHUNK><<<nb, BT, 0, st>>>(V, v0, nv, n4, w, partial, nv);
  return n;
}

// out[i] (+)= sum over blocks of partial[b][i], fixed order.
__global__ void reduce_partials_kernel(const double2* partial, int nb, int nv, double2* out, int accumulate) {
  int i = blockIdx.x;
  double sx = 0, sy = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) { sx += partial[(long long)b * nv + i].x; sy += partial[(long long)b * nv + i].y; }
  __shared__ double shx[256], shy[256];
  shx[threadIdx.x] = sx;
  shy[threadIdx.x] = sy;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { shx[threadIdx.x] += shx[threadIdx.x + o]; shy[threadIdx.x] += shy[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (accumulate) { out[i].x += shx[0]; out[i].y += shy[0]; }
    else out[i] = make_double2(shx[0], shy[0]);
  }
}

void launch_reduce_partials(const double2* partial, int nv, double2* out, int accumulate, cudaStream_t st) {
  reduce_partials_kernel<<<nv, 256, 0, st>>>(partial, blas_partials_blocks(), nv, out, accumulate);
}

// |x|^2 of an FP64 field (double2 units); exact FP64 arithmetic throughout.
__global__ void __launch_bounds__(BT) norm2_64_kernel(const double2* x, long long n2, double2* partial) {
  double s = 0;
  for (long long q = blockIdx.x * (long long)BT + threadIdx.x; q < n2; q += (long long)gridDim.x * BT) {
    double2 a = x[q];
    s += a.x * a.x + a.y * a.y;
  }
  double2 acc[1] = {make_double2(s, 0.0)};
  __shared__ double2 out[1];
  block_reduce<1>(acc, out);
  if (threadIdx.x == 0) partial[blockIdx.x] = out[0];
}
void launch_norm2_64(const double2* x, long long n2, double2* partial, cudaStream_t st) {
  norm2_64_kernel<<<blas_partials_blocks(), BT, 0, st>>>(x, n2, partial);
}

// x += sum_i y_i Z_i (Z FP32, x FP64): the sum is formed in FP32, added in FP64.
__global__ void __launch_bounds__(BT) x_update_kernel(double2* x, const float4* Z, int nz, long long n4, const double2* y) {
  __shared__ float2 ys[64];
  if (threadIdx.x < nz) ys[threadIdx.x] = make_float2((float)y[threadIdx.x].x, (float)y[threadIdx.x].y);
  __syncthreads();
  for (long long q = blockIdx.x * (long long)BT + threadIdx.x; q < n4; q += (long long)gridDim.x * BT) {
    float4 a = make_float4(0, 0, 0, 0);
    for (int i = 0; i < nz; ++i) {
      float4 v = Z[(long long)i * n4 + q];
      float2 c = ys[i];
      a.x += c.x * v.x - c.y * v.y;
      a.y += c.x * v.y + c.y * v.x;
      a.z += c.x * v.z - c.y * v.w;
      a.w += c.x * v.w + c.y * v.z;
    }
    double2 x0 = x[2 * q], x1 = x[2 * q + 1];
    x[2 * q] = make_double2(x0.x + a.x, x0.y + a.y);
    x[2 * q + 1] = make_double2(x1.x + a.z, x1.y + a.w);
  }
}
void launch_x_update(double2* x, const float4* Z, int nz, long long n4, const double2* y, cudaStream_t st) {
  x_update_kernel<<<blas_partials_blocks(), BT, 0, st>>>(x, Z, nz, n4, y);
}

// v = r / sqrt(nrm2) in FP32 (the FP64 and FP32 layouts hold the same complex numbers
// in the same order: double2 unit 2q and 2q+1 <-> float4 unit q).
__global__ void r64_to_v32_kernel(float4* v, const double2* r, long long n4, const double2* nrm2, const int* gate) {
  if (gate && *gate != 1) return;
  double s = 1.0 / sqrt(nrm2->x);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    double2 a = r[2 * q], b = r[2 * q + 1];
    v[q] = make_float4((float)(a.x * s), (float)(a.y * s), (float)(b.x * s), (float)(b.y * s));
  }
}
void launch_r64_to_v32(float4* v, const double2* r, long long n4, const double2* nrm2, cudaStream_t st,
                       const int* gate) {
  r64_to_v32_kernel<<<blas_partials_blocks(), BT, 0, st>>>(v, r, n4, nrm2, gate);
}

// out_l = sum_i P[i + l ldp] V_i for l < nout (P complex FP64, column-major).  One pass
// produces NO outputs (instantiated for every count up to 16, so a deflated restart with
// k <= 15 reads each basis once and holds no unused accumulators); each loop trip issues
// RU independent input loads per thread, which is what keeps HBM busy here.  out may be
// V itself (in-place recombination): a thread reads all inputs at q before it writes
// the outputs at q, and no other thread touches q.
constexpr int RBT = 128, RU = 8;
template <int NO, typename VT>
__global__ void __launch_bounds__(RBT) recombine_kernel(VT* out, const VT* V, int nv, int l0, long long n4,
                                                        const double2* P, int ldp, const int* gate,
                                                        const float* vscale, float oscale) {
  if (gate && *gate != 1) return;
  __shared__ float2 ps[64][NO];
  for (int t = threadIdx.x; t < nv * NO; t += RBT) {
    int i = t / NO, l = t % NO;
    const double2 c = P[i + (long long)(l0 + l) * ldp];
    const double sc = vscale ? (double)vscale[i] : 1.0;   // stored V_i = v_i / vscale[i]
    ps[i][l] = make_float2((float)(c.x * sc), (float)(c.y * sc));
  }
  __syncthreads();
  for (long long q = blockIdx.x * (long long)RBT + threadIdx.x; q < n4; q += (long long)gridDim.x * RBT) {
    float4 a[NO];
#pragma unroll
    for (int l = 0; l < NO; ++l) a[l] = make_float4(0, 0, 0, 0);
    auto fma_in = [&](int i, float4 v) {
#pragma unroll
      for (int l = 0; l < NO; ++l) {
        float2 c = ps[i][l];
        a[l].x += c.x * v.x - c.y * v.y;
        a[l].y += c.x * v.y + c.y * v.x;
        a[l].z += c.x * v.z - c.y * v.w;
        a[l].w += c.x * v.w + c.y * v.z;
      }
    };
    int i = 0;
    for (; i + RU <= nv; i += RU) {
      float4 v[RU];
#pragma unroll
      for (int u = 0; u < RU; ++u) v[u] = ldv(V, (long long)(i + u) * n4 + q);
#pragma unroll
      for (int u = 0; u < RU; ++u) fma_in(i + u, v[u]);
    }
    for (; i < nv; ++i) fma_in(i, ldv(V, (long long)i * n4 + q));
#pragma unroll
    for (int l = 0; l < NO; ++l) stv(out, (long long)(l0 + l) * n4 + q, a[l], oscale);
  }
}

template <int NO, typename VT>
static void recombine_launch(int nl, VT* out, const VT* V, int nv, int l0, long long n4, const double2* P, int ldp,
                             cudaStream_t st, const int* gate, const float* vscale, float oscale) {
  if constexpr (NO > 1) {
    if (nl < NO) return recombine_launch<NO - 1, VT>(nl, out, V, nv, l0, n4, P, ldp, st, gate, vscale, oscale);
  }
  recombine_kernel<NO, VT><<<2 * blas_partials_blocks(), RBT, 0, st>>>(out, V, nv, l0, n4, P, ldp, gate, vscale,
                                                                      oscale);
}

int launch_recombine(float4* out, const float4* V, int nv, int nout, long long n4, const double2* P, int ldp,
                     cudaStream_t st, const int* gate, const float* vscale) {
  int n = 0;
  for (int l0 = 0; l0 < nout; l0 += 16, ++n)
    recombine_launch<16, float4>(nout - l0 < 16 ? nout - l0 : 16, out, V, nv, l0, n4, P, ldp, st, gate, vscale, 1.f);
  return n;
}

int launch_recombine(uint2* out, const uint2* V, int nv, int nout, long long n4, const double2* P, int ldp,
                     cudaStream_t st, const int* gate, const float* vscale, float oscale) {
  int n = 0;
  for (int l0 = 0; l0 < nout; l0 += 16, ++n)
    recombine_launch<16, uint2>(nout - l0 < 16 ? nout - l0 : 16, out, V, nv, l0, n4, P, ldp, st, gate, vscale,
                                oscale);
  return n;
}

// ------------------------------------------------------------------ Gram-Schmidt passes
// Classical Gram-Schmidt with selective reorthogonalisation, gated on the device so no
// host round trip is needed.  Pass 1 forms h = V^H w and |w|^2 in one read of the basis;
// the projection pass writes w - V h and its exact squared norm; a second projection runs
// only when the first cancelled more than half of |w|^2.
//
// One launch covers every basis vector.  Block b takes the chunk b % nch of NV vectors
// and the q-slice b / nch, so blocks that read the same elements of w are adjacent in
// launch order and all but the first find them in L2.  Each loop trip handles U elements
// per vector, (NV + 1) * U independent 16-byte loads per thread, which keeps enough bytes
// in flight for HBM even for the short last chunk.
template <int NV, int U>
__global__ void __launch_bounds__(BT, 2) gs_dot_kernel(const float4* __restrict__ V, int nv, int nch, long long n4,
                                                       const float4* __restrict__ w, double2* partial, int ldp,
                                                       const int* gate, int want, const float* vscale) {
  if (gate && *gate != want) return;
  const int chunk = blockIdx.x % nch, qb = blockIdx.x / nch, nqb = gridDim.x / nch;
  const int v0 = chunk * NV, nvc = min(NV, nv - v0);
  const bool self = chunk == 0;
  float re[NV], im[NV], ww = 0.f;
#pragma unroll
  for (int i = 0; i < NV; ++i) re[i] = im[i] = 0.f;
  const long long stride = (long long)nqb * BT;
  const float4* Vc = V + (long long)v0 * n4;
  long long q = (long long)qb * BT + threadIdx.x;
  for (; q + (U - 1) * stride < n4; q += U * stride) {
    float4 wq[U], vq[NV][U];
#pragma unroll
    for (int u = 0; u < U; ++u) wq[u] = w[q + u * stride];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvc)
#pragma unroll
        for (int u = 0; u < U; ++u) vq[i][u] = ldv(Vc, (long long)i * n4 + q + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (self) ww += wq[u].x * wq[u].x + wq[u].y * wq[u].y + wq[u].z * wq[u].z + wq[u].w * wq[u].w;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nvc) {
          cx<float> d = dot4(vq[i][u], wq[u]);
          re[i] += d.re;
          im[i] += d.im;
        }
    }
  }
  for (; q < n4; q += stride) {
    float4 wq = w[q];
    if (self) ww += wq.x * wq.x + wq.y * wq.y + wq.z * wq.z + wq.w * wq.w;
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvc) {
        cx<float> d = dot4(ldv(Vc, (long long)i * n4 + q), wq);
        re[i] += d.re;
        im[i] += d.im;
      }
  }
  double2 acc[NV + 1];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    // stored V_i = v_i / vscale[i]: the product with v_i is the stored one times vscale[i]
    const double sc = (vscale && i < nvc) ? (double)vscale[v0 + i] : 1.0;
    acc[i] = make_double2(re[i] * sc, im[i] * sc);
  }
  acc[NV] = make_double2(ww, 0.0);
  __shared__ double2 out[NV + 1];
  block_reduce<NV + 1>(acc, out);
  if ((int)threadIdx.x < nvc) partial[(long long)qb * ldp + v0 + threadIdx.x] = out[threadIdx.x];
  if (self && threadIdx.x == 0) partial[(long long)qb * ldp + nv] = out[NV];
}

// partial layout [q-slice][nv + 1]: entries 0..nv-1 are V^H w, entry nv is |w|^2.
int launch_gs_dot(const float4* V, int nv, long long n4, const float4* w, double2* partial, const int* gate, int want,
                  cudaStream_t st, const float* vscale) {
  const int nch = nv > 0 ? (nv + 7) / 8 : 1;
  gs_dot_kernel<8, 2><<<blas_partials_blocks() * nch, BT, 0, st>>>(V, nv, nch, n4, w, partial, nv + 1, gate, want,
                                                                   vscale);
  return 1;
}

// The FP16-basis forms read the basis in 16-byte loads of two units (four complex numbers)
// and w as the matching two float4, so each load moves as many bytes as in the FP32 forms.
__device__ inline void unpack_pair(uint4 u, float4& lo, float4& hi) {
  const float2 a = h2f(u.x), b = h2f(u.y), c = h2f(u.z), d = h2f(u.w);
  lo = make_float4(a.x, a.y, b.x, b.y);
  hi = make_float4(c.x, c.y, d.x, d.y);
}

template <int NV, int U>
__global__ void __launch_bounds__(BT, 2) gs_dot16_kernel(const uint4* __restrict__ V, int nv, int nch, long long n8,
                                                         const float4* __restrict__ w, double2* partial, int ldp,
                                                         const int* gate, int want, const float* vscale) {
  if (gate && *gate != want) return;
  const int chunk = blockIdx.x % nch, qb = blockIdx.x / nch, nqb = gridDim.x / nch;
  const int v0 = chunk * NV, nvc = min(NV, nv - v0);
  const bool self = chunk == 0;
  float re[NV], im[NV], ww = 0.f;
#pragma unroll
  for (int i = 0; i < NV; ++i) re[i] = im[i] = 0.f;
  const long long stride = (long long)nqb * BT;
  const uint4* Vc = V + (long long)v0 * n8;
  for (long long q = (long long)qb * BT + threadIdx.x; q < n8; q += U * stride) {
    float4 wl[U], wh[U];
    uint4 vq[NV][U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long e = q + u * stride;
      ok[u] = e < n8;
      wl[u] = ok[u] ? w[2 * e] : make_float4(0.f, 0.f, 0.f, 0.f);
      wh[u] = ok[u] ? w[2 * e + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvc)
#pragma unroll
        for (int u = 0; u < U; ++u) vq[i][u] = ok[u] ? Vc[(long long)i * n8 + q + u * stride] : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (self)
        ww += wl[u].x * wl[u].x + wl[u].y * wl[u].y + wl[u].z * wl[u].z + wl[u].w * wl[u].w +
              wh[u].x * wh[u].x + wh[u].y * wh[u].y + wh[u].z * wh[u].z + wh[u].w * wh[u].w;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nvc) {
          float4 lo, hi;
          unpack_pair(vq[i][u], lo, hi);
          const cx<float> d0 = dot4(lo, wl[u]), d1 = dot4(hi, wh[u]);
          re[i] += d0.re + d1.re;
          im[i] += d0.im + d1.im;
        }
    }
  }
  double2 acc[NV + 1];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double sc = (vscale && i < nvc) ? (double)vscale[v0 + i] : 1.0;
    acc[i] = make_double2(re[i] * sc, im[i] * sc);
  }
  acc[NV] = make_double2(ww, 0.0);
  __shared__ double2 out[NV + 1];
  block_reduce<NV + 1>(acc, out);
  if ((int)threadIdx.x < nvc) partial[(long long)qb * ldp + v0 + threadIdx.x] = out[threadIdx.x];
  if (self && threadIdx.x == 0) partial[(long long)qb * ldp + nv] = out[NV];
}

int launch_gs_dot(const uint2* V, int nv, long long n4, const float4* w, double2* partial, const int* gate, int want,
                  cudaStream_t st, const float* vscale) {
  const int nch = nv > 0 ? (nv + 7) / 8 : 1;
  // n4 is even (six units per site): the basis is read as n4 / 2 pairs of units
  gs_dot16_kernel<8, 2><<<blas_partials_blocks() * nch, BT, 0, st>>>(reinterpret_cast<const uint4*>(V), nv, nch,
                                                                     n4 / 2, w, partial, nv + 1, gate, want, vscale);
  return 1;
}

__global__ void gs_reduce_kernel(const double2* partial, int nb, int ld, double2* out, const int* gate, int want) {
  if (gate && *gate != want) return;
  int i = blockIdx.x;
  double sx = 0, sy = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) { sx += partial[(long long)b * ld + i].x; sy += partial[(long long)b * ld + i].y; }
  __shared__ double shx[256], shy[256];
  shx[threadIdx.x] = sx;
  shy[threadIdx.x] = sy;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { shx[threadIdx.x] += shx[threadIdx.x + o]; shy[threadIdx.x] += shy[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = make_double2(shx[0], shy[0]);
}

void launch_gs_reduce(const double2* partial, int nv, double2* out, const int* gate, int want, cudaStream_t st) {
  gs_reduce_kernel<<<nv + 1, 256, 0, st>>>(partial, blas_partials_blocks(), nv + 1, out, gate, want);
}

// out = w - V h with |out|^2 partials per block (exact norm of the projected vector).
// in_place: out aliases w (each thread reads w[q] before it writes out[q]).
// Each thread carries GP_U elements and loads GP_B basis vectors for all of them before the
// products, so 8 independent 16-byte loads are in flight per thread (one vector at a time
// reached ~4.9 TB/s; this form reaches the copy bandwidth).  Every element still subtracts
// h_0 v_0, h_1 v_1, ... in that order, so the result does not depend on the unrolling.
constexpr int GP_U = 2, GP_B = 4;
__global__ void __launch_bounds__(BT) gs_project_kernel(float4* out, const float4* w, const float4* __restrict__ V,
                                                        int nv, long long n4, const double2* h,
                                                        double2* norm_partial, const int* gate, int want,
                                                        const float* vscale) {
  if (gate && *gate != want) return;
  __shared__ float2 hs[64];
  for (int i = threadIdx.x; i < nv; i += BT) {
    const double sc = vscale ? (double)vscale[i] : 1.0;   // h_i v_i = (h_i vscale[i]) V_i
    hs[i] = make_float2((float)(h[i].x * sc), (float)(h[i].y * sc));
  }
  __syncthreads();
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long stride = (long long)gridDim.x * BT;
  float nrm = 0.f;
  for (long long q0 = blockIdx.x * (long long)BT + threadIdx.x; q0 < n4; q0 += GP_U * stride) {
    float4 a[GP_U];
    long long q[GP_U];
    bool ok[GP_U];
#pragma unroll
    for (int u = 0; u < GP_U; ++u) {
      q[u] = q0 + u * stride;
      ok[u] = q[u] < n4;
      a[u] = ok[u] ? w[q[u]] : zero;
    }
    int i = 0;
    for (; i + GP_B <= nv; i += GP_B) {
      float4 v[GP_B][GP_U];
#pragma unroll
      for (int b = 0; b < GP_B; ++b)
#pragma unroll
        for (int u = 0; u < GP_U; ++u) v[b][u] = ok[u] ? ldv(V, (long long)(i + b) * n4 + q[u]) : zero;
#pragma unroll
      for (int b = 0; b < GP_B; ++b) {
        const float2 c = hs[i + b];
#pragma unroll
        for (int u = 0; u < GP_U; ++u) {
          a[u].x -= c.x * v[b][u].x - c.y * v[b][u].y;
          a[u].y -= c.x * v[b][u].y + c.y * v[b][u].x;
          a[u].z -= c.x * v[b][u].z - c.y * v[b][u].w;
          a[u].w -= c.x * v[b][u].w + c.y * v[b][u].z;
        }
      }
    }
    for (; i < nv; ++i) {
      const float2 c = hs[i];
#pragma unroll
      for (int u = 0; u < GP_U; ++u) {
        if (!ok[u]) continue;
        const float4 x = ldv(V, (long long)i * n4 + q[u]);
        a[u].x -= c.x * x.x - c.y * x.y;
        a[u].y -= c.x * x.y + c.y * x.x;
        a[u].z -= c.x * x.z - c.y * x.w;
        a[u].w -= c.x * x.w + c.y * x.z;
      }
    }
#pragma unroll
    for (int u = 0; u < GP_U; ++u)
      if (ok[u]) {
        out[q[u]] = a[u];
        nrm += a[u].x * a[u].x + a[u].y * a[u].y + a[u].z * a[u].z + a[u].w * a[u].w;
      }
  }
  double2 acc[1] = {make_double2(nrm, 0.0)};
  __shared__ double2 o[1];
  block_reduce<1>(acc, o);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = o[0];
}

void launch_gs_project(float4* out, const float4* w, const float4* V, int nv, long long n4, const double2* h,
                       double2* norm_partial, const int* gate, int want, cudaStream_t st, const float* vscale) {
  gs_project_kernel<<<blas_partials_blocks(), BT, 0, st>>>(out, w, V, nv, n4, h, norm_partial, gate, want, vscale);
}

// out = w - V h over an FP16 basis read in unit pairs (see gs_dot16_kernel); in place
// allowed (out aliases w).
__global__ void __launch_bounds__(BT) gs_project16_kernel(float4* out, const float4* w, const uint4* __restrict__ V,
                                                          int nv, long long n8, const double2* h,
                                                          double2* norm_partial, const int* gate, int want,
                                                          const float* vscale) {
  if (gate && *gate != want) return;
  __shared__ float2 hs[64];
  for (int i = threadIdx.x; i < nv; i += BT) {
    const double sc = vscale ? (double)vscale[i] : 1.0;
    hs[i] = make_float2((float)(h[i].x * sc), (float)(h[i].y * sc));
  }
  __syncthreads();
  auto sub = [](float4& a, float2 c, float4 v) {
    a.x -= c.x * v.x - c.y * v.y;
    a.y -= c.x * v.y + c.y * v.x;
    a.z -= c.x * v.z - c.y * v.w;
    a.w -= c.x * v.w + c.y * v.z;
  };
  const long long stride = (long long)gridDim.x * BT;
  float nrm = 0.f;
  for (long long q0 = blockIdx.x * (long long)BT + threadIdx.x; q0 < n8; q0 += GP_U * stride) {
    float4 al[GP_U], ah[GP_U];
    long long q[GP_U];
    bool ok[GP_U];
#pragma unroll
    for (int u = 0; u < GP_U; ++u) {
      q[u] = q0 + u * stride;
      ok[u] = q[u] < n8;
      al[u] = ok[u] ? w[2 * q[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
      ah[u] = ok[u] ? w[2 * q[u] + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int i = 0;
    for (; i + GP_B <= nv; i += GP_B) {
      uint4 v[GP_B][GP_U];
#pragma unroll
      for (int b = 0; b < GP_B; ++b)
#pragma unroll
        for (int u = 0; u < GP_U; ++u) v[b][u] = ok[u] ? V[(long long)(i + b) * n8 + q[u]] : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int b = 0; b < GP_B; ++b) {
        const float2 c = hs[i + b];
#pragma unroll
        for (int u = 0; u < GP_U; ++u) {
          float4 lo, hi;
          unpack_pair(v[b][u], lo, hi);
          sub(al[u], c, lo);
          sub(ah[u], c, hi);
        }
      }
    }
    for (; i < nv; ++i) {
      const float2 c = hs[i];
#pragma unroll
      for (int u = 0; u < GP_U; ++u) {
        if (!ok[u]) continue;
        float4 lo, hi;
        unpack_pair(V[(long long)i * n8 + q[u]], lo, hi);
        sub(al[u], c, lo);
        sub(ah[u], c, hi);
      }
    }
#pragma unroll
    for (int u = 0; u < GP_U; ++u)
      if (ok[u]) {
        out[2 * q[u]] = al[u];
        out[2 * q[u] + 1] = ah[u];
        nrm += al[u].x * al[u].x + al[u].y * al[u].y + al[u].z * al[u].z + al[u].w * al[u].w +
               ah[u].x * ah[u].x + ah[u].y * ah[u].y + ah[u].z * ah[u].z + ah[u].w * ah[u].w;
      }
  }
  double2 acc[1] = {make_double2(nrm, 0.0)};
  __shared__ double2 o[1];
  block_reduce<1>(acc, o);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = o[0];
}

void launch_gs_project(float4* out, const float4* w, const uint2* V, int nv, long long n4, const double2* h,
                       double2* norm_partial, const int* gate, int want, cudaStream_t st, const float* vscale) {
  gs_project16_kernel<<<blas_partials_blocks(), BT, 0, st>>>(out, w, reinterpret_cast<const uint4*>(V), nv, n4 / 2, h,
                                                             norm_partial, gate, want, vscale);
}

// v16 = FP16 of s w / sqrt(*nu2) and v32 = w / sqrt(*nu2) (the FP32 copy the next Schwarz
// application reads); with a gate, only when *gate == 1.
__global__ void basis16_store_kernel(uint2* v16, float4* v32, const float4* w, long long n4, const double* nu2,
                                     float s, const int* gate) {
  if (gate && *gate != 1) return;
  const float inv = (float)(1.0 / sqrt(*nu2));
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    const float4 a = w[q];
    const float4 v = make_float4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
    if (v32) v32[q] = v;
    stv(v16, q, v, s);
  }
}
void launch_basis16_store(uint2* v16, float4* v32, const float4* w, long long n4, const double* nu2, float s,
                          cudaStream_t st, const int* gate) {
  basis16_store_kernel<<<blas_partials_blocks(), BT, 0, st>>>(v16, v32, w, n4, nu2, s, gate);
}

// v32 = FP32 of v16 * s
__global__ void basis16_load_kernel(float4* v32, const uint2* v16, long long n4, float s) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    const float4 a = ldv(v16, q);
    v32[q] = make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
  }
}
void launch_basis16_load(float4* v32, const uint2* v16, long long n4, float s, cudaStream_t st) {
  basis16_load_kernel<<<blas_partials_blocks(), BT, 0, st>>>(v32, v16, n4, s);
}

// v *= 1 / sqrt(*nu2)
__global__ void scale_inplace_kernel(float4* v, long long n4, const double* nu2) {
  float s = (float)(1.0 / sqrt(*nu2));
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    float4 a = v[q];
    v[q] = make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
  }
}
void launch_scale_inplace(float4* v, long long n4, const double* nu2, cudaStream_t st) {
  scale_inplace_kernel<<<blas_partials_blocks(), BT, 0, st>>>(v, n4, nu2);
}

}  // namespace dd

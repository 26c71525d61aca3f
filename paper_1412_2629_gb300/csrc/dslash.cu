// Full-lattice Wilson-clover operator A = 1/(2 kappa) - 1/2 D_w + D_cl (Eq. 1-3).
//
// One thread per site in the domain-major layout: consecutive threads are consecutive
// sites of one parity of one domain, so the site's own spinor, links and clover are read
// with fully coalesced 16-byte (8- or 4-byte for links) loads, and most neighbours are
// adjacent sites of the other parity (read through L1/L2).  Hops that leave the domain
// go to the neighbouring domain's block; the antiperiodic time boundary is already in
// the links.  The diagonal 1/(2 kappa) is folded into the stored clover.
// Bytes per site (algorithmic, each field read once): 4 links + clover + in + out =
// 192 reals; FP32 768 B, FP64 1536 B, FP16 384 B + 8 B of spinor norms.
#include <type_traits>

#include "dd_kernels.hpp"

namespace dd {

template <int MU, typename T>
__device__ inline void hop_pair(const Geom& g, const Site& st, long long s, const SpinorPtr<T>& in,
                                const LinkPtr<T>& U, Spinor<typename Arith<T>::type>& acc) {
  typedef typename Arith<T>::type R;
  Spinor<R> psi;
  Half<R> h, uh;
  Link<R> L;
  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
  long long sf = neighbour(g, st, MU, +1);
  in.load(g, sf, psi);
  project<MU, -1>(psi, h);
  U.load(g, s, MU, L);
  su3_mul(L, h, uh);
  accum_recon<MU, -1>(acc, uh);
  // backward: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
  long long sb = neighbour(g, st, MU, -1);
  in.load(g, sb, psi);
  project<MU, +1>(psi, h);
  U.load(g, sb, MU, L);
  su3_dag_mul(L, h, uh);
  accum_recon<MU, +1>(acc, uh);
}

template <typename T>
__global__ void __launch_bounds__(256) apply_A_kernel(Geom g, LinkPtr<T> U, CloverPtr<T> C, SpinorPtr<T> in,
                                                       SpinorPtr<T> out, SpinorPtr<T> f, int residual) {
  typedef typename Arith<T>::type R;
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Site st = decode(g, s);
  Spinor<R> hop;
  zero(hop);
  hop_pair<0, T>(g, st, s, in, U, hop);
  hop_pair<1, T>(g, st, s, in, U, hop);
  hop_pair<2, T>(g, st, s, in, U, hop);
  hop_pair<3, T>(g, st, s, in, U, hop);
  Spinor<R> x, y;
  in.load(g, s, x);
  R m[72];
  C.load(g, s, m);
  clover_mul(m, x, y);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) y.c[a][b] = y.c[a][b] - R(0.5) * hop.c[a][b];
  if (residual) {
    Spinor<R> fv;
    f.load(g, s, fv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) y.c[a][b] = fv.c[a][b] - y.c[a][b];
  }
  out.store(g, s, y);
}

// ------------------------------------------------------------------ FP32, shape known at compile time
// The same one-thread-per-site operator for FP32 fields with the domain shape as
// compile-time constants (SHAPE 1: 8x4x4x4, 2: 4x4x4x4): the site decoding and every
// neighbour and unit address then fold into shifts and immediate offsets, which takes the
// integer work off the issue slots that the loads need.  Two CTAs of 256 per SM: the
// compiler may then use 128 registers, and spends them on keeping more of the neighbour
// and link loads in flight (measured 20 % faster than the same code at 88 registers).
template <int SHAPE>
__global__ void __launch_bounds__(256, 2) apply_A_shape_kernel(Geom g0, LinkPtr<float> U, CloverPtr<float> C,
                                                            SpinorPtr<float> in, SpinorPtr<float> out,
                                                            SpinorPtr<float> f, int residual) {
  const Geom g = fixed_shape<SHAPE>(g0);
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Site st = decode(g, s);
  Spinor<float> hop;
  zero(hop);
  hop_pair<0, float>(g, st, s, in, U, hop);
  hop_pair<1, float>(g, st, s, in, U, hop);
  hop_pair<2, float>(g, st, s, in, U, hop);
  hop_pair<3, float>(g, st, s, in, U, hop);
  Spinor<float> x, y;
  in.load(g, s, x);
  float m[72];
  C.load(g, s, m);
  clover_mul(m, x, y);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) y.c[a][b] = y.c[a][b] - 0.5f * hop.c[a][b];
  if (residual) {
    Spinor<float> fv;
    f.load(g, s, fv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) y.c[a][b] = fv.c[a][b] - y.c[a][b];
  }
  out.store(g, s, y);
}

void launch_apply_A(const Geom& g, GaugeView U, CloverView C, FieldView in, FieldView out, const FieldView* f,
                    cudaStream_t st) {
  unsigned nb = (unsigned)((g.V + 255) / 256);
  int res = f != nullptr;
  if (in.prec == P32 && domain_shape_id(g) != 0) {
    const LinkPtr<float> L{(const float2*)U.links};
    const CloverPtr<float> Cp{(const float4*)C.m};
    const SpinorPtr<float> vi{(float4*)in.data}, vo{(float4*)out.data}, fi{res ? (float4*)f->data : nullptr};
    if (domain_shape_id(g) == 1) apply_A_shape_kernel<1><<<nb, 256, 0, st>>>(g, L, Cp, vi, vo, fi, res);
    else apply_A_shape_kernel<2><<<nb, 256, 0, st>>>(g, L, Cp, vi, vo, fi, res);
    return;
  }
  if (in.prec == P64) {
    SpinorPtr<double> fi{res ? (double2*)f->data : nullptr};
    apply_A_kernel<double><<<nb, 256, 0, st>>>(g, LinkPtr<double>{(const double2*)U.links},
                                               CloverPtr<double>{(const double2*)C.m},
                                               SpinorPtr<double>{(double2*)in.data},
                                               SpinorPtr<double>{(double2*)out.data}, fi, res);
  } else if (in.prec == P32) {
    SpinorPtr<float> fi{res ? (float4*)f->data : nullptr};
    apply_A_kernel<float><<<nb, 256, 0, st>>>(g, LinkPtr<float>{(const float2*)U.links},
                                              CloverPtr<float>{(const float4*)C.m},
                                              SpinorPtr<float>{(float4*)in.data}, SpinorPtr<float>{(float4*)out.data},
                                              fi, res);
  } else {
    SpinorPtr<__half> fi{res ? (uint4*)f->data : nullptr, res ? f->norm : nullptr};
    apply_A_kernel<__half><<<nb, 256, 0, st>>>(g, LinkPtr<__half>{(const uint32_t*)U.links},
                                               CloverPtr<__half>{(const uint4*)C.m},
                                               SpinorPtr<__half>{(uint4*)in.data, in.norm},
                                               SpinorPtr<__half>{(uint4*)out.data, out.norm}, fi, res);
  }
}

}  // namespace dd

namespace dd {

// ------------------------------------------------------------------ several right-hand sides
__device__ inline void shift_norm(SpinorPtr<float>&, long long) {}
__device__ inline void shift_norm(SpinorPtr<__half>& p, long long d) { p.norm += d; }

// Thread per site, NR right-hand sides per thread: every link and the clover block are
// loaded once and applied to NR spinors, so per right-hand side the operator moves
// (4 links + clover) / NR + in + out bytes instead of all 192 reals.
template <int MU, typename T, int NR>
__device__ inline void hop_pair_multi(const Geom& g, const Site& st, long long s, const SpinorPtr<T>* in,
                                      const LinkPtr<T>& U, Spinor<typename Arith<T>::type>* acc) {
  typedef typename Arith<T>::type R;
  Spinor<R> psi;
  Half<R> h, uh;
  Link<R> L;
  long long sf = neighbour(g, st, MU, +1);
  U.load(g, s, MU, L);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    in[r].load(g, sf, psi);
    project<MU, -1>(psi, h);
    su3_mul(L, h, uh);
    accum_recon<MU, -1>(acc[r], uh);
  }
  long long sb = neighbour(g, st, MU, -1);
  U.load(g, sb, MU, L);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    in[r].load(g, sb, psi);
    project<MU, +1>(psi, h);
    su3_dag_mul(L, h, uh);
    accum_recon<MU, +1>(acc[r], uh);
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(128) apply_A_multi_kernel(Geom g, LinkPtr<T> U, CloverPtr<T> C, SpinorPtr<T> in0,
                                                             SpinorPtr<T> out0, long long unit_stride,
                                                             long long norm_stride, int nrhs,
                                                             const float4* const* in_list, float4* const* out_list) {
  typedef typename Arith<T>::type R;
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int r0 = blockIdx.y * NR;
  SpinorPtr<T> in[NR], out[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    int rr = r0 + r < nrhs ? r0 + r : nrhs - 1;   // a short last group repeats the last field
    in[r] = in0;
    out[r] = out0;
    in[r].p += rr * unit_stride;
    out[r].p += rr * unit_stride;
    shift_norm(in[r], rr * norm_stride);
    shift_norm(out[r], rr * norm_stride);
    if constexpr (std::is_same<T, float>::value) {
      if (in_list) {   // FP32 fields anywhere in memory
        in[r].p = const_cast<float4*>(in_list[rr]);
        out[r].p = out_list[rr];
      }
    }
  }
  Site st = decode(g, s);
  Spinor<R> acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) zero(acc[r]);
  hop_pair_multi<0, T, NR>(g, st, s, in, U, acc);
  hop_pair_multi<1, T, NR>(g, st, s, in, U, acc);
  hop_pair_multi<2, T, NR>(g, st, s, in, U, acc);
  hop_pair_multi<3, T, NR>(g, st, s, in, U, acc);
  R m[72];
  C.load(g, s, m);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r0 + r >= nrhs) break;
    Spinor<R> x, y;
    in[r].load(g, s, x);
    clover_mul(m, x, y);
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 3; ++b2) y.c[a2][b2] = y.c[a2][b2] - R(0.5) * acc[r].c[a2][b2];
    out[r].store(g, s, y);
  }
}

void launch_apply_A_multi(const Geom& g, GaugeView U, CloverView C, FieldView in, FieldView out, int nrhs,
                          cudaStream_t st) {
  const int NR = 2;
  dim3 grid((unsigned)((g.V + 127) / 128), (unsigned)((nrhs + NR - 1) / NR));
  if (in.prec == P32) {
    apply_A_multi_kernel<float, NR><<<grid, 128, 0, st>>>(
        g, LinkPtr<float>{(const float2*)U.links}, CloverPtr<float>{(const float4*)C.m},
        SpinorPtr<float>{(float4*)in.data}, SpinorPtr<float>{(float4*)out.data}, g.V * 6, 0, nrhs, nullptr, nullptr);
  } else {
    // FP16 fields are V * 52 bytes each (values, then the per-site norms) and follow each
    // other: 13 V / 4 uint4 units or 13 V floats apart (V is a multiple of 64)
    apply_A_multi_kernel<__half, NR><<<grid, 128, 0, st>>>(
        g, LinkPtr<__half>{(const uint32_t*)U.links}, CloverPtr<__half>{(const uint4*)C.m},
        SpinorPtr<__half>{(uint4*)in.data, in.norm}, SpinorPtr<__half>{(uint4*)out.data, out.norm}, 13 * g.V / 4,
        13 * g.V, nrhs, nullptr, nullptr);
  }
}

void launch_apply_A_multi_list(const Geom& g, GaugeView U, CloverView C, const float4* const* in,
                               float4* const* out, int nrhs, cudaStream_t st) {
  const int NR = 2;
  dim3 grid((unsigned)((g.V + 127) / 128), (unsigned)((nrhs + NR - 1) / NR));
  apply_A_multi_kernel<float, NR><<<grid, 128, 0, st>>>(
      g, LinkPtr<float>{(const float2*)U.links}, CloverPtr<float>{(const float4*)C.m}, SpinorPtr<float>{nullptr},
      SpinorPtr<float>{nullptr}, 0, 0, nrhs, in, out);
}

}  // namespace dd

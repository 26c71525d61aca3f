// Two-level aggregation multigrid with the Schwarz method as its smoother (the use of
// domain-decomposition preconditioners that the paper's related work, Sec. V, points to:
// aggregation-based algebraic multigrid whose smoother is a Schwarz method).
//
// Aggregates are the Schwarz domains.  Each aggregate and chirality (spins 0, 1 and 2, 3:
// gamma_5 = +1 / -1 in the chiral basis) carries n_tv coarse degrees of freedom, so the
// interpolation P commutes with gamma_5 and the coarse operator D_c = P^H A P is a
// nearest-neighbour stencil on the lattice of domains.
//
// Layouts (device memory):
//   P: n_tv FP32 fields in the internal layout, one after another (stride n4 float4).
//      Field k holds column (chirality 0, k) in units 0-2 (spins 0, 1) and column
//      (chirality 1, k) in units 3-5 (spins 2, 3) of every domain: the two columns have
//      disjoint supports.  A domain's chirality-c piece is 3 Vd consecutive float4.
//   coarse vectors: complex FP32 (float2) [domain][chirality][k], nc = 2 n_tv per domain.
//   D_c: float2 [domain][dir][j][i] with dir 0 = the domain itself, 1 + 2 mu = its +mu
//      neighbour, 2 + 2 mu = its -mu neighbour; (D_c x)_(d, i) = sum_dir sum_j
//      D_c[d][dir][j][i] x_(nb(d, dir), j).  With two domains in a direction the +mu and
//      -mu neighbours coincide and both blocks act on the same coarse site.
#include "dd_kernels.hpp"

namespace dd {

constexpr int MGT = 256;   // threads per block of the restriction / prolongation kernels

// conj(p) . v over the two complex numbers of a float4 unit
__device__ inline void cdot_acc(float& re, float& im, float4 p, float4 v) {
  re += p.x * v.x + p.y * v.y + p.z * v.z + p.w * v.w;
  im += p.x * v.y - p.y * v.x + p.z * v.w - p.w * v.z;
}

// Sum of n <= N complex values over the block (blockDim.x a multiple of 32, <= 1024);
// thread t < n receives total t in (sr, si).  Every thread must call it.
template <int N>
__device__ inline void block_sum_cplx(float (&re)[N], float (&im)[N], int n, float& sr, float& si) {
  __shared__ float2 sh[32][N];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i >= n) break;
    float a = re[i], b = im[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) sh[w][i] = make_float2(a, b);
  }
  __syncthreads();
  sr = si = 0.f;
  if ((int)threadIdx.x < n) {
    for (int q = 0; q < nw; ++q) {
      sr += sh[q][threadIdx.x].x;
      si += sh[q][threadIdx.x].y;
    }
  }
  __syncthreads();
}

// FP64 complex sum over the block, returned to every thread.
__device__ inline double2 block_sum_d2(double2 v) {
  __shared__ double2 sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  for (int q = 0; q < nw; ++q) { t.x += sh[q].x; t.y += sh[q].y; }
  __syncthreads();
  return t;
}

// ------------------------------------------------------------------ restriction / prolongation
// rc_(d, c, k) = sum over the domain's chirality-c piece of conj(P_k) . in, times *vscale
// when given.  One block per (domain, chirality).
__global__ void __launch_bounds__(MGT) mg_restrict_kernel(const float4* __restrict__ in, const float4* __restrict__ P,
                                                          int ntv, long long n4, int lgVd, float2* rc,
                                                          const float* vscale) {
  const int d = blockIdx.x >> 1, chi = blockIdx.x & 1;
  const long long base = ((long long)d * 6 + 3 * chi) << lgVd;
  const int len = 3 << lgVd;
  float re[MG_MAXTV], im[MG_MAXTV];
#pragma unroll
  for (int k = 0; k < MG_MAXTV; ++k) re[k] = im[k] = 0.f;
  for (int e = threadIdx.x; e < len; e += MGT) {
    const float4 v = in[base + e];
#pragma unroll
    for (int k = 0; k < MG_MAXTV; ++k)
      if (k < ntv) cdot_acc(re[k], im[k], P[k * n4 + base + e], v);
  }
  float sr, si;
  block_sum_cplx<MG_MAXTV>(re, im, ntv, sr, si);
  if ((int)threadIdx.x < ntv) {
    const float sc = vscale ? *vscale : 1.f;
    rc[((long long)d * 2 + chi) * ntv + threadIdx.x] = make_float2(sc * sr, sc * si);
  }
}

// out = P ec over the domain's chirality-c piece.  One block per (domain, chirality).
__global__ void __launch_bounds__(MGT) mg_prolong_kernel(const float2* ec, const float4* __restrict__ P, int ntv,
                                                         long long n4, int lgVd, float4* out) {
  const int d = blockIdx.x >> 1, chi = blockIdx.x & 1;
  const long long base = ((long long)d * 6 + 3 * chi) << lgVd;
  const int len = 3 << lgVd;
  __shared__ float2 es[MG_MAXTV];
  if ((int)threadIdx.x < ntv) es[threadIdx.x] = ec[((long long)d * 2 + chi) * ntv + threadIdx.x];
  __syncthreads();
  for (int e = threadIdx.x; e < len; e += MGT) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < MG_MAXTV; ++k) {
      if (k < ntv) {
        const float4 p = P[k * n4 + base + e];
        const float2 c = es[k];
        a.x += c.x * p.x - c.y * p.y;
        a.y += c.x * p.y + c.y * p.x;
        a.z += c.x * p.z - c.y * p.w;
        a.w += c.x * p.w + c.y * p.z;
      }
    }
    out[base + e] = a;
  }
}

void launch_mg_restrict(const Geom& g, const float4* in, const float4* P, int ntv, float2* rc, const float* vscale,
                        cudaStream_t st) {
  mg_restrict_kernel<<<2 * g.ND, MGT, 0, st>>>(in, P, ntv, g.V * 6, g.lgVd, rc, vscale);
}

void launch_mg_prolong(const Geom& g, const float2* ec, const float4* P, int ntv, float4* out, cudaStream_t st) {
  mg_prolong_kernel<<<2 * g.ND, MGT, 0, st>>>(ec, P, ntv, g.V * 6, g.lgVd, out);
}

// ------------------------------------------------------------------ interpolation (set-up)
// Gram-Schmidt of the test vectors on every (domain, chirality) piece, in order, twice per
// vector (modified Gram-Schmidt, FP64 sums of FP32 values), then normalised: the columns
// of a QR factorisation with positive diagonal.  In place on P.  status[0] is set when a
// piece has no component left (the test vectors are linearly dependent there).
__global__ void __launch_bounds__(MGT) mg_orthonormalize_kernel(float4* P, int ntv, long long n4, int lgVd,
                                                                int* status) {
  const int d = blockIdx.x >> 1, chi = blockIdx.x & 1;
  const long long base = ((long long)d * 6 + 3 * chi) << lgVd;
  const int len = 3 << lgVd;
  for (int k = 0; k < ntv; ++k) {
    float4* pk = P + k * n4 + base;
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < k; ++i) {
        const float4* pi = P + i * n4 + base;
        double2 h = make_double2(0.0, 0.0);
        for (int e = threadIdx.x; e < len; e += MGT) {
          const float4 a = pi[e], b = pk[e];
          h.x += (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z + (double)a.w * b.w;
          h.y += (double)a.x * b.y - (double)a.y * b.x + (double)a.z * b.w - (double)a.w * b.z;
        }
        h = block_sum_d2(h);
        const float hr = (float)h.x, hi = (float)h.y;
        for (int e = threadIdx.x; e < len; e += MGT) {
          const float4 a = pi[e];
          float4 b = pk[e];
          b.x -= hr * a.x - hi * a.y;
          b.y -= hr * a.y + hi * a.x;
          b.z -= hr * a.z - hi * a.w;
          b.w -= hr * a.w + hi * a.z;
          pk[e] = b;
        }
      }
    }
    double2 n2 = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < len; e += MGT) {
      const float4 b = pk[e];
      n2.x += (double)b.x * b.x + (double)b.y * b.y + (double)b.z * b.z + (double)b.w * b.w;
    }
    n2 = block_sum_d2(n2);
    if (!(n2.x > 0.0) || !isfinite(n2.x)) {
      if (threadIdx.x == 0) atomicExch(status, 1);
      return;
    }
    const float s = (float)(1.0 / sqrt(n2.x));
    for (int e = threadIdx.x; e < len; e += MGT) {
      float4 b = pk[e];
      pk[e] = make_float4(b.x * s, b.y * s, b.z * s, b.w * s);
    }
  }
}

void launch_mg_orthonormalize(const Geom& g, float4* P, int ntv, int* status, cudaStream_t st) {
  mg_orthonormalize_kernel<<<2 * g.ND, MGT, 0, st>>>(P, ntv, g.V * 6, g.lgVd, status);
}

// ------------------------------------------------------------------ coarse operator (set-up)
// P_k at site s with the spins of the other chirality set to zero: column (chi, k).
__device__ inline void load_column(const Geom& g, const float4* P, long long n4, int k, int chi, long long s,
                                   Spinor<float>& v) {
  const SpinorPtr<float> f{const_cast<float4*>(P + k * n4)};
  f.load(g, s, v);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if ((sp >> 1) != chi) v.c[sp][c] = mk(0.f, 0.f);
}

// acc += (1 - gamma_mu) U_mu(x) psi (forward, psi taken at x + mu) or
// acc += (1 + gamma_mu) U_mu(x - mu)^dag psi (backward, psi taken at sn = x - mu)
template <int MU>
__device__ inline void hop_term(const Geom& g, const LinkPtr<float>& U, long long s, long long sn, int fw,
                                const Spinor<float>& psi, Spinor<float>& acc) {
  Half<float> h, uh;
  Link<float> L;
  if (fw) {
    project<MU, -1>(psi, h);
    U.load(g, s, MU, L);
    su3_mul(L, h, uh);
    accum_recon<MU, -1>(acc, uh);
  } else {
    project<MU, +1>(psi, h);
    U.load(g, sn, MU, L);
    su3_dag_mul(L, h, uh);
    accum_recon<MU, +1>(acc, uh);
  }
}

__device__ inline void hop_term_rt(int mu, const Geom& g, const LinkPtr<float>& U, long long s, long long sn, int fw,
                                   const Spinor<float>& psi, Spinor<float>& acc) {
  switch (mu) {
    case 0: hop_term<0>(g, U, s, sn, fw, psi, acc); break;
    case 1: hop_term<1>(g, U, s, sn, fw, psi, acc); break;
    case 2: hop_term<2>(g, U, s, sn, fw, psi, acc); break;
    default: hop_term<3>(g, U, s, sn, fw, psi, acc); break;
  }
}

// D_c[d][dir][j][:] = P_d^H (A restricted to the coupling dir) P_nb(d,dir) e_j.  One block
// per domain, one thread per site of the domain.  dir 0: the clover term (with 1/(2 kappa))
// and the hops that stay inside the domain; dir 1 + 2 mu / 2 + 2 mu: the hops that cross the
// domain's +mu / -mu face.  FP32 links, clover and arithmetic.
__global__ void __launch_bounds__(512) mg_coarse_build_kernel(Geom g, LinkPtr<float> U, CloverPtr<float> C,
                                                              const float4* P, int ntv, float2* Dc) {
  const long long n4 = g.V * 6;
  const int d = blockIdx.x, r = threadIdx.x, nc = 2 * ntv;
  const long long s = ((long long)d << g.lgVd) + r;
  const Site st = decode(g, s);
  long long nb[8];
  unsigned inside = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    nb[q] = neighbour(g, st, q >> 1, (q & 1) ? -1 : +1);
    if ((nb[q] >> g.lgVd) == d) inside |= 1u << q;
  }
  for (int dir = 0; dir < 9; ++dir) {
    for (int j = 0; j < nc; ++j) {
      const int cj = j / ntv, kj = j % ntv;
      Spinor<float> w;
      zero(w);
      if (dir == 0) {
        Spinor<float> x, hop;
        load_column(g, P, n4, kj, cj, s, x);
        float m[72];
        C.load(g, s, m);
        clover_mul(m, x, w);
        zero(hop);
        for (int q = 0; q < 8; ++q) {
          if (!((inside >> q) & 1u)) continue;
          Spinor<float> psi;
          load_column(g, P, n4, kj, cj, nb[q], psi);
          hop_term_rt(q >> 1, g, U, s, nb[q], !(q & 1), psi, hop);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) w.c[a][b] = w.c[a][b] - 0.5f * hop.c[a][b];
      } else {
        const int q = dir - 1;
        if (!((inside >> q) & 1u)) {
          Spinor<float> psi, hop;
          zero(hop);
          load_column(g, P, n4, kj, cj, nb[q], psi);
          hop_term_rt(q >> 1, g, U, s, nb[q], !(q & 1), psi, hop);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) w.c[a][b] = -0.5f * hop.c[a][b];
        }
      }
      float re[2 * MG_MAXTV], im[2 * MG_MAXTV];
#pragma unroll
      for (int i = 0; i < 2 * MG_MAXTV; ++i) re[i] = im[i] = 0.f;
      for (int i = 0; i < nc; ++i) {
        const int ci = i / ntv, ki = i % ntv;
        Spinor<float> p;
        load_column(g, P, n4, ki, ci, s, p);
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const cx<float> z = cjmul(p.c[sp][c], w.c[sp][c]);
            a += z.re;
            b += z.im;
          }
        // registers indexed at run time: keep the totals in a fixed slot order
#pragma unroll
        for (int t = 0; t < 2 * MG_MAXTV; ++t)
          if (t == i) { re[t] = a; im[t] = b; }
      }
      float sr, si;
      block_sum_cplx<2 * MG_MAXTV>(re, im, nc, sr, si);
      if (r < nc) Dc[(((long long)d * 9 + dir) * nc + j) * nc + r] = make_float2(sr, si);
    }
  }
}

void launch_mg_coarse_build(const Geom& g, const float2* U32, const float4* C32, const float4* P, int ntv, float2* Dc,
                            cudaStream_t st) {
  mg_coarse_build_kernel<<<g.ND, g.Vd, 0, st>>>(g, LinkPtr<float>{U32}, CloverPtr<float>{C32}, P, ntv, Dc);
}

// ------------------------------------------------------------------ coarse operator
// y = D_c x (b == nullptr) or y = b - D_c x; one thread per coarse row (domain, i), for row
// lengths without a compiled nine-thread form below.  Skipped when *gate != 0.
__global__ void __launch_bounds__(256) mg_coarse_apply_kernel(Geom g, const float2* __restrict__ Dc, int nc,
                                                              const float2* __restrict__ x, float2* y,
                                                              const float2* b, const int* gate) {
  if (gate && *gate) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)g.ND * nc) return;
  const int d = (int)(t / nc), i = (int)(t % nc);
  int n[4];
  domain_coords(g, d, n);
  float ar = 0.f, ai = 0.f;
  for (int dir = 0; dir < 9; ++dir) {
    const int dn = dir == 0 ? d : neighbour_domain(g, d, n, (dir - 1) >> 1, ((dir - 1) & 1) ? -1 : +1);
    const float2* D = Dc + ((long long)d * 9 + dir) * nc * nc + i;
    const float2* xv = x + (long long)dn * nc;
    for (int j = 0; j < nc; ++j) {
      const float2 a = D[(long long)j * nc], v = xv[j];
      ar += a.x * v.x - a.y * v.y;
      ai += a.x * v.y + a.y * v.x;
    }
  }
  y[t] = b ? make_float2(b[t].x - ar, b[t].y - ai) : make_float2(ar, ai);
}

// The same product with nine threads per coarse row, one per coupling (dir): one block per
// domain of 9 nc threads (the row length compiled in), each summing NC terms, then the nine
// partial sums of a row added in a fixed order through shared memory.  Nine times the
// threads of the one-thread-per-row form keeps enough loads in flight for short rows.
template <int NC>
__global__ void __launch_bounds__(9 * 32) mg_coarse_apply9_kernel(Geom g, const float2* __restrict__ Dc,
                                                                  const float2* __restrict__ x, float2* y,
                                                                  const float2* b, const int* gate) {
  if (gate && *gate) return;
  __shared__ float2 part[9][NC];
  const int d = blockIdx.x, dir = threadIdx.x / NC, i = threadIdx.x % NC;
  int n[4];
  domain_coords(g, d, n);
  const int dn = dir == 0 ? d : neighbour_domain(g, d, n, (dir - 1) >> 1, ((dir - 1) & 1) ? -1 : +1);
  const float2* D = Dc + ((long long)d * 9 + dir) * NC * NC + i;
  const float2* xv = x + (long long)dn * NC;
  float ar = 0.f, ai = 0.f;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const float2 a = D[(long long)j * NC], v = xv[j];
    ar += a.x * v.x - a.y * v.y;
    ai += a.x * v.y + a.y * v.x;
  }
  part[dir][i] = make_float2(ar, ai);
  __syncthreads();
  if (dir == 0) {
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      sr += part[q][i].x;
      si += part[q][i].y;
    }
    const long long t = (long long)d * NC + i;
    y[t] = b ? make_float2(b[t].x - sr, b[t].y - si) : make_float2(sr, si);
  }
}

void launch_mg_coarse_apply(const Geom& g, const float2* Dc, int nc, const float2* x, float2* y, const float2* b,
                            const int* gate, cudaStream_t st) {
  switch (nc) {
    case 8: mg_coarse_apply9_kernel<8><<<g.ND, 72, 0, st>>>(g, Dc, x, y, b, gate); return;
    case 16: mg_coarse_apply9_kernel<16><<<g.ND, 144, 0, st>>>(g, Dc, x, y, b, gate); return;
    case 24: mg_coarse_apply9_kernel<24><<<g.ND, 216, 0, st>>>(g, Dc, x, y, b, gate); return;
    case 32: mg_coarse_apply9_kernel<32><<<g.ND, 288, 0, st>>>(g, Dc, x, y, b, gate); return;
    default: break;
  }
  const long long n = (long long)g.ND * nc;
  mg_coarse_apply_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, Dc, nc, x, y, b, gate);
}

// ------------------------------------------------------------------ coarse-vector BLAS
// Coarse vectors are short (ND nc complex numbers), so a Gram-Schmidt pass costs mostly
// launches and reductions.  Each pass is one launch: every block stores its partial sums,
// and the last block to finish (a device-scope ticket taken after a fence; nobody waits)
// reduces them in block order in FP64 and runs the pass's scalar step.  The ticket is
// reset by that last block, so consecutive launches on one stream reuse it.
constexpr int CT = 256;

// The Hessenberg column j from the two passes' coefficients and |v_{j+1}|^2, its Givens
// update, and nu = 1 / h_{j+1,j}; a column whose subdiagonal entry vanishes against |w|
// (invariant subspace) is the last one: state[0] = 1 stops the remaining steps.
__device__ inline void hcol_step(zd* R, int ldh, int j, const double2* hA, const double2* hB, double n2,
                                 LsqState* lsq, zd* g, double* nu, int* state) {
  zd* col = R + (long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = Z(hA[i].x + hB[i].x, hA[i].y + hB[i].y);
  const double h = sqrt(fmax(n2, 0.0));
  col[j + 1] = Z(h);
  lsq_add_column(*lsq, R, ldh, j, j + 2, g);
  state[1] = j + 1;
  const double w2 = hA[j + 1].x;   // |w|^2 before the projection
  if (!(h * h > 1e-24 * w2) || !isfinite(h)) state[0] = 1;
  nu[0] = state[0] == 0 ? 1.0 / h : 0.0;
}

// h_out[i] = conj(V_i) . w for i < nv and h_out[nv] = |w|^2 (FP64 over blocks).  partial:
// gridDim.x (nv + 1) double2.  Skipped when *gate != 0.
__global__ void __launch_bounds__(CT) mg_cdot_kernel(const float4* __restrict__ V, int nv, long long n4,
                                                     const float4* __restrict__ w, double2* partial,
                                                     double2* h_out, int* ticket, const int* gate) {
  if (gate && *gate) return;
  const long long stride = (long long)gridDim.x * CT;
  const int ld = nv + 1;
  const int nch = nv > 0 ? (nv + 7) / 8 : 1;
  for (int ch = 0; ch < nch; ++ch) {
    const int v0 = ch * 8, nvc = min(8, nv - v0);
    float re[9], im[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) re[i] = im[i] = 0.f;
    for (long long q = blockIdx.x * (long long)CT + threadIdx.x; q < n4; q += stride) {
      const float4 wq = w[q];
      float4 vq[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < nvc) vq[i] = V[(long long)(v0 + i) * n4 + q];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < nvc) cdot_acc(re[i], im[i], vq[i], wq);
      if (ch == 0) re[8] += wq.x * wq.x + wq.y * wq.y + wq.z * wq.z + wq.w * wq.w;
    }
    float sr, si;
    block_sum_cplx<9>(re, im, 9, sr, si);
    const int t = threadIdx.x;
    if (t < nvc) partial[(long long)blockIdx.x * ld + v0 + t] = make_double2(sr, si);
    if (ch == 0 && t == 8) partial[(long long)blockIdx.x * ld + nv] = make_double2(sr, 0.0);
  }
  __threadfence();   // this block's partial sums are visible before its ticket is taken
  __syncthreads();
  __shared__ int last;
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i <= nv; i += CT) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const double2 p = __ldcg(partial + (long long)b * ld + i);   // other blocks' sums, not through L1
      s.x += p.x;
      s.y += p.y;
    }
    h_out[i] = s;
  }
  if (threadIdx.x == 0) *ticket = 0;
}

// out = w - V h (in place allowed: out may alias w); |out|^2 over blocks in FP64 into
// n2_out; with hc != 0 the last block also runs hcol_step for column j.  norm_partial:
// gridDim.x doubles.  Skipped when *gate != 0.
struct HcolArgs {
  int hc, j, ldh;
  zd* R;
  const double2 *hA, *hB;
  LsqState* lsq;
  zd* g;
  double* nu;
  int* state;
};
__global__ void __launch_bounds__(CT) mg_cproject_kernel(float4* out, const float4* w, const float4* __restrict__ V,
                                                         int nv, long long n4, const double2* h, double* norm_partial,
                                                         double* n2_out, int* ticket, const int* gate, HcolArgs hc) {
  if (gate && *gate) return;
  __shared__ float2 hs[64];
  for (int i = threadIdx.x; i < nv; i += CT) hs[i] = make_float2((float)h[i].x, (float)h[i].y);
  __syncthreads();
  float nrm = 0.f;
  for (long long q = blockIdx.x * (long long)CT + threadIdx.x; q < n4; q += (long long)gridDim.x * CT) {
    float4 a = w[q];
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      float4 v[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) v[b] = V[(long long)(i + b) * n4 + q];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float2 c = hs[i + b];
        a.x -= c.x * v[b].x - c.y * v[b].y;
        a.y -= c.x * v[b].y + c.y * v[b].x;
        a.z -= c.x * v[b].z - c.y * v[b].w;
        a.w -= c.x * v[b].w + c.y * v[b].z;
      }
    }
    for (; i < nv; ++i) {
      const float4 v = V[(long long)i * n4 + q];
      const float2 c = hs[i];
      a.x -= c.x * v.x - c.y * v.y;
      a.y -= c.x * v.y + c.y * v.x;
      a.z -= c.x * v.z - c.y * v.w;
      a.w -= c.x * v.w + c.y * v.z;
    }
    out[q] = a;
    nrm += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
  }
  const double2 s = block_sum_d2(make_double2(nrm, 0.0));
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = s.x;
  __threadfence();
  __syncthreads();
  __shared__ int last;
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double n2 = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) n2 += __ldcg(norm_partial + b);
  if (n2_out) *n2_out = n2;
  if (hc.hc && hc.state[0] == 0) hcol_step(hc.R, hc.ldh, hc.j, hc.hA, hc.hB, n2, hc.lsq, hc.g, hc.nu, hc.state);
  *ticket = 0;
}

static int coarse_blocks() { return blas_partials_blocks() / 2; }   // 2 per SM

void launch_mg_cdot(const float4* V, int nv, long long n4, const float4* w, double2* partial, double2* h_out,
                    int* ticket, const int* gate, cudaStream_t st) {
  mg_cdot_kernel<<<coarse_blocks(), CT, 0, st>>>(V, nv, n4, w, partial, h_out, ticket, gate);
}

void launch_mg_cproject(float4* out, const float4* w, const float4* V, int nv, long long n4, const double2* h,
                        double* norm_partial, double* n2_out, int* ticket, const int* gate, int hcol, zd* R, int ldh,
                        int j, const double2* hA, const double2* hB, LsqState* lsq, zd* g, double* nu, int* state,
                        cudaStream_t st) {
  HcolArgs a{hcol, j, ldh, R, hA, hB, lsq, g, nu, state};
  mg_cproject_kernel<<<coarse_blocks(), CT, 0, st>>>(out, w, V, nv, n4, h, norm_partial, n2_out, ticket, gate, a);
}

// ------------------------------------------------------------------ coarse GMRES small steps
// Start of a cycle: beta = |r| from its squared norm; g = beta e_1; the Givens state is
// reset; state[0] = 1 (nothing to do) when beta = 0; nu = 1 / beta for the scaling of v_1.
__global__ void mg_beta_kernel(const double2* nrm, zd* g, int ng, double* nu, int* state, LsqState* lsq) {
  const double b = sqrt(fmax(nrm[0].x, 0.0));
  for (int i = 0; i < ng; ++i) g[i] = Z(0.0);
  g[0] = Z(b);
  lsq->nrot = 0;
  state[0] = (b > 0.0 && isfinite(b)) ? 0 : 1;
  state[1] = 0;
  nu[0] = state[0] == 0 ? 1.0 / b : 0.0;
}

// y = R^{-1} g over the completed columns; the rest of y is zero.
__global__ void mg_lsq_kernel(const zd* R, int ldh, int mc, const zd* g, const int* state, zd* y) {
  const int n = state[1];
  lsq_solve(R, ldh, n, g, y);
  for (int i = n; i < mc; ++i) y[i] = Z(0.0);
}

// v *= nu[0] (skipped when *gate != 0)
__global__ void mg_scale_kernel(float4* v, long long n4, const double* nu, const int* gate) {
  if (gate && *gate) return;
  const float s = (float)nu[0];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    const float4 a = v[q];
    v[q] = make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
  }
}

// x += a t
__global__ void mg_axpy_kernel(float4* x, const float4* t, long long n4, float a) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    const float4 u = x[q], v = t[q];
    x[q] = make_float4(u.x + a * v.x, u.y + a * v.y, u.z + a * v.z, u.w + a * v.w);
  }
}

// z = sc (x + e) with sc = *vscale (1 when null) and e optional
__global__ void mg_combine_kernel(float4* z, const float4* x, const float4* e, long long n4, const float* vscale) {
  const float s = vscale ? *vscale : 1.f;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    float4 a = x[q];
    if (e) {
      const float4 b = e[q];
      a = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
    z[q] = make_float4(s * a.x, s * a.y, s * a.z, s * a.w);
  }
}

static unsigned grid_for(long long n4) {
  const long long b = (n4 + 255) / 256;
  const long long cap = 4LL * blas_partials_blocks();
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

void launch_mg_beta(const double2* nrm, zd* g, int ng, double* nu, int* state, LsqState* lsq, cudaStream_t st) {
  mg_beta_kernel<<<1, 1, 0, st>>>(nrm, g, ng, nu, state, lsq);
}
void launch_mg_lsq(const zd* R, int ldh, int mc, const zd* g, const int* state, zd* y, cudaStream_t st) {
  mg_lsq_kernel<<<1, 1, 0, st>>>(R, ldh, mc, g, state, y);
}
void launch_mg_scale(float4* v, long long n4, const double* nu, const int* gate, cudaStream_t st) {
  mg_scale_kernel<<<grid_for(n4), 256, 0, st>>>(v, n4, nu, gate);
}
void launch_mg_axpy(float4* x, const float4* t, long long n4, float a, cudaStream_t st) {
  mg_axpy_kernel<<<grid_for(n4), 256, 0, st>>>(x, t, n4, a);
}
void launch_mg_combine(float4* z, const float4* x, const float4* e, long long n4, const float* vscale,
                       cudaStream_t st) {
  mg_combine_kernel<<<grid_for(n4), 256, 0, st>>>(z, x, e, n4, vscale);
}

}  // namespace dd

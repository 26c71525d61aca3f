// Layout transforms (canonical lexicographic <-> domain-major) and the clover build.
//
// Canonical layouts (the library's public formats):
//   spinor: [t][z][y][x][spin 4][colour 3][re, im]   (FP64 or FP32)
//   gauge:  [t][z][y][x][mu 4][row 3][col 3][re, im] (FP64), forward links U_mu(x).
// The antiperiodic time boundary of the fermion field is folded into the internal copy
// of the links: U_t(x) at t = L_t - 1 is stored negated.  Every plaquette that crosses
// the boundary holds two such links, so the clover term is unaffected; it is built here
// from the canonical (unsigned) links.
#include "dd_kernels.hpp"

namespace dd {

__device__ inline void site_global(const Geom& g, const Site& st, int x[4]) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) x[mu] = st.n[mu] * g.b[mu] + st.l[mu];
}

__device__ inline long long canon_index(const Geom& g, const int x[4]) {
  return x[0] + (long long)g.L[0] * (x[1] + (long long)g.L[1] * (x[2] + (long long)g.L[2] * x[3]));
}

template <typename C, typename T>
__global__ void pack_spinor_kernel(Geom g, const C* canon, SpinorPtr<T> out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Site st = decode(g, s);
  int x[4];
  site_global(g, st, x);
  const C* q = canon + 24 * canon_index(g, x);
  Spinor<typename Arith<T>::type> v;
#pragma unroll
  for (int k = 0; k < 12; ++k) v.c[k / 3][k % 3] = mk<typename Arith<T>::type>(q[2 * k], q[2 * k + 1]);
  out.store(g, s, v);
}

template <typename T, typename C>
__global__ void unpack_spinor_kernel(Geom g, SpinorPtr<T> in, C* canon) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Site st = decode(g, s);
  int x[4];
  site_global(g, st, x);
  Spinor<typename Arith<T>::type> v;
  in.load(g, s, v);
  C* q = canon + 24 * canon_index(g, x);
#pragma unroll
  for (int k = 0; k < 12; ++k) { q[2 * k] = (C)v.c[k / 3][k % 3].re; q[2 * k + 1] = (C)v.c[k / 3][k % 3].im; }
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename C>
static void pack_dispatch(const Geom& g, const C* canon, FieldView out, cudaStream_t st) {
  unsigned nb = nblk(g.V, 256);
  if (out.prec == P64) pack_spinor_kernel<C, double><<<nb, 256, 0, st>>>(g, canon, SpinorPtr<double>{(double2*)out.data});
  else if (out.prec == P32) pack_spinor_kernel<C, float><<<nb, 256, 0, st>>>(g, canon, SpinorPtr<float>{(float4*)out.data});
  else pack_spinor_kernel<C, __half><<<nb, 256, 0, st>>>(g, canon, SpinorPtr<__half>{(uint4*)out.data, out.norm});
}

void launch_pack_spinor(const Geom& g, const void* canon, int canon_prec, FieldView out, cudaStream_t st) {
  if (canon_prec == P64) pack_dispatch(g, (const double*)canon, out, st);
  else pack_dispatch(g, (const float*)canon, out, st);
}

template <typename C>
static void unpack_dispatch(const Geom& g, FieldView in, C* canon, cudaStream_t st) {
  unsigned nb = nblk(g.V, 256);
  if (in.prec == P64) unpack_spinor_kernel<double, C><<<nb, 256, 0, st>>>(g, SpinorPtr<double>{(double2*)in.data}, canon);
  else if (in.prec == P32) unpack_spinor_kernel<float, C><<<nb, 256, 0, st>>>(g, SpinorPtr<float>{(float4*)in.data}, canon);
  else unpack_spinor_kernel<__half, C><<<nb, 256, 0, st>>>(g, SpinorPtr<__half>{(uint4*)in.data, in.norm}, canon);
}

void launch_unpack_spinor(const Geom& g, FieldView in, void* canon, int canon_prec, cudaStream_t st) {
  if (canon_prec == P64) unpack_dispatch(g, in, (double*)canon, st);
  else unpack_dispatch(g, in, (float*)canon, st);
}

__global__ void pack_gauge_kernel(Geom g, const double* canon, int anti, double2* u64, float2* u32, uint32_t* u16) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Site st = decode(g, s);
  int x[4];
  site_global(g, st, x);
  const double* q = canon + 72 * canon_index(g, x);
  long long d = st.d, r = s & (g.Vd - 1);
  for (int mu = 0; mu < 4; ++mu) {
    double sg = (anti && mu == 3 && x[3] == g.L[3] - 1) ? -1.0 : 1.0;
    for (int j = 0; j < 9; ++j) {
      double re = sg * q[18 * mu + 2 * j], im = sg * q[18 * mu + 2 * j + 1];
      long long a = (((d * 4 + mu) * 9 + j) << g.lgVd) + r;
      u64[a] = make_double2(re, im);
      u32[a] = make_float2((float)re, (float)im);
      u16[a] = f2h((float)re, (float)im);
    }
  }
}

void launch_pack_gauge(const Geom& g, const double* canon, int anti, double2* u64, float2* u32, uint32_t* u16,
                       cudaStream_t st) {
  pack_gauge_kernel<<<nblk(g.V, 128), 128, 0, st>>>(g, canon, anti, u64, u32, u16);
}

// ------------------------------------------------------------------ clover build (FP64)
struct M3 { cx<double> e[3][3]; };

__device__ inline M3 m3_mul(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cx<double> v = mk(0.0, 0.0);
      for (int k = 0; k < 3; ++k) v = v + cmul(a.e[i][k], b.e[k][j]);
      c.e[i][j] = v;
    }
  return c;
}
__device__ inline M3 m3_dag(const M3& a) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.e[i][j] = mk(a.e[j][i].re, -a.e[j][i].im);
  return c;
}

struct CanonLinks {
  Geom g;
  const double* U;
  __device__ M3 get(const int xin[4], int mu) const {
    int x[4];
    for (int k = 0; k < 4; ++k) x[k] = (xin[k] % g.L[k] + g.L[k]) % g.L[k];
    const double* q = U + 72 * canon_index(g, x) + 18 * mu;
    M3 m;
    for (int j = 0; j < 9; ++j) m.e[j / 3][j % 3] = mk(q[2 * j], q[2 * j + 1]);
    return m;
  }
};

// Sum of the four plaquette leaves in the (mu, nu) plane at x, oriented mu -> nu.
__device__ M3 leaves(const CanonLinks& L, const int x[4], int mu, int nu) {
  int xm[4], xn[4], xmm[4], xnm[4], xmmnm[4], xmmn[4], xmnm[4];
  for (int k = 0; k < 4; ++k) {
    int em = (k == mu), en = (k == nu);
    xm[k] = x[k] + em;           // x + mu
    xn[k] = x[k] + en;           // x + nu
    xmm[k] = x[k] - em;          // x - mu
    xnm[k] = x[k] - en;          // x - nu
    xmmnm[k] = x[k] - em - en;   // x - mu - nu
    xmmn[k] = x[k] - em + en;    // x - mu + nu
    xmnm[k] = x[k] + em - en;    // x + mu - nu
  }
  M3 Umx = L.get(x, mu), Unx = L.get(x, nu);
  M3 l1 = m3_mul(m3_mul(Umx, L.get(xm, nu)), m3_mul(m3_dag(L.get(xn, mu)), m3_dag(Unx)));
  M3 Um_mm = L.get(xmm, mu);
  M3 l2 = m3_mul(m3_mul(Unx, m3_dag(L.get(xmmn, mu))), m3_mul(m3_dag(L.get(xmm, nu)), Um_mm));
  M3 l3 = m3_mul(m3_mul(m3_dag(Um_mm), m3_dag(L.get(xmmnm, nu))), m3_mul(L.get(xmmnm, mu), L.get(xnm, nu)));
  M3 Un_nm = L.get(xnm, nu);
  M3 l4 = m3_mul(m3_mul(m3_dag(Un_nm), L.get(xnm, mu)), m3_mul(L.get(xmnm, nu), m3_dag(Umx)));
  M3 q;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q.e[i][j] = l1.e[i][j] + l2.e[i][j] + l3.e[i][j] + l4.e[i][j];
  return q;
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting.  Returns the
// smallest pivot magnitude relative to the largest entry.
__device__ double inv6(cx<double> a[6][6], cx<double> inv[6][6]) {
  double amax = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      inv[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
      amax = fmax(amax, hypot(a[i][j].re, a[i][j].im));
    }
  double minpiv = 1e300;
  for (int c = 0; c < 6; ++c) {
    int pr = c;
    double best = -1;
    for (int r = c; r < 6; ++r) {
      double v = hypot(a[r][c].re, a[r][c].im);
      if (v > best) { best = v; pr = r; }
    }
    minpiv = fmin(minpiv, best);
    if (best == 0.0) return 0.0;
    if (pr != c)
      for (int j = 0; j < 6; ++j) {
        cx<double> t = a[c][j]; a[c][j] = a[pr][j]; a[pr][j] = t;
        t = inv[c][j]; inv[c][j] = inv[pr][j]; inv[pr][j] = t;
      }
    cx<double> p = a[c][c];
    double pn = p.re * p.re + p.im * p.im;
    cx<double> pi = mk(p.re / pn, -p.im / pn);
    for (int j = 0; j < 6; ++j) { a[c][j] = cmul(a[c][j], pi); inv[c][j] = cmul(inv[c][j], pi); }
    for (int r = 0; r < 6; ++r) {
      if (r == c) continue;
      cx<double> f = a[r][c];
      for (int j = 0; j < 6; ++j) {
        a[r][j] = a[r][j] - cmul(f, a[c][j]);
        inv[r][j] = inv[r][j] - cmul(f, inv[c][j]);
      }
    }
  }
  return amax > 0 ? minpiv / amax : 0.0;
}

// Pack a Hermitian 6x6 block (its lower triangle and real diagonal) into 36 reals.
__device__ inline void pack_block(cx<double> a[6][6], double* out) {
  for (int i = 0; i < 6; ++i) out[i] = a[i][i].re;
  for (int i = 1; i < 6; ++i)
    for (int j = 0; j < i; ++j) {
      // Hermitian part of the pair (i, j), (j, i)
      out[6 + 2 * tri(i, j)] = 0.5 * (a[i][j].re + a[j][i].re);
      out[6 + 2 * tri(i, j) + 1] = 0.5 * (a[i][j].im - a[j][i].im);
    }
}

__global__ void __launch_bounds__(128) build_clover_kernel(Geom g, const double* canon, double kappa, double csw,
                                                           double2* c64, float4* c32, uint4* c16, float4* s32,
                                                           uint4* s16, int* status) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Site st = decode(g, s);
  int x[4];
  site_global(g, st, x);
  CanonLinks L{g, canon};
  // F(mu, nu) = Q_mu,nu - Q_mu,nu^dag for the six planes, needed as i F (Hermitian).
  // Plane order: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
  M3 F[6];
  const int pm[6] = {0, 0, 0, 1, 1, 2}, pn[6] = {1, 2, 3, 2, 3, 3};
  for (int k = 0; k < 6; ++k) {
    M3 Q = leaves(L, x, pm[k], pn[k]);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) F[k].e[i][j] = Q.e[i][j] - mk(Q.e[j][i].re, -Q.e[j][i].im);
  }
  // Chiral blocks: D_cl = -(c_sw/16) sum_{mu<nu} gamma_mu gamma_nu (x) F_mu,nu.  With
  // E = (F_yz, -F_xz, F_xy), G = (F_xt, F_yt, F_zt) and X_l = i (E_l -/+ G_l) for the
  // upper / lower chirality, each block is -(c_sw/16) [[X3, X1 - i X2], [X1 + i X2, -X3]].
  double cl[72], sm[72];   // clover (all sites); Schwarz matrix (clover on even, inverse on odd)
  double minrel = 1e300;
  for (int blk = 0; blk < 2; ++blk) {
    double sg = blk == 0 ? -1.0 : 1.0;
    M3 X[3];
    const M3* E[3] = {&F[3], &F[1], &F[0]};
    const double es[3] = {1.0, -1.0, 1.0};
    const M3* G[3] = {&F[2], &F[4], &F[5]};
    for (int l = 0; l < 3; ++l)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cx<double> v = es[l] * E[l]->e[i][j] + sg * G[l]->e[i][j];
          X[l].e[i][j] = ti(v);
        }
    cx<double> B[6][6];
    const double c = -csw / 16.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        B[a][b] = c * X[2].e[a][b];
        B[3 + a][3 + b] = (-c) * X[2].e[a][b];
        B[a][3 + b] = c * (X[0].e[a][b] + tmi(X[1].e[a][b]));
        B[3 + a][b] = c * (X[0].e[a][b] + ti(X[1].e[a][b]));
      }
    for (int i = 0; i < 6; ++i) B[i][i].re += 1.0 / (2.0 * kappa);
    pack_block(B, cl + 36 * blk);
    cx<double> Bc[6][6], Bi[6][6];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Bc[i][j] = B[i][j];
    minrel = fmin(minrel, inv6(Bc, Bi));
    if (st.p == 0) pack_block(B, sm + 36 * blk);
    else pack_block(Bi, sm + 36 * blk);
  }
  if (!(minrel >= 1e-12)) atomicAdd(status, 1);
  for (int u = 0; u < 36; ++u) c64[unit_addr(g, s, 36, u)] = make_double2(cl[2 * u], cl[2 * u + 1]);
  for (int u = 0; u < 18; ++u) {
    c32[unit_addr(g, s, 18, u)] = make_float4((float)cl[4 * u], (float)cl[4 * u + 1], (float)cl[4 * u + 2], (float)cl[4 * u + 3]);
    s32[unit_addr(g, s, 18, u)] = make_float4((float)sm[4 * u], (float)sm[4 * u + 1], (float)sm[4 * u + 2], (float)sm[4 * u + 3]);
  }
  for (int u = 0; u < 9; ++u) {
    uint32_t w[4], v[4];
    for (int e = 0; e < 4; ++e) {
      w[e] = f2h((float)cl[8 * u + 2 * e], (float)cl[8 * u + 2 * e + 1]);
      v[e] = f2h((float)sm[8 * u + 2 * e], (float)sm[8 * u + 2 * e + 1]);
    }
    c16[unit_addr(g, s, 9, u)] = make_uint4(w[0], w[1], w[2], w[3]);
    s16[unit_addr(g, s, 9, u)] = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

void launch_build_clover(const Geom& g, const double* canon, double kappa, double csw, double2* c64, float4* c32,
                         uint4* c16, float4* s32, uint4* s16, int* status, cudaStream_t st) {
  build_clover_kernel<<<nblk(g.V, 128), 128, 0, st>>>(g, canon, kappa, csw, c64, c32, c16, s32, s16, status);
}

}  // namespace dd

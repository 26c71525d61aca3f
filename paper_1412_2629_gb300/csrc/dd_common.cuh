// Device-side building blocks shared by the kernels of the GB300 solver library:
// lattice geometry in the domain-major layout, complex arithmetic, spin projection
// and reconstruction for the hopping term of Eq. 2, SU(3) products, packed Hermitian
// 6x6 clover blocks (Eq. 3), and typed loads/stores of every field format.
//
// Layout (all fields, every precision): sites are ordered domain-major.  A site with
// global coordinates (x, y, z, t) lies in domain d = nx + Nx (ny + Ny (nz + Nz nt)),
// n_mu = x_mu / b_mu, at local coordinates l_mu = x_mu mod b_mu.  Inside the domain
// it has parity p = (x + y + z + t) mod 2 (equal to the local parity because every b_mu
// is even) and index i = lex >> 1, lex = lx + bx (ly + by (lz + bz lt)).  Its internal
// index is s = d Vd + p Hd + i with Vd = prod b_mu and Hd = Vd / 2; r = s mod Vd.
// Every field is stored as 16-byte (or, for links, 8- or 4-byte) units in
// [domain][unit][r] order, so consecutive threads touch consecutive addresses.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dd {

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];      // lattice extents Lx, Ly, Lz, Lt
  int b[4];      // domain extents (powers of two, even)
  int N[4];      // domains per direction, L / b (even, >= 2)
  int lgb[4];    // log2 b
  int bstride[4];  // 1, bx, bx by, bx by bz: lex strides inside a domain
  int dstride[4];  // 1, Nx, Nx Ny, Nx Ny Nz: domain index strides
  int Vd, Hd, lgVd;
  int ND;        // number of domains
  long long V;   // lattice volume
  int face_n[4];     // sites on a face normal to mu: Vd / b_mu
  int face_off[8];   // offset of face (mu, side) inside a domain's face block, in sites
  int face_block;    // sites in all eight faces of one domain
};

struct Site {
  int d;          // domain
  int n[4];       // domain coordinates
  int l[4];       // local coordinates
  int lex, p, i;  // local lexicographic index, parity, index within parity
};

__host__ __device__ inline void domain_coords(const Geom& g, int d, int n[4]) {
  n[0] = d % g.N[0];
  int q = d / g.N[0];
  n[1] = q % g.N[1];
  q /= g.N[1];
  n[2] = q % g.N[2];
  n[3] = q / g.N[2];
}

// Decode (domain, parity, index-within-parity) into local coordinates.
__host__ __device__ inline void local_coords(const Geom& g, int p, int i, int l[4]) {
  const int hxl = g.lgb[0] - 1;           // log2(bx / 2)
  int ix = i & ((1 << hxl) - 1);
  int row = i >> hxl;
  l[1] = row & (g.b[1] - 1);
  row >>= g.lgb[1];
  l[2] = row & (g.b[2] - 1);
  l[3] = row >> g.lgb[2];
  l[0] = 2 * ix + ((p + l[1] + l[2] + l[3]) & 1);
}

__host__ __device__ inline Site decode(const Geom& g, long long s) {
  Site st;
  st.d = (int)(s >> g.lgVd);
  int r = (int)(s & (g.Vd - 1));
  st.p = r >= g.Hd;
  st.i = r - st.p * g.Hd;
  domain_coords(g, st.d, st.n);
  local_coords(g, st.p, st.i, st.l);
  st.lex = st.l[0] + g.bstride[1] * st.l[1] + g.bstride[2] * st.l[2] + g.bstride[3] * st.l[3];
  return st;
}

__host__ __device__ inline long long encode_global(const Geom& g, const int x[4]) {
  int n[4], l[4];
  for (int mu = 0; mu < 4; ++mu) {
    n[mu] = x[mu] >> g.lgb[mu];
    l[mu] = x[mu] & (g.b[mu] - 1);
  }
  int d = n[0] + g.dstride[1] * n[1] + g.dstride[2] * n[2] + g.dstride[3] * n[3];
  int lex = l[0] + g.bstride[1] * l[1] + g.bstride[2] * l[2] + g.bstride[3] * l[3];
  int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  return ((long long)d << g.lgVd) + p * g.Hd + (lex >> 1);
}

// Domain index of the neighbour domain in direction mu (dir = +1 / -1), periodic.
__host__ __device__ inline int neighbour_domain(const Geom& g, int d, const int n[4], int mu, int dir) {
  if (dir > 0) return n[mu] + 1 < g.N[mu] ? d + g.dstride[mu] : d - (g.N[mu] - 1) * g.dstride[mu];
  return n[mu] > 0 ? d - g.dstride[mu] : d + (g.N[mu] - 1) * g.dstride[mu];
}

// Internal index of the nearest neighbour x + dir mu_hat of a decoded site.
__host__ __device__ inline long long neighbour(const Geom& g, const Site& st, int mu, int dir) {
  int d = st.d, lex = st.lex;
  if (dir > 0) {
    if (st.l[mu] + 1 < g.b[mu]) lex += g.bstride[mu];
    else { d = neighbour_domain(g, st.d, st.n, mu, +1); lex -= (g.b[mu] - 1) * g.bstride[mu]; }
  } else {
    if (st.l[mu] > 0) lex -= g.bstride[mu];
    else { d = neighbour_domain(g, st.d, st.n, mu, -1); lex += (g.b[mu] - 1) * g.bstride[mu]; }
  }
  return ((long long)d << g.lgVd) + (1 - st.p) * g.Hd + (lex >> 1);
}

// Index of a face site inside the face normal to mu: lexicographic over the other three
// local coordinates in the order x, y, z, t.
__host__ __device__ inline int face_index(const Geom& g, const int l[4], int mu) {
  int idx = 0, stride = 1;
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    idx += l[nu] * stride;
    stride *= g.b[nu];
  }
  return idx;
}

// Domain shapes the hot kernels are also compiled for (SHAPE 1: 8x4x4x4, 2: 4x4x4x4; 0:
// shape read at run time).  With the shape known at compile time every local stride, site
// count and buffer offset is a constant, so addresses fold into immediate offsets and
// most index arithmetic disappears.
template <int SHAPE> struct ShapeOf;
template <> struct ShapeOf<1> {
  __host__ __device__ static constexpr int b(int mu) { return mu == 0 ? 8 : 4; }
  __host__ __device__ static constexpr int lg(int mu) { return mu == 0 ? 3 : 2; }
};
template <> struct ShapeOf<2> {
  __host__ __device__ static constexpr int b(int) { return 4; }
  __host__ __device__ static constexpr int lg(int) { return 2; }
};

inline int domain_shape_id(const Geom& g) {
  if (g.b[0] == 8 && g.b[1] == 4 && g.b[2] == 4 && g.b[3] == 4) return 1;
  if (g.b[0] == 4 && g.b[1] == 4 && g.b[2] == 4 && g.b[3] == 4) return 2;
  return 0;
}

// The geometry with the domain fields replaced by compile-time constants (SHAPE != 0).
template <int SHAPE>
__device__ __forceinline__ Geom fixed_shape(const Geom& in) {
  Geom g = in;
  if constexpr (SHAPE != 0) {
    using S = ShapeOf<SHAPE>;
    constexpr int vd = S::b(0) * S::b(1) * S::b(2) * S::b(3);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      g.b[mu] = S::b(mu);
      g.lgb[mu] = S::lg(mu);
      g.face_n[mu] = vd / S::b(mu);
    }
    g.bstride[0] = 1;
    g.bstride[1] = S::b(0);
    g.bstride[2] = S::b(0) * S::b(1);
    g.bstride[3] = S::b(0) * S::b(1) * S::b(2);
    g.Vd = vd;
    g.Hd = vd / 2;
    g.lgVd = S::lg(0) + S::lg(1) + S::lg(2) + S::lg(3);
  }
  return g;
}

// ------------------------------------------------------------------ complex
template <typename R> struct cx { R re, im; };

template <typename R> __host__ __device__ inline cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <typename R> __host__ __device__ inline cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ inline cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ inline cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R> __host__ __device__ inline cx<R> cmul(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// conj(a) * b
template <typename R> __host__ __device__ inline cx<R> cjmul(cx<R> a, cx<R> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <typename R> __host__ __device__ inline cx<R> ti(cx<R> a) { return mk(-a.im, a.re); }    //  i a
template <typename R> __host__ __device__ inline cx<R> tmi(cx<R> a) { return mk(a.im, -a.re); }   // -i a

// Spinor in registers: psi[spin][colour]; spin 0,1 = upper chirality.
template <typename R> struct Spinor { cx<R> c[4][3]; };
template <typename R> struct Half { cx<R> c[2][3]; };
template <typename R> struct Link { cx<R> e[3][3]; };

template <typename R> __device__ inline void zero(Spinor<R>& s) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s.c[a][b] = mk<R>(0, 0);
}

// ------------------------------------------------------------------ spin projection
// Chiral basis: gamma_mu = [[0, B_mu], [B_mu^dag, 0]] with B_x = -i s1, B_y = -i s2,
// B_z = -i s3, B_t = 1.  (1 + S gamma_mu) psi has upper half h = psi_up + S B_mu psi_dn
// and lower half S B_mu^dag h, so a hop only needs the 6 complex numbers of h.
template <int MU, int S, typename R>
__device__ inline void project(const Spinor<R>& p, Half<R>& h) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (MU == 0) {        // B psi_dn = (-i p3, -i p2)
      h.c[0][a] = S > 0 ? p.c[0][a] + tmi(p.c[3][a]) : p.c[0][a] + ti(p.c[3][a]);
      h.c[1][a] = S > 0 ? p.c[1][a] + tmi(p.c[2][a]) : p.c[1][a] + ti(p.c[2][a]);
    } else if (MU == 1) { // B psi_dn = (-p3, p2)
      h.c[0][a] = S > 0 ? p.c[0][a] - p.c[3][a] : p.c[0][a] + p.c[3][a];
      h.c[1][a] = S > 0 ? p.c[1][a] + p.c[2][a] : p.c[1][a] - p.c[2][a];
    } else if (MU == 2) { // B psi_dn = (-i p2, i p3)
      h.c[0][a] = S > 0 ? p.c[0][a] + tmi(p.c[2][a]) : p.c[0][a] + ti(p.c[2][a]);
      h.c[1][a] = S > 0 ? p.c[1][a] + ti(p.c[3][a]) : p.c[1][a] + tmi(p.c[3][a]);
    } else {              // B psi_dn = (p2, p3)
      h.c[0][a] = S > 0 ? p.c[0][a] + p.c[2][a] : p.c[0][a] - p.c[2][a];
      h.c[1][a] = S > 0 ? p.c[1][a] + p.c[3][a] : p.c[1][a] - p.c[3][a];
    }
  }
}

// acc += (upper = h, lower = S B_mu^dag h)
template <int MU, int S, typename R>
__device__ inline void accum_recon(Spinor<R>& acc, const Half<R>& h) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc.c[0][a] = acc.c[0][a] + h.c[0][a];
    acc.c[1][a] = acc.c[1][a] + h.c[1][a];
    cx<R> l2, l3;
    if (MU == 0) { l2 = ti(h.c[1][a]); l3 = ti(h.c[0][a]); }              // B^dag = i s1
    else if (MU == 1) { l2 = h.c[1][a]; l3 = mk<R>(-h.c[0][a].re, -h.c[0][a].im); }  // i s2
    else if (MU == 2) { l2 = ti(h.c[0][a]); l3 = tmi(h.c[1][a]); }        // i s3
    else { l2 = h.c[0][a]; l3 = h.c[1][a]; }                                // 1
    if (S > 0) { acc.c[2][a] = acc.c[2][a] + l2; acc.c[3][a] = acc.c[3][a] + l3; }
    else       { acc.c[2][a] = acc.c[2][a] - l2; acc.c[3][a] = acc.c[3][a] - l3; }
  }
}

// out = U h  (both spin rows)
template <typename R>
__device__ inline void su3_mul(const Link<R>& U, const Half<R>& h, Half<R>& o) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> v = cmul(U.e[a][0], h.c[s][0]);
      v = v + cmul(U.e[a][1], h.c[s][1]);
      v = v + cmul(U.e[a][2], h.c[s][2]);
      o.c[s][a] = v;
    }
}

// out = U^dag h
template <typename R>
__device__ inline void su3_dag_mul(const Link<R>& U, const Half<R>& h, Half<R>& o) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> v = cjmul(U.e[0][a], h.c[s][0]);
      v = v + cjmul(U.e[1][a], h.c[s][1]);
      v = v + cjmul(U.e[2][a], h.c[s][2]);
      o.c[s][a] = v;
    }
}

// ------------------------------------------------------------------ clover blocks
// 72 reals per site: two packed Hermitian 6x6 blocks (block 0 acts on spins 0,1,
// block 1 on spins 2,3; index 3 s + colour).  Per block: 6 real diagonal entries,
// then the 15 strictly lower entries L(i, j), i > j, in the order i = 1..5, j = 0..i-1,
// each as (re, im).
__host__ __device__ inline int tri(int i, int j) { return i * (i - 1) / 2 + j; }

template <typename R>
__device__ inline void clover_block_mul(const R* m, const cx<R> v[6], cx<R> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = m[i] * v[i];
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      cx<R> L = mk(m[6 + 2 * tri(i, j)], m[6 + 2 * tri(i, j) + 1]);
      y[i] = y[i] + cmul(L, v[j]);
      y[j] = y[j] + cjmul(L, v[i]);
    }
}

template <typename R>
__device__ inline void clover_mul(const R* m72, const Spinor<R>& x, Spinor<R>& y) {
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    cx<R> v[6], w[6];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) v[3 * s + a] = x.c[2 * b + s][a];
    clover_block_mul(m72 + 36 * b, v, w);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) y.c[2 * b + s][a] = w[3 * s + a];
  }
}

// ------------------------------------------------------------------ field access
// Spinor storage types.  FP64: 6 units of two double2; FP32: 6 float4 units; FP16: 3
// uint4 units of 8 halves each, scaled by a per-site FP32 norm (max |component|).
__device__ inline long long unit_addr(const Geom& g, long long s, int nunits, int u) {
  long long d = s >> g.lgVd;
  long long r = s & (g.Vd - 1);
  return ((d * nunits + u) << g.lgVd) + r;
}

template <typename T> struct SpinorPtr;

// FP64 spinors use the FP32 unit structure (6 units of two complex numbers, here 32 B
// each), so the flat index of a complex number is the same in both precisions: double2
// 2q and 2q + 1 hold the two complex numbers of float4 q.  Vector kernels that mix the
// precisions rely on this.
template <> struct SpinorPtr<double> {
  double2* p;
  __device__ void load(const Geom& g, long long s, Spinor<double>& v) const {
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      long long a = 2 * unit_addr(g, s, 6, u);
      double2 q0 = p[a], q1 = p[a + 1];
      v.c[(2 * u) / 3][(2 * u) % 3] = mk(q0.x, q0.y);
      v.c[(2 * u + 1) / 3][(2 * u + 1) % 3] = mk(q1.x, q1.y);
    }
  }
  __device__ void store(const Geom& g, long long s, const Spinor<double>& v) const {
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      long long a = 2 * unit_addr(g, s, 6, u);
      p[a] = make_double2(v.c[(2 * u) / 3][(2 * u) % 3].re, v.c[(2 * u) / 3][(2 * u) % 3].im);
      p[a + 1] = make_double2(v.c[(2 * u + 1) / 3][(2 * u + 1) % 3].re, v.c[(2 * u + 1) / 3][(2 * u + 1) % 3].im);
    }
  }
};

template <> struct SpinorPtr<float> {
  float4* p;
  __device__ void load(const Geom& g, long long s, Spinor<float>& v) const {
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      float4 q = p[unit_addr(g, s, 6, u)];
      int k = 2 * u;
      v.c[k / 3][k % 3] = mk(q.x, q.y);
      v.c[(k + 1) / 3][(k + 1) % 3] = mk(q.z, q.w);
    }
  }
  __device__ void store(const Geom& g, long long s, const Spinor<float>& v) const {
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      int k = 2 * u;
      p[unit_addr(g, s, 6, u)] = make_float4(v.c[k / 3][k % 3].re, v.c[k / 3][k % 3].im,
                                             v.c[(k + 1) / 3][(k + 1) % 3].re, v.c[(k + 1) / 3][(k + 1) % 3].im);
    }
  }
};

__device__ inline float2 h2f(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
__device__ inline uint32_t f2h(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

template <> struct SpinorPtr<__half> {
  uint4* p;
  float* norm;
  __device__ void load(const Geom& g, long long s, Spinor<float>& v) const {
    float n = norm[s];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      uint4 q = p[unit_addr(g, s, 3, u)];
      uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float2 f = h2f(w[e]);
        int k = 4 * u + e;
        v.c[k / 3][k % 3] = mk(f.x * n, f.y * n);
      }
    }
  }
  __device__ void store(const Geom& g, long long s, const Spinor<float>& v) const {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) m = fmaxf(m, fmaxf(fabsf(v.c[a][b].re), fabsf(v.c[a][b].im)));
    float inv = m > 0.f ? 1.f / m : 0.f;
    norm[s] = m;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int k = 4 * u + e;
        w[e] = f2h(v.c[k / 3][k % 3].re * inv, v.c[k / 3][k % 3].im * inv);
      }
      p[unit_addr(g, s, 3, u)] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
};

// Arithmetic type for a storage type.
template <typename T> struct Arith { typedef float type; };
template <> struct Arith<double> { typedef double type; };

// Gauge links: [domain][mu][9][r] of (double2 | float2 | half2); entry j = 3 a + b.
template <typename T> struct LinkPtr;
template <> struct LinkPtr<double> {
  const double2* p;
  __device__ void load(const Geom& g, long long s, int mu, Link<double>& U) const {
    long long d = s >> g.lgVd, r = s & (g.Vd - 1);
    const double2* q = p + (((d * 4 + mu) * 9) << g.lgVd) + r;
#pragma unroll
    for (int j = 0; j < 9; ++j) { double2 v = q[(long long)j << g.lgVd]; U.e[j / 3][j % 3] = mk(v.x, v.y); }
  }
};
template <> struct LinkPtr<float> {
  const float2* p;
  __device__ void load(const Geom& g, long long s, int mu, Link<float>& U) const {
    long long d = s >> g.lgVd, r = s & (g.Vd - 1);
    const float2* q = p + (((d * 4 + mu) * 9) << g.lgVd) + r;
#pragma unroll
    for (int j = 0; j < 9; ++j) { float2 v = __ldg(q + ((long long)j << g.lgVd)); U.e[j / 3][j % 3] = mk(v.x, v.y); }
  }
};
template <> struct LinkPtr<__half> {
  const uint32_t* p;
  __device__ void load(const Geom& g, long long s, int mu, Link<float>& U) const {
    long long d = s >> g.lgVd, r = s & (g.Vd - 1);
    const uint32_t* q = p + (((d * 4 + mu) * 9) << g.lgVd) + r;
#pragma unroll
    for (int j = 0; j < 9; ++j) { float2 v = h2f(__ldg(q + ((long long)j << g.lgVd))); U.e[j / 3][j % 3] = mk(v.x, v.y); }
  }
};

// Clover (72 reals per site): FP64 36 double2 units, FP32 18 float4, FP16 9 uint4.
template <typename T> struct CloverPtr;
template <> struct CloverPtr<double> {
  const double2* p;
  __device__ void load(const Geom& g, long long s, double m[72]) const {
#pragma unroll
    for (int u = 0; u < 36; ++u) { double2 v = p[unit_addr(g, s, 36, u)]; m[2 * u] = v.x; m[2 * u + 1] = v.y; }
  }
};
template <> struct CloverPtr<float> {
  const float4* p;
  __device__ void load(const Geom& g, long long s, float m[72]) const {
#pragma unroll
    for (int u = 0; u < 18; ++u) {
      float4 v = __ldg(p + unit_addr(g, s, 18, u));
      m[4 * u] = v.x; m[4 * u + 1] = v.y; m[4 * u + 2] = v.z; m[4 * u + 3] = v.w;
    }
  }
};
template <> struct CloverPtr<__half> {
  const uint4* p;
  __device__ void load(const Geom& g, long long s, float m[72]) const {
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      uint4 v = __ldg(p + unit_addr(g, s, 9, u));
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) { float2 f = h2f(w[e]); m[8 * u + 2 * e] = f.x; m[8 * u + 2 * e + 1] = f.y; }
    }
  }
};

}  // namespace dd

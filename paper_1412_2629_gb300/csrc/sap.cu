// Multiplicative Schwarz (SAP) half-sweep: every domain of one colour is solved
// approximately in one launch, one CTA per domain (Sec. II-D, Table I).
//
// Formulation.  Per site the state is u (accumulated solution) and, on even sites only,
// the residual r of the last solve of its domain (the odd residual after a solve is
// exactly zero, Eq. 5).  Between two visits of a domain its neighbours (all of the other
// colour) changed their solution by delta'; their face buffers hold the half-spinors of
// delta' that enter the coupling R.  A visit does:
//   1. r = stored r (or the input v on the first sweep); r -= R delta' from the faces.
//   2. even-odd: t_o = A_oo^{-1} r_o;  f_e = r_e - D_eo t_o.
//   3. MR on D~_ee = A_ee - D_eo A_oo^{-1} D_oe, I_domain steps from x = 0.
//   4. delta_e = x, delta_o = A_oo^{-1} (r_o - D_oe x); u += delta; store r = MR residual.
//   5. write the projected half-spinors of delta on the eight faces.
// D_eo, D_oe are the hops inside the domain with factor -1/2; A_ee is the clover block
// (diagonal 1/(2 kappa) included), A_oo^{-1} its per-site inverse.
//
// Data movement.  The domain's links and Schwarz matrices (clover on even sites,
// inverse on odd sites) form contiguous blocks in HBM; when they fit, one thread
// stages both into shared memory with bulk asynchronous copies (TMA engine,
// completion on an mbarrier) while the others load the residual.  The even-site and
// odd-site work vectors live in shared memory as FP32; the thread for local index i
// owns even site i and odd site i and keeps x, rho and r_o in registers, so every MR
// step runs on chip.  The MR inner products are reduced with warp shuffles and one
// exchange through shared memory.
#include <mutex>
#include <type_traits>

#include "dd_kernels.hpp"

namespace dd {

// ------------------------------------------------------------------ matrix views
template <typename MT> struct MatBlock;

template <> struct MatBlock<__half> {
  const uint32_t* lk;  // [mu][9][Vd] half2
  const uint4* cm;     // [9][Vd]     8 halves
  int Vd;
  __device__ void link(int mu, int r, Link<float>& U) const {
#pragma unroll
    for (int j = 0; j < 9; ++j) { float2 v = h2f(lk[(mu * 9 + j) * Vd + r]); U.e[j / 3][j % 3] = mk(v.x, v.y); }
  }
  __device__ void mat(int r, float m[72]) const {
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      uint4 v = cm[u * Vd + r];
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) { float2 f = h2f(w[e]); m[8 * u + 2 * e] = f.x; m[8 * u + 2 * e + 1] = f.y; }
    }
  }
  static constexpr int link_bytes_per_site = 4 * 9 * 4;
  static constexpr int mat_bytes_per_site = 9 * 16;
};

template <> struct MatBlock<float> {
  const float2* lk;    // [mu][9][Vd]
  const float4* cm;    // [18][Vd]
  int Vd;
  __device__ void link(int mu, int r, Link<float>& U) const {
#pragma unroll
    for (int j = 0; j < 9; ++j) { float2 v = lk[(mu * 9 + j) * Vd + r]; U.e[j / 3][j % 3] = mk(v.x, v.y); }
  }
  __device__ void mat(int r, float m[72]) const {
#pragma unroll
    for (int u = 0; u < 18; ++u) {
      float4 v = cm[u * Vd + r];
      m[4 * u] = v.x; m[4 * u + 1] = v.y; m[4 * u + 2] = v.z; m[4 * u + 3] = v.w;
    }
  }
  static constexpr int link_bytes_per_site = 4 * 9 * 8;
  static constexpr int mat_bytes_per_site = 18 * 16;
};

// ------------------------------------------------------------------ work buffers
__device__ inline void ld_buf(const float4* buf, int Hd, int i, Spinor<float>& v) {
#pragma unroll
  for (int u = 0; u < 6; ++u) {
    float4 q = buf[u * Hd + i];
    int k = 2 * u;
    v.c[k / 3][k % 3] = mk(q.x, q.y);
    v.c[(k + 1) / 3][(k + 1) % 3] = mk(q.z, q.w);
  }
}
__device__ inline void st_buf(float4* buf, int Hd, int i, const Spinor<float>& v) {
#pragma unroll
  for (int u = 0; u < 6; ++u) {
    int k = 2 * u;
    buf[u * Hd + i] = make_float4(v.c[k / 3][k % 3].re, v.c[k / 3][k % 3].im, v.c[(k + 1) / 3][(k + 1) % 3].re,
                                  v.c[(k + 1) / 3][(k + 1) % 3].im);
  }
}

// Even-site residual store: per domain Hd sites.
template <typename VT> struct EvenStore;
template <> struct EvenStore<float> {
  float4* p;
  float* unused;
  __device__ void load(long long d, int Hd, int i, Spinor<float>& v) const { ld_buf(p + d * 6 * Hd, Hd, i, v); }
  __device__ void store(long long d, int Hd, int i, const Spinor<float>& v) const { st_buf(p + d * 6 * Hd, Hd, i, v); }
};
template <> struct EvenStore<__half> {
  uint4* p;
  float* norm;
  __device__ void load(long long d, int Hd, int i, Spinor<float>& v) const {
    float n = norm[d * Hd + i];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      uint4 q = p[(d * 3 + u) * Hd + i];
      uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float2 f = h2f(w[e]);
        int k = 4 * u + e;
        v.c[k / 3][k % 3] = mk(f.x * n, f.y * n);
      }
    }
  }
  __device__ void store(long long d, int Hd, int i, const Spinor<float>& v) const {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) m = fmaxf(m, fmaxf(fabsf(v.c[a][b].re), fabsf(v.c[a][b].im)));
    float inv = m > 0.f ? 1.f / m : 0.f;
    norm[d * Hd + i] = m;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int k = 4 * u + e;
        w[e] = f2h(v.c[k / 3][k % 3].re * inv, v.c[k / 3][k % 3].im * inv);
      }
      p[(d * 3 + u) * Hd + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
};

template <typename VT> struct VecPtr;
template <> struct VecPtr<float> {
  typedef SpinorPtr<float> type;
  __device__ static type make(void* p, float*) { return type{(float4*)p}; }
};
template <> struct VecPtr<__half> {
  typedef SpinorPtr<__half> type;
  __device__ static type make(void* p, float* n) { return type{(uint4*)p, n}; }
};

// ------------------------------------------------------------------ hop helpers
// acc += sum of the hops of one site that stay inside its domain (no -1/2 factor).
// src holds the other parity's vector; links come from the domain's block.
template <int MU, typename MT>
__device__ inline void inside_hop_mu(const Geom& g, const int l[4], int lex, int p, int r_self, const float4* src,
                                     const MatBlock<MT>& M, Spinor<float>& acc) {
  Spinor<float> psi;
  Half<float> h, uh;
  Link<float> L;
  if (l[MU] + 1 < g.b[MU]) {
    int j = (lex + g.bstride[MU]) >> 1;
    ld_buf(src, g.Hd, j, psi);
    project<MU, -1>(psi, h);
    M.link(MU, r_self, L);
    su3_mul(L, h, uh);
    accum_recon<MU, -1>(acc, uh);
  }
  if (l[MU] > 0) {
    int j = (lex - g.bstride[MU]) >> 1;
    ld_buf(src, g.Hd, j, psi);
    project<MU, +1>(psi, h);
    M.link(MU, (1 - p) * g.Hd + j, L);
    su3_dag_mul(L, h, uh);
    accum_recon<MU, +1>(acc, uh);
  }
}

template <typename MT>
__device__ inline void inside_hops(const Geom& g, const int l[4], int lex, int p, int r_self, const float4* src,
                                   const MatBlock<MT>& M, Spinor<float>& acc) {
  inside_hop_mu<0>(g, l, lex, p, r_self, src, M, acc);
  inside_hop_mu<1>(g, l, lex, p, r_self, src, M, acc);
  inside_hop_mu<2>(g, l, lex, p, r_self, src, M, acc);
  inside_hop_mu<3>(g, l, lex, p, r_self, src, M, acc);
}

__device__ inline void ld_half(const float4* q, Half<float>& h) {
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    float4 v = q[u];
    int k = 2 * u;
    h.c[k / 3][k % 3] = mk(v.x, v.y);
    h.c[(k + 1) / 3][(k + 1) % 3] = mk(v.z, v.w);
  }
}
__device__ inline void st_half(float4* q, const Half<float>& h) {
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    int k = 2 * u;
    q[u] = make_float4(h.c[k / 3][k % 3].re, h.c[k / 3][k % 3].im, h.c[(k + 1) / 3][(k + 1) % 3].re,
                       h.c[(k + 1) / 3][(k + 1) % 3].im);
  }
}

// acc += hops from the neighbouring domains, read from their face buffers.
//   +mu face of this domain: neighbour d+mu wrote P^-_mu delta on its -mu face;
//     the hop is (1 - gamma_mu) U_mu(x) delta(x + mu).
//   -mu face: neighbour d-mu wrote U_mu(y)^dag P^+_mu delta(y) on its +mu face.
template <int MU, typename MT>
__device__ inline void face_hop_mu(const Geom& g, int d, const int n[4], const int l[4], int r_self,
                                   const float4* faces, const MatBlock<MT>& M, Spinor<float>& acc) {
  Half<float> h, uh;
  if (l[MU] == g.b[MU] - 1) {
    long long dn = neighbour_domain(g, d, n, MU, +1);
    const float4* q = faces + (dn * g.face_block + g.face_off[2 * MU] + face_index(g, l, MU)) * 3;
    ld_half(q, h);
    Link<float> L;
    M.link(MU, r_self, L);
    su3_mul(L, h, uh);
    accum_recon<MU, -1>(acc, uh);
  }
  if (l[MU] == 0) {
    long long dn = neighbour_domain(g, d, n, MU, -1);
    const float4* q = faces + (dn * g.face_block + g.face_off[2 * MU + 1] + face_index(g, l, MU)) * 3;
    ld_half(q, h);
    accum_recon<MU, +1>(acc, h);
  }
}

template <typename MT>
__device__ inline void face_hops(const Geom& g, int d, const int n[4], const int l[4], int r_self,
                                 const float4* faces, const MatBlock<MT>& M, Spinor<float>& acc) {
  face_hop_mu<0>(g, d, n, l, r_self, faces, M, acc);
  face_hop_mu<1>(g, d, n, l, r_self, faces, M, acc);
  face_hop_mu<2>(g, d, n, l, r_self, faces, M, acc);
  face_hop_mu<3>(g, d, n, l, r_self, faces, M, acc);
}

template <int MU, typename MT>
__device__ inline void face_write_mu(const Geom& g, long long d, const int l[4], int r_self, float4* faces,
                                     const MatBlock<MT>& M, const Spinor<float>& dl) {
  Half<float> h, uh;
  if (l[MU] == 0) {
    project<MU, -1>(dl, h);
    st_half(faces + (d * g.face_block + g.face_off[2 * MU] + face_index(g, l, MU)) * 3, h);
  }
  if (l[MU] == g.b[MU] - 1) {
    project<MU, +1>(dl, h);
    Link<float> L;
    M.link(MU, r_self, L);
    su3_dag_mul(L, h, uh);
    st_half(faces + (d * g.face_block + g.face_off[2 * MU + 1] + face_index(g, l, MU)) * 3, uh);
  }
}

template <typename MT>
__device__ inline void face_write(const Geom& g, long long d, const int l[4], int r_self, float4* faces,
                                  const MatBlock<MT>& M, const Spinor<float>& dl) {
  face_write_mu<0>(g, d, l, r_self, faces, M, dl);
  face_write_mu<1>(g, d, l, r_self, faces, M, dl);
  face_write_mu<2>(g, d, l, r_self, faces, M, dl);
  face_write_mu<3>(g, d, l, r_self, faces, M, dl);
}

// ------------------------------------------------------------------ TMA bulk copy + mbarrier
__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ inline unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the given phase parity of the barrier, for at most limit_ns nanoseconds;
// returns false if the limit ran out.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t phase, unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    uint32_t ok = 0;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (ok) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

struct SapArgs {
  Geom g;
  int colour, first, use_faces, last, i_domain;
  const void* links;
  const void* smat;
  void* r_store;
  float* r_norm;
  void* u_store;
  float* u_norm;
  float4* faces;       // face buffers read by the couplings
  float4* faces_out;   // face buffers written (== faces except in the additive form)
  int both_colours;    // additive form: the grid covers the domains of both colours
  const float4* v;
  float4* z;
  const float* vscale;   // if set: the input is v * (*vscale) (a basis vector stored unnormalised)
  const float4* const* vptr;   // if set: input / output of right-hand side r at vptr[r] / zptr[r]
  float4* const* zptr;
  int* err;
  // Bound of the wait for the staged matrices, and extra bytes the barrier is told to
  // expect: 0 normally; a test sets it so the wait runs out and the error path is taken.
  unsigned long long wait_ns;
  unsigned extra_tx;
  // several right-hand sides per launch (two-threads-per-site kernel): strides between
  // consecutive right-hand sides of v / z (float4), faces (float4), residual and solution
  // storage (bytes) and their FP16 norms (floats)
  int nrhs;
  long long v_stride, f_stride, r_bytes, u_bytes, rn_stride, un_stride;
};

constexpr int SAP_MAX_THREADS = 256;

template <typename MT, typename VT, bool MSMEM>
__global__ void __launch_bounds__(SAP_MAX_THREADS, 1) sap_kernel(SapArgs a) {
  const Geom& g = a.g;
  extern __shared__ float4 smem[];
  __shared__ uint64_t mbar, mbar_inj;   // staged copies; injected bytes (test hook)
  __shared__ float4 red[SAP_MAX_THREADS / 32];
  const int tid = threadIdx.x;
  const int Hd = g.Hd, Vd = g.Vd;

  // domain of this CTA: the blockIdx.x-th domain of the given colour
  int n[4];
  {
    int half = g.N[0] >> 1;
    int j = blockIdx.x % half;
    int row = blockIdx.x / half;
    n[1] = row % g.N[1];
    n[2] = (row / g.N[1]) % g.N[2];
    n[3] = row / (g.N[1] * g.N[2]);
    n[0] = 2 * j + ((a.colour + n[1] + n[2] + n[3]) & 1);
  }
  const long long d = n[0] + (long long)g.dstride[1] * n[1] + (long long)g.dstride[2] * n[2] +
                      (long long)g.dstride[3] * n[3];

  const size_t lk_elems = (size_t)4 * 9 * Vd;
  const size_t lk_bytes = (size_t)MatBlock<MT>::link_bytes_per_site * Vd;
  const size_t cm_bytes = (size_t)MatBlock<MT>::mat_bytes_per_site * Vd;
  char* sbase = reinterpret_cast<char*>(smem);
  MatBlock<MT> M;
  M.Vd = Vd;
  typedef typename std::remove_const<typename std::remove_pointer<decltype(M.lk)>::type>::type LkT;
  typedef typename std::remove_const<typename std::remove_pointer<decltype(M.cm)>::type>::type CmT;
  const LkT* glk = reinterpret_cast<const LkT*>(a.links) + d * lk_elems;
  const CmT* gcm = reinterpret_cast<const CmT*>(a.smat) + d * (cm_bytes / sizeof(CmT));
  float4* sE;
  if (MSMEM) {
    M.lk = reinterpret_cast<const LkT*>(sbase);
    M.cm = reinterpret_cast<const CmT*>(sbase + lk_bytes);
    sE = reinterpret_cast<float4*>(sbase + lk_bytes + cm_bytes);
    if (tid == 0) {
      mbar_init(&mbar, 1);
      mbar_init(&mbar_inj, 1);
    }
    __syncthreads();
    if (tid == 0) {
      mbar_expect_tx(&mbar, (uint32_t)(lk_bytes + cm_bytes));
      bulk_g2s(sbase, glk, (uint32_t)lk_bytes, &mbar);
      bulk_g2s(sbase + lk_bytes, gcm, (uint32_t)cm_bytes, &mbar);
      // test hook: bytes that nobody sends, on a barrier of their own
      if (a.extra_tx) mbar_expect_tx(&mbar_inj, a.extra_tx);
    }
  } else {
    M.lk = glk;
    M.cm = gcm;
    sE = smem;
  }
  float4* sO = sE + 6 * Hd;

  int le[4], lo[4];
  local_coords(g, 0, tid, le);
  local_coords(g, 1, tid, lo);
  const int lex_e = le[0] + g.bstride[1] * le[1] + g.bstride[2] * le[2] + g.bstride[3] * le[3];
  const int lex_o = lo[0] + g.bstride[1] * lo[1] + g.bstride[2] * lo[2] + g.bstride[3] * lo[3];
  const long long s_e = (d << g.lgVd) + tid, s_o = s_e + Hd;
  const int r_e = tid, r_o = Hd + tid;

  // 1. residual
  Spinor<float> re, ro;
  const SpinorPtr<float> vin{const_cast<float4*>(a.v)};
  EvenStore<VT> rst{reinterpret_cast<decltype(EvenStore<VT>::p)>(a.r_store), a.r_norm};
  if (a.first) {
    vin.load(g, s_e, re);
    vin.load(g, s_o, ro);
    if (a.vscale) {
      const float sc = *a.vscale;
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          re.c[sp][c] = sc * re.c[sp][c];
          ro.c[sp][c] = sc * ro.c[sp][c];
        }
    }
  } else {
    rst.load(d, Hd, tid, re);
    zero(ro);
  }
  if (MSMEM) {
    bool ok = mbar_wait(&mbar, 0, a.wait_ns);
    if (a.extra_tx) ok = mbar_wait(&mbar_inj, 0, a.wait_ns) && ok;
    if (__syncthreads_or(!ok)) {
      // a wait ran out: flag it; then wait (bounded) for the staged copies themselves,
      // which were issued and will land, so none is left writing into this CTA's shared
      // memory after it exits
      if (tid == 0) atomicExch(a.err, 1);
      mbar_wait(&mbar, 0, a.wait_ns);
      return;
    }
  }
  if (a.use_faces) {
    Spinor<float> ae, ao;
    zero(ae);
    zero(ao);
    face_hops(g, (int)d, n, le, r_e, a.faces, M, ae);
    face_hops(g, (int)d, n, lo, r_o, a.faces, M, ao);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        re.c[s][c] = re.c[s][c] + 0.5f * ae.c[s][c];
        ro.c[s][c] = ro.c[s][c] + 0.5f * ao.c[s][c];
      }
  }

  // 2. even-odd preparation
  float m[72];
  Spinor<float> t, acc, rho, x;
  M.mat(r_o, m);
  clover_mul(m, ro, t);
  st_buf(sO, Hd, tid, t);
  __syncthreads();
  zero(acc);
  inside_hops(g, le, lex_e, 0, r_e, sO, M, acc);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rho.c[s][c] = re.c[s][c] + 0.5f * acc.c[s][c];
      x.c[s][c] = mk(0.f, 0.f);
    }
  st_buf(sE, Hd, tid, rho);
  __syncthreads();

  // 3. MR on the Schur complement
  const int nwarp = (Hd + 31) >> 5;
  for (int it = 0; it < a.i_domain; ++it) {
    // odd sites: t = A_oo^{-1} H_oe rho
    zero(acc);
    inside_hops(g, lo, lex_o, 1, r_o, sE, M, acc);
    M.mat(r_o, m);
    clover_mul(m, acc, t);
    st_buf(sO, Hd, tid, t);
    __syncthreads();
    // even sites: p = A_ee rho - 1/4 H_eo t
    zero(acc);
    inside_hops(g, le, lex_e, 0, r_e, sO, M, acc);
    Spinor<float> pv;
    M.mat(r_e, m);
    clover_mul(m, rho, pv);
    float pr_re = 0.f, pr_im = 0.f, pp = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv.c[s][c] = pv.c[s][c] - 0.25f * acc.c[s][c];
        cx<float> q = cjmul(pv.c[s][c], rho.c[s][c]);
        pr_re += q.re;
        pr_im += q.im;
        pp += pv.c[s][c].re * pv.c[s][c].re + pv.c[s][c].im * pv.c[s][c].im;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pr_re += __shfl_xor_sync(0xffffffffu, pr_re, o);
      pr_im += __shfl_xor_sync(0xffffffffu, pr_im, o);
      pp += __shfl_xor_sync(0xffffffffu, pp, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = make_float4(pr_re, pr_im, pp, 0.f);
    __syncthreads();
    float sr = 0.f, si = 0.f, sp = 0.f;
    for (int w = 0; w < nwarp; ++w) {
      float4 q = red[w];
      sr += q.x;
      si += q.y;
      sp += q.z;
    }
    cx<float> alpha = sp > 0.f ? mk(sr / sp, si / sp) : mk(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x.c[s][c] = x.c[s][c] + cmul(alpha, rho.c[s][c]);
        rho.c[s][c] = rho.c[s][c] - cmul(alpha, pv.c[s][c]);
      }
    st_buf(sE, Hd, tid, rho);
    __syncthreads();
  }

  // 4. odd reconstruction: delta_o = A_oo^{-1} (r_o + 1/2 H_oe x)
  st_buf(sE, Hd, tid, x);
  __syncthreads();
  zero(acc);
  inside_hops(g, lo, lex_o, 1, r_o, sE, M, acc);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.c[s][c] = ro.c[s][c] + 0.5f * acc.c[s][c];
  Spinor<float> dlo;
  M.mat(r_o, m);
  clover_mul(m, acc, dlo);

  // solution and residual
  typename VecPtr<VT>::type ust = VecPtr<VT>::make(a.u_store, a.u_norm);
  Spinor<float> ue, uo;
  if (a.first) {
    ue = x;
    uo = dlo;
  } else {
    ust.load(g, s_e, ue);
    ust.load(g, s_o, uo);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ue.c[s][c] = ue.c[s][c] + x.c[s][c];
        uo.c[s][c] = uo.c[s][c] + dlo.c[s][c];
      }
  }
  if (a.last) {
    SpinorPtr<float> zo{a.z};
    zo.store(g, s_e, ue);
    zo.store(g, s_o, uo);
  } else {
    ust.store(g, s_e, ue);
    ust.store(g, s_o, uo);
    rst.store(d, Hd, tid, rho);
  }
  // 5. faces for the other colour (not needed after the very last half-sweep)
  if (!(a.last && a.colour == 1)) {
    face_write(g, d, le, r_e, a.faces, M, x);
    face_write(g, d, lo, r_o, a.faces, M, dlo);
  }
}

// ------------------------------------------------------------------ two threads per site
// Same algorithm with 2 Hd threads per domain.  In the MR phases thread (h, i) works on
// even site i and odd site i: h = 0 computes the hops along x and y, h = 1 along z and t,
// and each keeps chirality half h (spins 2h, 2h+1) of x, rho and r_o.  Because the clover
// block and its inverse act within one chirality, the only exchange is of the two
// threads' partial hop sums, half by half, through the shared work buffer that the phase
// does not otherwise read.  Prologue and epilogue run one thread per site (h = parity).

// Half h of a site vector in a work buffer: units 3h .. 3h+2.
__device__ inline void ld_hbuf(const float4* buf, int Hd, int i, int h, Half<float>& v) {
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    float4 q = buf[(3 * h + u) * Hd + i];
    int k = 2 * u;
    v.c[k / 3][k % 3] = mk(q.x, q.y);
    v.c[(k + 1) / 3][(k + 1) % 3] = mk(q.z, q.w);
  }
}
__device__ inline void st_hbuf(float4* buf, int Hd, int i, int h, const Half<float>& v) {
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    int k = 2 * u;
    buf[(3 * h + u) * Hd + i] = make_float4(v.c[k / 3][k % 3].re, v.c[k / 3][k % 3].im, v.c[(k + 1) / 3][(k + 1) % 3].re,
                                            v.c[(k + 1) / 3][(k + 1) % 3].im);
  }
}
__device__ inline void half_of(const Spinor<float>& s, int h, Half<float>& o) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) o.c[a][c] = h ? s.c[2 + a][c] : s.c[a][c];
}

// Clover block H (36 reals) of site r.
template <typename MT> struct BlockLoad;
template <> struct BlockLoad<__half> {
  template <int H>
  __device__ static void load(const MatBlock<__half>& M, int r, float m[36]) {
    // 72 halves in 9 units of 8; block H holds halves 36 H .. 36 H + 35 (units 4 H .. 4 H + 4)
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      uint4 v = M.cm[(4 * H + u) * M.Vd + r];
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float2 f = h2f(w[e]);
        const int k = 8 * u + 2 * e - 4 * H;   // position inside the block
        if (k >= 0 && k < 36) { m[k] = f.x; m[k + 1] = f.y; }
      }
    }
  }
};
template <> struct BlockLoad<float> {
  template <int H>
  __device__ static void load(const MatBlock<float>& M, int r, float m[36]) {
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      float4 v = M.cm[(9 * H + u) * M.Vd + r];
      m[4 * u] = v.x; m[4 * u + 1] = v.y; m[4 * u + 2] = v.z; m[4 * u + 3] = v.w;
    }
  }
};

template <typename MT>
__device__ inline void block_apply(const MatBlock<MT>& M, int r, int h, const Half<float>& x, Half<float>& y) {
  float m[36];
  if (h == 0) BlockLoad<MT>::template load<0>(M, r, m);
  else BlockLoad<MT>::template load<1>(M, r, m);
  cx<float> v[6], w[6];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) v[3 * s + c] = x.c[s][c];
  clover_block_mul(m, v, w);
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) y.c[s][c] = w[3 * s + c];
}

// acc: this thread's partial sum over its two directions.  The other thread of the site
// holds the rest.  Returns the full sum of chirality half h.  buf is scratch here.
__device__ inline void exchange(const Spinor<float>& acc, int h, float4* buf, int Hd, int i, Half<float>& own) {
  Half<float> give, mine, got;
  half_of(acc, 1 - h, give);
  half_of(acc, h, mine);
  st_hbuf(buf, Hd, i, 1 - h, give);
  __syncthreads();
  ld_hbuf(buf, Hd, i, h, got);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) own.c[a][c] = mine.c[a][c] + got.c[a][c];
}

// Store half h of the even-site residual; FP16 needs the norm of the whole site, which
// the two threads share through nrm (2 Hd floats of shared memory).
template <typename VT> struct EvenHalfStore;
template <> struct EvenHalfStore<float> {
  __device__ static void store(const EvenStore<float>& E, float*, long long d, int Hd, int i, int h,
                               const Half<float>& v) {
    st_hbuf(E.p + d * 6 * Hd, Hd, i, h, v);
  }
};
template <> struct EvenHalfStore<__half> {
  __device__ static void store(const EvenStore<__half>& E, float* nrm, long long d, int Hd, int i, int h,
                               const Half<float>& v) {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) m = fmaxf(m, fmaxf(fabsf(v.c[a][c].re), fabsf(v.c[a][c].im)));
    nrm[h * Hd + i] = m;
    __syncthreads();
    m = fmaxf(nrm[i], nrm[Hd + i]);
    float inv = m > 0.f ? 1.f / m : 0.f;
    if (h == 0) E.norm[d * Hd + i] = m;
    uint2* q = reinterpret_cast<uint2*>(E.p);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int k = 2 * t;            // complex pair (k, k+1) of this half
      int pair = 3 * h + t;     // pair number inside the site's 12 complex numbers
      int u = pair >> 1, j = pair & 1;
      q[((d * 3 + u) * Hd + i) * 2 + j] =
          make_uint2(f2h(v.c[k / 3][k % 3].re * inv, v.c[k / 3][k % 3].im * inv),
                     f2h(v.c[(k + 1) / 3][(k + 1) % 3].re * inv, v.c[(k + 1) / 3][(k + 1) % 3].im * inv));
    }
  }
};

// ------------------------------------------------------------------ face code, run-time direction
// Face coupling and face output run once per visit; with the direction as a loop variable
// (only the spin projection and reconstruction are selected per direction, warp-uniform)
// their code stays small.
__device__ inline void project_rt(int mu, int dir, const Spinor<float>& p, Half<float>& h) {
  // forward hop uses (1 - gamma_mu), backward (1 + gamma_mu)
  switch (2 * mu + (dir < 0)) {
    case 0: project<0, -1>(p, h); break;
    case 1: project<0, +1>(p, h); break;
    case 2: project<1, -1>(p, h); break;
    case 3: project<1, +1>(p, h); break;
    case 4: project<2, -1>(p, h); break;
    case 5: project<2, +1>(p, h); break;
    case 6: project<3, -1>(p, h); break;
    default: project<3, +1>(p, h); break;
  }
}
__device__ inline void recon_rt(int mu, int dir, Spinor<float>& acc, const Half<float>& h) {
  switch (2 * mu + (dir < 0)) {
    case 0: accum_recon<0, -1>(acc, h); break;
    case 1: accum_recon<0, +1>(acc, h); break;
    case 2: accum_recon<1, -1>(acc, h); break;
    case 3: accum_recon<1, +1>(acc, h); break;
    case 4: accum_recon<2, -1>(acc, h); break;
    case 5: accum_recon<2, +1>(acc, h); break;
    case 6: accum_recon<3, -1>(acc, h); break;
    default: accum_recon<3, +1>(acc, h); break;
  }
}

// U_mu(site r) for dir > 0, U_mu(site r)^dag for dir < 0.
template <typename MT>
__device__ inline void link_rt(const MatBlock<MT>& M, int mu, int r, int dir, Link<float>& U) {
  Link<float> L;
  M.link(mu, r, L);
  if (dir > 0) {
    U = L;
  } else {
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 3; ++b2) U.e[a2][b2] = mk(L.e[b2][a2].re, -L.e[b2][a2].im);
  }
}

// Masks of the directions whose forward / backward neighbour is inside the domain.
__device__ inline void inside_masks(const Geom& g, const int l[4], unsigned& fwd, unsigned& bwd) {
  fwd = bwd = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    fwd |= (l[mu] + 1 < g.b[mu] ? 1u : 0u) << mu;
    bwd |= (l[mu] > 0 ? 1u : 0u) << mu;
  }
}

// acc += couplings to the neighbouring domains from their face buffers (see face_hop_mu).
template <typename MT>
__device__ inline void face_hops_rt(const Geom& g, int d, const int n[4], const int l[4], unsigned fwd, unsigned bwd,
                                    int r_self, const float4* faces, const MatBlock<MT>& M, Spinor<float>& acc) {
  int fidx[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) fidx[mu] = face_index(g, l, mu);
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const int dir = (k & 1) ? -1 : 1;
    if ((((dir > 0 ? fwd : bwd) >> mu) & 1u)) continue;   // neighbour inside: not a face hop
    long long dn;
    int fi;
    switch (mu) {   // register arrays are only indexed with constants
      case 0: dn = neighbour_domain(g, d, n, 0, dir); fi = fidx[0]; break;
      case 1: dn = neighbour_domain(g, d, n, 1, dir); fi = fidx[1]; break;
      case 2: dn = neighbour_domain(g, d, n, 2, dir); fi = fidx[2]; break;
      default: dn = neighbour_domain(g, d, n, 3, dir); fi = fidx[3]; break;
    }
    const float4* q = faces + (dn * g.face_block + g.face_off[2 * mu + (dir > 0 ? 0 : 1)] + fi) * 3;
    Half<float> h, uh;
    ld_half(q, h);
    if (dir > 0) {
      Link<float> U;
      M.link(mu, r_self, U);
      su3_mul(U, h, uh);
    } else {
      uh = h;
    }
    recon_rt(mu, dir, acc, uh);
  }
}

// Projected half-spinors of dl on this site's faces (see face_write_mu).
template <typename MT>
__device__ inline void face_write_rt(const Geom& g, long long d, const int l[4], unsigned fwd, unsigned bwd,
                                     int r_self, float4* faces, const MatBlock<MT>& M, const Spinor<float>& dl) {
  int fidx[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) fidx[mu] = face_index(g, l, mu);
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const int side = k & 1;          // 0: -mu face (l_mu = 0), 1: +mu face (l_mu = b_mu - 1)
    if (side == 0 ? ((bwd >> mu) & 1u) : ((fwd >> mu) & 1u)) continue;
    int fi;
    switch (mu) {
      case 0: fi = fidx[0]; break;
      case 1: fi = fidx[1]; break;
      case 2: fi = fidx[2]; break;
      default: fi = fidx[3]; break;
    }
    Half<float> h, uh;
    // -mu face: P^-_mu dl for the neighbour's forward hop; +mu face: U^dag P^+_mu dl
    project_rt(mu, side == 0 ? 1 : -1, dl, h);
    if (side == 1) {
      Link<float> U;
      link_rt(M, mu, r_self, -1, U);
      su3_mul(U, h, uh);
    } else {
      uh = h;
    }
    st_half(faces + (d * g.face_block + g.face_off[2 * mu + side] + fi) * 3, uh);
  }
}

// ------------------------------------------------------------------ packed FP16 arithmetic
// Optional form of the domain solve's two products, in half2 arithmetic (two FP16 lanes
// per instruction) straight from the FP16 links and Schwarz matrices in shared memory.
//  - SU(3) times a half-spinor is spin-vectorised: the two spin rows of one colour share
//    a half2 (re = (s0.re, s1.re), im = (s0.im, s1.im)), so each link element, broadcast
//    to both lanes, enters four fused multiply-adds that cover both spins.
//  - A Hermitian 6x6 block times a 6-vector keeps (re, im) in a half2 and a copy of i x
//    per input entry, (-im, re); an entry L enters y_i += Lr x_j + Li (i x_j) and, as
//    conj(L), y_j += Lr x_i - Li (i x_i).
// Hop sums, MR reductions and vector updates stay FP32; values are scaled per domain into
// FP16's range before they meet these products (sap_pair_body).
struct HalfH2 {
  __half2 re[3], im[3];   // colour c: (spin 0, spin 1) of the real and imaginary parts
};

__device__ inline __half2 as_h2(uint32_t w) { return *reinterpret_cast<__half2*>(&w); }

__device__ inline void pack_h2(const Half<float>& h, HalfH2& o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.re[c] = __floats2half2_rn(h.c[0][c].re, h.c[1][c].re);
    o.im[c] = __floats2half2_rn(h.c[0][c].im, h.c[1][c].im);
  }
}
__device__ inline void unpack_h2(const HalfH2& o, Half<float>& h) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 r = __half22float2(o.re[c]), i = __half22float2(o.im[c]);
    h.c[0][c] = mk(r.x, i.x);
    h.c[1][c] = mk(r.y, i.y);
  }
}

// o = U h (DAG false) or U^dag h (DAG true); u: the 9 (re, im) words of U, stride Vd.
template <bool DAG>
__device__ inline void su3_h2(const __half2* u, int Vd, const HalfH2& h, HalfH2& o) {
  __half2 U[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) U[e] = u[e * Vd];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    __half2 re, im;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const __half2 e = DAG ? U[3 * b + a] : U[3 * a + b];
      const __half2 er = __low2half2(e), ei = __high2half2(e);
      // U h:     re += er h.re - ei h.im,  im += er h.im + ei h.re
      // U^dag h: re += er h.re + ei h.im,  im += er h.im - ei h.re
      if (b == 0) {
        re = __hmul2(er, h.re[b]);
        im = __hmul2(er, h.im[b]);
      } else {
        re = __hfma2(er, h.re[b], re);
        im = __hfma2(er, h.im[b], im);
      }
      re = __hfma2(DAG ? ei : __hneg2(ei), h.im[b], re);
      im = __hfma2(DAG ? __hneg2(ei) : ei, h.re[b], im);
    }
    o.re[a] = re;
    o.im[a] = im;
  }
}

// y = H x for block H of site r; the block's 18 words are 3 pairs of diagonal entries
// and the 15 lower entries (re, im) in the order of tri(i, j).
template <int H>
__device__ inline void clover_block_h2(const MatBlock<__half>& M, int r, const __half2 x[6], __half2 y[6]) {
  uint32_t w[20];   // units 4H .. 4H+4 of the site; block word k is w[2H + k]
#pragma unroll
  for (int u = 0; u < 5; ++u) {
    uint4 v = M.cm[(4 * H + u) * M.Vd + r];
    w[4 * u] = v.x;
    w[4 * u + 1] = v.y;
    w[4 * u + 2] = v.z;
    w[4 * u + 3] = v.w;
  }
  const __half2 sgn = __floats2half2_rn(-1.f, 1.f);
  __half2 xs[6];   // i x = (-im, re)
#pragma unroll
  for (int j = 0; j < 6; ++j) xs[j] = __hmul2(__lowhigh2highlow(x[j]), sgn);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const __half2 d = as_h2(w[2 * H + i / 2]);
    y[i] = __hmul2((i & 1) ? __high2half2(d) : __low2half2(d), x[i]);
  }
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const __half2 L = as_h2(w[2 * H + 3 + tri(i, j)]);
      const __half2 lr = __low2half2(L), li = __high2half2(L);
      y[i] = __hfma2(lr, x[j], y[i]);
      y[i] = __hfma2(li, xs[j], y[i]);
      y[j] = __hfma2(lr, x[i], y[j]);
      y[j] = __hfma2(__hneg2(li), xs[i], y[j]);
    }
}

template <typename MT, bool H2>
__device__ inline void block_apply_pair(const MatBlock<MT>& M, int r, int h, const Half<float>& x, Half<float>& y) {
  if constexpr (H2) {
    __half2 xv[6], yv[6];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) xv[3 * s + c] = __floats2half2_rn(x.c[s][c].re, x.c[s][c].im);
    if (h == 0) clover_block_h2<0>(M, r, xv, yv);
    else clover_block_h2<1>(M, r, xv, yv);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 f = __half22float2(yv[3 * s + c]);
        y.c[s][c] = mk(f.x, f.y);
      }
  } else {
    block_apply(M, r, h, x, y);
  }
}

// Hops of one direction with the inside-the-domain test taken from bit masks, so the
// phase loop carries four small integers instead of two coordinate arrays.
template <int MU, typename MT, bool H2>
__device__ inline void hop_mask_mu(const Geom& g, unsigned fwd, unsigned bwd, int lex, int p, int r_self,
                                   const float4* src, const MatBlock<MT>& M, Spinor<float>& acc) {
  Spinor<float> psi;
  Half<float> h, uh;
  if ((fwd >> MU) & 1u) {
    int j = (lex + g.bstride[MU]) >> 1;
    ld_buf(src, g.Hd, j, psi);
    project<MU, -1>(psi, h);
    if constexpr (H2) {
      HalfH2 hh, oh;
      pack_h2(h, hh);
      su3_h2<false>(reinterpret_cast<const __half2*>(M.lk) + MU * 9 * g.Vd + r_self, g.Vd, hh, oh);
      unpack_h2(oh, uh);
    } else {
      Link<float> L;
      M.link(MU, r_self, L);
      su3_mul(L, h, uh);
    }
    accum_recon<MU, -1>(acc, uh);
  }
  if ((bwd >> MU) & 1u) {
    int j = (lex - g.bstride[MU]) >> 1;
    ld_buf(src, g.Hd, j, psi);
    project<MU, +1>(psi, h);
    if constexpr (H2) {
      HalfH2 hh, oh;
      pack_h2(h, hh);
      su3_h2<true>(reinterpret_cast<const __half2*>(M.lk) + MU * 9 * g.Vd + (1 - p) * g.Hd + j, g.Vd, hh, oh);
      unpack_h2(oh, uh);
    } else {
      Link<float> L;
      M.link(MU, (1 - p) * g.Hd + j, L);
      su3_dag_mul(L, h, uh);
    }
    accum_recon<MU, +1>(acc, uh);
  }
}

template <typename MT, bool H2>
__device__ inline void hops_half_mask(int h, const Geom& g, unsigned fwd, unsigned bwd, int lex, int p, int r_self,
                                      const float4* src, const MatBlock<MT>& M, Spinor<float>& acc) {
  if (h == 0) {
    hop_mask_mu<0, MT, H2>(g, fwd, bwd, lex, p, r_self, src, M, acc);
    hop_mask_mu<1, MT, H2>(g, fwd, bwd, lex, p, r_self, src, M, acc);
  } else {
    hop_mask_mu<2, MT, H2>(g, fwd, bwd, lex, p, r_self, src, M, acc);
    hop_mask_mu<3, MT, H2>(g, fwd, bwd, lex, p, r_self, src, M, acc);
  }
}

// Two threads per site.  The MR iteration is a loop over hop phases, so the hop and
// clover code appears once (the whole kernel then fits the instruction cache):
//   phase 0:          even sites, src = t_o      -> rho = r_e + 1/2 H t_o, x = 0
//   phase 2k+1:       odd sites,  src = rho      -> t = A_oo^{-1} H rho
//   phase 2k+2:       even sites, src = t        -> p = A_ee rho - 1/4 H t, MR step
//   phase 2 I_d + 1:  odd sites,  src = x        -> delta_o = A_oo^{-1} (r_o + 1/2 H x)
// cta: index of the domain among the domains of the given colour.
// H2: hop and clover products in packed FP16 (see su3_h2); the domain's residual is then
// scaled by a power of two, 16 / 2^ceil(log2 max|r|), before it enters the work buffers,
// and everything that leaves them (the new residual, delta) is scaled back.  The MR
// iteration is invariant under that scaling and powers of two are exact in FP32.
template <typename MT, typename VT, bool MSMEM, bool H2, int SHAPE = 0>
__device__ __forceinline__ void sap_pair_body(const SapArgs& a, int cta) {
  // hop phases use g (constant domain fields when SHAPE != 0); the face code, which indexes
  // the face offsets at run time, reads the kernel parameters a.g directly
  const Geom g = fixed_shape<SHAPE>(a.g);
  extern __shared__ float4 smem[];
  __shared__ uint64_t mbar, mbar_inj;   // staged copies; injected bytes (test hook)
  __shared__ float4 red[2 * SAP_MAX_THREADS / 32];
  __shared__ float nrm[2 * SAP_MAX_THREADS];
  const int tid = threadIdx.x;
  const int Hd = g.Hd, Vd = g.Vd;
  const int h = tid >= Hd;          // MR phases: chirality half and hop directions; ends: parity
  const int i = tid - h * Hd;

  // Domain-independent set-up: this thread's sites (even site i and odd site i), their
  // local coordinates, hop masks and the shared-memory regions.
  const size_t lk_elems = (size_t)4 * 9 * Vd;
  const size_t lk_bytes = (size_t)MatBlock<MT>::link_bytes_per_site * Vd;
  const size_t cm_bytes = (size_t)MatBlock<MT>::mat_bytes_per_site * Vd;
  char* sbase = reinterpret_cast<char*>(smem);
  MatBlock<MT> M;
  M.Vd = Vd;
  typedef typename std::remove_const<typename std::remove_pointer<decltype(M.lk)>::type>::type LkT;
  typedef typename std::remove_const<typename std::remove_pointer<decltype(M.cm)>::type>::type CmT;
  float4* sE = MSMEM ? reinterpret_cast<float4*>(sbase + lk_bytes + cm_bytes) : smem;
  float4* sO = sE + 6 * Hd;
  if (MSMEM) {
    M.lk = reinterpret_cast<const LkT*>(sbase);
    M.cm = reinterpret_cast<const CmT*>(sbase + lk_bytes);
  }
  int le[4], lo[4];
  local_coords(g, 0, i, le);
  local_coords(g, 1, i, lo);
  const int lex_e = le[0] + g.bstride[1] * le[1] + g.bstride[2] * le[2] + g.bstride[3] * le[3];
  const int lex_o = lo[0] + g.bstride[1] * lo[1] + g.bstride[2] * lo[2] + g.bstride[3] * lo[3];
  unsigned fe, be, fo, bo;
  inside_masks(g, le, fe, be);
  inside_masks(g, lo, fo, bo);
  const int r_e = i, r_o = Hd + i;
  const int r_site = h * Hd + i;
  const unsigned fs = h ? fo : fe, bs = h ? bo : be;

  // This CTA's domain: the cta-th of the launch (the additive form runs both colours, colour
  // 0 first).  Its links and Schwarz matrices are copied into shared memory on an mbarrier
  // while the residual is loaded.
  const int ndom = a.both_colours ? g.ND : (g.ND >> 1);
  int n[4], colour;
  long long d;
  {
    colour = a.both_colours ? (cta >= (g.ND >> 1)) : a.colour;
    const int cidx = a.both_colours ? cta - colour * (g.ND >> 1) : cta;
    int hx = g.N[0] >> 1;
    int j = cidx % hx;
    int row = cidx / hx;
    n[1] = row % g.N[1];
    n[2] = (row / g.N[1]) % g.N[2];
    n[3] = row / (g.N[1] * g.N[2]);
    n[0] = 2 * j + ((colour + n[1] + n[2] + n[3]) & 1);
    d = n[0] + (long long)g.dstride[1] * n[1] + (long long)g.dstride[2] * n[2] + (long long)g.dstride[3] * n[3];
  }
  const LkT* glk = reinterpret_cast<const LkT*>(a.links) + d * lk_elems;
  const CmT* gcm = reinterpret_cast<const CmT*>(a.smat) + d * (cm_bytes / sizeof(CmT));
  if (cta >= ndom) return;
  if (MSMEM) {
    if (tid == 0) {
      mbar_init(&mbar, 1);
      mbar_init(&mbar_inj, 1);
    }
    __syncthreads();
    if (tid == 0) {
      mbar_expect_tx(&mbar, (uint32_t)(lk_bytes + cm_bytes));
      bulk_g2s(sbase, glk, (uint32_t)lk_bytes, &mbar);
      bulk_g2s(sbase + lk_bytes, gcm, (uint32_t)cm_bytes, &mbar);
      // test hook: bytes that nobody sends, on a barrier of their own
      if (a.extra_tx) mbar_expect_tx(&mbar_inj, a.extra_tx);
    }
  } else {
    M.lk = glk;
    M.cm = gcm;
  }
  const long long s_site = (d << g.lgVd) + h * Hd + i;

  // Right-hand sides share the staged matrices; each has its own input, output and state.
#pragma unroll 1
  for (int rhs = 0; rhs < a.nrhs; ++rhs) {
  float4* const fr = a.faces + rhs * a.f_stride;
  float4* const fw = a.faces_out + rhs * a.f_stride;
  float* const rnr = a.r_norm ? a.r_norm + rhs * a.rn_stride : nullptr;
  float* const unr = a.u_norm ? a.u_norm + rhs * a.un_stride : nullptr;
  float inv_sc = 1.f;   // H2: undoes the domain's scaling on the way out
  // 1. residual of site (parity h, index i), with the couplings to the other colour
  EvenStore<VT> rst{reinterpret_cast<decltype(EvenStore<VT>::p)>((char*)a.r_store + rhs * a.r_bytes), rnr};
  {
    Spinor<float> r;
    const SpinorPtr<float> vin{const_cast<float4*>(a.vptr ? a.vptr[rhs] : a.v + rhs * a.v_stride)};
    if (a.first) {
      vin.load(g, s_site, r);
      if (a.vscale) {
        const float sc = *a.vscale;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) r.c[sp][c] = sc * r.c[sp][c];
      }
    } else if (h == 0) {
      rst.load(d, Hd, i, r);
    } else {
      zero(r);
    }
    if (MSMEM && rhs == 0) {
      bool ok = mbar_wait(&mbar, 0, a.wait_ns);
      if (a.extra_tx) ok = mbar_wait(&mbar_inj, 0, a.wait_ns) && ok;
      if (__syncthreads_or(!ok)) {
        // as in sap_kernel: flag, then a bounded wait for the real copies before leaving
        if (tid == 0) atomicExch(a.err, 1);
        mbar_wait(&mbar, 0, a.wait_ns);
        return;
      }
    }
    if (a.use_faces) {
      Spinor<float> acc;
      zero(acc);
      if (h) face_hops_rt(a.g, (int)d, n, lo, fs, bs, r_site, fr, M, acc);
      else face_hops_rt(a.g, (int)d, n, le, fs, bs, r_site, fr, M, acc);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) r.c[s][c] = r.c[s][c] + 0.5f * acc.c[s][c];
    }
    if constexpr (H2) {
      float m = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) m = fmaxf(m, fmaxf(fabsf(r.c[s][c].re), fabsf(r.c[s][c].im)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((tid & 31) == 0) red[tid >> 5].x = m;
      __syncthreads();
      m = 0.f;
      for (int w = 0; w < (2 * Hd + 31) >> 5; ++w) m = fmaxf(m, red[w].x);
      int e = 0;
      frexpf(m, &e);   // m < 2^e
      const float sc = m > 0.f ? ldexpf(1.f, 4 - max(e, -100)) : 1.f;   // finite even for tiny m
      inv_sc = 1.f / sc;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) r.c[s][c] = mk(r.c[s][c].re * sc, r.c[s][c].im * sc);
    }
    st_buf(h ? sO : sE, Hd, i, r);
  }
  __syncthreads();
  Half<float> roh, t, own, rho, x;
  ld_hbuf(sE, Hd, i, h, rho);              // rho starts as r_e; phase 0 adds 1/2 H t_o
  ld_hbuf(sO, Hd, i, h, roh);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) x.c[s][c] = mk(0.f, 0.f);
  block_apply_pair<MT, H2>(M, r_o, h, roh, t);   // t_o = A_oo^{-1} r_o
  st_hbuf(sO, Hd, i, h, t);
  __syncthreads();

  // 2.-4. preparation, MR steps and odd reconstruction as one loop over hop phases
  const int nph = 2 * a.i_domain + 2;
  const int nwarp = (2 * Hd + 31) >> 5;
#pragma unroll 1
  for (int ph = 0; ph < nph; ++ph) {
    const int odd = ph & 1;
    Spinor<float> acc;
    zero(acc);
    // the hop code is specialised per direction pair (h) but appears once in the loop
    hops_half_mask<MT, H2>(h, g, odd ? fo : fe, odd ? bo : be, odd ? lex_o : lex_e, odd, odd ? r_o : r_e,
                           odd ? sE : sO, M, acc);
    exchange(acc, h, odd ? sO : sE, Hd, i, own);
    if (ph == 0) {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) rho.c[s][c] = rho.c[s][c] + 0.5f * own.c[s][c];
      st_hbuf(sE, Hd, i, h, rho);
    } else {
      // one clover-block application per phase: A_oo^{-1} on odd phases, A_ee rho on even
      Half<float> bin;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          bin.c[s][c] = !odd ? rho.c[s][c] : (ph == nph - 1 ? roh.c[s][c] + 0.5f * own.c[s][c] : own.c[s][c]);
      block_apply_pair<MT, H2>(M, odd ? r_o : r_e, h, bin, t);
      if (odd) st_hbuf(sO, Hd, i, h, t);
    }
    if (ph != 0 && !odd) {
      Half<float> pv = t;
      float pr_re = 0.f, pr_im = 0.f, pp = 0.f;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pv.c[s][c] = pv.c[s][c] - 0.25f * own.c[s][c];
          cx<float> q = cjmul(pv.c[s][c], rho.c[s][c]);
          pr_re += q.re;
          pr_im += q.im;
          pp += pv.c[s][c].re * pv.c[s][c].re + pv.c[s][c].im * pv.c[s][c].im;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        pr_re += __shfl_xor_sync(0xffffffffu, pr_re, o);
        pr_im += __shfl_xor_sync(0xffffffffu, pr_im, o);
        pp += __shfl_xor_sync(0xffffffffu, pp, o);
      }
      if ((tid & 31) == 0) red[tid >> 5] = make_float4(pr_re, pr_im, pp, 0.f);
      __syncthreads();
      // every warp sums the nwarp partial sums the same way (lane l holds entry l, a
      // butterfly over the lanes, lane 0's total broadcast), so all threads get one alpha
      float sr = 0.f, si = 0.f, sp = 0.f;
      {
        const int lane = tid & 31;
        if (lane < nwarp) {
          const float4 q = red[lane];
          sr = q.x;
          si = q.y;
          sp = q.z;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          if (o >= nwarp) break;
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
          sp += __shfl_xor_sync(0xffffffffu, sp, o);
        }
        sr = __shfl_sync(0xffffffffu, sr, 0);
        si = __shfl_sync(0xffffffffu, si, 0);
        sp = __shfl_sync(0xffffffffu, sp, 0);
      }
      cx<float> alpha = sp > 0.f ? mk(sr / sp, si / sp) : mk(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x.c[s][c] = x.c[s][c] + cmul(alpha, rho.c[s][c]);
          rho.c[s][c] = rho.c[s][c] - cmul(alpha, pv.c[s][c]);
        }
      // the last MR step hands x to the reconstruction phase instead of rho
      st_hbuf(sE, Hd, i, h, ph == nph - 2 ? x : rho);
    }
    __syncthreads();
  }
  if (!a.last) {
    if constexpr (H2) {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) rho.c[s][c] = mk(rho.c[s][c].re * inv_sc, rho.c[s][c].im * inv_sc);
    }
    EvenHalfStore<VT>::store(rst, nrm, d, Hd, i, h, rho);
    __syncthreads();
  }

  // 5. site (h, i): u += delta, faces of delta
  Spinor<float> dl;
  ld_buf(h ? sO : sE, Hd, i, dl);
  if constexpr (H2) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) dl.c[s][c] = mk(dl.c[s][c].re * inv_sc, dl.c[s][c].im * inv_sc);
  }
  typename VecPtr<VT>::type ust = VecPtr<VT>::make((char*)a.u_store + rhs * a.u_bytes, unr);
  Spinor<float> u;
  if (a.first) {
    u = dl;
  } else {
    ust.load(g, s_site, u);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) u.c[s][c] = u.c[s][c] + dl.c[s][c];
  }
  if (a.last) {
    SpinorPtr<float> zo{a.zptr ? a.zptr[rhs] : a.z + rhs * a.v_stride};
    zo.store(g, s_site, u);
  } else {
    ust.store(g, s_site, u);
  }
  // faces for the next half-sweep (none after the very last one)
  if (!(a.last && (a.both_colours || colour == 1))) {
    if (h) face_write_rt(a.g, d, lo, fs, bs, r_site, fw, M, dl);
    else face_write_rt(a.g, d, le, fs, bs, r_site, fw, M, dl);
  }
  __syncthreads();   // the work buffers are reused by the next right-hand side
  }
}

// One CTA per domain (measured faster on GB300 than a persistent grid walking its domains
// with the next domain's copies in flight: the round-robin tail and the extra live state
// cost more than the overlap gains).
template <typename MT, typename VT, bool MSMEM, bool H2, int SHAPE>
__global__ void __launch_bounds__(2 * SAP_MAX_THREADS, 1) sap_kernel_pair(SapArgs a) {
  sap_pair_body<MT, VT, MSMEM, H2, SHAPE>(a, blockIdx.x);
}

// Several lattices of the same domain shape in one launch: the grid is the concatenation
// of every lattice's domains of the colour; lattice l owns CTAs first[l] .. first[l+1]-1.
constexpr int SAP_MAX_LATTICES = 4;
struct SapLattices {
  SapArgs lat[SAP_MAX_LATTICES];
  int first[SAP_MAX_LATTICES + 1];
  int nlat;
};

template <typename MT, typename VT, bool MSMEM>
__global__ void __launch_bounds__(2 * SAP_MAX_THREADS, 1) sap_kernel_pair_lattices(SapLattices m) {
  int l = 0;
  while (l + 1 < m.nlat && (int)blockIdx.x >= m.first[l + 1]) ++l;
  switch (l) {   // constant indices keep the arguments in the parameter space
    case 0: sap_pair_body<MT, VT, MSMEM, false>(m.lat[0], blockIdx.x - m.first[0]); break;
    case 1: sap_pair_body<MT, VT, MSMEM, false>(m.lat[1], blockIdx.x - m.first[1]); break;
    case 2: sap_pair_body<MT, VT, MSMEM, false>(m.lat[2], blockIdx.x - m.first[2]); break;
    default: sap_pair_body<MT, VT, MSMEM, false>(m.lat[3], blockIdx.x - m.first[3]); break;
  }
}

size_t sap_smem_bytes(const Geom& g, int mat_prec, bool mat_in_smem) {
  size_t vec = (size_t)2 * 6 * g.Hd * 16;
  if (!mat_in_smem) return vec;
  size_t per = mat_prec == P16 ? (MatBlock<__half>::link_bytes_per_site + MatBlock<__half>::mat_bytes_per_site)
                               : (MatBlock<float>::link_bytes_per_site + MatBlock<float>::mat_bytes_per_site);
  return vec + per * g.Vd;
}

static int smem_optin();
bool sap_mat_fits_smem(const Geom& g, int mat_prec) {
  return sap_smem_bytes(g, mat_prec, true) + 1024 <= (size_t)smem_optin();
}

static int smem_optin() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return v;
}

int sap_max_domain_sites() { return 2 * SAP_MAX_THREADS; }

template <typename MT, typename VT, bool MSMEM, bool H2, int SHAPE>
static void launch_pair(const SapArgs& a, int grid, size_t smem, cudaStream_t st) {
  static int configured = 0;
  if (!configured) {
    // static shared memory (barriers, reduction slots) is a few KB; the rest may be dynamic
    cudaFuncSetAttribute(sap_kernel_pair<MT, VT, MSMEM, H2, SHAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem_optin() - 4096);
    configured = 1;
  }
  sap_kernel_pair<MT, VT, MSMEM, H2, SHAPE><<<grid, 2 * a.g.Hd, smem, st>>>(a);
}

template <typename MT, typename VT, bool MSMEM, bool H2 = false>
static int launch_one(const SapArgs& a, int grid, int pair, cudaStream_t st) {
  size_t smem = sap_smem_bytes(a.g, std::is_same<MT, __half>::value ? P16 : P32, MSMEM);
  if (pair) {
    switch (domain_shape_id(a.g)) {
      case 1: launch_pair<MT, VT, MSMEM, H2, 1>(a, grid, smem, st); break;
      case 2: launch_pair<MT, VT, MSMEM, H2, 2>(a, grid, smem, st); break;
      default: launch_pair<MT, VT, MSMEM, H2, 0>(a, grid, smem, st); break;
    }
  } else {
    static int configured = 0;
    if (!configured) {
      cudaFuncSetAttribute(sap_kernel<MT, VT, MSMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin() - 1024);
      configured = 1;
    }
    sap_kernel<MT, VT, MSMEM><<<grid, a.g.Hd, smem, st>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

static SapArgs make_args(const Geom& g, const SapState& S, int colour, int first, int use_faces, int last,
                         const float4* v, float4* z, int i_domain);

// All lattices' domains of one colour in one launch (FP16 storage, two threads per site,
// same domain shape everywhere).
int sap_half_sweep_lattices(const Geom* gs, const SapState* Ss, int nlat, int colour, int first, int use_faces,
                            int last, const float4* const* v, float4* const* z, int i_domain, cudaStream_t st) {
  if (nlat < 1 || nlat > SAP_MAX_LATTICES) return -1;
  SapLattices m;
  m.nlat = nlat;
  int total = 0;
  for (int l = 0; l < nlat; ++l) {
    const Geom& g = gs[l];
    if (g.Hd != gs[0].Hd || g.Hd > SAP_MAX_THREADS || (g.Hd & 31) || Ss[l].mat_prec != P16 || Ss[l].vec_prec != P16 ||
        Ss[l].mat_in_smem != Ss[0].mat_in_smem)
      return -1;
    m.lat[l] = make_args(g, Ss[l], colour, first, use_faces, last, v[l], z[l], i_domain);
    m.first[l] = total;
    total += g.ND / 2;
  }
  m.first[nlat] = total;
  const bool ms = Ss[0].mat_in_smem;
  size_t smem = sap_smem_bytes(gs[0], P16, ms);
  if (ms) {
    static int configured = 0;
    if (!configured) {
      cudaFuncSetAttribute(sap_kernel_pair_lattices<__half, __half, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem_optin() - 4096);
      configured = 1;
    }
    sap_kernel_pair_lattices<__half, __half, true><<<total, 2 * gs[0].Hd, smem, st>>>(m);
  } else {
    sap_kernel_pair_lattices<__half, __half, false><<<total, 2 * gs[0].Hd, smem, st>>>(m);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int sap_half_sweep(const Geom& g, const SapState& S, int colour, int first, int use_faces, int last,
                   const float4* v, float4* z, int i_domain, cudaStream_t st) {
  if (g.Hd > SAP_MAX_THREADS || (g.Hd & 31)) return -1;
  // only the pair kernel loops over right-hand sides and reads pointer lists
  if ((S.nrhs > 1 || S.vlist) && S.threads_per_site != 2) return -1;
  if (S.both_colours && S.threads_per_site != 2) return -1;   // the additive form: pair kernel only
  SapArgs a = make_args(g, S, colour, first, use_faces, last, v, z, i_domain);
  int grid = S.both_colours ? g.ND : g.ND / 2;
  bool ms = S.mat_in_smem;
  int pr = S.threads_per_site == 2;
  // matrices and vectors are stored in the same precision (FP16 or FP32)
  if (S.mat_prec != S.vec_prec) return -1;
  if (S.half_arith) {   // packed FP16 products: FP16 storage and the two-thread kernel only
    if (S.mat_prec != P16 || !pr) return -1;
    return ms ? launch_one<__half, __half, true, true>(a, grid, 1, st)
              : launch_one<__half, __half, false, true>(a, grid, 1, st);
  }
  if (S.mat_prec == P16)
    return ms ? launch_one<__half, __half, true>(a, grid, pr, st) : launch_one<__half, __half, false>(a, grid, pr, st);
  return ms ? launch_one<float, float, true>(a, grid, pr, st) : launch_one<float, float, false>(a, grid, pr, st);
}

static SapArgs make_args(const Geom& g, const SapState& S, int colour, int first, int use_faces, int last,
                         const float4* v, float4* z, int i_domain) {
  SapArgs a;
  a.g = g;
  a.colour = colour;
  a.first = first;
  a.use_faces = use_faces;
  a.last = last;
  a.i_domain = i_domain;
  a.links = S.links;
  a.smat = S.smat;
  a.r_store = S.r_store;
  a.r_norm = S.r_norm;
  a.u_store = S.u_store;
  a.u_norm = S.u_norm;
  a.faces = S.faces;
  a.faces_out = S.faces_out ? S.faces_out : S.faces;
  a.both_colours = S.both_colours ? 1 : 0;
  a.v = v;
  a.z = z;
  a.vscale = S.vscale;
  a.vptr = S.vlist;
  a.zptr = S.zlist;
  a.err = S.err;
  a.nrhs = S.nrhs;
  a.v_stride = g.V * 6;
  a.f_stride = (long long)g.ND * g.face_block * 3;
  a.r_bytes = S.r_bytes;
  a.u_bytes = S.u_bytes;
  a.rn_stride = g.V / 2;
  a.un_stride = g.V;
  a.extra_tx = S.inject_wait_timeout ? 16u : 0u;
  a.wait_ns = S.inject_wait_timeout ? 50000000ull : 2000000000ull;
  return a;
}

}  // namespace dd

// ------------------------------------------------------------------ allocation-free variant
// Scratch of dd_sap_precondition_noalloc: a fixed array in this module's global memory.
// Every GPU that loads the library holds it until the process exits; every call of the
// allocation-free entry point shares it.
namespace dd {

constexpr size_t SAP_NOALLOC_SCRATCH_BYTES = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_sap_noalloc_scratch[SAP_NOALLOC_SCRATCH_BYTES];

size_t sap_noalloc_scratch_bytes() { return SAP_NOALLOC_SCRATCH_BYTES; }

// Device address of the scratch array on the current device.  In host code the array's
// name is only a stand-in, so the address is looked up with cudaGetSymbolAddress, once per
// device, with that device current; a mutex makes the first lookups from several threads
// safe.  The address belongs to the device's context: after cudaDeviceReset the cache is
// stale, and the library (whose contexts are then invalid too) must not be used on that
// device again in this process.  Returns nullptr if the lookup fails.
void* sap_noalloc_scratch() {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sap_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace dd

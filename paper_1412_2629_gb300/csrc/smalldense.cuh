// Small dense complex FP64 algebra of the outer solver (FGMRES with deflated restarts).
// Everything here works on (m+1) x m problems with m <= DD_MAXM, in column-major
// arrays with leading dimension ld, and compiles for host and device.  The incremental
// least-squares solver runs on the device in one-thread kernels; the deflated restart
// (harmonic Ritz pairs and the new basis coefficients) is written for a team of threads
// that share every step: the solver runs it as one warp on the device, and the C ABI
// runs the same code with a team of one on the host so it can be checked without a GPU.
#pragma once

#include <math.h>

namespace dd {

#define DD_HD __host__ __device__
constexpr int DD_MAXM = 64;

struct zd { double re, im; };
DD_HD inline zd Z(double a, double b = 0.0) { zd z; z.re = a; z.im = b; return z; }
DD_HD inline zd operator+(zd a, zd b) { return Z(a.re + b.re, a.im + b.im); }
DD_HD inline zd operator-(zd a, zd b) { return Z(a.re - b.re, a.im - b.im); }
DD_HD inline zd operator-(zd a) { return Z(-a.re, -a.im); }
DD_HD inline zd operator*(zd a, zd b) { return Z(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
DD_HD inline zd operator*(double s, zd a) { return Z(s * a.re, s * a.im); }
DD_HD inline zd conj(zd a) { return Z(a.re, -a.im); }
DD_HD inline double abs2(zd a) { return a.re * a.re + a.im * a.im; }
// |a| without hypot's scaling: the entries here are far from the FP64 overflow and
// underflow limits, and a plain square root is several times cheaper on the device
DD_HD inline double zabs(zd a) { return sqrt(a.re * a.re + a.im * a.im); }
DD_HD inline zd zdiv(zd a, zd b) {
  double d = abs2(b);
  return Z((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// Plane rotation G = [[c, s], [-conj(s), c]], c real, acting on a pair (a, b).
struct Rot { double c; zd s; };

// Rotation with G [x; y] = [r; 0].
DD_HD inline Rot make_rot(zd x, zd y) {
  Rot g;
  double ax = zabs(x), ay = zabs(y);
  if (ay == 0.0) { g.c = 1.0; g.s = Z(0.0); return g; }
  if (ax == 0.0) { g.c = 0.0; g.s = Z(1.0); return g; }
  double nrm = sqrt(ax * ax + ay * ay);
  zd ph = Z(x.re / ax, x.im / ax);
  g.c = ax / nrm;
  g.s = (1.0 / nrm) * (ph * conj(y));
  return g;
}
DD_HD inline void rot_apply(const Rot& g, zd& a, zd& b) {
  zd a2 = g.c * a + g.s * b;
  zd b2 = g.c * b - conj(g.s) * a;
  a = a2;
  b = b2;
}
// [a, b] G^H  (the matching column operation)
DD_HD inline void rot_apply_right(const Rot& g, zd& a, zd& b) {
  zd a2 = g.c * a + conj(g.s) * b;
  zd b2 = g.c * b - g.s * a;
  a = a2;
  b = b2;
}

// ---------------------------------------------------------------- incremental least squares
// Least squares min |g - Hbar y| by plane rotations, one column at a time.  Column j of
// R (leading dimension ld) is rotated by every stored rotation, then the entries below
// row j are annihilated bottom-up; rows[] records which row pair each rotation acts on.
// Returns the residual norm |g[j+1 .. nrows-1]|.
struct LsqState {
  int nrot;
  int rows[DD_MAXM * DD_MAXM / 2 + DD_MAXM];
  Rot rot[DD_MAXM * DD_MAXM / 2 + DD_MAXM];
};

DD_HD inline double lsq_add_column(LsqState& S, zd* R, int ld, int j, int nrows, zd* g) {
  zd* col = R + (long)j * ld;
  for (int k = 0; k < S.nrot; ++k) rot_apply(S.rot[k], col[S.rows[k]], col[S.rows[k] + 1]);
  for (int i = nrows - 2; i >= j; --i) {
    Rot r = make_rot(col[i], col[i + 1]);
    rot_apply(r, col[i], col[i + 1]);
    col[i + 1] = Z(0.0);
    rot_apply(r, g[i], g[i + 1]);
    S.rows[S.nrot] = i;
    S.rot[S.nrot] = r;
    S.nrot++;
  }
  double res = 0.0;
  for (int i = j + 1; i < nrows; ++i) res += abs2(g[i]);
  return sqrt(res);
}

// Back substitution R[0:n, 0:n] y = g[0:n].
DD_HD inline void lsq_solve(const zd* R, int ld, int n, const zd* g, zd* y) {
  for (int i = n - 1; i >= 0; --i) {
    zd s = g[i];
    for (int j = i + 1; j < n; ++j) s = s - R[i + (long)j * ld] * y[j];
    y[i] = zdiv(s, R[i + (long)i * ld]);
  }
}

// ---------------------------------------------------------------- cooperative team
// The threads that share the deflated restart: thread tid of nt; sync() separates steps
// (a barrier of the CTA on the device, nothing on the host, where nt = 1).  Every member
// runs the same control flow: decisions are taken from data that all of them read after
// the same barrier.
struct Team {
  int tid, nt;
  DD_HD void sync() const {
#ifdef __CUDA_ARCH__
    __syncthreads();
#endif
  }
};

// ---------------------------------------------------------------- Hessenberg LU
// In place LU of the upper Hessenberg A (n x n, ld) with partial pivoting between the two
// rows that can hold column c's pivot: step c swaps rows c, c+1 when |A(c+1, c)| is the
// larger (piv[c] = 1) and subtracts l[c] times row c from row c+1.  An exactly zero pivot
// is replaced by `tiny` (inverse iteration factors matrices that are singular up to
// rounding).  The strictly lower part of A is left undefined.
DD_HD inline void hess_lu(const Team& T, zd* A, int n, int ld, int* piv, zd* l, double tiny) {
  auto a = [&](int i, int j) -> zd& { return A[i + (long)j * ld]; };
  for (int c = 0; c + 1 < n; ++c) {
    const bool sw = abs2(a(c + 1, c)) > abs2(a(c, c));
    T.sync();   // every member has read the pivot candidates
    if (sw)
      for (int j = c + T.tid; j < n; j += T.nt) { zd t = a(c, j); a(c, j) = a(c + 1, j); a(c + 1, j) = t; }
    T.sync();
    zd d = a(c, c);
    if (abs2(d) == 0.0) d = Z(tiny);
    const zd f = zdiv(a(c + 1, c), d);
    T.sync();   // every member has read row c + 1's first entry
    for (int j = c + 1 + T.tid; j < n; j += T.nt) a(c + 1, j) = a(c + 1, j) - f * a(c, j);
    if (T.tid == 0) {
      a(c, c) = d;
      piv[c] = sw ? 1 : 0;
      l[c] = f;
    }
    T.sync();
  }
  if (T.tid == 0 && abs2(a(n - 1, n - 1)) == 0.0) a(n - 1, n - 1) = Z(tiny);
  T.sync();
}

// x <- U^{-1} x for the upper triangle U of A (column-oriented back substitution).
DD_HD inline void upper_solve(const Team& T, const zd* A, int n, int ld, zd* x) {
  for (int i = n - 1; i >= 0; --i) {
    if (T.tid == 0) x[i] = zdiv(x[i], A[i + (long)i * ld]);
    T.sync();
    for (int r = T.tid; r < i; r += T.nt) x[r] = x[r] - A[r + (long)i * ld] * x[i];
    T.sync();
  }
}

// x <- (A^H)^{-1} x for the factored Hessenberg A = (L-steps)^{-1} U: first U^H g = x by
// forward substitution, then the adjoint of every elimination and swap, last step first.
DD_HD inline void hess_solve_adjoint(const Team& T, const zd* A, int n, int ld, const int* piv, const zd* l, zd* x) {
  for (int i = 0; i < n; ++i) {
    if (T.tid == 0) x[i] = zdiv(x[i], conj(A[i + (long)i * ld]));
    T.sync();
    for (int r = i + 1 + T.tid; r < n; r += T.nt) x[r] = x[r] - conj(A[i + (long)r * ld]) * x[i];
    T.sync();
  }
  if (T.tid == 0)
    for (int c = n - 2; c >= 0; --c) {
      x[c] = x[c] - conj(l[c]) * x[c + 1];
      if (piv[c]) { zd t = x[c]; x[c] = x[c + 1]; x[c + 1] = t; }
    }
  T.sync();
}

// x <- A^{-1} x for the factored Hessenberg A: the swaps and eliminations in order, then U.
DD_HD inline void hess_solve(const Team& T, const zd* A, int n, int ld, const int* piv, const zd* l, zd* x) {
  if (T.tid == 0)
    for (int c = 0; c + 1 < n; ++c) {
      if (piv[c]) { zd t = x[c]; x[c] = x[c + 1]; x[c + 1] = t; }
      x[c + 1] = x[c + 1] - l[c] * x[c];
    }
  T.sync();
  upper_solve(T, A, n, ld, x);
}

// ---------------------------------------------------------------- FP32 eigenvalue estimates
// The QR sweeps that locate the harmonic Ritz values run in FP32: each rotation is a short
// chain of square roots and divisions, and in FP64 on the device (GB300's FP64 rate is a
// small fraction of its FP32 rate) that chain dominates the whole restart.  The values only
// order the candidates and shift the inverse iteration, which then computes every kept
// vector and its Rayleigh quotient in FP64.
struct zf { float re, im; };
DD_HD inline zf Zf(float a, float b = 0.f) { zf z; z.re = a; z.im = b; return z; }
DD_HD inline zf operator+(zf a, zf b) { return Zf(a.re + b.re, a.im + b.im); }
DD_HD inline zf operator-(zf a, zf b) { return Zf(a.re - b.re, a.im - b.im); }
DD_HD inline zf operator*(zf a, zf b) { return Zf(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
DD_HD inline zf operator*(float s, zf a) { return Zf(s * a.re, s * a.im); }
DD_HD inline zf conj(zf a) { return Zf(a.re, -a.im); }
DD_HD inline float abs2(zf a) { return a.re * a.re + a.im * a.im; }
DD_HD inline float zabs(zf a) { return sqrtf(a.re * a.re + a.im * a.im); }

struct Rotf { float c; zf s; };
DD_HD inline Rotf make_rot(zf x, zf y) {
  Rotf g;
  const float ax2 = abs2(x), ay2 = abs2(y);
  if (ay2 == 0.f) { g.c = 1.f; g.s = Zf(0.f); return g; }
  if (ax2 == 0.f) { g.c = 0.f; g.s = Zf(1.f); return g; }
  const float ax = sqrtf(ax2), inv = 1.f / sqrtf(ax2 + ay2);
  g.c = ax * inv;
  g.s = (inv / ax) * (x * conj(y));
  return g;
}
DD_HD inline void rot_apply(const Rotf& g, zf& a, zf& b) {
  zf a2 = g.c * a + g.s * b;
  zf b2 = g.c * b - conj(g.s) * a;
  a = a2;
  b = b2;
}
DD_HD inline void rot_apply_right(const Rotf& g, zf& a, zf& b) {
  zf a2 = g.c * a + conj(g.s) * b;
  zf b2 = g.c * b - g.s * a;
  a = a2;
  b = b2;
}

// Eigenvalues of the upper Hessenberg A (n x n, ld) by the implicit single-shift QR
// iteration with Wilkinson shifts (an exceptional shift every 11th step), each sweep
// restricted to the active block [lo, hi], in FP32: A's diagonal holds them on return.
// Returns the number of sweeps, or -1 if the iteration did not converge.
DD_HD inline int hess_eigenvalues_f32(const Team& T, zf* A, int n, int ld) {
  auto a = [&](int i, int j) -> zf& { return A[i + (long)j * ld]; };
  const float eps = 1.1920929e-7f;
  int total = 0, hi = n - 1, iter = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      float s = zabs(a(lo - 1, lo - 1)) + zabs(a(lo, lo));
      if (s == 0.f) s = 1.f;
      if (zabs(a(lo, lo - 1)) <= eps * s) break;
      --lo;
    }
    T.sync();
    if (lo > 0 && T.tid == 0) a(lo, lo - 1) = Zf(0.f);
    T.sync();
    if (lo == hi) { --hi; iter = 0; continue; }
    if (++iter > 60 * n) return -1;
    ++total;
    zf aa = a(hi - 1, hi - 1), bb = a(hi - 1, hi), cc = a(hi, hi - 1), dd = a(hi, hi);
    zf tr2 = 0.5f * (aa + dd);
    zf disc = tr2 * tr2 - (aa * dd - bb * cc);
    const float rr = zabs(disc);
    const float sre = sqrtf(0.5f * (rr + disc.re)), sim = sqrtf(fmaxf(0.f, 0.5f * (rr - disc.re)));
    zf sq = Zf(sre, disc.im < 0.f ? -sim : sim);
    zf l1 = tr2 + sq, l2 = tr2 - sq;
    zf mu = abs2(l1 - dd) < abs2(l2 - dd) ? l1 : l2;
    if (iter % 11 == 10) mu = dd + Zf(zabs(a(hi, hi - 1)), 0.f);
    zf x = a(lo, lo) - mu, y = a(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
      const Rotf r = make_rot(x, y);
      const int c0 = k > lo ? k - 1 : lo;
      T.sync();
      for (int j = c0 + T.tid; j <= hi; j += T.nt) rot_apply(r, a(k, j), a(k + 1, j));
      T.sync();
      const int r1 = k + 2 < hi ? k + 2 : hi;
      for (int i = lo + T.tid; i <= r1; i += T.nt) rot_apply_right(r, a(i, k), a(i, k + 1));
      T.sync();
      if (k > lo && T.tid == 0) a(k + 1, k - 1) = Zf(0.f);
      if (k + 1 < hi) { x = a(k + 1, k); y = a(k + 2, k); }
    }
    T.sync();
  }
  return total;
}

// Dense LU with partial pivoting of A (n x n, ld), applied to b on the way (A is
// overwritten by U, b by U^{-1} L^{-1} P b); then b <- A^{-1} b by back substitution.
// Returns false (all members alike) if a pivot is exactly zero.
DD_HD inline bool dense_solve(const Team& T, zd* A, int n, int ld, zd* b) {
  auto a = [&](int i, int j) -> zd& { return A[i + (long)j * ld]; };
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = -1.0;
    for (int r = c; r < n; ++r) {
      const double v = abs2(a(r, c));
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) return false;
    T.sync();   // every member has read column c
    if (p != c) {
      for (int j = c + T.tid; j < n; j += T.nt) { zd t = a(c, j); a(c, j) = a(p, j); a(p, j) = t; }
      if (T.tid == 0) { zd t = b[c]; b[c] = b[p]; b[p] = t; }
      T.sync();
    }
    for (int r = c + 1 + T.tid; r < n; r += T.nt) {
      const zd f = zdiv(a(r, c), a(c, c));
      for (int j = c + 1; j < n; ++j) a(r, j) = a(r, j) - f * a(c, j);
      b[r] = b[r] - f * b[c];
    }
    T.sync();
  }
  upper_solve(T, A, n, ld, b);
  return true;
}

// Reduction of A (n x n, ld) to upper Hessenberg form by plane rotations, A <- Q^H A Q,
// with Q (ld) accumulated from the identity.  Only nonzero entries below the first
// subdiagonal are rotated away (after a deflated restart that is the dense leading block).
DD_HD inline void hessenberg(const Team& T, zd* A, zd* Q, int n, int ld) {
  auto a = [&](int i, int j) -> zd& { return A[i + (long)j * ld]; };
  auto q = [&](int i, int j) -> zd& { return Q[i + (long)j * ld]; };
  for (int e = T.tid; e < n * n; e += T.nt) q(e % n, e / n) = Z(e % n == e / n ? 1.0 : 0.0);
  T.sync();
  for (int j = 0; j + 2 < n; ++j)
    for (int i = n - 1; i >= j + 2; --i) {
      if (abs2(a(i, j)) == 0.0) continue;   // same decision for every member
      const Rot r = make_rot(a(i - 1, j), a(i, j));
      T.sync();
      for (int k = T.tid; k < n; k += T.nt) rot_apply(r, a(i - 1, k), a(i, k));
      T.sync();
      for (int k = T.tid; k < n; k += T.nt) {
        rot_apply_right(r, a(k, i - 1), a(k, i));
        rot_apply_right(r, q(k, i - 1), q(k, i));
      }
      T.sync();
      if (T.tid == 0) a(i, j) = Z(0.0);
      T.sync();
    }
}

// Workspace of the deflated restart for basis size m: four m x m matrices (leading
// dimension m) and short vectors, carved from one buffer of deflate_bytes(m) bytes
// (host memory, device global memory or shared memory).
struct DeflateWork {
  zd *G, *G0, *M, *Q;
  zf* Gf;                     // FP32 copy for the eigenvalue estimates
  zd *f, *v, *w, *cls, *dot;
  zd* l;
  double *absth, *nrm;
  int *order, *piv;
  int ld;
};
DD_HD inline size_t deflate_bytes(int m) {
  return (size_t)4 * m * m * sizeof(zd) + (size_t)m * m * sizeof(zf) + 6 * (size_t)(DD_MAXM + 1) * sizeof(zd) +
         (DD_MAXM + 1) * sizeof(double) * 2 + 2 * (size_t)(DD_MAXM + 1) * sizeof(int);
}
DD_HD inline DeflateWork deflate_work(void* base, int m) {
  DeflateWork W;
  zd* z = (zd*)base;
  W.ld = m;
  W.G = z; z += m * m;
  W.G0 = z; z += m * m;
  W.M = z; z += m * m;
  W.Q = z; z += m * m;
  W.Gf = (zf*)z; z += (m * m + 1) / 2;
  W.f = z; z += DD_MAXM + 1;
  W.v = z; z += DD_MAXM + 1;
  W.w = z; z += DD_MAXM + 1;
  W.cls = z; z += DD_MAXM + 1;
  W.dot = z; z += DD_MAXM + 1;
  W.l = z; z += DD_MAXM + 1;
  double* d = (double*)z;
  W.absth = d; d += DD_MAXM + 1;
  W.nrm = d; d += DD_MAXM + 1;
  int* i = (int*)d;
  W.order = i; i += DD_MAXM + 1;
  W.piv = i;
  return W;
}

// p <- p - sum_t (p_t^H p) p_t over the first nprev columns of P (ld), twice, then p / |p|;
// returns |p| before the final scaling.
DD_HD inline double orthonormalise(const Team& T, zd* P, int ld, int nprev, int len, zd* p, DeflateWork& W) {
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = T.tid; t < nprev; t += T.nt) {
      const zd* pt = P + (long)t * ld;
      zd d = Z(0.0);
      for (int i = 0; i < len; ++i) d = d + conj(pt[i]) * p[i];
      W.dot[t] = d;
    }
    T.sync();
    for (int i = T.tid; i < len; i += T.nt) {
      zd s = p[i];
      for (int t = 0; t < nprev; ++t) s = s - W.dot[t] * P[i + (long)t * ld];
      p[i] = s;
    }
    T.sync();
  }
  if (T.tid == 0) {
    double n2 = 0;
    for (int i = 0; i < len; ++i) n2 += abs2(p[i]);
    W.nrm[0] = sqrt(n2);
  }
  T.sync();
  const double nrm = W.nrm[0];
  if (nrm > 0)
    for (int i = T.tid; i < len; i += T.nt) p[i] = (1.0 / nrm) * p[i];
  T.sync();
  return nrm;
}

// Deflated restart of flexible GMRES-DR (Sec. II-C; Morgan's GMRES-DR with flexible
// preconditioning).
// In:  Hbar (m+1) x m (ld = ldh), c (m+1), y (m): the cycle's least-squares solution.
//      After a deflated restart the leading (k+1) x k block of Hbar is dense; the rest is
//      upper Hessenberg.
// Out: P (m+1) x (k+1), ld = ldh: orthonormal basis of the k harmonic Ritz vectors of
//      smallest |theta| (padded with a zero row) followed by the least-squares residual
//      vector c - Hbar y; Hn = P^H Hbar P_k ((k+1) x k, ld = ldh); cn = P^H (c - Hbar y);
//      theta[0:m] harmonic Ritz values sorted by |theta| (stable).
// The harmonic Ritz pairs solve (H_m + |h_{m+1,m}|^2 f e_m^H) g = theta g with
// f = H_m^{-H} e_m.  That matrix is reduced to Hessenberg form (Q); FP32 QR sweeps give
// estimates of its eigenvalues, which order the candidates; each kept vector comes from two
// steps of FP64 inverse iteration on the Hessenberg form shifted by its estimate, mapped
// back by Q, and its value from the FP64 Rayleigh quotient (theta[0:k] are FP64 accurate,
// theta[k:m] are the FP32 estimates).  A vector that is not independent of those already
// kept (a repeated eigenvalue) is passed over for the next one in the order.  Returns 0 on success, nonzero if a step failed (the caller then
// restarts plainly); all members of the team return the same value.
DD_HD inline int deflate(const Team& T, const zd* Hbar, int ldh, int m, int k, const zd* c, const zd* y, zd* P, zd* Hn,
                         zd* cn, zd* theta, DeflateWork& W) {
  const int ld = W.ld;
  double hn2 = 0;   // max |H_ij|^2
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= m; ++i) hn2 = fmax(hn2, abs2(Hbar[i + (long)j * ldh]));
  const double hn = sqrt(hn2);
  if (!(hn > 0) || !isfinite(hn)) return 1;
  // f = H_m^{-H} e_m (dense: the leading block need not be Hessenberg)
  for (int q = T.tid; q < m * m; q += T.nt) W.M[q % m + (q / m) * ld] = conj(Hbar[q / m + (long)(q % m) * ldh]);
  for (int i = T.tid; i < m; i += T.nt) W.f[i] = Z(i == m - 1 ? 1.0 : 0.0);
  T.sync();
  if (!dense_solve(T, W.M, m, ld, W.f)) return 1;
  // G = H_m + |h_{m+1,m}|^2 f e_m^H, reduced to Hessenberg form G <- Q^H G Q
  const double h2 = abs2(Hbar[m + (long)(m - 1) * ldh]);
  for (int q = T.tid; q < m * m; q += T.nt) {
    const int i = q % m, j = q / m;
    zd g = Hbar[i + (long)j * ldh];
    if (j == m - 1) g = g + h2 * W.f[i];
    W.G[i + j * ld] = g;
  }
  T.sync();
  hessenberg(T, W.G, W.Q, m, ld);
  for (int q = T.tid; q < m * m; q += T.nt) {
    const zd g = W.G[q % m + (q / m) * ld];
    W.G0[q % m + (q / m) * ld] = g;
    W.Gf[q] = Zf((float)g.re, (float)g.im);
  }
  T.sync();
  // eigenvalue estimates (FP32 QR), ordered by modulus (stable insertion sort)
  if (hess_eigenvalues_f32(T, W.Gf, m, m) < 0) return 2;
  if (T.tid == 0) {
    for (int i = 0; i < m; ++i) { W.absth[i] = (double)zabs(W.Gf[i + i * m]); W.order[i] = i; }
    for (int i = 1; i < m; ++i) {
      int o = W.order[i];
      int j = i - 1;
      while (j >= 0 && W.absth[W.order[j]] > W.absth[o]) { W.order[j + 1] = W.order[j]; --j; }
      W.order[j + 1] = o;
    }
    for (int i = 0; i < m; ++i) {
      const zf t = W.Gf[W.order[i] + W.order[i] * m];
      theta[i] = Z((double)t.re, (double)t.im);
    }
  }
  T.sync();
  // columns of P: for the candidates in that order, two steps of FP64 inverse iteration on
  // the Hessenberg form shifted by the estimate, the Rayleigh quotient as the refined
  // value, the vector mapped back by Q; k independent ones are kept
  const double tiny = 1e-15 * hn;
  int kept = 0;
  for (int cand = 0; cand < m && kept < k; ++cand) {
    const zd th = theta[cand];
    for (int q = T.tid; q < m * m; q += T.nt) {
      const int i = q % m, j = q / m;
      W.M[i + j * ld] = i == j ? W.G0[i + j * ld] - th : W.G0[i + j * ld];
    }
    for (int i = T.tid; i < m; i += T.nt) W.v[i] = Z(1.0);
    T.sync();
    hess_lu(T, W.M, m, ld, W.piv, W.l, tiny);
    bool ok = true;
    for (int it = 0; it < 2 && ok; ++it) {
      if (it == 0) upper_solve(T, W.M, m, ld, W.v);      // U v = (1, ..., 1)
      else hess_solve(T, W.M, m, ld, W.piv, W.l, W.v);   // (G0 - theta) v = v
      if (T.tid == 0) {
        double n2 = 0;
        for (int i = 0; i < m; ++i) n2 += abs2(W.v[i]);
        W.nrm[0] = sqrt(n2);
      }
      T.sync();
      const double nrm = W.nrm[0];
      if (!(nrm > 0) || !isfinite(nrm)) { ok = false; break; }
      for (int i = T.tid; i < m; i += T.nt) W.v[i] = (1.0 / nrm) * W.v[i];
      T.sync();
    }
    if (!ok) continue;
    // Rayleigh quotient v^H G0 v (|v| = 1)
    for (int i = T.tid; i < m; i += T.nt) {
      zd s = Z(0.0);
      for (int j = (i > 0 ? i - 1 : 0); j < m; ++j) s = s + W.G0[i + j * ld] * W.v[j];
      W.w[i] = s;
    }
    T.sync();
    if (T.tid == 0) {
      zd rq = Z(0.0);
      for (int i = 0; i < m; ++i) rq = rq + conj(W.v[i]) * W.w[i];
      theta[cand] = rq;
    }
    // back to the basis of H_m: p = Q v
    zd* p = P + (long)kept * ldh;
    for (int i = T.tid; i <= m; i += T.nt) {
      zd s = Z(0.0);
      if (i < m)
        for (int j = 0; j < m; ++j) s = s + W.Q[i + j * ld] * W.v[j];
      p[i] = s;
    }
    T.sync();
    if (orthonormalise(T, P, ldh, kept, m + 1, p, W) > 1e-8) ++kept;
  }
  if (kept < k) return 3;
  // last column: least-squares residual c - Hbar y
  for (int i = T.tid; i <= m; i += T.nt) {
    zd s = c[i];
    for (int j = 0; j < m; ++j) s = s - Hbar[i + (long)j * ldh] * y[j];
    W.cls[i] = s;
    P[i + (long)k * ldh] = s;
  }
  T.sync();
  if (!(orthonormalise(T, P, ldh, k, m + 1, P + (long)k * ldh, W) > 0)) return 4;
  // Hn = (P^H Hbar) P_k, cn = P^H cls; the product P^H Hbar goes to M ((k+1) x m)
  for (int q = T.tid; q < (k + 1) * m; q += T.nt) {
    const int a = q % (k + 1), j = q / (k + 1);
    const zd* pa = P + (long)a * ldh;
    zd s = Z(0.0);
    for (int i = 0; i <= m; ++i) s = s + conj(pa[i]) * Hbar[i + (long)j * ldh];
    W.M[a + j * ld] = s;
  }
  for (int a = T.tid; a <= k; a += T.nt) {
    const zd* pa = P + (long)a * ldh;
    zd s = Z(0.0);
    for (int i = 0; i <= m; ++i) s = s + conj(pa[i]) * W.cls[i];
    cn[a] = s;
  }
  T.sync();
  for (int q = T.tid; q < (k + 1) * k; q += T.nt) {
    const int a = q % (k + 1), b = q / (k + 1);
    const zd* pb = P + (long)b * ldh;
    zd s = Z(0.0);
    for (int j = 0; j < m; ++j) s = s + W.M[a + j * ld] * pb[j];
    Hn[a + (long)b * ldh] = s;
  }
  T.sync();
  return 0;
}

}  // namespace dd

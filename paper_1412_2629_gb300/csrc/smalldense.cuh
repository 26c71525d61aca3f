// Small dense complex FP64 algebra of the outer solver (FGMRES with deflated restarts).
// Everything here works on (m+1) x m problems with m <= DD_MAXM, in column-major
// arrays with leading dimension ld, and compiles for host and device: the solver runs
// it on the device in a one-thread kernel; the C ABI also exposes the host build so it
// can be checked without a GPU.
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
DD_HD inline double zabs(zd a) { return hypot(a.re, a.im); }
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
  double nrm = hypot(ax, ay);
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

// ---------------------------------------------------------------- eigen-decomposition
// A (n x n, leading dimension ld) is overwritten by its Schur form T = Q^H A Q; Q (ld)
// receives the unitary factor.  Givens reduction to Hessenberg form, then the implicit
// single-shift QR iteration with Wilkinson shifts.  Returns the number of iterations or
// -1 if it did not converge.
DD_HD inline int schur(zd* A, zd* Q, int n, int ld) {
  auto a = [&](int i, int j) -> zd& { return A[i + (long)j * ld]; };
  auto q = [&](int i, int j) -> zd& { return Q[i + (long)j * ld]; };
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) q(i, j) = Z(i == j ? 1.0 : 0.0);
  // Hessenberg reduction: zero a(i, j) for i > j + 1 using rows (i - 1, i)
  for (int j = 0; j + 2 < n; ++j)
    for (int i = n - 1; i >= j + 2; --i) {
      if (abs2(a(i, j)) == 0.0) continue;
      Rot r = make_rot(a(i - 1, j), a(i, j));
      for (int k = 0; k < n; ++k) rot_apply(r, a(i - 1, k), a(i, k));
      for (int k = 0; k < n; ++k) rot_apply_right(r, a(k, i - 1), a(k, i));
      for (int k = 0; k < n; ++k) rot_apply_right(r, q(k, i - 1), q(k, i));
      a(i, j) = Z(0.0);
    }
  int total = 0;
  int hi = n - 1, iter = 0;
  const double eps = 2.220446049250313e-16;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      double s = zabs(a(lo - 1, lo - 1)) + zabs(a(lo, lo));
      if (s == 0.0) s = 1.0;
      if (zabs(a(lo, lo - 1)) <= eps * s) { a(lo, lo - 1) = Z(0.0); break; }
      --lo;
    }
    if (lo == hi) { --hi; iter = 0; continue; }
    if (++iter > 60 * n) return -1;
    ++total;
    // Wilkinson shift: eigenvalue of the trailing 2x2 block closest to a(hi, hi)
    zd aa = a(hi - 1, hi - 1), bb = a(hi - 1, hi), cc = a(hi, hi - 1), dd = a(hi, hi);
    zd tr2 = 0.5 * (aa + dd);
    zd det = aa * dd - bb * cc;
    zd disc = tr2 * tr2 - det;
    double rr = zabs(disc), th = atan2(disc.im, disc.re);
    zd sq = Z(sqrt(rr) * cos(0.5 * th), sqrt(rr) * sin(0.5 * th));
    zd l1 = tr2 + sq, l2 = tr2 - sq;
    zd mu = abs2(l1 - dd) < abs2(l2 - dd) ? l1 : l2;
    if (iter % 11 == 10) mu = dd + Z(zabs(a(hi, hi - 1)), 0.0);   // exceptional shift
    zd x = a(lo, lo) - mu, y = a(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
      Rot r = make_rot(x, y);
      int c0 = k > lo ? k - 1 : lo;
      for (int j = c0; j < n; ++j) rot_apply(r, a(k, j), a(k + 1, j));
      int r1 = k + 2 < hi ? k + 2 : hi;
      for (int i = 0; i <= r1; ++i) rot_apply_right(r, a(i, k), a(i, k + 1));
      for (int i = 0; i < n; ++i) rot_apply_right(r, q(i, k), q(i, k + 1));
      if (k > lo) a(k + 1, k - 1) = Z(0.0);
      if (k + 1 < hi) { x = a(k + 1, k); y = a(k + 2, k); }
    }
  }
  return total;
}

// Eigenvector of the upper triangular T for eigenvalue T(e, e), mapped back by Q and
// normalised; written to v[0:n].
DD_HD inline void schur_eigvec(const zd* T, const zd* Q, int n, int ld, int e, zd* y, zd* v) {
  double tn = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) tn = fmax(tn, zabs(T[i + (long)j * ld]));
  const double small = 1e-15 * (tn > 0 ? tn : 1.0);
  zd lam = T[e + (long)e * ld];
  for (int i = 0; i < n; ++i) y[i] = Z(0.0);
  y[e] = Z(1.0);
  for (int i = e - 1; i >= 0; --i) {
    zd s = Z(0.0);
    for (int j = i + 1; j <= e; ++j) s = s + T[i + (long)j * ld] * y[j];
    zd d = T[i + (long)i * ld] - lam;
    if (zabs(d) < small) d = Z(small);
    y[i] = -zdiv(s, d);
  }
  double nrm = 0;
  for (int i = 0; i < n; ++i) {
    zd s = Z(0.0);
    for (int j = 0; j <= e; ++j) s = s + Q[i + (long)j * ld] * y[j];
    v[i] = s;
    nrm += abs2(s);
  }
  nrm = sqrt(nrm);
  for (int i = 0; i < n; ++i) v[i] = (1.0 / nrm) * v[i];
}

// Solve M x = b (n x n, column-major, overwritten) by Gaussian elimination with
// partial pivoting.  Returns false if a pivot is exactly zero.
DD_HD inline bool dense_solve(zd* M, int n, int ld, zd* b) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = -1;
    for (int r = c; r < n; ++r) if (zabs(M[r + (long)c * ld]) > best) { best = zabs(M[r + (long)c * ld]); p = r; }
    if (best == 0.0) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) { zd t = M[c + (long)j * ld]; M[c + (long)j * ld] = M[p + (long)j * ld]; M[p + (long)j * ld] = t; }
      zd t = b[c]; b[c] = b[p]; b[p] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      zd f = zdiv(M[r + (long)c * ld], M[c + (long)c * ld]);
      for (int j = c; j < n; ++j) M[r + (long)j * ld] = M[r + (long)j * ld] - f * M[c + (long)j * ld];
      b[r] = b[r] - f * b[c];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    zd s = b[i];
    for (int j = i + 1; j < n; ++j) s = s - M[i + (long)j * ld] * b[j];
    b[i] = zdiv(s, M[i + (long)i * ld]);
  }
  return true;
}

// Workspace for the deflated restart, sized for DD_MAXM.
struct DeflateWork {
  zd G[DD_MAXM * DD_MAXM];
  zd Q[DD_MAXM * DD_MAXM];
  zd M[DD_MAXM * DD_MAXM];
  zd f[DD_MAXM + 1];
  zd y[DD_MAXM + 1];
  zd v[DD_MAXM + 1];
  zd cls[DD_MAXM + 1];
  double absth[DD_MAXM];
  int order[DD_MAXM];
};

// Deflated restart of flexible GMRES-DR.
// In:  Hbar (m+1) x m (ld = ldh), c (m+1), y (m): the cycle's least-squares solution.
// Out: P (m+1) x (k+1), ld = ldh: orthonormal basis of the k harmonic Ritz vectors of
//      smallest |theta| (padded with a zero row) followed by the least-squares residual
//      vector c - Hbar y; Hn = P^H Hbar P_k ((k+1) x k, ld = ldh); cn = P^H (c - Hbar y);
//      theta[0:m] harmonic Ritz values sorted by |theta|.
// Returns 0 on success, nonzero if a step failed (the caller then restarts plainly).
DD_HD inline int deflate(const zd* Hbar, int ldh, int m, int k, const zd* c, const zd* y, zd* P, zd* Hn, zd* cn,
                         zd* theta, DeflateWork& W) {
  const int ld = DD_MAXM;
  // f = H_m^{-H} e_m
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) W.M[i + j * ld] = conj(Hbar[j + (long)i * ldh]);
  for (int i = 0; i < m; ++i) W.f[i] = Z(0.0);
  W.f[m - 1] = Z(1.0);
  if (!dense_solve(W.M, m, ld, W.f)) return 1;
  // G = H_m + |h_{m+1,m}|^2 f e_m^H
  double h2 = abs2(Hbar[m + (long)(m - 1) * ldh]);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) W.G[i + j * ld] = Hbar[i + (long)j * ldh];
  for (int i = 0; i < m; ++i) W.G[i + (m - 1) * ld] = W.G[i + (m - 1) * ld] + h2 * W.f[i];
  if (schur(W.G, W.Q, m, ld) < 0) return 2;
  // order by |theta| (stable insertion sort)
  for (int i = 0; i < m; ++i) { W.absth[i] = zabs(W.G[i + i * ld]); W.order[i] = i; }
  for (int i = 1; i < m; ++i) {
    int o = W.order[i];
    int j = i - 1;
    while (j >= 0 && W.absth[W.order[j]] > W.absth[o]) { W.order[j + 1] = W.order[j]; --j; }
    W.order[j + 1] = o;
  }
  for (int i = 0; i < m; ++i) theta[i] = W.G[W.order[i] + W.order[i] * ld];
  // columns of P: harmonic Ritz vectors (zero last row), orthonormalised twice
  for (int l = 0; l < k; ++l) {
    schur_eigvec(W.G, W.Q, m, ld, W.order[l], W.y, W.v);
    zd* p = P + (long)l * ldh;
    for (int i = 0; i < m; ++i) p[i] = W.v[i];
    p[m] = Z(0.0);
    for (int pass = 0; pass < 2; ++pass)
      for (int t = 0; t < l; ++t) {
        const zd* pt = P + (long)t * ldh;
        zd d = Z(0.0);
        for (int i = 0; i <= m; ++i) d = d + conj(pt[i]) * p[i];
        for (int i = 0; i <= m; ++i) p[i] = p[i] - d * pt[i];
      }
    double nrm = 0;
    for (int i = 0; i <= m; ++i) nrm += abs2(p[i]);
    nrm = sqrt(nrm);
    if (!(nrm > 1e-12)) return 3;
    for (int i = 0; i <= m; ++i) p[i] = (1.0 / nrm) * p[i];
  }
  // last column: least-squares residual c - Hbar y
  for (int i = 0; i <= m; ++i) {
    zd s = c[i];
    for (int j = 0; j < m; ++j) s = s - Hbar[i + (long)j * ldh] * y[j];
    W.cls[i] = s;
  }
  zd* p = P + (long)k * ldh;
  for (int i = 0; i <= m; ++i) p[i] = W.cls[i];
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < k; ++t) {
      const zd* pt = P + (long)t * ldh;
      zd d = Z(0.0);
      for (int i = 0; i <= m; ++i) d = d + conj(pt[i]) * p[i];
      for (int i = 0; i <= m; ++i) p[i] = p[i] - d * pt[i];
    }
  double nrm = 0;
  for (int i = 0; i <= m; ++i) nrm += abs2(p[i]);
  nrm = sqrt(nrm);
  if (!(nrm > 0)) return 4;
  for (int i = 0; i <= m; ++i) p[i] = (1.0 / nrm) * p[i];
  // Hn = P^H Hbar P_k, cn = P^H cls
  for (int a = 0; a <= k; ++a) {
    const zd* pa = P + (long)a * ldh;
    for (int b = 0; b < k; ++b) {
      const zd* pb = P + (long)b * ldh;
      zd s = Z(0.0);
      for (int j = 0; j < m; ++j) {
        zd hp = Z(0.0);
        for (int i = 0; i <= m; ++i) hp = hp + conj(pa[i]) * Hbar[i + (long)j * ldh];
        s = s + hp * pb[j];
      }
      Hn[a + (long)b * ldh] = s;
    }
    zd s = Z(0.0);
    for (int i = 0; i <= m; ++i) s = s + conj(pa[i]) * W.cls[i];
    cn[a] = s;
  }
  return 0;
}

}  // namespace dd

/*
 * dd.h -- C ABI of a GB300 (sm_103a) solver for the Wilson-clover Dirac equation with
 * the domain-decomposition method of Heybrock et al., "Lattice QCD with Domain
 * Decomposition on Intel Xeon Phi Co-Processors" (SC14): a multiplicative Schwarz
 * (SAP) preconditioner whose domain solves are minimal-residual iterations on the
 * even-odd Schur complement, inside flexible GMRES with deflated restarts.
 *
 * Conventions for every entry point:
 *   - Every function returns a dd_status; DD_OK is 0.  Nothing aborts or exits.  After
 *     a failure dd_last_error(ctx) returns a message (valid until the next call).
 *   - The caller owns every buffer it passes and keeps ownership.  The context owns
 *     its internal copies (gauge field, clover, Schwarz state, Krylov basis).
 *   - All work is issued on the stream given to dd_create (NULL = legacy stream) and
 *     the functions return after that work has completed, unless stated otherwise.
 *   - One context per stream; contexts are not thread safe.
 *
 * Canonical layouts (host or device memory, little endian IEEE):
 *   spinor  [t][z][y][x][spin 4][colour 3][re, im]    FP64 (double) or FP32 (float)
 *   gauge   [t][z][y][x][mu 4][row 3][col 3][re, im]  FP64, mu = x, y, z, t; entry
 *           (mu, a, b) of site x is U_mu(x)_ab, the forward link from x to x + mu.
 *   Site x = (x, y, z, t); lexicographic index x + Lx (y + Ly (z + Lz t)).
 * Internal layout: domain-major (see dd_spinor_bytes); only needed for the fastest
 *   device-to-device calls.  dd_pack_spinor / dd_unpack_spinor convert.
 *
 * Operator (Sec. II-B, Eq. 1-3):  A = 1/(2 kappa) - 1/2 D_w + D_cl with
 *   D_w psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)
 *   D_cl(x)   = -(c_sw/32) sum_{mu != nu} gamma_mu gamma_nu (Q_mu,nu(x) - Q_nu,mu(x)),
 *   Q_mu,nu the sum of the four plaquettes in the (mu, nu) plane at x; N_d + m = 1/(2 kappa).
 *   Gamma matrices: chiral basis, gamma_5 = diag(1, 1, -1, -1), gamma_k = [[0, -i s_k],
 *   [i s_k, 0]] for k = x, y, z, gamma_t = [[0, 1], [1, 0]].  Boundary conditions:
 *   periodic in x, y, z; antiperiodic in t when t_antiperiodic != 0.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_ctx dd_ctx;
typedef int dd_status;

enum {
  DD_OK = 0,
  DD_ERR_INVALID = 1,          /* null pointer or out-of-range argument */
  DD_ERR_DIMS = 2,             /* lattice / domain shape not allowed */
  DD_ERR_NO_GAUGE = 3,         /* dd_load_gauge has not been called */
  DD_ERR_NO_CLOVER = 4,        /* dd_build_clover has not been called */
  DD_ERR_SINGULAR_CLOVER = 5,  /* a 6x6 clover block is (numerically) singular */
  DD_ERR_NOT_CONVERGED = 6,    /* iteration limit reached; info is still filled */
  DD_ERR_NONFINITE = 7,        /* NaN or Inf met in a norm */
  DD_ERR_TIMEOUT = 8,          /* a bounded device wait ran out */
  DD_ERR_OOM = 9,              /* device allocation failed */
  DD_ERR_CUDA = 10             /* other CUDA runtime error */
};

enum { DD_PREC_FP64 = 0, DD_PREC_FP32 = 1, DD_PREC_FP16 = 2, DD_PREC_FP16_H2 = 3 };
enum { DD_HOST = 0, DD_DEVICE = 1 };
enum { DD_LAYOUT_CANONICAL = 0, DD_LAYOUT_INTERNAL = 1 };

/* Schwarz preconditioner parameters (Sec. II-D, Table I). */
typedef struct {
  int i_schwarz;      /* Schwarz iterations; one iteration = black then white half-sweep (paper: 16) */
  int i_domain;       /* MR steps per domain solve (paper: 4-5) */
  int storage_prec;   /* DD_PREC_FP16: FP16 links, Schwarz matrices and spinors (FP32 arithmetic);
                         DD_PREC_FP16_H2: FP16 storage as above, and the domain solve's SU(3) and
                           clover-block products in packed FP16 arithmetic (half2), each domain's
                           residual scaled into FP16 range by a power of two; hop sums, MR
                           reductions and updates stay FP32.  Not part of the paper (which keeps
                           single-precision arithmetic); needs threads_per_site 0 or 2;
                         DD_PREC_FP32: everything FP32 */
  int threads_per_site; /* 1 or 2 GPU threads per lattice site in the domain solve; 0 = default (2) */
  int additive;       /* 0: multiplicative Schwarz (block Gauss-Seidel over the two colours, the
                         paper's choice, Table I); 1: additive Schwarz (block Jacobi, Sec. II-D,
                         Eq. 4): every domain of both colours solves with the residual of the same
                         iterate, one launch per sweep; needs threads_per_site 0 or 2, and is not
                         available in dd_sap_precondition_lattices or
                         dd_sap_precondition_noalloc (DD_ERR_INVALID) */
} dd_sap_params;

/* Outer solver parameters (flexible GMRES with deflated restarts, Table I). */
typedef struct {
  double tol;         /* target |f - A x| / |f|, recomputed in FP64 (paper: 1e-10) */
  int m;              /* basis size, 1 <= m <= 63 (else DD_ERR_INVALID) */
  int k;              /* deflation vectors kept at a restart, 0 <= k < m */
  int max_iter;       /* total Arnoldi steps allowed */
  dd_sap_params sap;
  int basis_fp16;     /* dd_solve with one right-hand side at a time: 1 stores the basis V in FP16
                         (one power-of-two scale for the whole basis; Gram-Schmidt, recombination and
                         the preconditioner's input read it in FP32 arithmetic), halving its bytes;
                         0 (default) FP32.  Not part of the paper.  Other solvers ignore it */
} dd_solve_params;

/* Result of dd_solve (for nrhs > 1: summed counts and times, worst residual). */
typedef struct {
  int status;
  int iterations;         /* Arnoldi steps = applications of the preconditioner */
  int restarts;           /* cycles after the first */
  int reliable_updates;   /* FP64 true-residual recomputations */
  int deflated_restarts;
  double true_rel_residual;  /* |f - A x| / |f| in FP64 at exit */
  double t_total, t_A, t_M, t_GS, t_other;  /* seconds (device time of each part) */
  double flops_nominal;   /* 1848 flop/site per A and per D application, paper's convention */
} dd_solve_info;

/* Create a context for a lattice dims = {Lx, Ly, Lz, Lt} split into domains of shape
 * domain = {bx, by, bz, bt}.  Each b_mu must be a power of two >= 2 and divide L_mu,
 * each L_mu / b_mu must be even (two-colouring of the domains, Sec. IV-B, Eq. 6) and >= 2, and
 * the Schwarz kernel needs 64 <= prod(b) <= 512.  stream: a cudaStream_t or NULL.
 * Allocates its device memory with cudaMalloc. */
dd_status dd_create(dd_ctx** out, const int dims[4], const int domain[4], int t_antiperiodic, void* stream);
dd_status dd_destroy(dd_ctx* ctx);
const char* dd_last_error(const dd_ctx* ctx);

/* Load the gauge field U_mu(x) of the hopping term (Sec. II-B, Eq. 2; canonical FP64
 * layout, host or device memory per `where`).  It is copied; FP64, FP32 and FP16 copies
 * in the domain-major layout are made (Sec. III-A: each domain's data contiguous), with
 * the antiperiodic time boundary folded into the links U_t(x) at t = L_t - 1.  The
 * caller's buffer is not retained.  Returns DD_ERR_OOM if the copies cannot be allocated. */
dd_status dd_load_gauge(dd_ctx* ctx, const double* U, int where);

/* Build the clover term (Eq. 3) with the diagonal 1/(2 kappa) folded in, in FP64, and
 * each 6x6 block's inverse for the even-odd domain solves (Eq. 5); store FP64/FP32/FP16
 * copies.  Returns DD_ERR_SINGULAR_CLOVER (after building) if a block is singular. */
dd_status dd_build_clover(dd_ctx* ctx, double kappa, double c_sw);

/* out = A in (Eq. 1) for device buffers.  prec: DD_PREC_FP64 / FP32 (canonical or
 * internal layout) or DD_PREC_FP16 (internal layout only: FP16 storage, FP32
 * arithmetic).  in and out must not overlap. */
dd_status dd_apply_D(dd_ctx* ctx, const void* in, void* out, int prec, int layout);

/* out = M in: the multiplicative Schwarz preconditioner (Table I, Sec. II-D) with
 * I_Schwarz black/white sweeps of even-odd MR domain solves.  in/out: FP32 device
 * buffers in `layout`; they may not overlap. */
dd_status dd_sap_precondition(dd_ctx* ctx, const float* in, float* out, const dd_sap_params* p, int layout);

/* Several right-hand sides in one launch (batching of the many solves of an analysis,
 * Sec. IV-C).  in/out hold nrhs fields in the internal layout, one after another
 * (stride dd_spinor_bytes(ctx, prec, DD_LAYOUT_INTERNAL)); they may not overlap.
 * dd_sap_precondition_batch: out_r = M in_r, FP32 fields; each domain's links and Schwarz
 * matrices are staged into shared memory once and used for all right-hand sides
 * (threads_per_site must be 0 or 2).  dd_apply_D_batch: out_r = A in_r for FP32 or FP16
 * fields, two right-hand sides per thread, so each link and clover block is loaded once
 * per pair. */
dd_status dd_sap_precondition_batch(dd_ctx* ctx, const float* in, float* out, int nrhs, const dd_sap_params* p);
/* Lattices of different volume in one launch per half-sweep (Sec. IV-C: the many
 * independent solves of an analysis): out_{l,r} = M_l in_{l,r} for the nlat <= 4 contexts
 * ctxs[l] (their own gauge fields, clover and kappa) and nrhs right-hand sides each, all
 * with the same domain volume, FP16 storage and two threads per site.  The launch walks a
 * work list of (lattice, domain) and every CTA loops over the nrhs right-hand sides with
 * its domain's links and Schwarz matrices staged once.  in[l] / out[l]: nrhs FP32
 * internal fields of lattice l one after another (stride dd_spinor_bytes(ctxs[l],
 * DD_PREC_FP32, DD_LAYOUT_INTERNAL)).  Work is issued on ctxs[0]'s stream. */
dd_status dd_sap_precondition_lattices(dd_ctx** ctxs, const float* const* in, float* const* out, int nlat, int nrhs,
                                       const dd_sap_params* p);
dd_status dd_apply_D_batch(dd_ctx* ctx, const void* in, void* out, int nrhs, int prec);

/* out = M in like dd_sap_precondition, but without allocating: the paper has no
 * counterpart to this entry point.  It is for callers that cannot call cudaMalloc when
 * they apply the preconditioner: frameworks that own all device memory through their own
 * pool (a cudaMalloc behind the pool's back can fail or fragment it), and loops that
 * cannot afford cudaMalloc's device-wide synchronisation.
 * in/out: FP32 device buffers in the internal layout (see dd_pack_spinor); the context's
 * gauge field and clover must already be built (dd_load_gauge / dd_build_clover allocate,
 * this call does not).  The Schwarz working state lives in one fixed 64 MiB array in the
 * library's device memory, held by every GPU that loads the library until the process
 * exits; lattices whose state does not fit are rejected with DD_ERR_INVALID and a message
 * giving both sizes (about 160 bytes per site with FP16 storage, 230 with FP32: up to
 * ~4e5 sites).  All calls share that array, so calls that overlap on the GPU (other
 * streams, other contexts, other threads) race and must be serialised by the caller.
 * The first call on each device looks up the array's address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The call is
 * synchronous like the others: it reads the kernel's error word back and waits for the
 * stream before it returns. */
dd_status dd_sap_precondition_noalloc(dd_ctx* ctx, const float* in, float* out, const dd_sap_params* p);

/* Solve A x = f (Sec. II-C, Table I) for nrhs right-hand sides stored one after another
 * in the canonical FP64 layout (host or device memory per `where`).  x holds the
 * initial guess on entry (zeros are fine) and the solution on exit.  Outer FGMRES-DR
 * in FP32 vectors with FP64 Hessenberg, Gram-Schmidt coefficients and least squares;
 * x accumulated in FP64 and the residual recomputed with the FP64 operator at every
 * restart (reliable update).  info may be NULL.
 * With nrhs > 1 (and threads_per_site 0 or 2) the right-hand sides are solved in
 * lockstep: each keeps its own basis, restarts and stopping point, while every Arnoldi
 * step applies M and A to all unconverged ones in one launch each (per Schwarz
 * half-sweep); this holds nrhs copies of the solver's buffers.  DD_SEQUENTIAL_RHS=1 in
 * the environment solves them one after another instead.  info sums iterations,
 * restarts and updates over the right-hand sides; true_rel_residual is the largest. */
dd_status dd_solve(dd_ctx* ctx, const double* f, double* x, int nrhs, int where, const dd_solve_params* p,
                   dd_solve_info* info);

/* Lockstep solves over nlat <= 4 lattices of different volume (the many independent
 * solves of an analysis, Sec. IV-C), nrhs right-hand sides each: f[l] / x[l] hold lattice
 * l's nrhs canonical FP64 fields one after another (host or device per `where`).  Every
 * (lattice, right-hand side) is solved as by dd_solve (FGMRES-DR with reliable updates,
 * its own basis, restarts and stopping point); every Arnoldi step applies the Schwarz
 * preconditioner to all unconverged ones in one launch per half-sweep over the lattices'
 * (domain, right-hand side) work, and the operator in one launch per lattice.  The
 * contexts need the same domain volume; FP16 storage, two threads per site and the
 * multiplicative form (else DD_ERR_INVALID).  All work runs on ctxs[0]'s stream; each
 * context holds nrhs copies of the solver's buffers.  info sums over all solves;
 * true_rel_residual is the largest. */
dd_status dd_solve_lattices(dd_ctx** ctxs, int nlat, const double* const* f, double* const* x, int nrhs, int where,
                            const dd_solve_params* p, dd_solve_info* info);

/* A x = f with flexible GCR(m) around the same Schwarz preconditioner: the outer solver
 * of Luescher's SAP-GCR, which the paper contrasts with its FGMRES-DR (Sec. V).  Per step
 * z_k = M r, w_k = A z_k orthonormalised against w_0..w_{k-1} (classical Gram-Schmidt with
 * a second pass when the first cancels more than half, FP64-reduced; the coefficients are
 * applied to z_k too), alpha_k = <w_k, r>, r -= alpha_k w_k.  After at most p->m steps
 * x += sum alpha_k z_k in FP64 and the residual is recomputed with the FP64 operator
 * (restart).  FP32 vectors, canonical FP64 f and x (host or device per `where`), one
 * right-hand side; p->k is ignored.  Uses the context's solver buffers (sized by m). */
dd_status dd_solve_gcr(dd_ctx* ctx, const double* f, double* x, int where, const dd_solve_params* p,
                       dd_solve_info* info);

/* Standard (not domain-decomposed) comparison solver, the kind the paper measures its
 * solver against (Sec. IV-C, Table III: BiCGstab in double precision; mixed-precision
 * Richardson iteration around BiCGstab).  Solves A x = f like dd_solve (canonical FP64
 * layout, host or device memory per `where`; x holds the initial guess on entry):
 *   precision DD_PREC_FP64: BiCGstab in FP64 on the FP64 operator; its recursive residual
 *     drifts from the true one, so the true residual is recomputed (FP64) whenever the
 *     recursion reports convergence, and BiCGstab resumes from it if needed;
 *   precision DD_PREC_FP32: Richardson iteration (defect correction) in FP64: r = f - A x
 *     in FP64, a correction e from BiCGstab in FP32 on the FP32 operator for A e = r / |r|
 *     to relative residual inner_tol, x += |r| e in FP64, until |f - A x| / |f| <= tol.
 * max_iter bounds the BiCGstab iterations in total (two operator applications each).
 * info: iterations = BiCGstab iterations, restarts = Richardson corrections after the
 * first, reliable_updates = FP64 residuals, t_A = operator time, t_M = t_GS = 0.
 * Temporary device memory (3 FP64 fields, 7 fields of the iteration's precision) is
 * allocated per call and released before returning.  Returns DD_ERR_NOT_CONVERGED with
 * info filled when max_iter is reached. */
typedef struct {
  double tol;        /* target |f - A x| / |f| (FP64-recomputed) */
  int max_iter;      /* BiCGstab iterations in total */
  int precision;     /* DD_PREC_FP64 or DD_PREC_FP32 (mixed Richardson) */
  double inner_tol;  /* DD_PREC_FP32: residual reduction of each inner solve, 0 < inner_tol < 1 */
} dd_bicgstab_params;
dd_status dd_solve_bicgstab(dd_ctx* ctx, const double* f, double* x, int where, const dd_bicgstab_params* p,
                            dd_solve_info* info);

/* Two-level aggregation multigrid with the Schwarz method as its smoother.  The paper lists
 * this use of domain-decomposition preconditioners among related work (Sec. V: algebraic
 * multigrid solvers whose smoother is a Schwarz method); the method here is the plain
 * two-level form of those works:
 *   - aggregates are the context's Schwarz domains; each aggregate and chirality (spins
 *     0, 1: gamma_5 = +1; spins 2, 3: gamma_5 = -1) has n_tv coarse degrees of freedom, so
 *     the coarse lattice is the lattice of domains with nc = 2 n_tv unknowns per site;
 *   - the interpolation P is built from n_tv test vectors, each first replaced setup_iters
 *     times by M_sap v (setup_mode 0: inverse iteration with the smoother's Schwarz method,
 *     at least one cycle) or by v - M_sap A v (setup_mode 1: the smoother run on A v = 0,
 *     which keeps the low modes of A), then made orthonormal in order on every (aggregate,
 *     chirality) (Gram-Schmidt: the Q of a QR factorisation with positive diagonal);
 *   - the coarse operator is D_c = P^H A P, a nearest-neighbour stencil of nc x nc blocks
 *     on the lattice of domains, built in FP32;
 *   - one application of the preconditioner to v: e_c ~ D_c^{-1} P^H v by coarse_cycles
 *     cycles of GMRES(coarse_m) from zero (FP32 vectors, FP64 sums and least squares, a
 *     fixed number of steps), x = P e_c, then z = x + M_sap (v - A x) with the smoother's
 *     i_schwarz Schwarz cycles (0: no smoothing).
 * Coarse vectors (device, FP32 complex as re, im pairs): [domain][chirality][k], domains
 * numbered like the internal layout (x fastest over L_mu / b_mu domains per direction). */
typedef struct {
  int n_tv;            /* test vectors, 1..16 */
  int setup_iters;     /* Schwarz applications to each test vector before P is built (>= 0) */
  int coarse_m;        /* GMRES steps per coarse cycle, 1..63 */
  int coarse_cycles;   /* coarse GMRES cycles per application (>= 1) */
  dd_sap_params smoother;   /* Schwarz form of the smoother and of the set-up; i_schwarz >= 0 */
  int setup_mode;      /* 0: v <- M_sap v; 1: v <- v - M_sap A v */
} dd_mg_params;

/* Build P and D_c from n_tv test vectors tv (canonical FP64 fields one after another, host
 * or device per `where`; the caller chooses them, e.g. Gaussian noise) with the context's
 * gauge field and clover.  Replaces any earlier set-up (and drops the outer solver's
 * captured steps).  Allocates n_tv + 3 FP32 fields, D_c (9 nc^2 complex per domain) and
 * the coarse solver's buffers.  seconds (may be NULL): device time of the set-up.
 * DD_ERR_NONFINITE when the test vectors are linearly dependent on some aggregate. */
dd_status dd_mg_setup(dd_ctx* ctx, const double* tv, int where, const dd_mg_params* p, double* seconds);
/* out = P^H in (in: FP32 internal-layout field; out: coarse vector), out = P in (in: coarse
 * vector; out: FP32 internal field), y = D_c x (coarse vectors, x != y) and x ~ D_c^{-1} b
 * (the coarse solve of one application).  Device buffers; synchronous. */
dd_status dd_mg_restrict(dd_ctx* ctx, const float* in, float* out);
dd_status dd_mg_prolong(dd_ctx* ctx, const float* in, float* out);
dd_status dd_mg_coarse_apply(dd_ctx* ctx, const float* x, float* y);
dd_status dd_mg_coarse_solve(dd_ctx* ctx, const float* b, float* x);
/* out = B in, one application of the two-level preconditioner; FP32 device fields in
 * `layout`, in != out. */
dd_status dd_mg_precondition(dd_ctx* ctx, const float* in, float* out, int layout);
/* A x = f with the outer solver of dd_solve (FGMRES-DR, FP64 reliable updates) and the
 * two-level preconditioner in place of the Schwarz method; one right-hand side; p->sap is
 * ignored.  dd_mg_setup must have been called.  t_M in info is the preconditioner's time. */
dd_status dd_solve_mg(dd_ctx* ctx, const double* f, double* x, int where, const dd_solve_params* p,
                      dd_solve_info* info);

/* Bytes of one spinor field for a precision and layout (FP16 internal: values and norms). */
size_t dd_spinor_bytes(const dd_ctx* ctx, int prec, int layout);

/* Convert between the canonical layout (FP64 or FP32, device) and the internal layout
 * (FP64, FP32 or FP16, device).  For FP16 the per-site norms follow the values in the
 * same buffer (see dd_spinor_bytes). */
dd_status dd_pack_spinor(dd_ctx* ctx, const void* canonical, int canonical_prec, void* internal, int internal_prec);
dd_status dd_unpack_spinor(dd_ctx* ctx, const void* internal, int internal_prec, void* canonical, int canonical_prec);

/* Number of kernels this context has launched since it was created. */
long long dd_launch_count(const dd_ctx* ctx);

/* Measured FP32 CUDA-core peak of the current device (the roofline denominator of the
 * Schwarz kernel, which is bound by FP32 arithmetic): back-to-back launches of a kernel
 * whose threads run eight independent FFMA chains each (no memory traffic), for at least
 * duration_ms milliseconds of device time after one warm-up launch.  burst_tflops: the
 * fastest launch; sustained_tflops: all launches together (clocks settle under the power
 * limit).  2 flop per FFMA.  Uses its own stream and a 16-byte buffer; changes no device
 * setting. */
dd_status dd_fp32_peak(int duration_ms, double* burst_tflops, double* sustained_tflops);
/* The same for FP64 fused multiply-adds (DFMA chains): the denominator of the FP64 operator
 * that recomputes the true residual at every restart (Sec. II-C: reliable updates), which
 * GB300's FP64 rate bounds.  Arguments and behaviour as dd_fp32_peak. */
dd_status dd_fp64_peak(int duration_ms, double* burst_tflops, double* sustained_tflops);

/* Wave-quantisation load of the Schwarz kernel, the GPU analogue of Eq. 6-7: with
 * n = number of domains of one colour and `slots` CTAs resident at once,
 * load = n / (slots * ceil(n / slots)).  Pure host function. */
double dd_load_model(long long n_domains_per_colour, int slots);

/* Autotuner (Sec. IV-B: the domain size and I_domain are chosen by the overall
 * time-to-solution; Eq. 6-7 give the load of a domain count).  Picks a domain shape,
 * I_Schwarz, I_domain and threads per site for this lattice with the context's gauge
 * field and clover; the context's own shape is not changed.  Every candidate runs a short
 * FGMRES-DR(16, 4) solve from x = 0 of a fixed pseudo-random source on the device (12
 * Arnoldi steps in the shape stage, 48 afterwards) and is scored by its device time per
 * e-fold of true-residual reduction.  Stages: (1) every allowed shape with extents 2, 4 or
 * 8 at I_Schwarz 4, I_domain 4, two threads per site, keeping the four best; (2) I_domain
 * 2..6 x threads per site 1, 2 on those shapes; (3) I_Schwarz in {1, 2, 4, 8, 16}, then
 * I_domain again, at the best shape.  On entry, out->i_schwarz, out->i_domain and
 * out->threads_per_site > 0 fix that parameter (threads_per_site 2 is needed for
 * several right-hand sides in lockstep), and out->additive (0 or 1) selects the Schwarz
 * form that is tuned; storage_prec: DD_PREC_FP16, DD_PREC_FP16_H2 or
 * DD_PREC_FP32 (else DD_ERR_INVALID).  Writes the best shape to domain_out and its
 * parameters to out.  Temporary device memory (two FP64 fields here, one context per
 * candidate) is released before returning.  Returns the first candidate error other than
 * a refused shape or a diverging solve, or DD_ERR_NOT_CONVERGED if no candidate reduced
 * the residual.  With DD_TRACE set, one line per candidate gives its iterations, time,
 * residual, score and the load model's estimate (dd_load_model) for that shape. */
dd_status dd_autotune(dd_ctx* ctx, int storage_prec, int domain_out[4], dd_sap_params* out);

/* The small dense step of a deflated restart (Sec. II-C, Table I; GMRES-DR with flexible
 * preconditioning), run on the host by the same code that dd_solve runs as one warp on
 * the device (a team of one thread here), so it can be checked without a GPU.  Given the
 * (m+1) x m Hessenberg matrix Hbar (column-major, leading dimension m+1, complex as
 * re, im pairs), the cycle's right-hand side c (m+1) and least-squares solution y (m),
 * return the orthonormal (m+1) x (k+1) basis P, Hn = P^H Hbar P_k ((k+1) x k, ld m+1),
 * cn = P^H (c - Hbar y) and the harmonic Ritz values theta (m, sorted by modulus).
 * All arrays are host memory owned by the caller; 1 <= k < m < 64 (else DD_ERR_INVALID);
 * DD_ERR_NONFINITE when a step fails (the solver then restarts without deflation). */
dd_status dd_deflate_host(int m, int k, const double* Hbar, const double* c, const double* y, double* P, double* Hn,
                          double* cn, double* theta);
/* The same step as dd_solve runs it (one warp on the current device), for checks and
 * timing: arguments as dd_deflate_host but in device memory; ms (host, may be NULL)
 * receives the kernel's device time.  Allocates and frees its scratch; synchronous. */
dd_status dd_deflate_device(int m, int k, const double* Hbar, const double* c, const double* y, double* P, double* Hn,
                            double* cn, double* theta, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* DD_H */

// Host-callable launchers for every device kernel of the library.  All launches are
// asynchronous on the given stream; none of them allocates memory.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dd_common.cuh"
#include "smalldense.cuh"

namespace dd {

enum Prec { P64 = 0, P32 = 1, P16 = 2 };

// Opaque views of one spinor field in the internal layout.
struct FieldView {
  void* data;     // double2[] | float4[] | uint4[]
  float* norm;    // FP16 only: per-site scale
  int prec;
};

// Gauge / clover storage in the internal layout for one precision.
struct GaugeView { const void* links; int prec; };
struct CloverView { const void* m; int prec; };

// ---- layout (layout_clover.cu)
void launch_pack_spinor(const Geom& g, const void* canon, int canon_prec, FieldView out, cudaStream_t st);
void launch_unpack_spinor(const Geom& g, FieldView in, void* canon, int canon_prec, cudaStream_t st);
void launch_pack_gauge(const Geom& g, const double* canon, int t_antiperiodic, double2* u64, float2* u32,
                       uint32_t* u16, cudaStream_t st);
// Builds clover (all sites, with the 1/(2 kappa) diagonal) in FP64/FP32/FP16 and the
// Schwarz matrices (even sites: clover block; odd sites: its inverse) in FP32/FP16.
// status[0] counts sites with a (near-)singular block.
void launch_build_clover(const Geom& g, const double* canon, double kappa, double csw, double2* c64,
                         float4* c32, uint4* c16, float4* s32, uint4* s16, int* status, cudaStream_t st);

// ---- Wilson-clover operator (dslash.cu)
// Several right-hand sides per thread (nrhs fields of one precision, one after another,
// stride = one field): each link and clover block is loaded once per site.
void launch_apply_A_multi(const Geom& g, GaugeView U, CloverView C, FieldView in, FieldView out, int nrhs,
                          cudaStream_t st);
// The same for FP32 fields given by device arrays of nrhs input and output pointers.
void launch_apply_A_multi_list(const Geom& g, GaugeView U, CloverView C, const float4* const* in,
                               float4* const* out, int nrhs, cudaStream_t st);
// out = A in, or out = f - A in when f != nullptr.  FP64 and FP32 fields use the matching
// gauge/clover precision; FP16 fields use FP16 gauge/clover and FP32 arithmetic.
void launch_apply_A(const Geom& g, GaugeView U, CloverView C, FieldView in, FieldView out, const FieldView* f,
                    cudaStream_t st);

// ---- Schwarz sweep (sap.cu)
struct SapState {
  int mat_prec;        // P32 or P16: gauge and Schwarz matrices
  int vec_prec;        // P32 or P16: stored residual and solution
  const void* links;   // gauge in mat_prec
  const void* smat;    // Schwarz matrices in mat_prec
  void* r_store;       // even-site residual, Hd sites per domain, vec_prec
  float* r_norm;
  void* u_store;       // solution, Vd sites per domain, vec_prec
  float* u_norm;
  float4* faces;       // projected half-spinors on the 8 faces of every domain (FP32)
  int* err;            // set to 1 when a bounded device wait runs out
  bool mat_in_smem;    // stage links and Schwarz matrices in shared memory
  int threads_per_site = 2;   // 1: one thread per site; 2: hop directions and chirality split
  bool inject_wait_timeout = false;   // test hook: make the bounded wait run out (no fault)
  int nrhs = 1;                // right-hand sides in one launch (their buffers follow each other)
  bool half_arith = false;     // FP16 storage with packed FP16 hop and clover products
  // device arrays of nrhs input / output pointers (FP32 internal fields), instead of v and
  // z with their fixed stride; two threads per site only
  const float4* const* vlist = nullptr;
  float4* const* zlist = nullptr;
  long long r_bytes = 0;       // bytes of one right-hand side's residual / solution storage
  long long u_bytes = 0;
  // additive form (block Jacobi): one launch per sweep over both colours, reading the
  // faces of the previous sweep from `faces` and writing this sweep's to faces_out
  bool both_colours = false;
  float4* faces_out = nullptr;
  // single right-hand side: the input is v * (*vscale) (device scalar), when set
  const float* vscale = nullptr;
};
// One half-sweep: all domains of `colour`.  first: the residual is the input v (both
// parities) and u = 0; use_faces: subtract the couplings to the other colour from the
// face buffers; last: write u (FP32) into z.
int sap_half_sweep(const Geom& g, const SapState& S, int colour, int first, int use_faces, int last,
                   const float4* v, float4* z, int i_domain, cudaStream_t st);
// Several lattices (same domain shape, FP16 storage) in one launch per half-sweep.
int sap_half_sweep_lattices(const Geom* gs, const SapState* Ss, int nlat, int colour, int first, int use_faces,
                            int last, const float4* const* v, float4* const* z, int i_domain, cudaStream_t st);
size_t sap_smem_bytes(const Geom& g, int mat_prec, bool mat_in_smem);
bool sap_mat_fits_smem(const Geom& g, int mat_prec);
int sap_max_domain_sites();
// Fixed scratch array of the allocation-free Schwarz entry point (size, device address).
size_t sap_noalloc_scratch_bytes();
void* sap_noalloc_scratch();

// ---- BLAS on FP32 / FP64 internal vectors (blas.cu).  n4 = number of float4 (or
// double2) units in one vector; vectors of a basis are contiguous, stride n4.
int blas_partials_blocks();
int launch_multi_dot(const float4* V, int nv, long long n4, const float4* w, double2* partial, cudaStream_t st);
void launch_reduce_partials(const double2* partial, int nv, double2* out, int accumulate, cudaStream_t st);
void launch_norm2_64(const double2* x, long long n2, double2* partial, cudaStream_t st);
void launch_x_update(double2* x, const float4* Z, int nz, long long n4, const double2* y, cudaStream_t st);
// v = r / sqrt(nrm2); with a gate, only when *gate == 1
void launch_r64_to_v32(float4* v, const double2* r, long long n4, const double2* nrm2, cudaStream_t st,
                       const int* gate = nullptr);
// out_l = sum_i P(i, l) v_i for l < nout (in place allowed); with a gate, only when
// *gate == 1.  vscale (optional, device): the stored vectors are V_i = v_i / vscale[i].
int launch_recombine(float4* out, const float4* V, int nv, int nout, long long n4, const double2* P, int ldp,
                     cudaStream_t st, const int* gate = nullptr, const float* vscale = nullptr);
// FP16 basis (uint2 = two complex numbers as half2): the outputs are stored times oscale
int launch_recombine(uint2* out, const uint2* V, int nv, int nout, long long n4, const double2* P, int ldp,
                     cudaStream_t st, const int* gate, const float* vscale, float oscale);

// Classical Gram-Schmidt passes with device-gated reorthogonalisation (blas.cu).  A kernel
// given a gate runs only when *gate == want.  vscale (optional, device): the basis holds
// V_i = v_i / vscale[i] (a vector whose normalisation is deferred to its readers); dots and
// projections are taken against v_i.
int launch_gs_dot(const float4* V, int nv, long long n4, const float4* w, double2* partial, const int* gate, int want,
                  cudaStream_t st, const float* vscale = nullptr);
void launch_gs_reduce(const double2* partial, int nv, double2* out, const int* gate, int want, cudaStream_t st);
void launch_gs_project(float4* out, const float4* w, const float4* V, int nv, long long n4, const double2* h,
                       double2* norm_partial, const int* gate, int want, cudaStream_t st,
                       const float* vscale = nullptr);
void launch_scale_inplace(float4* v, long long n4, const double* nu2, cudaStream_t st);
// The same passes over an FP16 basis (w and the projection's output stay FP32), and the
// FP16 basis store / load: v16 = FP16(s w / sqrt(nu2)) with the FP32 copy w / sqrt(nu2) in
// v32 (optional; gate as r64_to_v32); v32 = s v16.
int launch_gs_dot(const uint2* V, int nv, long long n4, const float4* w, double2* partial, const int* gate, int want,
                  cudaStream_t st, const float* vscale);
void launch_gs_project(float4* out, const float4* w, const uint2* V, int nv, long long n4, const double2* h,
                       double2* norm_partial, const int* gate, int want, cudaStream_t st, const float* vscale);
void launch_basis16_store(uint2* v16, float4* v32, const float4* w, long long n4, const double* nu2, float s,
                          cudaStream_t st, const int* gate = nullptr);
void launch_basis16_load(float4* v32, const uint2* v16, long long n4, float s, cudaStream_t st);

// ---- BiCGstab comparison solver (krylov.cu).  U = float4 (FP32 fields) or double2 (FP64
// fields); sc: the recurrence's scalars on the device (see krylov.cu); partial: at least
// 2 blas_partials_blocks() double2.
template <typename U>
struct BicgKernels {
  // sc[slot] = <a, b>; with c, d also sc[slot + 1] = <c, d>
  static void dot(const Geom& g, const U* a, const U* b, const U* c, const U* d, double2* partial, zd* sc, int slot,
                  cudaStream_t st);
  static void p_update(const Geom& g, U* p, const U* r, const U* v, const zd* sc, cudaStream_t st);
  static void s_update(const Geom& g, U* s, const U* r, const U* v, const zd* sc, cudaStream_t st);
  // x += alpha p + omega s, r = s - omega t, sc[8] = |r|^2
  static void xr_update(const Geom& g, U* x, U* r, const U* p, const U* s, const U* t, zd* sc, double2* partial,
                        cudaStream_t st);
  static void copy(const Geom& g, U* dst, const U* src, cudaStream_t st);   // src null: zero
};
void launch_bicg_scalars(zd* sc, int stage, cudaStream_t st);
void launch_bicg_reset(zd* sc, cudaStream_t st);
// ---- two-level multigrid with the Schwarz smoother (mg.cu).  Aggregates are the domains;
// P: n_tv FP32 internal fields (column (chirality c, k) of a domain in field k's units
// 3c..3c+2); coarse vectors float2 [domain][chirality][k]; D_c float2 [domain][9][j][i].
constexpr int MG_MAXTV = 16;
void launch_mg_restrict(const Geom& g, const float4* in, const float4* P, int ntv, float2* rc, const float* vscale,
                        cudaStream_t st);
void launch_mg_prolong(const Geom& g, const float2* ec, const float4* P, int ntv, float4* out, cudaStream_t st);
void launch_mg_orthonormalize(const Geom& g, float4* P, int ntv, int* status, cudaStream_t st);
void launch_mg_coarse_build(const Geom& g, const float2* U32, const float4* C32, const float4* P, int ntv, float2* Dc,
                            cudaStream_t st);
// y = D_c x, or y = b - D_c x when b != nullptr; skipped when gate && *gate != 0
void launch_mg_coarse_apply(const Geom& g, const float2* Dc, int nc, const float2* x, float2* y, const float2* b,
                            const int* gate, cudaStream_t st);
// coarse-vector Gram-Schmidt passes, one launch each (the last block reduces the partial
// sums in FP64): h_out[0..nv-1] = V^H w, h_out[nv] = |w|^2; the projection out = w - V h
// leaves |out|^2 in *n2_out (if not null) and, with hcol != 0, runs the Hessenberg column
// j's update (Givens, nu = 1 / h_{j+1,j}, state).  ticket: a device int, zero between
// launches.  partial: 2 blas_partials_blocks() (nv + 1) double2; norm_partial: as many doubles.
void launch_mg_cdot(const float4* V, int nv, long long n4, const float4* w, double2* partial, double2* h_out,
                    int* ticket, const int* gate, cudaStream_t st);
void launch_mg_cproject(float4* out, const float4* w, const float4* V, int nv, long long n4, const double2* h,
                        double* norm_partial, double* n2_out, int* ticket, const int* gate, int hcol, zd* R, int ldh,
                        int j, const double2* hA, const double2* hB, LsqState* lsq, zd* g, double* nu, int* state,
                        cudaStream_t st);
// coarse GMRES one-thread steps: start of a cycle (state[0] != 0 stops a cycle, state[1] =
// columns done) and the final least squares
void launch_mg_beta(const double2* nrm, zd* g, int ng, double* nu, int* state, LsqState* lsq, cudaStream_t st);
void launch_mg_lsq(const zd* R, int ldh, int mc, const zd* g, const int* state, zd* y, cudaStream_t st);
void launch_mg_scale(float4* v, long long n4, const double* nu, const int* gate, cudaStream_t st);
void launch_mg_axpy(float4* x, const float4* t, long long n4, float a, cudaStream_t st);   // x += a t
// z = vscale (x + e); e and vscale optional
void launch_mg_combine(float4* z, const float4* x, const float4* e, long long n4, const float* vscale,
                       cudaStream_t st);
}  // namespace dd

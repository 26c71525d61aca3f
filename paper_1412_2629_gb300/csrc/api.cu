// C ABI of the library (include/dd.h): context, gauge and clover set-up, the operator,
// the Schwarz preconditioner and the outer solver.
//
// Outer solver (Table I): flexible GMRES with deflated restarts.  Krylov vectors V, Z are
// FP32 fields; Gram-Schmidt coefficients, the Hessenberg matrix, its least-squares
// problem and the m x m harmonic-Ritz eigenproblem of a deflated restart are FP64 on the
// device (the last one in a one-warp kernel beside the reliable update), as is the basis
// recombination; the solution is accumulated in FP64 and at every restart the residual is
// recomputed with the FP64 operator (reliable update), which is what makes the 1e-10
// target reachable with FP32 Krylov vectors.  A deflated restart keeps the k harmonic Ritz vectors of smallest modulus;
// its right-hand side is the projection of the recomputed FP64 residual onto the new
// basis, and the restart falls back to a plain one when that projection misses more
// than `defl_tol` of the residual.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "dd.h"
#include "dd_kernels.hpp"
#include "smalldense.cuh"

using namespace dd;

struct SapBuffers {
  void* r_store = nullptr;
  float* r_norm = nullptr;
  void* u_store = nullptr;
  float* u_norm = nullptr;
  float4* faces = nullptr;
  float4* faces2 = nullptr;    // second face buffer of the additive form (allocated on first use)
  int cap = 0;                 // right-hand sides the buffers hold
  long long r_bytes = 0, u_bytes = 0;
};

// A launch sequence of the outer solver captured as a CUDA graph: key = (part, step j,
// I_Schwarz, I_domain, storage precision, threads per site, m, additive).
typedef std::array<int, 8> GraphKey;
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;     // kernels per replay
  int seen = 0;
};

struct SolverBuffers {
  int m = 0;                 // capacity (basis size)
  cudaStream_t stream = nullptr;       // private stream of dd_solve (capturable)
  cudaEvent_t ev_in = nullptr;
  cudaStream_t side = nullptr;         // second branch of an Arnoldi step (small dense work)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::map<GraphKey, GraphEntry> graphs;
  float4* V = nullptr;                 // m+1 basis vectors (recombined in place at a restart)
  float4* Z = nullptr;                 // m preconditioned vectors
  float4* w = nullptr;
  double2 *x64 = nullptr, *f64 = nullptr, *r64 = nullptr;
  double2* canon64 = nullptr;          // canonical FP64 staging (one field)
  // device scalars
  zd *H = nullptr, *R = nullptr, *g = nullptr, *c0 = nullptr, *y = nullptr;
  zd *hA = nullptr, *hB = nullptr, *P = nullptr, *Hn = nullptr, *cn = nullptr, *theta = nullptr, *cp = nullptr;
  double2* partial = nullptr;
  double2* partial2 = nullptr;         // per-block norm partials of the Gram-Schmidt projection
  double2* nrm2 = nullptr;
  double* status = nullptr;            // [0] residual estimate, [1] deflate status
  double* h_status = nullptr;          // pinned host mirror
  LsqState* lsq = nullptr;
  int* flag = nullptr;                 // Gram-Schmidt: 1 when a second projection is needed
  double* nu2 = nullptr;               // squared norm of the projected vector
  // 1 / |v_i| of the basis vectors as stored: the single-right-hand-side solver leaves each
  // new vector unnormalised (its exact norm comes out of the projection pass) and its
  // readers apply the scale, which saves a read and a write of the vector per step
  float* vscale = nullptr;
  // FP16 basis (dd_solve_params.basis_fp16): V16 replaces V, holding s v_i in FP16 with one
  // power-of-two scale s for the whole basis (vscale[i] = 1 / s); vin is the FP32 copy of
  // the newest basis vector, the next preconditioner application's input
  bool v16 = false;
  float v16_scale = 1.f;
  uint2* V16 = nullptr;
  float4* vin = nullptr;
  double* one = nullptr;          // device 1.0
  // deflated restart on the device: workspace and flags ([0] deflation status, [1] the
  // recombination gate: deflation succeeded and the residual is above target)
  void* dW = nullptr;            // deflate_bytes(m) of global scratch (when shared memory is too small)
  int* dflags = nullptr;
};

struct dd_ctx {
  Geom g;
  int anti = 1;
  cudaStream_t st = nullptr;
  std::string err;
  long long launches = 0;
  bool trace = false;   // DD_TRACE=1 in the environment: one line per solver step on stderr
  // DD_INJECT_WAIT_TIMEOUT=1 at dd_create: the Schwarz kernel's bounded wait for its staged
  // data is made to run out (it expects 16 bytes nobody sends, limit 50 ms), to exercise
  // the DD_ERR_TIMEOUT path without any fault
  bool inject_wait_timeout = false;
  bool use_graphs = true;   // DD_NO_GRAPHS=1: launch the outer solver's kernels directly
  // gauge
  double* Ucanon = nullptr;
  double2* U64 = nullptr;
  float2* U32 = nullptr;
  uint32_t* U16 = nullptr;
  bool have_gauge = false;
  // clover
  double2* C64 = nullptr;
  float4* C32 = nullptr;
  uint4* C16 = nullptr;
  float4* S32 = nullptr;
  uint4* S16 = nullptr;
  int* dstatus = nullptr;
  bool have_clover = false;
  double kappa = 0, csw = 0;
  // schwarz
  SapBuffers sap[3];
  int* sap_err = nullptr;
  // scratch fields for canonical-layout calls
  void* scratch_in = nullptr;
  void* scratch_out = nullptr;
  SolverBuffers sv;
  // lockstep solves: one set of solver buffers per right-hand side, and the device / pinned
  // host arrays of per-right-hand-side pointers handed to the batched launches
  std::vector<SolverBuffers> lock;
  void** lock_ptrs = nullptr;
  void** h_lock_ptrs = nullptr;
  int lock_cap = 0;
  // two-level multigrid (dd_mg_setup): interpolation, coarse operator and the coarse
  // solver's buffers; mg_active: dd_solve_mg's outer solver applies it instead of M_sap
  struct Mg {
    int ntv = 0, nc = 0, mc = 0, cycles = 0;
    dd_sap_params smoother{};
    bool ready = false;
    float4* P = nullptr;                  // ntv FP32 internal fields
    float2* Dc = nullptr;                 // [domain][9][nc][nc]
    float4 *cb = nullptr, *cx = nullptr, *ct = nullptr, *cV = nullptr;   // coarse vectors, mc + 1 basis
    double2 *partial = nullptr, *partial2 = nullptr, *hA = nullptr, *hB = nullptr, *nrm = nullptr;
    zd *R = nullptr, *gv = nullptr, *y = nullptr;
    LsqState* lsq = nullptr;
    double* nu = nullptr;
    int* state = nullptr;
    int* ticket = nullptr;                // last-block ticket of the coarse Gram-Schmidt passes
    float4 *xf = nullptr, *rf = nullptr, *ef = nullptr;   // fine work fields
  } mg;
  bool mg_active = false;
  std::vector<void*> allocs;
};

// ------------------------------------------------------------------ helpers
static dd_status fail(dd_ctx* c, dd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

static dd_status cuda_check(dd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DD_OK;
  if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA;
}

template <typename T>
static dd_status dalloc(dd_ctx* c, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DD_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  c->allocs.push_back(q);
  *p = (T*)q;
  return DD_OK;
}

#define TRY(x)                         \
  do {                                 \
    dd_status _s = (x);                \
    if (_s != DD_OK) return _s;        \
  } while (0)

static dd_status launched(dd_ctx* c, int n = 1) {
  c->launches += n;
  cudaError_t e = cudaGetLastError();
  return cuda_check(c, e, "kernel launch");
}

static size_t field_bytes(const Geom& g, int prec) {
  if (prec == P64) return (size_t)g.V * 24 * 8;
  if (prec == P32) return (size_t)g.V * 24 * 4;
  return (size_t)g.V * 24 * 2 + (size_t)g.V * 4;
}

static FieldView view(const Geom& g, void* p, int prec) {
  FieldView f;
  f.data = p;
  f.prec = prec;
  f.norm = prec == P16 ? (float*)((char*)p + (size_t)g.V * 48) : nullptr;
  return f;
}

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

// ------------------------------------------------------------------ create / destroy
extern "C" dd_status dd_create(dd_ctx** out, const int dims[4], const int domain[4], int t_antiperiodic,
                               void* stream) {
  if (!out || !dims || !domain) return DD_ERR_INVALID;
  *out = nullptr;
  Geom g;
  memset(&g, 0, sizeof(g));
  g.V = 1;
  g.Vd = 1;
  g.ND = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = dims[mu];
    g.b[mu] = domain[mu];
    if (dims[mu] <= 0 || domain[mu] < 2 || ilog2(domain[mu]) < 0 || dims[mu] % domain[mu]) return DD_ERR_DIMS;
    g.N[mu] = dims[mu] / domain[mu];
    if (g.N[mu] < 2 || g.N[mu] % 2) return DD_ERR_DIMS;
    g.lgb[mu] = ilog2(domain[mu]);
    g.V *= dims[mu];
    g.Vd *= domain[mu];
    g.ND *= g.N[mu];
  }
  if (g.Vd < 64 || g.Vd > sap_max_domain_sites()) return DD_ERR_DIMS;
  g.Hd = g.Vd / 2;
  g.lgVd = ilog2(g.Vd);
  g.bstride[0] = 1;
  g.dstride[0] = 1;
  for (int mu = 1; mu < 4; ++mu) {
    g.bstride[mu] = g.bstride[mu - 1] * g.b[mu - 1];
    g.dstride[mu] = g.dstride[mu - 1] * g.N[mu - 1];
  }
  int off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    g.face_n[mu] = g.Vd / g.b[mu];
    g.face_off[2 * mu] = off;
    off += g.face_n[mu];
    g.face_off[2 * mu + 1] = off;
    off += g.face_n[mu];
  }
  g.face_block = off;
  dd_ctx* c = new dd_ctx();
  c->g = g;
  c->anti = t_antiperiodic ? 1 : 0;
  c->st = (cudaStream_t)stream;
  const char* tr = getenv("DD_TRACE");
  c->trace = tr && tr[0] && tr[0] != '0';
  const char* inj = getenv("DD_INJECT_WAIT_TIMEOUT");
  c->inject_wait_timeout = inj && inj[0] && inj[0] != '0';
  const char* ng = getenv("DD_NO_GRAPHS");
  c->use_graphs = !(ng && ng[0] && ng[0] != '0');
  if (dalloc(c, &c->dstatus, 64) != DD_OK || dalloc(c, &c->sap_err, 64) != DD_OK) {
    for (void* p : c->allocs) cudaFree(p);
    delete c;
    return DD_ERR_OOM;
  }
  cudaMemsetAsync(c->dstatus, 0, 64, c->st);
  cudaMemsetAsync(c->sap_err, 0, 64, c->st);
  *out = c;
  return DD_OK;
}

static void release_solver(dd_ctx* c);

extern "C" dd_status dd_destroy(dd_ctx* c) {
  if (!c) return DD_ERR_INVALID;
  cudaStreamSynchronize(c->st);
  release_solver(c);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
  return DD_OK;
}

extern "C" const char* dd_last_error(const dd_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" long long dd_launch_count(const dd_ctx* c) { return c ? c->launches : 0; }

extern "C" size_t dd_spinor_bytes(const dd_ctx* c, int prec, int layout) {
  if (!c) return 0;
  if (layout == DD_LAYOUT_CANONICAL) return (size_t)c->g.V * 24 * (prec == DD_PREC_FP64 ? 8 : 4);
  return field_bytes(c->g, prec);
}

// ------------------------------------------------------------------ gauge / clover
extern "C" dd_status dd_load_gauge(dd_ctx* c, const double* U, int where) {
  if (!c || !U) return DD_ERR_INVALID;
  const Geom& g = c->g;
  size_t n = (size_t)g.V * 72;
  if (!c->Ucanon) {
    TRY(dalloc(c, &c->Ucanon, n * 8));
    TRY(dalloc(c, &c->U64, n * 8));
    TRY(dalloc(c, &c->U32, n * 4));
    TRY(dalloc(c, &c->U16, n * 2));
  }
  TRY(cuda_check(c, cudaMemcpyAsync(c->Ucanon, U, n * 8, where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st),
                 "gauge copy"));
  launch_pack_gauge(g, c->Ucanon, c->anti, c->U64, c->U32, c->U16, c->st);
  TRY(launched(c));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "load_gauge"));
  c->have_gauge = true;
  c->have_clover = false;
  return DD_OK;
}

extern "C" dd_status dd_build_clover(dd_ctx* c, double kappa, double csw) {
  if (!c) return DD_ERR_INVALID;
  if (!c->have_gauge) return fail(c, DD_ERR_NO_GAUGE, "no gauge field loaded");
  if (!(kappa > 0)) return fail(c, DD_ERR_INVALID, "kappa must be positive");
  const Geom& g = c->g;
  if (!c->C64) {
    TRY(dalloc(c, &c->C64, (size_t)g.V * 72 * 8));
    TRY(dalloc(c, &c->C32, (size_t)g.V * 72 * 4));
    TRY(dalloc(c, &c->C16, (size_t)g.V * 72 * 2));
    TRY(dalloc(c, &c->S32, (size_t)g.V * 72 * 4));
    TRY(dalloc(c, &c->S16, (size_t)g.V * 72 * 2));
  }
  cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->st);
  launch_build_clover(g, c->Ucanon, kappa, csw, c->C64, c->C32, c->C16, c->S32, c->S16, c->dstatus, c->st);
  TRY(launched(c));
  int bad = 0;
  TRY(cuda_check(c, cudaMemcpyAsync(&bad, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st), "clover status"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "build_clover"));
  c->kappa = kappa;
  c->csw = csw;
  c->have_clover = true;
  if (bad) return fail(c, DD_ERR_SINGULAR_CLOVER, std::to_string(bad) + " sites with a singular clover block");
  return DD_OK;
}

// ------------------------------------------------------------------ operator
static GaugeView gauge_view(dd_ctx* c, int prec) {
  GaugeView v;
  v.prec = prec;
  v.links = prec == P64 ? (const void*)c->U64 : prec == P32 ? (const void*)c->U32 : (const void*)c->U16;
  return v;
}
static CloverView clover_view(dd_ctx* c, int prec) {
  CloverView v;
  v.prec = prec;
  v.m = prec == P64 ? (const void*)c->C64 : prec == P32 ? (const void*)c->C32 : (const void*)c->C16;
  return v;
}

static dd_status ensure_scratch(dd_ctx* c) {
  if (!c->scratch_in) {
    TRY(dalloc(c, &c->scratch_in, field_bytes(c->g, P64)));
    TRY(dalloc(c, &c->scratch_out, field_bytes(c->g, P64)));
  }
  return DD_OK;
}

static dd_status apply_internal(dd_ctx* c, const void* in, void* out, int prec, const void* f = nullptr) {
  FieldView vi = view(c->g, (void*)in, prec), vo = view(c->g, out, prec), vf = view(c->g, (void*)f, prec);
  launch_apply_A(c->g, gauge_view(c, prec), clover_view(c, prec), vi, vo, f ? &vf : nullptr, c->st);
  return launched(c);
}

extern "C" dd_status dd_apply_D(dd_ctx* c, const void* in, void* out, int prec, int layout) {
  if (!c || !in || !out || prec < 0 || prec > 2) return DD_ERR_INVALID;
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (layout == DD_LAYOUT_INTERNAL) {
    TRY(apply_internal(c, in, out, prec));
  } else {
    if (prec == P16) return fail(c, DD_ERR_INVALID, "FP16 needs the internal layout");
    TRY(ensure_scratch(c));
    launch_pack_spinor(c->g, in, prec, view(c->g, c->scratch_in, prec), c->st);
    TRY(launched(c));
    TRY(apply_internal(c, c->scratch_in, c->scratch_out, prec));
    launch_unpack_spinor(c->g, view(c->g, c->scratch_out, prec), out, prec, c->st);
    TRY(launched(c));
  }
  return cuda_check(c, cudaStreamSynchronize(c->st), "apply_D");
}

extern "C" dd_status dd_pack_spinor(dd_ctx* c, const void* canon, int cprec, void* internal, int iprec) {
  if (!c || !canon || !internal || cprec < 0 || cprec > 1 || iprec < 0 || iprec > 2) return DD_ERR_INVALID;
  launch_pack_spinor(c->g, canon, cprec, view(c->g, internal, iprec), c->st);
  TRY(launched(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "pack");
}

extern "C" dd_status dd_unpack_spinor(dd_ctx* c, const void* internal, int iprec, void* canon, int cprec) {
  if (!c || !canon || !internal || cprec < 0 || cprec > 1 || iprec < 0 || iprec > 2) return DD_ERR_INVALID;
  launch_unpack_spinor(c->g, view(c->g, (void*)internal, iprec), canon, cprec, c->st);
  TRY(launched(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "unpack");
}

// ------------------------------------------------------------------ Schwarz preconditioner
static void release(dd_ctx* c, void* p);

// The outer solver's captured graphs hold the addresses of the Schwarz state; they are
// destroyed whenever that state is reallocated, so no replay touches freed memory.
static void drop_graphs(dd_ctx* c) {
  for (auto& kv : c->sv.graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  c->sv.graphs.clear();
}

// Schwarz state (residual, solution, faces) for nrhs right-hand sides, one after another.
static dd_status ensure_sap(dd_ctx* c, int prec, int nrhs = 1) {
  SapBuffers& b = c->sap[prec];
  if (b.faces && b.cap >= nrhs) return DD_OK;
  if (b.faces) {
    cudaStreamSynchronize(c->st);
    drop_graphs(c);
    for (void* q : {(void*)b.r_store, (void*)b.r_norm, (void*)b.u_store, (void*)b.u_norm, (void*)b.faces,
                    (void*)b.faces2})
      release(c, q);
    b = SapBuffers();
  }
  const Geom& g = c->g;
  size_t half_sites = (size_t)g.V / 2, n = (size_t)nrhs;
  if (prec == P16) {
    TRY(dalloc(c, &b.r_store, n * half_sites * 48));
    TRY(dalloc(c, &b.r_norm, n * half_sites * 4));
    TRY(dalloc(c, &b.u_store, n * (size_t)g.V * 48));
    TRY(dalloc(c, &b.u_norm, n * (size_t)g.V * 4));
    b.r_bytes = (long long)half_sites * 48;
    b.u_bytes = (long long)g.V * 48;
  } else {
    TRY(dalloc(c, &b.r_store, n * half_sites * 96));
    TRY(dalloc(c, &b.u_store, n * (size_t)g.V * 96));
    b.r_bytes = (long long)half_sites * 96;
    b.u_bytes = (long long)g.V * 96;
  }
  TRY(dalloc(c, &b.faces, n * (size_t)g.ND * g.face_block * 48));
  b.cap = nrhs;
  return DD_OK;
}

// Storage precision of the Schwarz state for a dd_sap_params::storage_prec value.
static int sap_prec(int storage_prec) { return storage_prec == DD_PREC_FP32 ? P32 : P16; }

static SapState sap_state(dd_ctx* c, int prec, const dd_sap_params* p, int nrhs) {
  SapBuffers& b = c->sap[prec];
  SapState S;
  S.nrhs = nrhs;
  S.r_bytes = b.r_bytes;
  S.u_bytes = b.u_bytes;
  S.mat_prec = prec;
  S.vec_prec = prec;
  S.links = prec == P16 ? (const void*)c->U16 : (const void*)c->U32;
  S.smat = prec == P16 ? (const void*)c->S16 : (const void*)c->S32;
  S.r_store = b.r_store;
  S.r_norm = b.r_norm;
  S.u_store = b.u_store;
  S.u_norm = b.u_norm;
  S.faces = b.faces;
  S.err = c->sap_err;
  S.mat_in_smem = sap_mat_fits_smem(c->g, prec);
  S.threads_per_site = p->threads_per_site ? p->threads_per_site : 2;
  S.inject_wait_timeout = c->inject_wait_timeout;
  S.half_arith = p->storage_prec == DD_PREC_FP16_H2;
  return S;
}

// The launches of one Schwarz application on state S.  Multiplicative: I_Schwarz x (black,
// white) half-sweeps on one face buffer.  Additive: I_Schwarz launches over both colours,
// sweep s reading the faces of sweep s - 1 from one buffer and writing its own to the other.
static dd_status sap_sweeps(dd_ctx* c, SapState& S, const dd_sap_params* p, const float4* v, float4* z,
                            float4* faces2) {
  if (p->additive) {
    float4* fb[2] = {S.faces, faces2};
    S.both_colours = true;
    for (int s = 0; s < p->i_schwarz; ++s) {
      S.faces = fb[(s + 1) & 1];
      S.faces_out = fb[s & 1];
      if (sap_half_sweep(c->g, S, 0, s == 0, s > 0, s == p->i_schwarz - 1, v, z, p->i_domain, c->st))
        return fail(c, DD_ERR_CUDA, std::string("Schwarz launch failed: ") + cudaGetErrorString(cudaGetLastError()));
      TRY(launched(c));
    }
    return DD_OK;
  }
  for (int s = 0; s < p->i_schwarz; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      int first = s == 0, use_faces = !(s == 0 && colour == 0), last = s == p->i_schwarz - 1;
      if (sap_half_sweep(c->g, S, colour, first, use_faces, last, v, z, p->i_domain, c->st))
        return fail(c, DD_ERR_CUDA, std::string("Schwarz launch failed: ") + cudaGetErrorString(cudaGetLastError()));
      TRY(launched(c));
    }
  return DD_OK;
}

// The additive form's second face buffer, allocated on first use.
static dd_status ensure_faces2(dd_ctx* c, int prec) {
  SapBuffers& b = c->sap[prec];
  if (!b.faces2) TRY(dalloc(c, &b.faces2, (size_t)b.cap * c->g.ND * c->g.face_block * 48));
  return DD_OK;
}

// vscale (device scalar, single right-hand side): the input is v * (*vscale)
static dd_status sap_run(dd_ctx* c, const float4* v, float4* z, const dd_sap_params* p, int nrhs = 1,
                         const float* vscale = nullptr) {
  int prec = sap_prec(p->storage_prec);
  TRY(ensure_sap(c, prec, nrhs));
  if (p->additive) TRY(ensure_faces2(c, prec));
  SapState S = sap_state(c, prec, p, nrhs);
  S.vscale = vscale;
  return sap_sweeps(c, S, p, v, z, c->sap[prec].faces2);
}

static dd_status check_sap_params(dd_ctx* c, const dd_sap_params* p) {
  if (!p || p->i_schwarz < 1 || p->i_domain < 0 ||
      (p->storage_prec != DD_PREC_FP16 && p->storage_prec != DD_PREC_FP32 && p->storage_prec != DD_PREC_FP16_H2) ||
      p->threads_per_site < 0 || p->threads_per_site > 2 || p->additive < 0 || p->additive > 1)
    return fail(c, DD_ERR_INVALID, "bad Schwarz parameters");
  if (p->additive && p->threads_per_site == 1)
    return fail(c, DD_ERR_INVALID, "the additive form needs two threads per site");
  if (p->storage_prec == DD_PREC_FP16_H2 && p->threads_per_site == 1)
    return fail(c, DD_ERR_INVALID, "packed FP16 arithmetic needs two threads per site");
  return DD_OK;
}

static dd_status sap_error_flag(dd_ctx* c) {
  int e = 0;
  TRY(cuda_check(c, cudaMemcpyAsync(&e, c->sap_err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "sap status"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "sap"));
  if (e) {
    cudaMemsetAsync(c->sap_err, 0, sizeof(int), c->st);
    return fail(c, DD_ERR_TIMEOUT, "a bounded wait for the domain's staged data ran out");
  }
  return DD_OK;
}

extern "C" dd_status dd_sap_precondition(dd_ctx* c, const float* in, float* out, const dd_sap_params* p, int layout) {
  if (!c || !in || !out) return DD_ERR_INVALID;
  TRY(check_sap_params(c, p));
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (p->i_domain == 0) return fail(c, DD_ERR_INVALID, "i_domain must be >= 1");
  if (layout == DD_LAYOUT_INTERNAL) {
    TRY(sap_run(c, (const float4*)in, (float4*)out, p));
  } else {
    TRY(ensure_scratch(c));
    launch_pack_spinor(c->g, in, P32, view(c->g, c->scratch_in, P32), c->st);
    TRY(launched(c));
    TRY(sap_run(c, (const float4*)c->scratch_in, (float4*)c->scratch_out, p));
    launch_unpack_spinor(c->g, view(c->g, c->scratch_out, P32), out, P32, c->st);
    TRY(launched(c));
  }
  return sap_error_flag(c);
}

// ------------------------------------------------------------------ several right-hand sides
extern "C" dd_status dd_sap_precondition_batch(dd_ctx* c, const float* in, float* out, int nrhs,
                                               const dd_sap_params* p) {
  if (!c || !in || !out || nrhs < 1) return DD_ERR_INVALID;
  TRY(check_sap_params(c, p));
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (p->i_domain == 0) return fail(c, DD_ERR_INVALID, "i_domain must be >= 1");
  if (p->threads_per_site == 1 && nrhs > 1) return fail(c, DD_ERR_INVALID, "batches need threads_per_site 2");
  TRY(sap_run(c, (const float4*)in, (float4*)out, p, nrhs));
  return sap_error_flag(c);
}

extern "C" dd_status dd_sap_precondition_lattices(dd_ctx** ctxs, const float* const* in, float* const* out, int nlat,
                                                  int nrhs, const dd_sap_params* p) {
  if (!ctxs || !in || !out || nlat < 1 || nlat > 4 || nrhs < 1) return DD_ERR_INVALID;
  dd_ctx* c0 = ctxs[0];
  if (!c0) return DD_ERR_INVALID;
  TRY(check_sap_params(c0, p));
  if (p->storage_prec != DD_PREC_FP16 || p->threads_per_site == 1 || p->i_domain < 1 || p->additive)
    return fail(c0, DD_ERR_INVALID,
                "lattice batches need FP16 storage, two threads per site, i_domain >= 1 and the multiplicative form");
  Geom gs[4];
  SapState Ss[4];
  for (int l = 0; l < nlat; ++l) {
    dd_ctx* c = ctxs[l];
    if (!c || !in[l] || !out[l]) return DD_ERR_INVALID;
    if (!c->have_clover) return fail(c0, DD_ERR_NO_CLOVER, "clover not built on lattice " + std::to_string(l));
    if (c->g.Vd != c0->g.Vd || c->g.Hd != c0->g.Hd)
      return fail(c0, DD_ERR_DIMS, "lattices of one launch need the same domain volume");
    TRY(ensure_sap(c, P16, nrhs));
    gs[l] = c->g;
    Ss[l] = sap_state(c, P16, p, nrhs);
    if (Ss[l].mat_in_smem != Ss[0].mat_in_smem) return fail(c0, DD_ERR_DIMS, "mixed domain shapes");
  }
  for (int l = 0; l < nlat; ++l) cudaStreamSynchronize(ctxs[l]->st);   // inputs written on the lattices' streams
  for (int s = 0; s < p->i_schwarz; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      int first = s == 0, use_faces = !(s == 0 && colour == 0), last = s == p->i_schwarz - 1;
      if (sap_half_sweep_lattices(gs, Ss, nlat, colour, first, use_faces, last, (const float4* const*)in,
                                  (float4* const*)out, p->i_domain, c0->st))
        return fail(c0, DD_ERR_CUDA, std::string("Schwarz launch failed: ") + cudaGetErrorString(cudaGetLastError()));
      TRY(launched(c0));
    }
  TRY(cuda_check(c0, cudaStreamSynchronize(c0->st), "sap_lattices"));
  for (int l = 0; l < nlat; ++l) TRY(sap_error_flag(ctxs[l]));
  return DD_OK;
}

extern "C" dd_status dd_apply_D_batch(dd_ctx* c, const void* in, void* out, int nrhs, int prec) {
  if (!c || !in || !out || nrhs < 1 || (prec != DD_PREC_FP32 && prec != DD_PREC_FP16)) return DD_ERR_INVALID;
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  launch_apply_A_multi(c->g, gauge_view(c, prec), clover_view(c, prec), view(c->g, (void*)in, prec),
                       view(c->g, out, prec), nrhs, c->st);
  TRY(launched(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "apply_D_batch");
}

// ------------------------------------------------------------------ small dense kernels
__global__ void fill_value_kernel(float* v, int n, float x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}

__global__ void fill_ones_kernel(float* v, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 1.f;
}

// vscale[0] = 1 / sqrt(nu2): the scale of a vector stored unnormalised
__global__ void set_vscale_kernel(float* vscale, const double* nu2) { vscale[0] = (float)(1.0 / sqrt(*nu2)); }

// After the first projection: |w - V h|^2 is known exactly; ask for a second projection
// when it is below half of |w|^2.
__global__ void gs_decide_kernel(const zd* hA, int nv, const double2* nrm_a, zd* hB, int* flag, double* nu2) {
  double ww = hA[nv].re, v = nrm_a->x;
  for (int i = 0; i <= nv; ++i) hB[i] = Z(0.0);
  *nu2 = v;
  *flag = v < 0.5 * ww ? 1 : 0;
}

__global__ void gs_decide2_kernel(const int* flag, const double2* nrm_b, double* nu2) {
  if (*flag) *nu2 = nrm_b->x;
}

__global__ void arnoldi_finish_kernel(zd* H, zd* R, int ldh, int j, const zd* hA, const zd* hB, const double* nu2,
                                      LsqState* lsq, zd* g, double* status) {
  zd* col = H + (long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = hA[i] + hB[i];
  double h = sqrt(*nu2);
  col[j + 1] = Z(h);
  zd* rc = R + (long)j * ldh;
  for (int i = 0; i <= j + 1; ++i) rc[i] = col[i];
  status[0] = lsq_add_column(*lsq, R, ldh, j, j + 2, g);
  status[2] = h;
  status[3] = abs2(hB[0]) > 0 ? 1.0 : 0.0;
}

__global__ void lsq_solve_kernel(const zd* R, int ldh, int n, const zd* g, zd* y) { lsq_solve(R, ldh, n, g, y); }

// After a deflated restart: H <- Hn (k+1 x k), g <- cp, and the rotations of the dense
// block are rebuilt.
__global__ void restart_lsq_kernel(zd* H, zd* R, int ldh, int m, int k, const zd* Hn, const zd* cp, zd* g, zd* c0,
                                   LsqState* lsq, double* status, float* vscale) {
  for (int i = 0; i <= k; ++i) vscale[i] = 1.f;   // the recombined vectors are normalised
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= m; ++i) { H[i + (long)j * ldh] = Z(0.0); R[i + (long)j * ldh] = Z(0.0); }
  for (int i = 0; i <= m; ++i) g[i] = c0[i] = Z(0.0);
  for (int i = 0; i <= k; ++i) g[i] = c0[i] = cp[i];
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= k; ++i) H[i + (long)j * ldh] = R[i + (long)j * ldh] = Hn[i + (long)j * ldh];
  lsq->nrot = 0;
  double res = 0;
  for (int j = 0; j < k; ++j) res = lsq_add_column(*lsq, R, ldh, j, k + 1, g);
  status[0] = res;
}

__global__ void plain_restart_kernel(zd* H, zd* R, int ldh, int m, const double2* nrm2, zd* g, zd* c0, LsqState* lsq,
                                     float* vscale) {
  vscale[0] = 1.f;   // v_1 = r / |r| is stored normalised
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= m; ++i) { H[i + (long)j * ldh] = Z(0.0); R[i + (long)j * ldh] = Z(0.0); }
  for (int i = 0; i <= m; ++i) g[i] = c0[i] = Z(0.0);
  g[0] = c0[0] = Z(sqrt(nrm2->x));
  lsq->nrot = 0;
}

// The deflated restart's small dense step (harmonic Ritz pairs, P, Hn, cn) by one warp.
// Its workspace sits in shared memory when deflate_bytes(mm) fits (in_smem), else in the
// global scratch.
__global__ void deflate_kernel(const zd* H, int ldh, int mm, int k, const zd* c0, const zd* y, zd* P, zd* Hn, zd* cn,
                               zd* theta, void* gscratch, int in_smem, int* flags) {
  extern __shared__ __align__(16) unsigned char deflate_smem[];
  DeflateWork W = deflate_work(in_smem ? (void*)deflate_smem : gscratch, mm);
  const Team T{(int)threadIdx.x, (int)blockDim.x};
  const int rc = deflate(T, H, ldh, mm, k, c0, y, P, Hn, cn, theta, W);
  if (threadIdx.x == 0) flags[0] = rc;
}

static void launch_deflate(const zd* H, int ldh, int mm, int k, const zd* c0, const zd* y, zd* P, zd* Hn, zd* cn,
                           zd* theta, void* gscratch, int* flags, cudaStream_t st) {
  constexpr size_t smem_cap = 200 * 1024;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(deflate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap);
    configured = true;
  }
  const size_t b = deflate_bytes(mm);
  const int in_smem = b <= smem_cap;
  deflate_kernel<<<1, 32, in_smem ? b : 0, st>>>(H, ldh, mm, k, c0, y, P, Hn, cn, theta, gscratch, in_smem, flags);
}

// flags[1] = 1 when the basis is to be recombined: a deflation was computed and succeeded,
// and the recomputed residual is still above target (|r|^2 > tol2).
__global__ void restart_gate_kernel(int* flags, int want, const double2* nrm2, double tol2) {
  flags[1] = (want && flags[0] == 0 && nrm2->x > tol2) ? 1 : 0;
}

// After the projection cp = V_{k+1}^H (r / rho): cp <- rho cp, and whether the deflated
// restart keeps enough of r: |r - V_{k+1} cp| <= defl_tol |r|.  status[8..11] = |r|^2,
// decision, the part of r that the projection misses, deflation status.
__global__ void restart_decide_kernel(const int* flags, int want, int k, zd* cp, const double2* nrm2, double defl_tol,
                                      double* status) {
  const double rho2 = nrm2->x;
  int dec = 0;
  double miss = 1.0;
  if (want && flags[1]) {
    const double rho = sqrt(rho2);
    double pc = 0;
    for (int i = 0; i <= k; ++i) {
      cp[i] = rho * cp[i];
      pc += abs2(cp[i]);
    }
    miss = sqrt(fmax(0.0, 1.0 - pc / rho2));
    dec = miss <= defl_tol ? 1 : 0;
  }
  status[8] = rho2;
  status[9] = dec;
  status[10] = miss;
  status[11] = want ? (double)flags[0] : -1.0;
}

// ------------------------------------------------------------------ solver
static void release(dd_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      cudaFree(p);
      c->allocs.erase(c->allocs.begin() + i);
      return;
    }
}

// Free the outer solver's buffers (they are sized by the basis size m).
static void free_solver_buffers(dd_ctx* c, SolverBuffers& s) {
  cudaStreamSynchronize(c->st);
  for (void* p : {(void*)s.V, (void*)s.Z, (void*)s.w, (void*)s.x64,
                  (void*)s.f64, (void*)s.r64, (void*)s.canon64, (void*)s.H, (void*)s.R, (void*)s.P, (void*)s.Hn,
                  (void*)s.g, (void*)s.c0, (void*)s.y, (void*)s.hA, (void*)s.hB, (void*)s.cn, (void*)s.theta,
                  (void*)s.cp, (void*)s.partial, (void*)s.partial2, (void*)s.nrm2, (void*)s.status, (void*)s.lsq,
                  (void*)s.flag, (void*)s.nu2, (void*)s.dW, (void*)s.dflags, (void*)s.vscale, (void*)s.V16,
                  (void*)s.vin, (void*)s.one})
    release(c, p);
  if (s.h_status) cudaFreeHost(s.h_status);
  for (auto& kv : s.graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (s.stream) cudaStreamDestroy(s.stream);
  if (s.side) cudaStreamDestroy(s.side);
  for (cudaEvent_t e : {s.ev_in, s.ev_fork, s.ev_join})
    if (e) cudaEventDestroy(e);
  s = SolverBuffers();
}

static void release_solver(dd_ctx* c) {
  free_solver_buffers(c, c->sv);
  for (SolverBuffers& b : c->lock) free_solver_buffers(c, b);
  c->lock.clear();
  release(c, c->lock_ptrs);
  c->lock_ptrs = nullptr;
  if (c->h_lock_ptrs) cudaFreeHost(c->h_lock_ptrs);
  c->h_lock_ptrs = nullptr;
  c->lock_cap = 0;
}

// Krylov basis, FP64 fields and small dense buffers for basis size m; streams and events
// only for the context's own solver (the lockstep right-hand sides run on its stream).
static dd_status alloc_solver_buffers(dd_ctx* c, SolverBuffers& s, int m, bool streams, bool v16 = false) {
  const Geom& g = c->g;
  long long n4 = g.V * 6;
  size_t vb = (size_t)n4 * 16;
  if (v16) {
    TRY(dalloc(c, &s.V16, (size_t)n4 * 8 * (m + 1)));
    TRY(dalloc(c, &s.vin, vb));
    TRY(dalloc(c, &s.one, 16));
    const double one = 1.0;
    TRY(cuda_check(c, cudaMemcpy(s.one, &one, sizeof(double), cudaMemcpyHostToDevice), "constant"));
    // components of a unit vector have rms 1 / sqrt(24 V); s puts them near 2^-4, far from
    // both ends of the FP16 range
    s.v16_scale = ldexpf(1.f, (int)lrint(0.5 * log2(24.0 * (double)g.V)) - 4);
  } else {
    TRY(dalloc(c, &s.V, vb * (m + 1)));
  }
  s.v16 = v16;
  TRY(dalloc(c, &s.Z, vb * m));
  TRY(dalloc(c, &s.w, vb));
  TRY(dalloc(c, &s.x64, field_bytes(g, P64)));
  TRY(dalloc(c, &s.f64, field_bytes(g, P64)));
  TRY(dalloc(c, &s.r64, field_bytes(g, P64)));
  TRY(dalloc(c, &s.canon64, field_bytes(g, P64)));
  int ld = m + 1;
  size_t hm = (size_t)ld * (m + 1) * sizeof(zd);
  TRY(dalloc(c, &s.H, hm));
  TRY(dalloc(c, &s.R, hm));
  TRY(dalloc(c, &s.P, hm));
  TRY(dalloc(c, &s.Hn, hm));
  for (zd** p : {&s.g, &s.c0, &s.y, &s.hA, &s.hB, &s.cn, &s.theta, &s.cp}) TRY(dalloc(c, p, (m + 2) * sizeof(zd)));
  TRY(dalloc(c, &s.partial, (size_t)blas_partials_blocks() * (m + 2) * sizeof(double2)));
  TRY(dalloc(c, &s.partial2, (size_t)blas_partials_blocks() * sizeof(double2)));
  TRY(dalloc(c, &s.nrm2, 4 * sizeof(double2)));
  TRY(dalloc(c, &s.status, 16 * sizeof(double)));
  TRY(dalloc(c, &s.lsq, sizeof(LsqState)));
  TRY(dalloc(c, &s.flag, 16));
  TRY(dalloc(c, &s.nu2, 16));
  TRY(dalloc(c, &s.dW, deflate_bytes(m)));
  TRY(dalloc(c, &s.vscale, (m + 2) * sizeof(float)));
  fill_value_kernel<<<1, 64, 0, c->st>>>(s.vscale, m + 2, v16 ? 1.f / s.v16_scale : 1.f);
  TRY(launched(c));
  TRY(dalloc(c, &s.dflags, 16 * sizeof(int)));
  if (cudaMallocHost(&s.h_status, 8 * sizeof(double)) != cudaSuccess) return fail(c, DD_ERR_OOM, "pinned status");
  if (streams && (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming) != cudaSuccess))
    return fail(c, DD_ERR_CUDA, "solver stream");
  s.m = m;
  return DD_OK;
}

static dd_status ensure_solver(dd_ctx* c, int m, bool v16 = false) {
  if (c->sv.m >= m && c->sv.v16 == v16) return DD_OK;
  if (c->sv.m) {
    drop_graphs(c);   // captured steps hold the old buffers
    release_solver(c);
  }
  return alloc_solver_buffers(c, c->sv, m, true, v16);
}

// Run a launch sequence of the outer solver: directly on its first use, captured into a
// CUDA graph on its second (so one-time set-up inside the sequence stays out of the
// capture), replayed from the graph afterwards.  If capture is not possible the
// sequence keeps running directly.
template <typename F>
static dd_status graphed(dd_ctx* c, const GraphKey& key, F&& fn) {
  SolverBuffers& s = c->sv;
  GraphEntry& e = s.graphs[key];
  if (e.exec) {
    TRY(cuda_check(c, cudaGraphLaunch(e.exec, c->st), "graph launch"));
    c->launches += e.kernels;
    return DD_OK;
  }
  if (!c->use_graphs || e.seen == 0 || c->st != s.stream) {
    e.seen++;
    return fn();
  }
  cudaGraph_t gr = nullptr;
  TRY(cuda_check(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal), "begin capture"));
  long long l0 = c->launches;
  dd_status st = fn();
  cudaError_t ce = cudaStreamEndCapture(c->st, &gr);
  long long kernels = c->launches - l0;
  c->launches = l0;
  cudaGraphExec_t ex = nullptr;
  if (st == DD_OK && ce == cudaSuccess && gr && cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess) {
    cudaGraphDestroy(gr);
    e.exec = ex;
    e.kernels = kernels;
    TRY(cuda_check(c, cudaGraphLaunch(ex, c->st), "graph launch"));
    c->launches += kernels;
    return DD_OK;
  }
  if (gr) cudaGraphDestroy(gr);
  cudaGetLastError();
  c->use_graphs = false;   // capture unavailable: stay with direct launches
  if (st != DD_OK) return st;
  return fn();
}

static dd_status read_status(dd_ctx* c, int n = 4) {
  SolverBuffers& s = c->sv;
  TRY(cuda_check(c, cudaMemcpyAsync(s.h_status, s.status, n * sizeof(double), cudaMemcpyDeviceToHost, c->st), "status"));
  return cuda_check(c, cudaStreamSynchronize(c->st), "solver step");
}

// rho2 = |f - A x|^2 into s.nrm2 (device) and return it on the host (s: the context's own
// solver buffers unless given).
static dd_status true_residual(dd_ctx* c, double* rho2, SolverBuffers* sp = nullptr) {
  SolverBuffers& s = sp ? *sp : c->sv;
  TRY(apply_internal(c, s.x64, s.r64, P64, s.f64));
  launch_norm2_64(s.r64, c->g.V * 12, s.partial, c->st);
  launch_reduce_partials(s.partial, 1, s.nrm2, 0, c->st);
  TRY(launched(c, 2));
  double2 h;
  TRY(cuda_check(c, cudaMemcpyAsync(&h, s.nrm2, sizeof(double2), cudaMemcpyDeviceToHost, c->st), "norm"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "norm"));
  *rho2 = h.x;
  return DD_OK;
}

// End of a cycle after mm Arnoldi steps, on the device: y from the least-squares problem;
// the deflated restart's small dense step (one warp, on the second stream beside the
// reliable update when `side` is set); x64 += Z y; r64 = f - A64 x64 and |r64|^2; then,
// when the deflation succeeded and |r64| is still above target, V <- V P_{k+1} and
// Z <- Z P_k in place and the projection of r64 onto the new V_{k+1}.  The one host read
// returns |r64|^2 and whether the deflated restart keeps enough of r64.
struct CycleEnd {
  double rho2 = 0, miss = 1;
  bool deflate = false;
  int defl_rc = -1;
};

static dd_status end_cycle(dd_ctx* c, SolverBuffers& s, int mm, const dd_solve_params* p, double nf, bool side,
                           CycleEnd* out) {
  const long long n4 = c->g.V * 6;
  const int m = p->m, k = p->k, ldh = m + 1;
  const double defl_tol = 1e-2;
  const int want = k > 0 && mm > k;
  lsq_solve_kernel<<<1, 1, 0, c->st>>>(s.R, ldh, mm, s.g, s.y);
  int nk = 1;
  cudaStream_t ds = c->st;
  if (want) {
    if (side && s.side) {
      cudaEventRecord(s.ev_fork, c->st);
      cudaStreamWaitEvent(s.side, s.ev_fork, 0);
      ds = s.side;
    }
    launch_deflate(s.H, ldh, mm, k, s.c0, s.y, s.P, s.Hn, s.cn, s.theta, s.dW, s.dflags, ds);
    nk++;
    if (ds != c->st) cudaEventRecord(s.ev_join, ds);
  }
  launch_x_update(s.x64, s.Z, mm, n4, (const double2*)s.y, c->st);
  nk++;
  TRY(launched(c, nk));
  TRY(apply_internal(c, s.x64, s.r64, P64, s.f64));
  launch_norm2_64(s.r64, c->g.V * 12, s.partial, c->st);
  launch_reduce_partials(s.partial, 1, s.nrm2, 0, c->st);
  nk = 2;
  if (want && ds != c->st) cudaStreamWaitEvent(c->st, s.ev_join, 0);
  const double tol2 = (p->tol * nf) * (p->tol * nf);
  restart_gate_kernel<<<1, 1, 0, c->st>>>(s.dflags, want, s.nrm2, tol2);
  nk++;
  if (want) {
    // V <- V P_{k+1}, Z <- Z P_k in place: every output element depends only on the inputs
    // at the same position, which its thread reads before writing
    const int* gate = s.dflags + 1;
    if (s.v16)
      nk += launch_recombine(s.V16, s.V16, mm + 1, k + 1, n4, (const double2*)s.P, ldh, c->st, gate, s.vscale,
                             s.v16_scale);
    else
      nk += launch_recombine(s.V, s.V, mm + 1, k + 1, n4, (const double2*)s.P, ldh, c->st, gate, s.vscale);
    nk += launch_recombine(s.Z, s.Z, mm, k, n4, (const double2*)s.P, ldh, c->st, gate);
    launch_r64_to_v32(s.w, s.r64, n4, s.nrm2, c->st, gate);
    if (s.v16)
      nk += 1 + launch_gs_dot(s.V16, k + 1, n4, s.w, s.partial, gate, 1, c->st, s.vscale);
    else
      nk += 1 + launch_gs_dot(s.V, k + 1, n4, s.w, s.partial, gate, 1, c->st);
    launch_gs_reduce(s.partial, k + 1, (double2*)s.cp, gate, 1, c->st);
    nk++;
  }
  restart_decide_kernel<<<1, 1, 0, c->st>>>(s.dflags, want, k, s.cp, s.nrm2, defl_tol, s.status);
  nk++;
  TRY(launched(c, nk));
  TRY(cuda_check(c, cudaMemcpyAsync(s.h_status, s.status + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st),
                 "restart status"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "restart"));
  out->rho2 = s.h_status[0];
  out->deflate = s.h_status[1] != 0.0;
  out->miss = s.h_status[2];
  out->defl_rc = (int)s.h_status[3];
  return DD_OK;
}

// ------------------------------------------------------------------ two-level multigrid
// The Schwarz method as the smoother of an aggregation-based two-level method (the use of
// domain-decomposition preconditioners in the multigrid solvers of the paper's related
// work, Sec. V).  Aggregates are the Schwarz domains; kernels in mg.cu.
static void mg_free(dd_ctx* c) {
  dd_ctx::Mg& M = c->mg;
  cudaStreamSynchronize(c->st);
  for (void* p : {(void*)M.P, (void*)M.Dc, (void*)M.cb, (void*)M.cx, (void*)M.ct, (void*)M.cV, (void*)M.partial,
                  (void*)M.partial2, (void*)M.hA, (void*)M.hB, (void*)M.nrm, (void*)M.R, (void*)M.gv, (void*)M.y,
                  (void*)M.lsq, (void*)M.nu, (void*)M.state, (void*)M.ticket, (void*)M.xf, (void*)M.rf,
                  (void*)M.ef})
    release(c, p);
  M = dd_ctx::Mg();
}

static dd_status mg_alloc(dd_ctx* c, int ntv, int mc) {
  dd_ctx::Mg& M = c->mg;
  const Geom& g = c->g;
  const long long n4 = g.V * 6;
  const int nc = 2 * ntv;
  const long long n4c = (long long)g.ND * nc / 2;
  M.ntv = ntv;
  M.nc = nc;
  M.mc = mc;
  TRY(dalloc(c, &M.P, (size_t)ntv * n4 * 16));
  TRY(dalloc(c, &M.Dc, (size_t)g.ND * 9 * nc * nc * sizeof(float2)));
  for (float4** q : {&M.cb, &M.cx, &M.ct}) TRY(dalloc(c, q, (size_t)n4c * 16));
  TRY(dalloc(c, &M.cV, (size_t)(mc + 1) * n4c * 16));
  // basis vectors past a breakdown are multiplied by zero coefficients: keep them finite
  TRY(cuda_check(c, cudaMemsetAsync(M.cV, 0, (size_t)(mc + 1) * n4c * 16, c->st), "coarse basis"));
  TRY(dalloc(c, &M.partial, (size_t)blas_partials_blocks() * (mc + 2) * sizeof(double2)));
  TRY(dalloc(c, &M.partial2, (size_t)blas_partials_blocks() * sizeof(double2)));
  for (double2** q : {&M.hA, &M.hB}) TRY(dalloc(c, q, (size_t)(mc + 2) * sizeof(double2)));
  TRY(dalloc(c, &M.nrm, 4 * sizeof(double2)));
  TRY(dalloc(c, &M.R, (size_t)(mc + 1) * (mc + 1) * sizeof(zd)));
  TRY(dalloc(c, &M.gv, (size_t)(mc + 2) * sizeof(zd)));
  TRY(dalloc(c, &M.y, (size_t)(mc + 1) * sizeof(zd)));
  TRY(dalloc(c, &M.lsq, sizeof(LsqState)));
  TRY(dalloc(c, &M.nu, 16));
  TRY(dalloc(c, &M.state, 16));
  TRY(dalloc(c, &M.ticket, 16));
  TRY(cuda_check(c, cudaMemsetAsync(M.ticket, 0, 16, c->st), "ticket"));
  for (float4** q : {&M.xf, &M.rf, &M.ef}) TRY(dalloc(c, q, (size_t)n4 * 16));
  return DD_OK;
}

// cx ~ D_c^{-1} cb: `cycles` cycles of GMRES(mc) from cx = 0 on the coarse operator, FP32
// vectors, classical Gram-Schmidt with a second pass (FP64 sums), FP64 Givens least
// squares.  A fixed launch sequence with no host synchronisation (a cycle that reaches an
// invariant subspace skips its remaining steps on the device), so it can be captured.
static dd_status mg_coarse_solve(dd_ctx* c) {
  dd_ctx::Mg& M = c->mg;
  const Geom& g = c->g;
  cudaStream_t st = c->st;
  const long long n4c = (long long)g.ND * M.nc / 2;
  auto Vc = [&](int i) { return M.cV + (long long)i * n4c; };
  const int ldh = M.mc + 1;
  double* nrm_part = (double*)M.partial2;   // per-block |v|^2 shares of a projection
  int nk = 0;
  for (int cyc = 0; cyc < M.cycles; ++cyc) {
    if (cyc == 0) {
      TRY(cuda_check(c, cudaMemcpyAsync(Vc(0), M.cb, (size_t)n4c * 16, cudaMemcpyDeviceToDevice, st), "coarse rhs"));
    } else {
      launch_mg_coarse_apply(g, M.Dc, M.nc, (const float2*)M.cx, (float2*)Vc(0), (const float2*)M.cb, nullptr, st);
      ++nk;
    }
    launch_mg_cdot(Vc(0), 0, n4c, Vc(0), M.partial, M.nrm, M.ticket, nullptr, st);   // |r|^2
    launch_mg_beta(M.nrm, M.gv, M.mc + 2, M.nu, M.state, M.lsq, st);
    launch_mg_scale(Vc(0), n4c, M.nu, M.state, st);
    nk += 3;
    // one step: w = D_c v_j; two classical Gram-Schmidt passes (coefficients, then the
    // projection); the second projection also forms the Hessenberg column, its Givens
    // update and 1 / h_{j+1,j}; then v_{j+1} is scaled
    for (int j = 0; j < M.mc; ++j) {
      launch_mg_coarse_apply(g, M.Dc, M.nc, (const float2*)Vc(j), (float2*)M.ct, nullptr, M.state, st);
      launch_mg_cdot(Vc(0), j + 1, n4c, M.ct, M.partial, M.hA, M.ticket, M.state, st);
      launch_mg_cproject(M.ct, M.ct, Vc(0), j + 1, n4c, M.hA, nrm_part, nullptr, M.ticket, M.state, 0, M.R, ldh, j,
                         M.hA, M.hB, M.lsq, M.gv, M.nu, M.state, st);
      launch_mg_cdot(Vc(0), j + 1, n4c, M.ct, M.partial, M.hB, M.ticket, M.state, st);
      launch_mg_cproject(Vc(j + 1), M.ct, Vc(0), j + 1, n4c, M.hB, nrm_part, nullptr, M.ticket, M.state, 1, M.R,
                         ldh, j, M.hA, M.hB, M.lsq, M.gv, M.nu, M.state, st);
      launch_mg_scale(Vc(j + 1), n4c, M.nu, M.state, st);
      nk += 6;
    }
    launch_mg_lsq(M.R, ldh, M.mc, M.gv, M.state, M.y, st);
    ++nk;
    if (cyc == 0) {
      nk += launch_recombine(M.cx, Vc(0), M.mc, 1, n4c, (const double2*)M.y, M.mc, st);
    } else {
      nk += launch_recombine(M.ct, Vc(0), M.mc, 1, n4c, (const double2*)M.y, M.mc, st);
      launch_mg_axpy(M.cx, M.ct, n4c, 1.f, st);
      ++nk;
    }
  }
  return launched(c, nk);
}

// z = B v, one application of the two-level preconditioner: coarse correction
// x = P D_c^{-1} P^H v (approximate coarse solve), then the smoother's Schwarz cycles on
// the remaining residual, z = x + M_sap (v - A x).  vscale (device scalar, optional): the
// input is v * (*vscale) (B is linear, so the scale is applied to z).
static dd_status mg_run(dd_ctx* c, const float4* v, float4* z, const float* vscale = nullptr) {
  dd_ctx::Mg& M = c->mg;
  const Geom& g = c->g;
  launch_mg_restrict(g, v, M.P, M.ntv, (float2*)M.cb, nullptr, c->st);
  TRY(launched(c));
  TRY(mg_coarse_solve(c));
  launch_mg_prolong(g, (const float2*)M.cx, M.P, M.ntv, M.xf, c->st);
  TRY(launched(c));
  const bool smooth = M.smoother.i_schwarz > 0;
  if (smooth) {
    TRY(apply_internal(c, M.xf, M.rf, P32, v));   // rf = v - A xf
    TRY(sap_run(c, M.rf, M.ef, &M.smoother));
  }
  launch_mg_combine(z, M.xf, smooth ? M.ef : nullptr, g.V * 6, vscale, c->st);
  return launched(c);
}

static dd_status solve_one(dd_ctx* c, const dd_solve_params* p, double nf2, dd_solve_info* info) {
  SolverBuffers& s = c->sv;
  const Geom& g = c->g;
  const long long n4 = g.V * 6;
  const int m = p->m, k = p->k, ldh = m + 1;
  const double tol = p->tol;
  const double nf = sqrt(nf2);
  const double defl_tol = 1e-2;
  cudaEvent_t e0, e1, e2, e3, e4;
  cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2); cudaEventCreate(&e3); cudaEventCreate(&e4);
  cudaEvent_t tstart, tend;
  cudaEventCreate(&tstart); cudaEventCreate(&tend);
  cudaEventRecord(tstart, c->st);
  double tA = 0, tM = 0, tGS = 0;
  int iters = 0, restarts = 0, reliable = 0, deflated = 0;
  dd_status rc = DD_OK;
  double rho2 = 0;
  auto Vv = [&](int i) { return s.V + (long long)i * n4; };
  auto Zv = [&](int i) { return s.Z + (long long)i * n4; };
  // FP16 basis: V16 holds s v_i (vscale[i] = 1 / s), vin the FP32 copy of the newest v
  const bool h16 = s.v16;
  const float vs16 = s.v16_scale;
  auto V16 = [&](int i) { return s.V16 + (long long)i * n4; };
  // v_1 = r / |r| (FP16 basis: into vin and, scaled, into V16)
  auto first_vector = [&]() -> dd_status {
    if (!h16) {
      launch_r64_to_v32(Vv(0), s.r64, n4, s.nrm2, c->st);
      plain_restart_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, ldh, m, s.nrm2, s.g, s.c0, s.lsq, s.vscale);
      return launched(c, 2);
    }
    launch_r64_to_v32(s.vin, s.r64, n4, s.nrm2, c->st);
    launch_basis16_store(V16(0), nullptr, s.vin, n4, s.one, vs16, c->st);
    plain_restart_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, ldh, m, s.nrm2, s.g, s.c0, s.lsq, s.vscale);
    fill_value_kernel<<<1, 64, 0, c->st>>>(s.vscale, m + 2, 1.f / vs16);
    return launched(c, 4);
  };

  TRY(true_residual(c, &rho2));
  reliable++;
  double rel = sqrt(rho2) / nf;
  if (!isfinite(rel)) rc = fail(c, DD_ERR_NONFINITE, "non-finite residual");
  int j0 = 0;
  if (rc == DD_OK && rel > tol) TRY(first_vector());
  while (rc == DD_OK && rel > tol) {
    if (iters >= p->max_iter) { rc = fail(c, DD_ERR_NOT_CONVERGED, "iteration limit reached"); break; }
    int mm = m;
    double rho_cycle = sqrt(rho2);
    for (int j = j0; j < m; ++j) {
      // one Arnoldi step = three device-only launch sequences, each replayed from a CUDA
      // graph once it has been captured (keyed by step and parameters)
      const GraphKey kbase = {0, j, p->sap.i_schwarz, p->sap.i_domain, p->sap.storage_prec,
                              p->sap.threads_per_site, m, p->sap.additive};
      GraphKey k0 = kbase, k1 = kbase, k2 = kbase;
      const int part0 = h16 ? 20 : 0;   // the FP16-basis steps are other launch sequences
      k0[0] = part0;
      k1[0] = part0 + 1;
      k2[0] = part0 + 2;
      // the preconditioner's input: the stored v_j with its scale, or the FP32 copy
      const float4* vj = h16 ? s.vin : Vv(j);
      const float* vjs = h16 ? nullptr : s.vscale + j;
      cudaEventRecord(e0, c->st);
      if (c->mg_active) {
        k0[0] = part0 + 7;
        TRY(graphed(c, k0, [&]() { return mg_run(c, vj, Zv(j), vjs); }));
      } else {
        TRY(graphed(c, k0, [&]() { return sap_run(c, vj, Zv(j), &p->sap, 1, vjs); }));
      }
      cudaEventRecord(e1, c->st);
      TRY(graphed(c, k1, [&]() { return apply_internal(c, Zv(j), s.w, P32); }));
      cudaEventRecord(e2, c->st);
      TRY(graphed(c, k2, [&]() {
        if (h16) {
          // the same Gram-Schmidt over the FP16 basis, projecting w in place; the new basis
          // vector is normalised on its way into V16 (and into vin for the next step)
          double2* nrm_a = s.nrm2 + 1;
          double2* nrm_b = s.nrm2 + 2;
          const float* sc = s.vscale;
          int nk = launch_gs_dot(V16(0), j + 1, n4, s.w, s.partial, nullptr, 0, c->st, sc);
          launch_gs_reduce(s.partial, j + 1, (double2*)s.hA, nullptr, 0, c->st);
          launch_gs_project(s.w, s.w, V16(0), j + 1, n4, (const double2*)s.hA, s.partial2, nullptr, 0, c->st, sc);
          launch_gs_reduce(s.partial2, 0, nrm_a, nullptr, 0, c->st);
          gs_decide_kernel<<<1, 1, 0, c->st>>>(s.hA, j + 1, nrm_a, s.hB, s.flag, s.nu2);
          nk += launch_gs_dot(V16(0), j + 1, n4, s.w, s.partial, s.flag, 1, c->st, sc);
          launch_gs_reduce(s.partial, j + 1, (double2*)s.hB, s.flag, 1, c->st);
          launch_gs_project(s.w, s.w, V16(0), j + 1, n4, (const double2*)s.hB, s.partial2, s.flag, 1, c->st, sc);
          launch_gs_reduce(s.partial2, 0, nrm_b, s.flag, 1, c->st);
          gs_decide2_kernel<<<1, 1, 0, c->st>>>(s.flag, nrm_b, s.nu2);
          cudaEventRecord(s.ev_fork, c->st);
          cudaStreamWaitEvent(s.side, s.ev_fork, 0);
          arnoldi_finish_kernel<<<1, 1, 0, s.side>>>(s.H, s.R, ldh, j, s.hA, s.hB, s.nu2, s.lsq, s.g, s.status);
          cudaEventRecord(s.ev_join, s.side);
          launch_basis16_store(V16(j + 1), s.vin, s.w, n4, s.nu2, vs16, c->st);
          cudaStreamWaitEvent(c->st, s.ev_join, 0);
          return launched(c, nk + 10);
        }
        // Gram-Schmidt: classical projection with the exact norm of the result, repeated
        // once when it cancels more than half of |w| (Daniel-Gragg-Kaufman-Stewart test)
        float4* vn = Vv(j + 1);
        double2* nrm_a = s.nrm2 + 1;
        double2* nrm_b = s.nrm2 + 2;
        // the basis vectors are read through their scales (vscale), and the new one stays
        // unnormalised: its exact norm comes out of the projection pass
        const float* sc = s.vscale;
        int nk = launch_gs_dot(Vv(0), j + 1, n4, s.w, s.partial, nullptr, 0, c->st, sc);
        launch_gs_reduce(s.partial, j + 1, (double2*)s.hA, nullptr, 0, c->st);
        launch_gs_project(vn, s.w, Vv(0), j + 1, n4, (const double2*)s.hA, s.partial2, nullptr, 0, c->st, sc);
        launch_gs_reduce(s.partial2, 0, nrm_a, nullptr, 0, c->st);
        gs_decide_kernel<<<1, 1, 0, c->st>>>(s.hA, j + 1, nrm_a, s.hB, s.flag, s.nu2);
        nk += launch_gs_dot(Vv(0), j + 1, n4, vn, s.partial, s.flag, 1, c->st, sc);
        launch_gs_reduce(s.partial, j + 1, (double2*)s.hB, s.flag, 1, c->st);
        launch_gs_project(vn, vn, Vv(0), j + 1, n4, (const double2*)s.hB, s.partial2, s.flag, 1, c->st, sc);
        launch_gs_reduce(s.partial2, 0, nrm_b, s.flag, 1, c->st);
        gs_decide2_kernel<<<1, 1, 0, c->st>>>(s.flag, nrm_b, s.nu2);
        // the Hessenberg column and its Givens update (one thread) beside the new vector's
        // scale; both only read nu2
        cudaEventRecord(s.ev_fork, c->st);
        cudaStreamWaitEvent(s.side, s.ev_fork, 0);
        arnoldi_finish_kernel<<<1, 1, 0, s.side>>>(s.H, s.R, ldh, j, s.hA, s.hB, s.nu2, s.lsq, s.g, s.status);
        cudaEventRecord(s.ev_join, s.side);
        set_vscale_kernel<<<1, 1, 0, c->st>>>(s.vscale + j + 1, s.nu2);
        cudaStreamWaitEvent(c->st, s.ev_join, 0);
        return launched(c, nk + 10);
      }));
      cudaEventRecord(e3, c->st);
      TRY(read_status(c));
      float ms;
      cudaEventElapsedTime(&ms, e0, e1); tM += ms * 1e-3;
      cudaEventElapsedTime(&ms, e1, e2); tA += ms * 1e-3;
      cudaEventElapsedTime(&ms, e2, e3); tGS += ms * 1e-3;
      iters++;
      double est = s.h_status[0];
      if (c->trace)
        fprintf(stderr, "[dd] it %d j %d est/rho %.3e h %.3e reorth %d\n", iters, j, est / rho_cycle, s.h_status[2],
                (int)s.h_status[3]);
      if (!isfinite(est) || !isfinite(s.h_status[2])) { rc = fail(c, DD_ERR_NONFINITE, "non-finite Arnoldi step"); break; }
      // stop the cycle when the target is met or FP32 vectors cannot resolve further
      if (est <= 0.5 * tol * nf || est <= 2e-6 * rho_cycle || iters >= p->max_iter) { mm = j + 1; break; }
    }
    if (rc != DD_OK) break;
    if (c->trace && getenv("DD_TRACE")[0] == '2' && !h16) {
      // orthogonality of the finished basis: max |V^H V - I|
      double dev = 0;
      std::vector<zd> row(mm + 1);
      std::vector<float> sc(mm + 1);
      cudaMemcpyAsync(sc.data(), s.vscale, (mm + 1) * sizeof(float), cudaMemcpyDeviceToHost, c->st);
      for (int i = 0; i <= mm; ++i) {
        launch_multi_dot(Vv(0), mm + 1, n4, Vv(i), s.partial, c->st);
        launch_reduce_partials(s.partial, mm + 1, (double2*)s.hB, 0, c->st);
        cudaMemcpyAsync(row.data(), s.hB, (mm + 1) * sizeof(zd), cudaMemcpyDeviceToHost, c->st);
        cudaStreamSynchronize(c->st);
        for (int l = 0; l <= mm; ++l)
          dev = fmax(dev, zabs(((double)sc[i] * sc[l]) * row[l] - Z(l == i ? 1.0 : 0.0)));
      }
      fprintf(stderr, "[dd] basis orthogonality max|V^H V - I| = %.3e over %d vectors\n", dev, mm + 1);
    }
    CycleEnd ce;
    TRY(end_cycle(c, s, mm, p, nf, true, &ce));
    rho2 = ce.rho2;
    reliable++;
    rel = sqrt(rho2) / nf;
    if (!isfinite(rel)) { rc = fail(c, DD_ERR_NONFINITE, "non-finite residual"); break; }
    if (rel <= tol) break;
    if (iters >= p->max_iter) { rc = fail(c, DD_ERR_NOT_CONVERGED, "iteration limit reached"); break; }
    restarts++;
    if (c->trace)
      fprintf(stderr, "[dd] restart: true residual %.3e, deflation status %d, misses %.3e\n", rel, ce.defl_rc, ce.miss);
    if (ce.deflate) {
      restart_lsq_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, ldh, m, k, s.Hn, s.cp, s.g, s.c0, s.lsq, s.status, s.vscale);
      TRY(launched(c));
      if (h16) {
        // the recombined basis is stored s v_i; the step at j = k reads v_k in FP32
        fill_value_kernel<<<1, 64, 0, c->st>>>(s.vscale, m + 2, 1.f / vs16);
        launch_basis16_load(s.vin, V16(k), n4, 1.f / vs16, c->st);
        TRY(launched(c, 2));
      }
      j0 = k;
      deflated++;
    } else {
      TRY(first_vector());
      j0 = 0;
    }
  }
  cudaEventRecord(tend, c->st);
  cudaEventSynchronize(tend);
  float ms = 0;
  cudaEventElapsedTime(&ms, tstart, tend);
  if (info) {
    info->iterations += iters;
    info->restarts += restarts;
    info->reliable_updates += reliable;
    info->deflated_restarts += deflated;
    info->true_rel_residual = fmax(info->true_rel_residual, rel);
    info->t_total += ms * 1e-3;
    info->t_A += tA;
    info->t_M += tM;
    info->t_GS += tGS;
    info->t_other += ms * 1e-3 - tA - tM - tGS;
    double V = (double)g.V;
    // paper's convention: 1848 flop per site per operator application; each Schwarz
    // half-sweep applies D once per MR step plus once for preparation and update
    info->flops_nominal += iters * (1848.0 * V + p->sap.i_schwarz * (p->sap.i_domain + 1) * 1848.0 * V) + reliable * 1848.0 * V;
  }
  for (cudaEvent_t e : {e0, e1, e2, e3, e4, tstart, tend}) cudaEventDestroy(e);
  if (rc == DD_OK) TRY(sap_error_flag(c));
  return rc;
}

// ------------------------------------------------------------------ lockstep right-hand sides
// Several right-hand sides solved together.  Each keeps its own Krylov basis, Hessenberg
// matrix, restarts and stopping point, with the same steps as solve_one; they share the
// two large applications of every Arnoldi step: the Schwarz preconditioner runs as one
// launch per half-sweep over all active right-hand sides (each CTA stages its domain's
// links and Schwarz matrices once for all of them) and the operator as one launch with
// two right-hand sides per thread.  Each right-hand side sits at its own step j, so both
// launches take device arrays of input and output pointers.
struct LockRhs {
  double nf = 0, rho2 = 0, rel = 0, rho_cycle = 0;
  int j = 0, j0 = 0;
  int iters = 0, restarts = 0, reliable = 0, deflated = 0;
  bool done = false;
  dd_status rc = DD_OK;
};

static dd_status ensure_lock(dd_ctx* c, int nrhs, int m) {
  bool ok = (int)c->lock.size() >= nrhs;
  for (int r = 0; ok && r < nrhs; ++r) ok = c->lock[r].m >= m;
  if (!ok) {
    for (SolverBuffers& b : c->lock) free_solver_buffers(c, b);
    c->lock.clear();
    c->lock.resize(nrhs);
    for (int r = 0; r < nrhs; ++r) TRY(alloc_solver_buffers(c, c->lock[r], m, false));
  }
  if (c->lock_cap < nrhs) {
    release(c, c->lock_ptrs);
    if (c->h_lock_ptrs) cudaFreeHost(c->h_lock_ptrs);
    c->lock_ptrs = nullptr;
    c->h_lock_ptrs = nullptr;
    TRY(dalloc(c, &c->lock_ptrs, 3 * (size_t)nrhs * sizeof(void*)));
    if (cudaMallocHost(&c->h_lock_ptrs, 3 * (size_t)nrhs * sizeof(void*)) != cudaSuccess)
      return fail(c, DD_ERR_OOM, "pinned pointer lists");
    c->lock_cap = nrhs;
  }
  return DD_OK;
}

// z_r = M v_r for na right-hand sides given by device pointer lists.
static dd_status sap_run_list(dd_ctx* c, const float4* const* vl, float4* const* zl, const dd_sap_params* p, int na) {
  int prec = sap_prec(p->storage_prec);
  TRY(ensure_sap(c, prec, na));
  if (p->additive) TRY(ensure_faces2(c, prec));
  SapState S = sap_state(c, prec, p, na);
  S.vlist = vl;
  S.zlist = zl;
  return sap_sweeps(c, S, p, nullptr, nullptr, c->sap[prec].faces2);
}

// Gram-Schmidt of step j and the Hessenberg update for one right-hand side (the sequence
// of solve_one, launched directly), then its status into the pinned mirror.
static dd_status lock_gs(dd_ctx* c, SolverBuffers& s, int j, int m) {
  const long long n4 = c->g.V * 6;
  const int ldh = m + 1;
  float4* vn = s.V + (long long)(j + 1) * n4;
  double2* nrm_a = s.nrm2 + 1;
  double2* nrm_b = s.nrm2 + 2;
  int nk = launch_gs_dot(s.V, j + 1, n4, s.w, s.partial, nullptr, 0, c->st);
  launch_gs_reduce(s.partial, j + 1, (double2*)s.hA, nullptr, 0, c->st);
  launch_gs_project(vn, s.w, s.V, j + 1, n4, (const double2*)s.hA, s.partial2, nullptr, 0, c->st);
  launch_gs_reduce(s.partial2, 0, nrm_a, nullptr, 0, c->st);
  gs_decide_kernel<<<1, 1, 0, c->st>>>(s.hA, j + 1, nrm_a, s.hB, s.flag, s.nu2);
  nk += launch_gs_dot(s.V, j + 1, n4, vn, s.partial, s.flag, 1, c->st);
  launch_gs_reduce(s.partial, j + 1, (double2*)s.hB, s.flag, 1, c->st);
  launch_gs_project(vn, vn, s.V, j + 1, n4, (const double2*)s.hB, s.partial2, s.flag, 1, c->st);
  launch_gs_reduce(s.partial2, 0, nrm_b, s.flag, 1, c->st);
  gs_decide2_kernel<<<1, 1, 0, c->st>>>(s.flag, nrm_b, s.nu2);
  launch_scale_inplace(vn, n4, s.nu2, c->st);
  arnoldi_finish_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, ldh, j, s.hA, s.hB, s.nu2, s.lsq, s.g, s.status);
  TRY(launched(c, nk + 10));
  return cuda_check(c, cudaMemcpyAsync(s.h_status, s.status, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st),
                    "status");
}

// End of a cycle of one right-hand side after mm Arnoldi steps: x64 += Z y, FP64 residual,
// then a deflated (or plain) restart, as in solve_one.
static dd_status lock_end_cycle(dd_ctx* c, SolverBuffers& s, LockRhs& R, int mm, const dd_solve_params* p) {
  const long long n4 = c->g.V * 6;
  const int m = p->m, k = p->k, ldh = m + 1;
  CycleEnd ce;
  TRY(end_cycle(c, s, mm, p, R.nf, false, &ce));
  R.rho2 = ce.rho2;
  R.reliable++;
  R.rel = sqrt(R.rho2) / R.nf;
  if (!isfinite(R.rel)) {
    R.rc = fail(c, DD_ERR_NONFINITE, "non-finite residual");
    R.done = true;
    return DD_OK;
  }
  if (R.rel <= p->tol) {
    R.done = true;
    return DD_OK;
  }
  if (R.iters >= p->max_iter) {
    R.rc = fail(c, DD_ERR_NOT_CONVERGED, "iteration limit reached");
    R.done = true;
    return DD_OK;
  }
  R.restarts++;
  if (ce.deflate) {
    restart_lsq_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, ldh, m, k, s.Hn, s.cp, s.g, s.c0, s.lsq, s.status, s.vscale);
    TRY(launched(c));
    R.j0 = k;
    R.deflated++;
  } else {
    launch_r64_to_v32(s.V, s.r64, n4, s.nrm2, c->st);
    plain_restart_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, ldh, m, s.nrm2, s.g, s.c0, s.lsq, s.vscale);
    TRY(launched(c, 2));
    R.j0 = 0;
  }
  R.j = R.j0;
  R.rho_cycle = sqrt(R.rho2);
  return DD_OK;
}

static dd_status solve_lockstep(dd_ctx* c, const double* f, double* x, int nrhs, int where, const dd_solve_params* p,
                                dd_solve_info* info) {
  const Geom& g = c->g;
  const long long n4 = g.V * 6;
  const int m = p->m;
  const double tol = p->tol;
  TRY(ensure_lock(c, nrhs, m));
  std::vector<LockRhs> R(nrhs);
  size_t cb = (size_t)g.V * 24 * 8;
  cudaMemcpyKind in_kind = where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyKind out_kind = where == DD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  cudaEvent_t e0, e1, e2, e3, tstart, tend;
  for (cudaEvent_t* e : {&e0, &e1, &e2, &e3, &tstart, &tend}) cudaEventCreate(e);
  cudaEventRecord(tstart, c->st);
  double tA = 0, tM = 0, tGS = 0;
  dd_status rc = DD_OK;
  // set-up: fields in, FP64 residual, first basis vector
  for (int r = 0; r < nrhs && rc == DD_OK; ++r) {
    SolverBuffers& s = c->lock[r];
    TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, f + (size_t)r * g.V * 24, cb, in_kind, c->st), "copy f"));
    launch_pack_spinor(g, s.canon64, P64, view(g, s.f64, P64), c->st);
    TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, x + (size_t)r * g.V * 24, cb, in_kind, c->st), "copy x"));
    launch_pack_spinor(g, s.canon64, P64, view(g, s.x64, P64), c->st);
    launch_norm2_64(s.f64, g.V * 12, s.partial, c->st);
    launch_reduce_partials(s.partial, 1, s.nrm2, 0, c->st);
    TRY(launched(c, 4));
    double2 h;
    TRY(cuda_check(c, cudaMemcpyAsync(&h, s.nrm2, sizeof(double2), cudaMemcpyDeviceToHost, c->st), "norm f"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->st), "norm f"));
    if (h.x == 0.0) {   // zero source: x = 0
      cudaMemsetAsync(s.x64, 0, field_bytes(g, P64), c->st);
      R[r].done = true;
      continue;
    }
    R[r].nf = sqrt(h.x);
    TRY(true_residual(c, &R[r].rho2, &s));
    R[r].reliable++;
    R[r].rel = sqrt(R[r].rho2) / R[r].nf;
    if (!isfinite(R[r].rel)) {
      R[r].rc = fail(c, DD_ERR_NONFINITE, "non-finite residual");
      R[r].done = true;
    } else if (R[r].rel <= tol) {
      R[r].done = true;
    } else {
      launch_r64_to_v32(s.V, s.r64, n4, s.nrm2, c->st);
      plain_restart_kernel<<<1, 1, 0, c->st>>>(s.H, s.R, m + 1, m, s.nrm2, s.g, s.c0, s.lsq, s.vscale);
      TRY(launched(c, 2));
      R[r].rho_cycle = sqrt(R[r].rho2);
    }
  }
  std::vector<int> act;
  const float4** vl = (const float4**)c->lock_ptrs;
  while (rc == DD_OK) {
    act.clear();
    for (int r = 0; r < nrhs; ++r)
      if (!R[r].done) act.push_back(r);
    if (act.empty()) break;
    const int na = (int)act.size();
    void** hp = c->h_lock_ptrs;
    for (int i = 0; i < na; ++i) {
      SolverBuffers& s = c->lock[act[i]];
      hp[i] = s.V + (long long)R[act[i]].j * n4;
      hp[na + i] = s.Z + (long long)R[act[i]].j * n4;
      hp[2 * na + i] = s.w;
    }
    TRY(cuda_check(c, cudaMemcpyAsync(c->lock_ptrs, hp, 3 * (size_t)na * sizeof(void*), cudaMemcpyHostToDevice, c->st),
                   "pointer lists"));
    cudaEventRecord(e0, c->st);
    TRY(sap_run_list(c, vl, (float4* const*)(c->lock_ptrs + na), &p->sap, na));
    cudaEventRecord(e1, c->st);
    launch_apply_A_multi_list(g, gauge_view(c, P32), clover_view(c, P32), (const float4* const*)(c->lock_ptrs + na),
                              (float4* const*)(c->lock_ptrs + 2 * na), na, c->st);
    TRY(launched(c));
    cudaEventRecord(e2, c->st);
    for (int r : act) TRY(lock_gs(c, c->lock[r], R[r].j, m));
    cudaEventRecord(e3, c->st);
    TRY(cuda_check(c, cudaStreamSynchronize(c->st), "lockstep step"));
    float ms;
    cudaEventElapsedTime(&ms, e0, e1); tM += ms * 1e-3;
    cudaEventElapsedTime(&ms, e1, e2); tA += ms * 1e-3;
    cudaEventElapsedTime(&ms, e2, e3); tGS += ms * 1e-3;
    for (int r : act) {
      LockRhs& Q = R[r];
      SolverBuffers& s = c->lock[r];
      Q.iters++;
      const double est = s.h_status[0];
      if (!isfinite(est) || !isfinite(s.h_status[2])) {
        Q.rc = fail(c, DD_ERR_NONFINITE, "non-finite Arnoldi step");
        Q.done = true;
        continue;
      }
      if (c->trace)
        fprintf(stderr, "[dd] rhs %d it %d j %d est/rho %.3e\n", r, Q.iters, Q.j, est / Q.rho_cycle);
      // the cycle ends when the target is met, FP32 vectors cannot resolve further, the
      // basis is full or the iteration budget is spent
      if (est <= 0.5 * tol * Q.nf || est <= 2e-6 * Q.rho_cycle || Q.iters >= p->max_iter || Q.j + 1 == m) {
        TRY(lock_end_cycle(c, s, Q, Q.j + 1, p));
      } else {
        Q.j++;
      }
    }
  }
  cudaEventRecord(tend, c->st);
  cudaEventSynchronize(tend);
  float ms_total = 0;
  cudaEventElapsedTime(&ms_total, tstart, tend);
  for (cudaEvent_t e : {e0, e1, e2, e3, tstart, tend}) cudaEventDestroy(e);
  dd_status worst = DD_OK;
  for (int r = 0; r < nrhs; ++r) {
    SolverBuffers& s = c->lock[r];
    launch_unpack_spinor(g, view(g, s.x64, P64), s.canon64, P64, c->st);
    TRY(launched(c));
    TRY(cuda_check(c, cudaMemcpyAsync(x + (size_t)r * g.V * 24, s.canon64, cb, out_kind, c->st), "copy x out"));
    if (R[r].rc != DD_OK && worst == DD_OK) worst = R[r].rc;
  }
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "solve"));
  if (info) {
    for (const LockRhs& Q : R) {
      info->iterations += Q.iters;
      info->restarts += Q.restarts;
      info->reliable_updates += Q.reliable;
      info->deflated_restarts += Q.deflated;
      info->true_rel_residual = fmax(info->true_rel_residual, Q.rel);
      const double V = (double)g.V;
      info->flops_nominal += Q.iters * (1848.0 * V + p->sap.i_schwarz * (p->sap.i_domain + 1) * 1848.0 * V) +
                             Q.reliable * 1848.0 * V;
    }
    info->t_total = ms_total * 1e-3;
    info->t_A = tA;
    info->t_M = tM;
    info->t_GS = tGS;
    info->t_other = ms_total * 1e-3 - tA - tM - tGS;
    info->status = worst;
  }
  if (worst == DD_OK) TRY(sap_error_flag(c));
  return worst;
}

// ------------------------------------------------------------------ lattices of different volume
// Lockstep solves over several lattices (the many independent solves of an analysis,
// Sec. IV-C): every (lattice, right-hand side) keeps its own basis, restarts and stopping
// point as in solve_lockstep; every Arnoldi step applies M to all unconverged ones in one
// launch per half-sweep over the lattices' (domain, right-hand side) work, and A in one
// launch per lattice.  All work runs on the first context's stream.
struct LatticeStreams {
  std::vector<dd_ctx*> ctxs;
  std::vector<cudaStream_t> saved;
  ~LatticeStreams() {
    if (!ctxs.empty()) cudaStreamSynchronize(ctxs[0]->st);
    for (size_t l = 0; l < ctxs.size(); ++l) ctxs[l]->st = saved[l];
  }
};

static dd_status solve_lattices(dd_ctx** ctxs, int nlat, const double* const* f, double* const* x, int nrhs, int where,
                                const dd_solve_params* p, dd_solve_info* info) {
  dd_ctx* c0 = ctxs[0];
  const cudaStream_t st = c0->st;
  LatticeStreams keep;
  for (int l = 0; l < nlat; ++l) {
    keep.ctxs.push_back(ctxs[l]);
    keep.saved.push_back(ctxs[l]->st);
    ctxs[l]->st = st;
  }
  const int m = p->m;
  const double tol = p->tol;
  cudaMemcpyKind in_kind = where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyKind out_kind = where == DD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  std::vector<std::vector<LockRhs>> R(nlat, std::vector<LockRhs>(nrhs));
  for (int l = 0; l < nlat; ++l) {
    TRY(ensure_lock(ctxs[l], nrhs, m));
    TRY(ensure_sap(ctxs[l], P16, nrhs));
  }
  cudaEvent_t e0, e1, e2, e3, tstart, tend;
  for (cudaEvent_t* e : {&e0, &e1, &e2, &e3, &tstart, &tend}) cudaEventCreate(e);
  struct EvFree {
    cudaEvent_t e[6];
    ~EvFree() { for (cudaEvent_t q : e) cudaEventDestroy(q); }
  } evf{{e0, e1, e2, e3, tstart, tend}};
  cudaEventRecord(tstart, st);
  double tA = 0, tM = 0, tGS = 0;
  // set-up: fields in, FP64 residual, first basis vector
  for (int l = 0; l < nlat; ++l) {
    dd_ctx* c = ctxs[l];
    const Geom& g = c->g;
    const size_t cb = (size_t)g.V * 24 * 8;
    for (int r = 0; r < nrhs; ++r) {
      SolverBuffers& s = c->lock[r];
      LockRhs& Q = R[l][r];
      TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, f[l] + (size_t)r * g.V * 24, cb, in_kind, st), "copy f"));
      launch_pack_spinor(g, s.canon64, P64, view(g, s.f64, P64), st);
      TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, x[l] + (size_t)r * g.V * 24, cb, in_kind, st), "copy x"));
      launch_pack_spinor(g, s.canon64, P64, view(g, s.x64, P64), st);
      launch_norm2_64(s.f64, g.V * 12, s.partial, st);
      launch_reduce_partials(s.partial, 1, s.nrm2, 0, st);
      TRY(launched(c, 4));
      double2 h;
      TRY(cuda_check(c, cudaMemcpyAsync(&h, s.nrm2, sizeof(double2), cudaMemcpyDeviceToHost, st), "norm f"));
      TRY(cuda_check(c, cudaStreamSynchronize(st), "norm f"));
      if (h.x == 0.0) {
        cudaMemsetAsync(s.x64, 0, field_bytes(g, P64), st);
        Q.done = true;
        continue;
      }
      Q.nf = sqrt(h.x);
      TRY(true_residual(c, &Q.rho2, &s));
      Q.reliable++;
      Q.rel = sqrt(Q.rho2) / Q.nf;
      if (!isfinite(Q.rel)) {
        Q.rc = fail(c0, DD_ERR_NONFINITE, "non-finite residual");
        Q.done = true;
      } else if (Q.rel <= tol) {
        Q.done = true;
      } else {
        launch_r64_to_v32(s.V, s.r64, g.V * 6, s.nrm2, st);
        plain_restart_kernel<<<1, 1, 0, st>>>(s.H, s.R, m + 1, m, s.nrm2, s.g, s.c0, s.lsq, s.vscale);
        TRY(launched(c, 2));
        Q.rho_cycle = sqrt(Q.rho2);
      }
    }
  }
  std::vector<std::vector<int>> act(nlat);
  while (true) {
    int total = 0, nl = 0;
    Geom gs[4];
    SapState Ss[4];
    int lat_of[4];
    for (int l = 0; l < nlat; ++l) {
      act[l].clear();
      for (int r = 0; r < nrhs; ++r)
        if (!R[l][r].done) act[l].push_back(r);
      const int na = (int)act[l].size();
      total += na;
      if (!na) continue;
      dd_ctx* c = ctxs[l];
      const long long n4 = c->g.V * 6;
      void** hp = c->h_lock_ptrs;
      for (int i = 0; i < na; ++i) {
        SolverBuffers& s = c->lock[act[l][i]];
        hp[i] = s.V + (long long)R[l][act[l][i]].j * n4;
        hp[na + i] = s.Z + (long long)R[l][act[l][i]].j * n4;
        hp[2 * na + i] = s.w;
      }
      TRY(cuda_check(c, cudaMemcpyAsync(c->lock_ptrs, hp, 3 * (size_t)na * sizeof(void*), cudaMemcpyHostToDevice, st),
                     "pointer lists"));
      gs[nl] = c->g;
      Ss[nl] = sap_state(c, P16, &p->sap, na);
      Ss[nl].vlist = (const float4* const*)c->lock_ptrs;
      Ss[nl].zlist = (float4* const*)(c->lock_ptrs + na);
      lat_of[nl++] = l;
    }
    if (!total) break;
    const float4* vnull[4] = {nullptr, nullptr, nullptr, nullptr};
    float4* znull[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEventRecord(e0, st);
    for (int sw = 0; sw < p->sap.i_schwarz; ++sw)
      for (int colour = 0; colour < 2; ++colour) {
        int first = sw == 0, use_faces = !(sw == 0 && colour == 0), last = sw == p->sap.i_schwarz - 1;
        if (sap_half_sweep_lattices(gs, Ss, nl, colour, first, use_faces, last, vnull, znull, p->sap.i_domain, st))
          return fail(c0, DD_ERR_CUDA, std::string("Schwarz launch failed: ") + cudaGetErrorString(cudaGetLastError()));
        TRY(launched(c0));
      }
    cudaEventRecord(e1, st);
    for (int q = 0; q < nl; ++q) {
      dd_ctx* c = ctxs[lat_of[q]];
      const int na = (int)act[lat_of[q]].size();
      launch_apply_A_multi_list(c->g, gauge_view(c, P32), clover_view(c, P32), (const float4* const*)(c->lock_ptrs + na),
                                (float4* const*)(c->lock_ptrs + 2 * na), na, st);
      TRY(launched(c));
    }
    cudaEventRecord(e2, st);
    for (int l = 0; l < nlat; ++l)
      for (int r : act[l]) TRY(lock_gs(ctxs[l], ctxs[l]->lock[r], R[l][r].j, m));
    cudaEventRecord(e3, st);
    TRY(cuda_check(c0, cudaStreamSynchronize(st), "lockstep step"));
    float ms;
    cudaEventElapsedTime(&ms, e0, e1); tM += ms * 1e-3;
    cudaEventElapsedTime(&ms, e1, e2); tA += ms * 1e-3;
    cudaEventElapsedTime(&ms, e2, e3); tGS += ms * 1e-3;
    for (int l = 0; l < nlat; ++l)
      for (int r : act[l]) {
        LockRhs& Q = R[l][r];
        SolverBuffers& s = ctxs[l]->lock[r];
        Q.iters++;
        const double est = s.h_status[0];
        if (!isfinite(est) || !isfinite(s.h_status[2])) {
          Q.rc = fail(c0, DD_ERR_NONFINITE, "non-finite Arnoldi step");
          Q.done = true;
          continue;
        }
        if (est <= 0.5 * tol * Q.nf || est <= 2e-6 * Q.rho_cycle || Q.iters >= p->max_iter || Q.j + 1 == m) {
          TRY(lock_end_cycle(ctxs[l], s, Q, Q.j + 1, p));
        } else {
          Q.j++;
        }
      }
  }
  cudaEventRecord(tend, st);
  cudaEventSynchronize(tend);
  float ms_total = 0;
  cudaEventElapsedTime(&ms_total, tstart, tend);
  dd_status worst = DD_OK;
  for (int l = 0; l < nlat; ++l) {
    dd_ctx* c = ctxs[l];
    const Geom& g = c->g;
    const size_t cb = (size_t)g.V * 24 * 8;
    for (int r = 0; r < nrhs; ++r) {
      SolverBuffers& s = c->lock[r];
      launch_unpack_spinor(g, view(g, s.x64, P64), s.canon64, P64, st);
      TRY(launched(c));
      TRY(cuda_check(c, cudaMemcpyAsync(x[l] + (size_t)r * g.V * 24, s.canon64, cb, out_kind, st), "copy x out"));
      if (R[l][r].rc != DD_OK && worst == DD_OK) worst = R[l][r].rc;
    }
  }
  TRY(cuda_check(c0, cudaStreamSynchronize(st), "solve"));
  if (info) {
    for (int l = 0; l < nlat; ++l)
      for (const LockRhs& Q : R[l]) {
        info->iterations += Q.iters;
        info->restarts += Q.restarts;
        info->reliable_updates += Q.reliable;
        info->deflated_restarts += Q.deflated;
        info->true_rel_residual = fmax(info->true_rel_residual, Q.rel);
        const double V = (double)ctxs[l]->g.V;
        info->flops_nominal += Q.iters * (1848.0 * V + p->sap.i_schwarz * (p->sap.i_domain + 1) * 1848.0 * V) +
                               Q.reliable * 1848.0 * V;
      }
    info->t_total = ms_total * 1e-3;
    info->t_A = tA;
    info->t_M = tM;
    info->t_GS = tGS;
    info->t_other = ms_total * 1e-3 - tA - tM - tGS;
    info->status = worst;
  }
  if (worst == DD_OK)
    for (int l = 0; l < nlat; ++l) TRY(sap_error_flag(ctxs[l]));
  return worst;
}

extern "C" dd_status dd_solve_lattices(dd_ctx** ctxs, int nlat, const double* const* f, double* const* x, int nrhs,
                                       int where, const dd_solve_params* p, dd_solve_info* info) {
  if (!ctxs || !f || !x || !p || nlat < 1 || nlat > 4 || nrhs < 1) return DD_ERR_INVALID;
  dd_ctx* c0 = ctxs[0];
  if (!c0) return DD_ERR_INVALID;
  if (p->m < 1 || p->m > DD_MAXM - 1 || p->k < 0 || p->k >= p->m || !(p->tol > 0) || p->max_iter < 1)
    return fail(c0, DD_ERR_INVALID, "bad solver parameters");
  TRY(check_sap_params(c0, &p->sap));
  if (p->sap.storage_prec != DD_PREC_FP16 || p->sap.threads_per_site == 1 || p->sap.i_domain < 1 || p->sap.additive)
    return fail(c0, DD_ERR_INVALID,
                "lattice batches need FP16 storage, two threads per site, i_domain >= 1 and the multiplicative form");
  for (int l = 0; l < nlat; ++l) {
    if (!ctxs[l] || !f[l] || !x[l]) return DD_ERR_INVALID;
    if (!ctxs[l]->have_clover) return fail(c0, DD_ERR_NO_CLOVER, "clover not built on lattice " + std::to_string(l));
    if (ctxs[l]->g.Vd != c0->g.Vd || sap_mat_fits_smem(ctxs[l]->g, P16) != sap_mat_fits_smem(c0->g, P16))
      return fail(c0, DD_ERR_DIMS, "lattices of one launch need the same domain volume");
    for (int q = 0; q < l; ++q)
      if (ctxs[q] == ctxs[l]) return fail(c0, DD_ERR_INVALID, "a context appears twice");
  }
  if (info) memset(info, 0, sizeof(*info));
  return solve_lattices(ctxs, nlat, f, x, nrhs, where, p, info);
}

extern "C" dd_status dd_solve(dd_ctx* c, const double* f, double* x, int nrhs, int where, const dd_solve_params* p,
                              dd_solve_info* info) {
  if (!c || !f || !x || !p || nrhs < 1) return DD_ERR_INVALID;
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (p->m < 1 || p->m > DD_MAXM - 1 || p->k < 0 || p->k >= p->m || !(p->tol > 0) || p->max_iter < 1)
    return fail(c, DD_ERR_INVALID, "bad solver parameters");
  TRY(check_sap_params(c, &p->sap));
  if (p->sap.i_domain < 1) return fail(c, DD_ERR_INVALID, "i_domain must be >= 1");
  if (p->basis_fp16 < 0 || p->basis_fp16 > 1) return fail(c, DD_ERR_INVALID, "basis_fp16 must be 0 or 1");
  const char* seq0 = getenv("DD_SEQUENTIAL_RHS");
  if (p->basis_fp16 && nrhs > 1 && p->sap.threads_per_site != 1 && !(seq0 && seq0[0] == '1'))
    return fail(c, DD_ERR_INVALID, "the FP16 basis is not available for right-hand sides in lockstep");
  TRY(ensure_solver(c, p->m, p->basis_fp16 != 0));
  if (info) memset(info, 0, sizeof(*info));
  SolverBuffers& s = c->sv;
  // Run on the solver's own stream (capturable into CUDA graphs even when the caller
  // uses the legacy default stream), ordered after the caller's stream; the call is
  // synchronous, so the caller's stream needs no event back.
  struct StreamSwap {
    dd_ctx* c;
    cudaStream_t user;
    ~StreamSwap() {
      cudaStreamSynchronize(c->st);
      c->st = user;
    }
  };
  cudaEventRecord(s.ev_in, c->st);
  cudaStreamWaitEvent(s.stream, s.ev_in, 0);
  StreamSwap swap{c, c->st};
  c->st = s.stream;
  // several right-hand sides in lockstep, unless the domain solve runs one thread per site
  // (no batched kernel) or DD_SEQUENTIAL_RHS=1 asks for one solve after another
  const char* seq = getenv("DD_SEQUENTIAL_RHS");
  if (nrhs > 1 && p->sap.threads_per_site != 1 && !(seq && seq[0] == '1'))
    return solve_lockstep(c, f, x, nrhs, where, p, info);
  const Geom& g = c->g;
  size_t cb = (size_t)g.V * 24 * 8;
  cudaMemcpyKind in_kind = where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyKind out_kind = where == DD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  dd_status worst = DD_OK;
  for (int r = 0; r < nrhs; ++r) {
    const double* fr = f + (size_t)r * g.V * 24;
    double* xr = x + (size_t)r * g.V * 24;
    TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, fr, cb, in_kind, c->st), "copy f"));
    launch_pack_spinor(g, s.canon64, P64, view(g, s.f64, P64), c->st);
    TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, xr, cb, in_kind, c->st), "copy x"));
    launch_pack_spinor(g, s.canon64, P64, view(g, s.x64, P64), c->st);
    launch_norm2_64(s.f64, g.V * 12, s.partial, c->st);
    launch_reduce_partials(s.partial, 1, s.nrm2, 0, c->st);
    TRY(launched(c, 4));
    double2 h;
    TRY(cuda_check(c, cudaMemcpyAsync(&h, s.nrm2, sizeof(double2), cudaMemcpyDeviceToHost, c->st), "norm f"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->st), "norm f"));
    dd_status st;
    if (h.x == 0.0) {
      cudaMemsetAsync(s.x64, 0, field_bytes(g, P64), c->st);
      st = DD_OK;
    } else {
      st = solve_one(c, p, h.x, info);
    }
    launch_unpack_spinor(g, view(g, s.x64, P64), s.canon64, P64, c->st);
    TRY(launched(c));
    TRY(cuda_check(c, cudaMemcpyAsync(xr, s.canon64, cb, out_kind, c->st), "copy x out"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->st), "solve"));
    if (st != DD_OK && worst == DD_OK) worst = st;
    if (st != DD_OK && st != DD_ERR_NOT_CONVERGED) break;
  }
  if (info) info->status = worst;
  return worst;
}

// ------------------------------------------------------------------ GCR outer solver
// Flexible GCR(m), the outer iteration of Luescher's SAP-GCR (the alternative to FGMRES-DR
// that the paper contrasts with its own choice, Sec. V): with r the current residual,
// z_k = M r, w_k = A z_k made orthonormal to w_0..w_{k-1} (the same coefficients applied
// to z_k keep A z_k = w_k), alpha_k = <w_k, r>, r -= alpha_k w_k; at the end of a cycle
// x += sum alpha_k z_k in FP64 and the residual is recomputed with the FP64 operator.
// W and Z use the solver's V and Z bases; r is the FP32 vector w, scaled by 1 / |r|.

// alpha <- rho alpha for the cycle's coefficients (r was normalised by rho)
__global__ void scale_by_norm_kernel(zd* a, int n, const double2* nrm2) {
  const double rho = sqrt(nrm2->x);
  for (int i = 0; i < n; ++i) a[i] = rho * a[i];
}
// status[0] = |r| after the step, status[2] = |w_k| before normalisation
__global__ void gcr_status_kernel(const double2* nrm_r, const double* nu2, double* status) {
  status[0] = sqrt(fmax(nrm_r->x, 0.0));
  status[2] = sqrt(*nu2);
  status[3] = 0.0;
}

static dd_status solve_gcr_one(dd_ctx* c, const dd_solve_params* p, double nf2, dd_solve_info* info) {
  SolverBuffers& s = c->sv;
  const Geom& g = c->g;
  const long long n4 = g.V * 6;
  const int m = p->m;
  const double tol = p->tol, nf = sqrt(nf2);
  cudaEvent_t e0, e1, e2, e3, tstart, tend;
  for (cudaEvent_t* e : {&e0, &e1, &e2, &e3, &tstart, &tend}) cudaEventCreate(e);
  cudaEventRecord(tstart, c->st);
  double tA = 0, tM = 0, tGS = 0;
  int iters = 0, restarts = 0, reliable = 0;
  dd_status rc = DD_OK;
  double rho2 = 0;
  auto Wv = [&](int i) { return s.V + (long long)i * n4; };
  auto Zv = [&](int i) { return s.Z + (long long)i * n4; };
  float4* r = s.w;
  float4* wk = s.V + (long long)m * n4;   // the (m+1)-th basis slot: the new direction
  zd* alpha = s.y;                          // m + 2 entries
  TRY(true_residual(c, &rho2));
  reliable++;
  double rel = sqrt(rho2) / nf;
  if (!isfinite(rel)) rc = fail(c, DD_ERR_NONFINITE, "non-finite residual");
  while (rc == DD_OK && rel > tol) {
    if (iters >= p->max_iter) { rc = fail(c, DD_ERR_NOT_CONVERGED, "iteration limit reached"); break; }
    launch_r64_to_v32(r, s.r64, n4, s.nrm2, c->st);   // r = r64 / |r64|
    TRY(launched(c));
    int mm = 0;
    for (int k = 0; k < m; ++k) {
      cudaEventRecord(e0, c->st);
      TRY(sap_run(c, r, Zv(k), &p->sap));
      cudaEventRecord(e1, c->st);
      TRY(apply_internal(c, Zv(k), wk, P32));
      cudaEventRecord(e2, c->st);
      // w_k <- w_k - W beta (classical, with the DGKS second pass); z_k <- z_k - Z beta
      double2* nrm_a = s.nrm2 + 1;
      double2* nrm_b = s.nrm2 + 2;
      int nk = launch_gs_dot(Wv(0), k, n4, wk, s.partial, nullptr, 0, c->st);
      launch_gs_reduce(s.partial, k, (double2*)s.hA, nullptr, 0, c->st);
      launch_gs_project(Wv(k), wk, Wv(0), k, n4, (const double2*)s.hA, s.partial2, nullptr, 0, c->st);
      launch_gs_reduce(s.partial2, 0, nrm_a, nullptr, 0, c->st);
      launch_gs_project(Zv(k), Zv(k), Zv(0), k, n4, (const double2*)s.hA, s.partial2, nullptr, 0, c->st);
      gs_decide_kernel<<<1, 1, 0, c->st>>>(s.hA, k, nrm_a, s.hB, s.flag, s.nu2);
      nk += launch_gs_dot(Wv(0), k, n4, Wv(k), s.partial, s.flag, 1, c->st);
      launch_gs_reduce(s.partial, k, (double2*)s.hB, s.flag, 1, c->st);
      launch_gs_project(Wv(k), Wv(k), Wv(0), k, n4, (const double2*)s.hB, s.partial2, s.flag, 1, c->st);
      launch_gs_reduce(s.partial2, 0, nrm_b, s.flag, 1, c->st);
      launch_gs_project(Zv(k), Zv(k), Zv(0), k, n4, (const double2*)s.hB, s.partial2, s.flag, 1, c->st);
      gs_decide2_kernel<<<1, 1, 0, c->st>>>(s.flag, nrm_b, s.nu2);
      launch_scale_inplace(Wv(k), n4, s.nu2, c->st);
      launch_scale_inplace(Zv(k), n4, s.nu2, c->st);
      // alpha_k = <w_k, r>; r <- r - alpha_k w_k with its exact norm
      nk += launch_gs_dot(Wv(k), 1, n4, r, s.partial, nullptr, 0, c->st);
      launch_gs_reduce(s.partial, 1, (double2*)(alpha + k), nullptr, 0, c->st);
      launch_gs_project(r, r, Wv(k), 1, n4, (const double2*)(alpha + k), s.partial2, nullptr, 0, c->st);
      launch_gs_reduce(s.partial2, 0, s.nrm2 + 3, nullptr, 0, c->st);
      gcr_status_kernel<<<1, 1, 0, c->st>>>(s.nrm2 + 3, s.nu2, s.status);
      TRY(launched(c, nk + 17));
      cudaEventRecord(e3, c->st);
      TRY(read_status(c));
      float ms;
      cudaEventElapsedTime(&ms, e0, e1); tM += ms * 1e-3;
      cudaEventElapsedTime(&ms, e1, e2); tA += ms * 1e-3;
      cudaEventElapsedTime(&ms, e2, e3); tGS += ms * 1e-3;
      iters++;
      mm = k + 1;
      const double est = s.h_status[0] * sqrt(rho2);
      if (c->trace) fprintf(stderr, "[dd] gcr it %d k %d est/rho %.3e |w| %.3e\n", iters, k, s.h_status[0], s.h_status[2]);
      if (!isfinite(est) || !isfinite(s.h_status[2])) { rc = fail(c, DD_ERR_NONFINITE, "non-finite GCR step"); break; }
      if (est <= 0.5 * tol * nf || s.h_status[0] <= 2e-6 || iters >= p->max_iter) break;
    }
    if (rc != DD_OK) break;
    // x += rho sum alpha_k z_k (FP64), then the FP64 residual
    scale_by_norm_kernel<<<1, 1, 0, c->st>>>(alpha, mm, s.nrm2);
    launch_x_update(s.x64, Zv(0), mm, n4, (const double2*)alpha, c->st);
    TRY(launched(c, 2));
    TRY(true_residual(c, &rho2));
    reliable++;
    rel = sqrt(rho2) / nf;
    if (!isfinite(rel)) { rc = fail(c, DD_ERR_NONFINITE, "non-finite residual"); break; }
    if (rel <= tol) break;
    restarts++;
    if (c->trace) fprintf(stderr, "[dd] gcr restart: true residual %.3e\n", rel);
  }
  cudaEventRecord(tend, c->st);
  cudaEventSynchronize(tend);
  float ms = 0;
  cudaEventElapsedTime(&ms, tstart, tend);
  if (info) {
    info->iterations += iters;
    info->restarts += restarts;
    info->reliable_updates += reliable;
    info->true_rel_residual = fmax(info->true_rel_residual, rel);
    info->t_total += ms * 1e-3;
    info->t_A += tA;
    info->t_M += tM;
    info->t_GS += tGS;
    info->t_other += ms * 1e-3 - tA - tM - tGS;
    const double V = (double)g.V;
    info->flops_nominal += iters * (1848.0 * V + p->sap.i_schwarz * (p->sap.i_domain + 1) * 1848.0 * V) +
                           reliable * 1848.0 * V;
  }
  for (cudaEvent_t e : {e0, e1, e2, e3, tstart, tend}) cudaEventDestroy(e);
  if (rc == DD_OK) TRY(sap_error_flag(c));
  return rc;
}

extern "C" dd_status dd_solve_gcr(dd_ctx* c, const double* f, double* x, int where, const dd_solve_params* p,
                                  dd_solve_info* info) {
  if (!c || !f || !x || !p) return DD_ERR_INVALID;
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (p->m < 1 || p->m > DD_MAXM - 1 || !(p->tol > 0) || p->max_iter < 1)
    return fail(c, DD_ERR_INVALID, "bad solver parameters");
  TRY(check_sap_params(c, &p->sap));
  if (p->sap.i_domain < 1) return fail(c, DD_ERR_INVALID, "i_domain must be >= 1");
  TRY(ensure_solver(c, p->m));
  if (info) memset(info, 0, sizeof(*info));
  const Geom& g = c->g;
  SolverBuffers& s = c->sv;
  const size_t cb = (size_t)g.V * 24 * 8;
  TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, f, cb, where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    c->st),
                 "copy f"));
  launch_pack_spinor(g, s.canon64, P64, view(g, s.f64, P64), c->st);
  TRY(cuda_check(c, cudaMemcpyAsync(s.canon64, x, cb, where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    c->st),
                 "copy x"));
  launch_pack_spinor(g, s.canon64, P64, view(g, s.x64, P64), c->st);
  launch_norm2_64(s.f64, g.V * 12, s.partial, c->st);
  launch_reduce_partials(s.partial, 1, s.nrm2, 0, c->st);
  TRY(launched(c, 4));
  double2 h;
  TRY(cuda_check(c, cudaMemcpyAsync(&h, s.nrm2, sizeof(double2), cudaMemcpyDeviceToHost, c->st), "norm f"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "norm f"));
  dd_status st = DD_OK;
  if (h.x == 0.0) cudaMemsetAsync(s.x64, 0, field_bytes(g, P64), c->st);
  else st = solve_gcr_one(c, p, h.x, info);
  launch_unpack_spinor(g, view(g, s.x64, P64), s.canon64, P64, c->st);
  TRY(launched(c));
  TRY(cuda_check(c, cudaMemcpyAsync(x, s.canon64, cb, where == DD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    c->st),
                 "copy x out"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "gcr"));
  if (info) info->status = st;
  return st;
}

// ------------------------------------------------------------------ BiCGstab comparison solver
// The standard, non-domain-decomposed solvers the paper compares against (Sec. IV-C,
// Table III): BiCGstab in FP64 on the FP64 operator, or an FP64 Richardson iteration
// (defect correction) whose corrections come from BiCGstab in FP32 on the FP32 operator.
namespace {
struct BicgRun {
  double tA = 0;
  int a_apps = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

// A in -> out (or f - A in with f) in precision prec, timed
dd_status bicg_apply(dd_ctx* c, BicgRun& R, const void* in, void* out, int prec, const void* f = nullptr) {
  cudaEventRecord(R.e0, c->st);
  TRY(apply_internal(c, in, out, prec, f));
  cudaEventRecord(R.e1, c->st);
  R.a_apps++;
  return DD_OK;
}

// BiCGstab on A x = b (b given through r = b - A x on entry, x updated in place) until
// |r| <= stop or iters reaches limit.  U: float4 (FP32) or double2 (FP64).  bnorm: |b|.
// Returns the iterations taken; *rel: the recursive |r| / bnorm at exit.
template <typename U>
dd_status bicgstab(dd_ctx* c, BicgRun& R, int prec, U* x, U* r, U* rh, U* pv, U* v, U* s, U* t, zd* sc, double2* part,
                   double* h_sc, double stop, int limit, int* iters, double* rnorm) {
  using K = BicgKernels<U>;
  const Geom& g = c->g;
  K::copy(g, rh, r, c->st);
  K::copy(g, pv, nullptr, c->st);
  K::copy(g, v, nullptr, c->st);
  launch_bicg_reset(sc, c->st);
  TRY(launched(c, 4));
  int it = 0;
  double rn = *rnorm;
  float ms = 0;
  while (it < limit && rn > stop) {
    K::dot(g, rh, r, nullptr, nullptr, part, sc, 4, c->st);
    launch_bicg_scalars(sc, 0, c->st);
    K::p_update(g, pv, r, v, sc, c->st);
    TRY(launched(c, 4));
    TRY(bicg_apply(c, R, pv, v, prec));
    cudaEventSynchronize(R.e1);
    cudaEventElapsedTime(&ms, R.e0, R.e1);
    R.tA += ms * 1e-3;
    K::dot(g, rh, v, nullptr, nullptr, part, sc, 5, c->st);
    launch_bicg_scalars(sc, 1, c->st);
    K::s_update(g, s, r, v, sc, c->st);
    TRY(launched(c, 4));
    TRY(bicg_apply(c, R, s, t, prec));
    K::dot(g, t, s, t, t, part, sc, 6, c->st);
    launch_bicg_scalars(sc, 2, c->st);
    K::xr_update(g, x, r, pv, s, t, sc, part, c->st);
    TRY(launched(c, 5));
    TRY(cuda_check(c, cudaMemcpyAsync(h_sc, sc + 8, 2 * sizeof(zd), cudaMemcpyDeviceToHost, c->st), "bicgstab"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->st), "bicgstab"));
    cudaEventElapsedTime(&ms, R.e0, R.e1);
    R.tA += ms * 1e-3;
    ++it;
    rn = sqrt(h_sc[0]);
    if (c->trace) fprintf(stderr, "[dd] bicgstab it %d |r| %.3e\n", it, rn);
    if (!isfinite(rn)) return fail(c, DD_ERR_NONFINITE, "non-finite BiCGstab residual");
    if (h_sc[2] != 0.0) {   // breakdown: restart the recurrence with rhat = r
      K::copy(g, rh, r, c->st);
      K::copy(g, pv, nullptr, c->st);
      K::copy(g, v, nullptr, c->st);
      launch_bicg_reset(sc, c->st);
      TRY(launched(c, 4));
    }
  }
  *iters = it;
  *rnorm = rn;
  return DD_OK;
}

__global__ void sqrt_to_coeff_kernel(double2* y, const double2* nrm2) { y[0] = make_double2(sqrt(nrm2->x), 0.0); }
}  // namespace

extern "C" dd_status dd_solve_bicgstab(dd_ctx* c, const double* f, double* x, int where, const dd_bicgstab_params* p,
                                       dd_solve_info* info) {
  if (!c || !f || !x || !p) return DD_ERR_INVALID;
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (!(p->tol > 0) || p->max_iter < 1 || (p->precision != DD_PREC_FP64 && p->precision != DD_PREC_FP32) ||
      (p->precision == DD_PREC_FP32 && !(p->inner_tol > 0 && p->inner_tol < 1)))
    return fail(c, DD_ERR_INVALID, "bad BiCGstab parameters");
  if (info) memset(info, 0, sizeof(*info));
  const Geom& g = c->g;
  const size_t b64 = field_bytes(g, P64), b32 = field_bytes(g, P32);
  const bool mixed = p->precision == DD_PREC_FP32;
  const size_t bw = mixed ? b32 : b64;
  std::vector<void*> bufs;
  auto alloc = [&](void** q, size_t n) -> dd_status {
    dd_status st = dalloc(c, q, n);
    if (st == DD_OK) bufs.push_back(*q);
    return st;
  };
  struct Cleanup {
    dd_ctx* c;
    std::vector<void*>* b;
    BicgRun* R;
    ~Cleanup() {
      cudaStreamSynchronize(c->st);
      for (void* q : *b) release(c, q);
      if (R->e0) cudaEventDestroy(R->e0);
      if (R->e1) cudaEventDestroy(R->e1);
    }
  };
  BicgRun R;
  Cleanup cleanup{c, &bufs, &R};
  void *x64, *f64, *r64, *canon, *xw, *r, *rh, *pv, *v, *s, *t, *part, *sc, *coef;
  TRY(alloc(&x64, b64));
  TRY(alloc(&f64, b64));
  TRY(alloc(&r64, b64));
  TRY(alloc(&canon, b64));
  for (void** q : {&xw, &r, &rh, &pv, &v, &s, &t}) TRY(alloc(q, bw));
  TRY(alloc(&part, 2 * (size_t)blas_partials_blocks() * sizeof(double2)));
  TRY(alloc(&sc, 16 * sizeof(zd)));
  TRY(alloc(&coef, 2 * sizeof(double2)));
  double* h_sc = nullptr;
  if (cudaMallocHost(&h_sc, 4 * sizeof(double)) != cudaSuccess) return fail(c, DD_ERR_OOM, "pinned scalars");
  struct HostFree { double* p; ~HostFree() { cudaFreeHost(p); } } hf{h_sc};
  cudaEventCreate(&R.e0);
  cudaEventCreate(&R.e1);
  cudaEvent_t tstart, tend;
  cudaEventCreate(&tstart);
  cudaEventCreate(&tend);
  struct EvFree { cudaEvent_t a, b; ~EvFree() { cudaEventDestroy(a); cudaEventDestroy(b); } } ef{tstart, tend};
  const size_t cb = (size_t)g.V * 24 * 8;
  cudaMemcpyKind in_kind = where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaEventRecord(tstart, c->st);
  TRY(cuda_check(c, cudaMemcpyAsync(canon, f, cb, in_kind, c->st), "copy f"));
  launch_pack_spinor(g, canon, P64, view(g, f64, P64), c->st);
  TRY(cuda_check(c, cudaMemcpyAsync(canon, x, cb, in_kind, c->st), "copy x"));
  launch_pack_spinor(g, canon, P64, view(g, x64, P64), c->st);
  TRY(launched(c, 2));
  // |f| and the FP64 residual
  double2* part2 = (double2*)part;
  auto norm64 = [&](const void* field, double* out) -> dd_status {
    launch_norm2_64((const double2*)field, g.V * 12, part2, c->st);
    launch_reduce_partials(part2, 1, (double2*)coef + 1, 0, c->st);
    TRY(launched(c, 2));
    double2 h;
    TRY(cuda_check(c, cudaMemcpyAsync(&h, (double2*)coef + 1, sizeof(h), cudaMemcpyDeviceToHost, c->st), "norm"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->st), "norm"));
    *out = h.x;
    return DD_OK;
  };
  double nf2 = 0;
  TRY(norm64(f64, &nf2));
  const double nf = sqrt(nf2);
  dd_status rc = DD_OK;
  int iters = 0, outer = 0, reliable = 0;
  double rel = 0;
  if (nf2 == 0.0) {
    cudaMemsetAsync(x64, 0, b64, c->st);
  } else {
    while (true) {
      // FP64 true residual
      TRY(bicg_apply(c, R, x64, r64, P64, f64));
      reliable++;
      double rho2 = 0;
      TRY(norm64(r64, &rho2));
      float ms = 0;
      cudaEventElapsedTime(&ms, R.e0, R.e1);
      R.tA += ms * 1e-3;
      rel = sqrt(rho2) / nf;
      if (c->trace) fprintf(stderr, "[dd] bicgstab outer %d true residual %.3e\n", outer, rel);
      if (!isfinite(rel)) { rc = fail(c, DD_ERR_NONFINITE, "non-finite residual"); break; }
      if (rel <= p->tol) break;
      if (iters >= p->max_iter) { rc = fail(c, DD_ERR_NOT_CONVERGED, "iteration limit reached"); break; }
      int it = 0;
      if (!mixed) {
        // FP64 BiCGstab on the true residual; its recursive residual drifts, so it stops a
        // little below the target and the loop recomputes the true one
        BicgKernels<double2>::copy(g, (double2*)r, (const double2*)r64, c->st);
        TRY(launched(c));
        double rn = sqrt(rho2);
        TRY(bicgstab<double2>(c, R, P64, (double2*)x64, (double2*)r, (double2*)rh, (double2*)pv, (double2*)v,
                              (double2*)s, (double2*)t, (zd*)sc, part2, h_sc, 0.5 * p->tol * nf,
                              p->max_iter - iters, &it, &rn));
      } else {
        // correction e from A32 e = r / |r| to inner_tol, then x += |r| e in FP64
        launch_norm2_64((const double2*)r64, g.V * 12, part2, c->st);
        launch_reduce_partials(part2, 1, (double2*)coef + 1, 0, c->st);
        launch_r64_to_v32((float4*)r, (const double2*)r64, g.V * 6, (const double2*)coef + 1, c->st);
        BicgKernels<float4>::copy(g, (float4*)xw, nullptr, c->st);
        TRY(launched(c, 4));
        double rn = 1.0;
        TRY(bicgstab<float4>(c, R, P32, (float4*)xw, (float4*)r, (float4*)rh, (float4*)pv, (float4*)v, (float4*)s,
                             (float4*)t, (zd*)sc, part2, h_sc, p->inner_tol, p->max_iter - iters, &it, &rn));
        sqrt_to_coeff_kernel<<<1, 1, 0, c->st>>>((double2*)coef, (const double2*)coef + 1);
        launch_x_update((double2*)x64, (const float4*)xw, 1, g.V * 6, (const double2*)coef, c->st);
        TRY(launched(c, 2));
      }
      iters += it;
      outer++;
      if (it == 0) { rc = fail(c, DD_ERR_NOT_CONVERGED, "BiCGstab made no progress"); break; }
    }
  }
  launch_unpack_spinor(g, view(g, x64, P64), canon, P64, c->st);
  TRY(launched(c));
  TRY(cuda_check(c, cudaMemcpyAsync(x, canon, cb, where == DD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    c->st),
                 "copy x out"));
  cudaEventRecord(tend, c->st);
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "bicgstab"));
  float ms = 0;
  cudaEventElapsedTime(&ms, tstart, tend);
  if (info) {
    info->status = rc;
    info->iterations = iters;
    info->restarts = outer > 0 ? outer - 1 : 0;
    info->reliable_updates = reliable;
    info->true_rel_residual = rel;
    info->t_total = ms * 1e-3;
    info->t_A = R.tA;
    info->t_other = ms * 1e-3 - R.tA;
    info->flops_nominal = 1848.0 * (double)g.V * R.a_apps;
  }
  return rc;
}

// ------------------------------------------------------------------ host utilities
extern "C" double dd_load_model(long long n, int slots) {
  if (n <= 0 || slots <= 0) return 0.0;
  long long waves = (n + slots - 1) / slots;
  return (double)n / ((double)slots * (double)waves);
}

extern "C" dd_status dd_deflate_host(int m, int k, const double* Hbar, const double* cvec, const double* yvec,
                                     double* P, double* Hn, double* cn, double* theta) {
  if (m < 1 || m >= DD_MAXM || k < 1 || k >= m || !Hbar || !cvec || !yvec || !P || !Hn || !cn || !theta)
    return DD_ERR_INVALID;
  std::vector<double2> buf(deflate_bytes(m) / sizeof(double2) + 1);
  DeflateWork W = deflate_work(buf.data(), m);
  const Team T{0, 1};
  int rc = deflate(T, (const zd*)Hbar, m + 1, m, k, (const zd*)cvec, (const zd*)yvec, (zd*)P, (zd*)Hn, (zd*)cn,
                   (zd*)theta, W);
  return rc == 0 ? DD_OK : DD_ERR_NONFINITE;
}

extern "C" dd_status dd_deflate_device(int m, int k, const double* Hbar, const double* cvec, const double* yvec,
                                       double* P, double* Hn, double* cn, double* theta, double* ms) {
  if (m < 1 || m >= DD_MAXM || k < 1 || k >= m || !Hbar || !cvec || !yvec || !P || !Hn || !cn || !theta)
    return DD_ERR_INVALID;
  void* scratch = nullptr;
  int* flags = nullptr;
  if (cudaMalloc(&scratch, deflate_bytes(m)) != cudaSuccess) return DD_ERR_OOM;
  if (cudaMalloc(&flags, 16) != cudaSuccess) { cudaFree(scratch); return DD_ERR_OOM; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, 0);
  launch_deflate((const zd*)Hbar, m + 1, m, k, (const zd*)cvec, (const zd*)yvec, (zd*)P, (zd*)Hn, (zd*)cn, (zd*)theta,
                 scratch, flags, 0);
  cudaEventRecord(e1, 0);
  int rc = -1;
  cudaError_t e = cudaMemcpy(&rc, flags, sizeof(int), cudaMemcpyDeviceToHost);
  float t = 0;
  cudaEventElapsedTime(&t, e0, e1);
  if (ms) *ms = t;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  cudaFree(flags);
  if (e != cudaSuccess) return DD_ERR_CUDA;
  return rc == 0 ? DD_OK : DD_ERR_NONFINITE;
}

// ------------------------------------------------------------------ autotuner
// Deterministic pseudo-random FP64 field (splitmix64 per real), for tuning runs only.
__global__ void fill_random64_kernel(double* v, long long n, unsigned long long seed) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(q + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[q] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

namespace {
// One candidate of the search and its measured score.
struct TuneCand {
  int b[4];
  int i_domain, i_schwarz, tps;
  double score = 1e300;   // seconds per e-fold of residual reduction (lower is better)
  double res = 1.0, t = 0.0;
  int iters = 0;
};

// A context of the candidate's domain shape with the tuned context's gauge field and
// clover; nullptr (status in *st) when the shape is not allowed or set-up failed.
dd_ctx* tune_ctx(dd_ctx* c, const int b[4], dd_status* st) {
  dd_ctx* t = nullptr;
  *st = dd_create(&t, c->g.L, b, c->anti, c->st);
  if (*st != DD_OK) return nullptr;
  *st = dd_load_gauge(t, c->Ucanon, DD_DEVICE);
  if (*st == DD_OK) *st = dd_build_clover(t, c->kappa, c->csw);
  if (*st != DD_OK) {
    if (*st == DD_ERR_SINGULAR_CLOVER) *st = DD_OK;   // same clover as the tuned context
    else { dd_destroy(t); return nullptr; }
  }
  return t;
}
}  // namespace

// Time-to-solution search (Sec. IV-B: I_domain and the domain size are chosen by the
// overall time-to-solution, Eq. 6-7 give the load of a domain count).  Each candidate runs
// a short solve from x = 0 of a fixed pseudo-random source; its score is the solve's
// device time divided by the number of e-folds by which it reduced the true residual.
extern "C" dd_status dd_autotune(dd_ctx* c, int storage_prec, int domain_out[4], dd_sap_params* out) {
  if (!c || !domain_out || !out) return DD_ERR_INVALID;
  if (storage_prec != DD_PREC_FP16 && storage_prec != DD_PREC_FP32 && storage_prec != DD_PREC_FP16_H2)
    return fail(c, DD_ERR_INVALID, "autotune: storage_prec must be DD_PREC_FP16, DD_PREC_FP16_H2 or DD_PREC_FP32");
  if (out->i_schwarz < 0 || out->i_domain < 0 || out->threads_per_site < 0 || out->threads_per_site > 2 ||
      (storage_prec == DD_PREC_FP16_H2 && out->threads_per_site == 1) || out->additive < 0 || out->additive > 1 ||
      (out->additive && out->threads_per_site == 1))
    return fail(c, DD_ERR_INVALID, "autotune: bad fixed parameters");
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  const int fix_is = out->i_schwarz, fix_id = out->i_domain;
  const int fix_tps = (storage_prec == DD_PREC_FP16_H2 || out->additive) ? 2 : out->threads_per_site;
  const long long nreal = c->g.V * 24;
  double *f = nullptr, *x = nullptr;
  TRY(dalloc(c, &f, (size_t)nreal * 8));
  dd_status st = dalloc(c, &x, (size_t)nreal * 8);
  if (st != DD_OK) { release(c, f); return st; }
  fill_random64_kernel<<<blas_partials_blocks(), 256, 0, c->st>>>(f, nreal, 12345);
  st = launched(c);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  dd_solve_params sp;
  memset(&sp, 0, sizeof(sp));
  sp.tol = 1e-7;
  sp.m = 16;
  sp.k = 4;
  sp.max_iter = 48;
  // score one candidate on context t (its shape), keeping the first hard error in st
  auto score = [&](dd_ctx* t, TuneCand& cd) {
    if (st != DD_OK) return;
    sp.sap.i_schwarz = cd.i_schwarz;
    sp.sap.i_domain = cd.i_domain;
    sp.sap.storage_prec = storage_prec;
    sp.sap.threads_per_site = cd.tps;
    sp.sap.additive = out->additive;
    dd_status s = cuda_check(c, cudaMemsetAsync(x, 0, (size_t)nreal * 8, c->st), "autotune x");
    dd_solve_info info;
    memset(&info, 0, sizeof(info));
    if (s == DD_OK) s = dd_solve(t, f, x, 1, DD_DEVICE, &sp, &info);
    c->launches += t->launches;
    t->launches = 0;
    if (s == DD_OK || s == DD_ERR_NOT_CONVERGED) {
      cd.res = info.true_rel_residual;
      cd.t = info.t_total;
      cd.iters = info.iterations;
      const double efold = -log(cd.res);
      cd.score = (isfinite(cd.res) && cd.res < 1.0 && efold > 1e-3) ? cd.t / efold : 1e300;
    } else if (s == DD_ERR_NONFINITE) {
      cd.score = 1e300;   // diverged: not a candidate
    } else {
      st = s;
      c->err = "autotune candidate failed: " + t->err;
    }
    if (c->trace) {
      const long long n = t->g.ND / 2;
      const bool big = sap_smem_bytes(t->g, sap_prec(storage_prec), sap_mat_fits_smem(t->g, sap_prec(storage_prec))) >
                       116 * 1024;
      fprintf(stderr,
              "[dd] autotune b %dx%dx%dx%d I_S %d I_d %d tps %d: %d it, %.3f ms, residual %.3e, %.4f ms/e-fold, "
              "load %.2f\n",
              cd.b[0], cd.b[1], cd.b[2], cd.b[3], cd.i_schwarz, cd.i_domain, cd.tps, cd.iters, 1e3 * cd.t, cd.res,
              1e3 * cd.score, dd_load_model(n, sms * (big ? 1 : 2)));
    }
  };
  TuneCand best;
  best.score = 1e300;
  // stage 1: every allowed domain shape (extents 2, 4 or 8) with a short solve at
  // provisional parameters; the four best shapes go on
  const int ext[3] = {2, 4, 8};
  const int is0 = fix_is > 0 ? fix_is : 4, id0 = fix_id > 0 ? fix_id : 4, tps0 = fix_tps > 0 ? fix_tps : 2;
  std::vector<TuneCand> shapes;
  sp.max_iter = 12;
  for (int a0 = 0; a0 < 3 && st == DD_OK; ++a0)
    for (int a1 = 0; a1 < 3 && st == DD_OK; ++a1)
      for (int a2 = 0; a2 < 3 && st == DD_OK; ++a2)
        for (int a3 = 0; a3 < 3 && st == DD_OK; ++a3) {
          TuneCand cd;
          const int b[4] = {ext[a0], ext[a1], ext[a2], ext[a3]};
          memcpy(cd.b, b, sizeof(b));
          cd.i_schwarz = is0;
          cd.i_domain = id0;
          cd.tps = tps0;
          dd_status cs;
          dd_ctx* t = tune_ctx(c, b, &cs);
          if (!t) {
            if (cs != DD_ERR_DIMS) { st = cs; c->err = "autotune: candidate set-up failed"; }
            continue;
          }
          score(t, cd);
          dd_destroy(t);
          if (cd.score < 1e300) shapes.push_back(cd);
        }
  std::sort(shapes.begin(), shapes.end(), [](const TuneCand& p, const TuneCand& q) { return p.score < q.score; });
  if (shapes.size() > 4) shapes.resize(4);
  // stage 2: I_domain x threads per site on the kept shapes, with longer solves
  sp.max_iter = 48;
  for (const TuneCand& sh : shapes) {
    if (st != DD_OK) break;
    dd_status cs;
    dd_ctx* t = tune_ctx(c, sh.b, &cs);
    if (!t) { st = cs == DD_OK ? DD_ERR_CUDA : cs; break; }
    for (int id = 2; id <= 6 && st == DD_OK; ++id) {
      if (fix_id > 0 && id != fix_id) continue;
      for (int tps = 1; tps <= 2 && st == DD_OK; ++tps) {
        if (fix_tps > 0 && tps != fix_tps) continue;
        TuneCand cd = sh;
        cd.i_domain = id;
        cd.tps = tps;
        score(t, cd);
        if (cd.score < best.score) best = cd;
      }
    }
    dd_destroy(t);
  }
  // stage 3: I_Schwarz, then I_domain again, at the chosen shape and threads per site
  if (st == DD_OK && best.score < 1e300 && (fix_is == 0 || fix_id == 0)) {
    dd_status cs;
    dd_ctx* t = tune_ctx(c, best.b, &cs);
    if (!t) {
      st = cs == DD_OK ? DD_ERR_CUDA : cs;
    } else {
      if (fix_is == 0) {
        const int is_set[5] = {1, 2, 4, 8, 16};
        const TuneCand base = best;
        for (int q = 0; q < 5 && st == DD_OK; ++q) {
          if (is_set[q] == base.i_schwarz) continue;
          TuneCand cd = base;
          cd.i_schwarz = is_set[q];
          score(t, cd);
          if (cd.score < best.score) best = cd;
        }
      }
      if (fix_id == 0) {
        const TuneCand base = best;
        for (int id = 2; id <= 6 && st == DD_OK; ++id) {
          if (id == base.i_domain) continue;
          TuneCand cd = base;
          cd.i_domain = id;
          score(t, cd);
          if (cd.score < best.score) best = cd;
        }
      }
      dd_destroy(t);
    }
  }
  cudaStreamSynchronize(c->st);
  release(c, f);
  release(c, x);
  if (st != DD_OK) return st;
  if (best.score >= 1e300)
    return fail(c, DD_ERR_NOT_CONVERGED, "autotune: no candidate reduced the residual");
  for (int mu = 0; mu < 4; ++mu) domain_out[mu] = best.b[mu];
  out->i_schwarz = best.i_schwarz;
  out->i_domain = best.i_domain;
  out->threads_per_site = best.tps;
  out->storage_prec = storage_prec;
  return cuda_check(c, cudaStreamSynchronize(c->st), "autotune");
}

// ------------------------------------------------------------------ allocation-free Schwarz
// Same preconditioner as dd_sap_precondition (internal FP32 layout), but its working
// state (stored residual, solution, face buffers, error word) lives in a fixed array of
// the library's global memory instead of context buffers made by cudaMalloc.  The first
// call on a device looks up that array's device address (cudaGetSymbolAddress) with the
// device current.  The call is synchronous: it reads the error word back and waits for
// the stream.
extern "C" dd_status dd_sap_precondition_noalloc(dd_ctx* c, const float* in, float* out, const dd_sap_params* p) {
  if (!c || !in || !out) return DD_ERR_INVALID;
  TRY(check_sap_params(c, p));
  if (p->additive) return fail(c, DD_ERR_INVALID, "the allocation-free entry point runs the multiplicative form only");
  if (p->i_domain == 0) return fail(c, DD_ERR_INVALID, "i_domain must be >= 1");
  const Geom& g = c->g;
  int prec = sap_prec(p->storage_prec);
  // carve the fixed array: residual (even sites), solution, faces, error word
  size_t half_sites = (size_t)g.V / 2;
  size_t r_bytes = prec == P16 ? half_sites * 48 : half_sites * 96;
  size_t rn_bytes = prec == P16 ? half_sites * 4 : 0;
  size_t u_bytes = prec == P16 ? (size_t)g.V * 48 : (size_t)g.V * 96;
  size_t un_bytes = prec == P16 ? (size_t)g.V * 4 : 0;
  size_t f_bytes = (size_t)g.ND * g.face_block * 48;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t need = up(r_bytes) + up(rn_bytes) + up(u_bytes) + up(un_bytes) + up(f_bytes) + 256;
  if (need > sap_noalloc_scratch_bytes())
    return fail(c, DD_ERR_INVALID, "lattice too large for the allocation-free Schwarz entry point: needs " +
                                       std::to_string(need) + " bytes of scratch, the fixed array holds " +
                                       std::to_string(sap_noalloc_scratch_bytes()));
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  char* base = (char*)sap_noalloc_scratch();
  if (!base) return fail(c, DD_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch array failed");
  SapState S;
  S.mat_prec = prec;
  S.vec_prec = prec;
  S.links = prec == P16 ? (const void*)c->U16 : (const void*)c->U32;
  S.smat = prec == P16 ? (const void*)c->S16 : (const void*)c->S32;
  size_t off = 0;
  S.r_store = base + off; off += up(r_bytes);
  S.r_norm = rn_bytes ? (float*)(base + off) : nullptr; off += up(rn_bytes);
  S.u_store = base + off; off += up(u_bytes);
  S.u_norm = un_bytes ? (float*)(base + off) : nullptr; off += up(un_bytes);
  S.faces = (float4*)(base + off); off += up(f_bytes);
  S.err = (int*)(base + off);
  S.mat_in_smem = sap_mat_fits_smem(g, prec);
  S.threads_per_site = p->threads_per_site ? p->threads_per_site : 2;
  S.half_arith = p->storage_prec == DD_PREC_FP16_H2;
  S.inject_wait_timeout = c->inject_wait_timeout;
  // the error word must start at zero; residual, solution and faces are written before
  // they are read within one call
  TRY(cuda_check(c, cudaMemsetAsync(S.err, 0, sizeof(int), c->st), "clear error word"));
  for (int s = 0; s < p->i_schwarz; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      int first = s == 0, use_faces = !(s == 0 && colour == 0), last = s == p->i_schwarz - 1;
      if (sap_half_sweep(g, S, colour, first, use_faces, last, (const float4*)in, (float4*)out, p->i_domain, c->st))
        return fail(c, DD_ERR_CUDA, std::string("Schwarz launch failed: ") + cudaGetErrorString(cudaGetLastError()));
      TRY(launched(c));
    }
  int e = 0;
  TRY(cuda_check(c, cudaMemcpyAsync(&e, S.err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "error word"));
  TRY(cuda_check(c, cudaStreamSynchronize(c->st), "sap_noalloc"));
  if (e) return fail(c, DD_ERR_TIMEOUT, "a bounded wait for the domain's staged data ran out");
  return DD_OK;
}

// ------------------------------------------------------------------ two-level multigrid: C ABI
extern "C" dd_status dd_mg_setup(dd_ctx* c, const double* tv, int where, const dd_mg_params* p, double* seconds) {
  if (!c || !tv || !p) return DD_ERR_INVALID;
  if (!c->have_clover) return fail(c, DD_ERR_NO_CLOVER, "clover not built");
  if (p->n_tv < 1 || p->n_tv > MG_MAXTV || p->setup_iters < 0 || p->coarse_m < 1 || p->coarse_m > DD_MAXM - 1 ||
      p->coarse_cycles < 1 || p->smoother.i_schwarz < 0 || p->setup_mode < 0 || p->setup_mode > 1)
    return fail(c, DD_ERR_INVALID, "bad multigrid parameters");
  // the smoother's Schwarz form (at least one cycle when the set-up smooths test vectors)
  dd_sap_params sm = p->smoother;
  if (sm.i_schwarz > 0 || p->setup_iters > 0) {
    dd_sap_params chk = sm;
    if (chk.i_schwarz < 1) chk.i_schwarz = 1;
    TRY(check_sap_params(c, &chk));
    if (chk.i_domain < 1) return fail(c, DD_ERR_INVALID, "i_domain must be >= 1");
  }
  const Geom& g = c->g;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, c->st);
  drop_graphs(c);   // captured solver steps may hold the previous set-up's buffers
  mg_free(c);
  TRY(mg_alloc(c, p->n_tv, p->coarse_m));
  dd_ctx::Mg& M = c->mg;
  M.cycles = p->coarse_cycles;
  M.smoother = sm;
  const long long n4 = g.V * 6;
  const size_t cb = (size_t)g.V * 24 * 8;
  double* stage = nullptr;
  TRY(dalloc(c, &stage, cb));
  dd_status rc = DD_OK;
  const cudaMemcpyKind kind = where == DD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int k = 0; k < p->n_tv && rc == DD_OK; ++k) {
    rc = cuda_check(c, cudaMemcpyAsync(stage, tv + (size_t)k * g.V * 24, cb, kind, c->st), "test vector");
    if (rc == DD_OK) {
      launch_pack_spinor(g, stage, P64, view(g, M.P + k * n4, P32), c->st);
      rc = launched(c);
    }
  }
  // test vectors <- M_sap v (inverse iteration) or v - M_sap A v (the smoother on A v = 0),
  // setup_iters times
  dd_sap_params ss = sm;
  if (ss.i_schwarz < 1) ss.i_schwarz = 1;
  for (int it = 0; it < p->setup_iters && rc == DD_OK; ++it)
    for (int k = 0; k < p->n_tv && rc == DD_OK; ++k) {
      float4* v = M.P + k * n4;
      if (p->setup_mode == 0) {
        rc = sap_run(c, v, M.ef, &ss);
        if (rc == DD_OK)
          rc = cuda_check(c, cudaMemcpyAsync(v, M.ef, (size_t)n4 * 16, cudaMemcpyDeviceToDevice, c->st),
                          "smoothed test vector");
      } else {
        rc = apply_internal(c, v, M.xf, P32);
        if (rc == DD_OK) rc = sap_run(c, M.xf, M.ef, &ss);
        if (rc == DD_OK) {
          launch_mg_axpy(v, M.ef, n4, -1.f, c->st);
          rc = launched(c);
        }
      }
    }
  if (rc == DD_OK && p->setup_iters > 0) rc = sap_error_flag(c);
  int bad = 0;
  if (rc == DD_OK) rc = cuda_check(c, cudaMemsetAsync(M.state, 0, 16, c->st), "status");
  if (rc == DD_OK) {
    launch_mg_orthonormalize(g, M.P, p->n_tv, M.state, c->st);
    rc = launched(c);
  }
  if (rc == DD_OK) rc = cuda_check(c, cudaMemcpyAsync(&bad, M.state, sizeof(int), cudaMemcpyDeviceToHost, c->st), "status");
  if (rc == DD_OK) rc = cuda_check(c, cudaStreamSynchronize(c->st), "orthonormalise");
  if (rc == DD_OK && bad) rc = fail(c, DD_ERR_NONFINITE, "test vectors are linearly dependent on a domain");
  if (rc == DD_OK) {
    launch_mg_coarse_build(g, c->U32, c->C32, M.P, p->n_tv, M.Dc, c->st);
    rc = launched(c);
  }
  cudaEventRecord(t1, c->st);
  if (rc == DD_OK) rc = cuda_check(c, cudaStreamSynchronize(c->st), "coarse operator");
  release(c, stage);
  float ms = 0;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (seconds) *seconds = ms * 1e-3;
  if (rc != DD_OK) {
    mg_free(c);
    return rc;
  }
  M.ready = true;
  return DD_OK;
}

static dd_status mg_ready(dd_ctx* c) {
  if (!c->mg.ready) return fail(c, DD_ERR_INVALID, "dd_mg_setup has not been called");
  return DD_OK;
}

extern "C" dd_status dd_mg_restrict(dd_ctx* c, const float* in, float* out) {
  if (!c || !in || !out) return DD_ERR_INVALID;
  TRY(mg_ready(c));
  launch_mg_restrict(c->g, (const float4*)in, c->mg.P, c->mg.ntv, (float2*)out, nullptr, c->st);
  TRY(launched(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "restrict");
}

extern "C" dd_status dd_mg_prolong(dd_ctx* c, const float* in, float* out) {
  if (!c || !in || !out) return DD_ERR_INVALID;
  TRY(mg_ready(c));
  launch_mg_prolong(c->g, (const float2*)in, c->mg.P, c->mg.ntv, (float4*)out, c->st);
  TRY(launched(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "prolong");
}

extern "C" dd_status dd_mg_coarse_apply(dd_ctx* c, const float* x, float* y) {
  if (!c || !x || !y || x == y) return DD_ERR_INVALID;
  TRY(mg_ready(c));
  launch_mg_coarse_apply(c->g, c->mg.Dc, c->mg.nc, (const float2*)x, (float2*)y, nullptr, nullptr, c->st);
  TRY(launched(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "coarse apply");
}

extern "C" dd_status dd_mg_coarse_solve(dd_ctx* c, const float* b, float* x) {
  if (!c || !b || !x) return DD_ERR_INVALID;
  TRY(mg_ready(c));
  const size_t bytes = (size_t)c->g.ND * c->mg.nc * sizeof(float2);
  TRY(cuda_check(c, cudaMemcpyAsync(c->mg.cb, b, bytes, cudaMemcpyDeviceToDevice, c->st), "coarse rhs"));
  TRY(mg_coarse_solve(c));
  TRY(cuda_check(c, cudaMemcpyAsync(x, c->mg.cx, bytes, cudaMemcpyDeviceToDevice, c->st), "coarse solution"));
  return cuda_check(c, cudaStreamSynchronize(c->st), "coarse solve");
}

extern "C" dd_status dd_mg_precondition(dd_ctx* c, const float* in, float* out, int layout) {
  if (!c || !in || !out || in == out) return DD_ERR_INVALID;
  TRY(mg_ready(c));
  if (layout == DD_LAYOUT_INTERNAL) {
    TRY(mg_run(c, (const float4*)in, (float4*)out));
  } else {
    TRY(ensure_scratch(c));
    launch_pack_spinor(c->g, in, P32, view(c->g, c->scratch_in, P32), c->st);
    TRY(launched(c));
    TRY(mg_run(c, (const float4*)c->scratch_in, (float4*)c->scratch_out));
    launch_unpack_spinor(c->g, view(c->g, c->scratch_out, P32), out, P32, c->st);
    TRY(launched(c));
  }
  if (c->mg.smoother.i_schwarz > 0) TRY(sap_error_flag(c));
  return cuda_check(c, cudaStreamSynchronize(c->st), "mg precondition");
}

extern "C" dd_status dd_solve_mg(dd_ctx* c, const double* f, double* x, int where, const dd_solve_params* p,
                                 dd_solve_info* info) {
  if (!c || !f || !x || !p) return DD_ERR_INVALID;
  TRY(mg_ready(c));
  dd_solve_params q = *p;
  // the smoother's parameters key the captured steps; the preconditioner is the two-level method
  q.sap = c->mg.smoother;
  if (q.sap.i_schwarz < 1) q.sap = dd_sap_params{1, 1, DD_PREC_FP16, 0, 0};
  c->mg_active = true;
  dd_status st = dd_solve(c, f, x, 1, where, &q, info);
  c->mg_active = false;
  return st;
}

// C ABI of the library (include/hrm.h): context management, the per-step CUDA
// graph and dispatch to the kernel tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hrm.h"
#include "hrm_batch.cuh"
#include "hrm_launch.h"
#include "hrm_learned.h"

using namespace hrm;

namespace {
constexpr int kMaxProf = 32;  // brackets of one step: 3 stages x (prim, 3 gates, sweeps, 3 sweeps, update) + finalize
}

struct hrm_ctx {
  int N = 0, D = 0, M = 0;
  int64_t nc = 0;                  // stored cells per plane (interior + Dirichlet slices)
  int64_t nint = 0;                // interior cells
  int bnd_need = 0, bnd_set = 0;   // Dirichlet sides (bit b = side b) and those given a state
  hrm_grid grid{};
  hrm_params params{};
  DevFluid fl{};
  DevGrid dg{};
  DevParams dp{};
  cudaStream_t stream = nullptr;   // caller's stream: every call is ordered on it
  cudaStream_t cap = nullptr;      // private stream used only to capture the step graph
  double* Wn = nullptr;            // state W^n (M planes)
  double* Ws = nullptr;            // RK stage state
  double* V = nullptr;             // primitive planes (M) -- also scratch for I/O
  double* AUX = nullptr;           // c, rho, rho c^2
  float* P32 = nullptr;            // FP32 planes of the precision form (M + D + 4 + N - 1)
  float* R32 = nullptr;            // FP32 residues of rho, u_d, p for the learned gate (D + 2)
  double* F[3] = {nullptr, nullptr, nullptr};  // midpoint fluxes per direction (M + N - 1 planes)
  StepState* st = nullptr;
  mlp::GateBlob* blob = nullptr;   // learned gate weights (hrm_set_detector)
  uint8_t* gate[3] = {nullptr, nullptr, nullptr};  // gate bytes per direction (midpoint grids)
  uint8_t* same = nullptr;         // FP64 form: per cell, the last update left W bit for bit as its source
  uint32_t* defer = nullptr;       // precision form: per direction, a worklist of deferred midpoints and its counter
  int64_t defer_cap = 0;           // worklist entries (the largest midpoint grid; 0: no worklist)
  hrm_alloc_fn alloc = nullptr;    // device memory source (hrm_set_allocator at creation; NULL: cudaMalloc)
  hrm_free_fn dealloc = nullptr;
  void* alloc_user = nullptr;
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};  // deferred midpoints overlap the next sweep here
  cudaEvent_t ev_fast[3] = {}, ev_fix[3] = {};
  // in 2D and 3D the sweeps of one stage run concurrently: direction d > 0 on par[d]
  cudaStream_t par[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {};
  int gate_set[3] = {0, 0, 0};     // fixed gate provided (hrm_set_gate)
  int gate_blocks = 0;             // persistent blocks of the gate kernel
  const CellKernels* ck = nullptr;
  const FaceKernels* fk = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_kernels = 0;
  int64_t launches = 0;
  // precision form in 2D: the step as three persistent stage launches (the
  // batched form's kernel over this one context), else the per-phase graph
  int step_path = 0;               // hrm_set_step_path: 1 persistent where eligible, 0 per-phase kernels
  bool persist = false;            // the current graph is the persistent one
  bool persist_refused = false;    // capturing the persistent launches failed once: per-phase graph
  BatchInst* p_inst = nullptr;     // this context as a one-instance batch
  WorkItem* p_cells = nullptr;
  WorkItem* p_tiles = nullptr;
  int p_ncell = 0, p_ntiles = 0, p_grid = 0;
  GridSync* p_sync = nullptr;
  unsigned int p_expired_seen = 0;
  // tracing: event pairs around every kernel of the captured step
  // W^n's interior cells all came out of this form's relaxation (relax_fast in
  // the precision form, relax_cell in FP64: a step that relaxed at its last
  // stage, and no state or parameter written since); the stage updates take
  // the relaxation's result from W^n for cells it would return unchanged only
  // then. Mirrored into StepState::wn_relaxed (wn_relaxed_dev: the value last
  // written there).
  bool wn_relaxed = false;
  int wn_relaxed_dev = 0;
  // precision form: the FP32 planes and the CFL maxima (StepState::tau_bits)
  // already hold W^n's, written by the last stage of the step just launched
  // (fuse_last), so that the next step's first primitive pass has nothing to
  // do; mirrored into StepState::planes_tau like wn_relaxed.
  bool planes_tau = false;
  int planes_tau_dev = 0;
  int profiling = 0;
  int nprof = 0;
  cudaEvent_t prof_ev[2 * kMaxProf] = {};
  int32_t prof_kind[kMaxProf] = {};
  std::string err;
};

namespace {

// NVTX range around an entry point (visible in Nsight timelines; no cost when no
// tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// Message of the last failed hrm_create on this thread (its context is gone).
thread_local std::string g_create_error = "null context";

// Allocator for contexts created from now on (hrm_set_allocator).
hrm_alloc_fn g_alloc = nullptr;
hrm_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;

// Device memory of a context: its allocator, else cudaMalloc.
cudaError_t ctx_malloc(hrm_ctx* c, void** p, size_t bytes) {
  if (!c->alloc) return cudaMalloc(p, bytes);
  *p = c->alloc(bytes, (void*)c->stream, c->alloc_user);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
template <typename T>
cudaError_t ctx_malloc(hrm_ctx* c, T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = ctx_malloc(c, &q, bytes);
  *p = static_cast<T*>(q);
  return e;
}
void ctx_free(hrm_ctx* c, void* p) {
  if (!p) return;
  if (c->dealloc)
    c->dealloc(p, (void*)c->stream, c->alloc_user);
  else if (!c->alloc)
    cudaFree(p);
}

hrm_status fail(hrm_ctx* c, hrm_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

hrm_status cuda_check(hrm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HRM_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? HRM_E_NOMEM : HRM_E_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

hrm_status last_launch(hrm_ctx* c, const char* what) { return cuda_check(c, cudaGetLastError(), what); }

hrm_status check_params(hrm_ctx* c, const hrm_params* p) {
  if (p->cfl <= 0.0) return fail(c, HRM_E_INVAL, "cfl must be positive");
  if (p->limiters && p->cfl > 0.5)
    return fail(c, HRM_E_INVAL, "cfl %.3g > 0.5 with the positivity limiters on (Sec. 4.1.2)", p->cfl);
  if (p->scheme < 0 || p->scheme > 1) return fail(c, HRM_E_INVAL, "unknown scheme %d", p->scheme);
  if (p->relax_mode < 0 || p->relax_mode > 2) return fail(c, HRM_E_INVAL, "unknown relax_mode %d", p->relax_mode);
  if (p->integrator < 0 || p->integrator > 2) return fail(c, HRM_E_INVAL, "unknown integrator %d", p->integrator);
  if (p->precision < 0 || p->precision > 1) return fail(c, HRM_E_INVAL, "unknown precision %d", p->precision);
  if (p->learned < 0 || p->learned > 2) return fail(c, HRM_E_INVAL, "unknown learned mode %d", p->learned);
  if (p->learned && !(p->learned_threshold > 0.0 && p->learned_threshold < 1.0))
    return fail(c, HRM_E_INVAL, "learned_threshold must lie in (0, 1)");
  if (p->learned == 1 && !c->blob) return fail(c, HRM_E_INVAL, "learned gate: call hrm_set_detector first");
  if (p->learned == 2)
    for (int d = 0; d < c->D; ++d)
      if (!c->gate_set[d]) return fail(c, HRM_E_INVAL, "fixed gate: call hrm_set_gate for direction %d", d);
  if (p->learned && p->scheme != HRM_SCHEME_WCNS)
    return fail(c, HRM_E_INVAL, "the gate acts on the WENO-IS interpolation (scheme WCNS only)");
  if (p->q_sensor < 1.0 || p->q_sensor != std::floor(p->q_sensor))
    return fail(c, HRM_E_INVAL, "q_sensor must be a positive integer");
  if (p->cfl_sound < 0 || p->cfl_sound > 1) return fail(c, HRM_E_INVAL, "unknown cfl_sound %d", p->cfl_sound);
  // the WENO-IS weights are formed as products of five (beta + eps) (App. C,
  // scaled by a common factor): eps well inside the FP64 range
  if (!(p->weno_eps > 0.0 && p->weno_eps <= 1e50)) return fail(c, HRM_E_INVAL, "weno_eps must lie in (0, 1e50]");
  return HRM_OK;
}

void fill_dev_params(hrm_ctx* c) {
  const hrm_params& p = c->params;
  DevParams& d = c->dp;
  d.limiters = p.limiters;
  d.blend = p.blend;
  d.scheme = p.scheme;
  d.qexp = (int)p.q_sensor;
  d.eps_ar = p.eps_ar;
  d.eps_a = p.eps_a;
  d.eps_rhoe = p.eps_rhoe;
  d.hs_ar = p.hs_ar;
  d.hs_a = p.hs_a;
  d.hs_rc2 = p.hs_rc2;
  d.hs_rhoe = p.hs_rhoe;
  d.weno_eps = p.weno_eps;
  d.Cs = p.Cs;
  fill_screen(d, p.screen);
}

void drop_graph(hrm_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->graph_kernels = 0;
}

// Launch one kernel of the step (or a group of launches, such as the
// concurrent sweeps of a stage); while profiling, bracket it with an event pair
// on s (captured as event-record nodes) and remember its kind (HRM_KERNEL_*).
// The slot is taken before launching, so brackets may nest.
template <typename F>
void traced(hrm_ctx* c, cudaStream_t s, int kind, F&& launch) {
  const int i = c->nprof;
  const bool on = c->profiling && i < kMaxProf;
  // external event-record nodes: recorded each time the graph runs
  if (on) {
    ++c->nprof;
    c->prof_kind[i] = kind;
    cudaEventRecordWithFlags(c->prof_ev[2 * i], s, cudaEventRecordExternal);
  }
  launch();
  if (on) cudaEventRecordWithFlags(c->prof_ev[2 * i + 1], s, cudaEventRecordExternal);
}

float gate_logit_threshold(const hrm_ctx* c) {
  const double t = c->params.learned_threshold;
  return (float)std::log(t / (1.0 - t));
}

// FP32 planes are written by the primitive kernel in the precision form and
// whenever the learned gate reads them.
float* p32_target(hrm_ctx* c) {
  return (c->params.precision == HRM_FP32 || c->params.learned == 1) ? c->P32 : nullptr;
}

float* r32_target(hrm_ctx* c) { return c->params.learned == 1 ? c->R32 : nullptr; }

// The gate of direction d's sweep: fixed bytes (learned 2: the caller's;
// learned 1: written by the detector's gate kernel just before the sweep).
// The precision form's sweep defers screen failures to a second kernel (one
// without the FP64 fallbacks inline), except with the first-order scheme or the
// screens off.
bool defer_sweep(const hrm_ctx* c) {
  return c->params.precision == HRM_FP32 && c->defer && c->params.scheme == HRM_SCHEME_WCNS && c->params.screen;
}

// Kernels one sweep launches.
int sweep_kernels(const hrm_ctx* c) { return defer_sweep(c) ? 2 : 1; }

GateArgs gate_of(const hrm_ctx* c, int d) {
  GateArgs g;
  if (defer_sweep(c)) {
    g.defer_list = c->defer + (size_t)d * (size_t)(c->defer_cap + 1);
    g.defer_count = g.defer_list + c->defer_cap;
  }
  if (c->params.learned) g.fixed = c->gate[d];
  if (c->params.learned == 1 && defer_sweep(c)) {  // the network inside the sweep
    g.net = c->blob;
    g.R32 = c->R32;
    g.zthr = gate_logit_threshold(c);
    g.out_gate = c->gate[d];
  }
  return g;
}

// With the learned detector, its gate kernel runs before each sweep, except in
// the precision form's screened sweep, which evaluates the network itself.
bool separate_gate(const hrm_ctx* c) { return c->params.learned == 1 && !defer_sweep(c); }

// CFL maxima of the prim kernels: 1 with the five-equation c, 2 with the
// four-equation HRM c (params.cfl_sound).
int tau_mode(const hrm_ctx* c) { return c->params.cfl_sound ? 2 : 1; }

// The precision form's last stage writes the next step's FP32 planes and CFL
// maxima itself: with the five-equation sound speed and without Dirichlet
// slices (whose cells the update does not cover).
bool fuse_last(const hrm_ctx* c) {
  return c->params.precision == HRM_FP32 && !c->params.cfl_sound && c->nint == c->nc;
}

// One RK stage: primitives of Wsrc, (gates,) midpoint fluxes, update into Wout.
// Precision form: the update of every stage but the last also writes the next
// stage's FP32 planes (k_update32p, fuse_next), and a stage whose planes were
// written so (prim_done) skips its primitive kernel.
// FP64 form within one step: same_out, the update marks the cells whose state it
// leaves bit for bit as in Wsrc; same_in, the primitive pass keeps those cells'
// primitives (the previous stage's update marked them, nothing wrote W since).
int enqueue_stage(hrm_ctx* c, cudaStream_t s, const double* Wsrc, double* Wout, double a, double b, int relax,
                  int count, bool first, bool prim_done = false, bool fuse_next = false, bool tau_next = false,
                  bool same_in = false, bool same_out = false) {
  uint8_t* same = c->params.precision == HRM_FP64 ? c->same : nullptr;
  int k = 0;
  float* p32 = p32_target(c);
  if (!prim_done) {
    traced(c, s, HRM_KERNEL_PRIM, [&] {
      if (c->params.precision == HRM_FP32)
        launch_prim32(c->N, c->D, Wsrc, c->P32, r32_target(c), c->dg, c->fl, c->st, first ? tau_mode(c) : 0, s);
      else
        c->ck->prim(Wsrc, c->V, c->AUX, p32, r32_target(c), c->dg, c->fl, c->st, first ? tau_mode(c) : 0,
                    same_in && !first ? same : nullptr, s);
    });
    ++k;
  }
  if (first) {
    traced(c, s, HRM_KERNEL_FINALIZE, [&] { launch_finalize(c->st, c->dg, c->D, c->params.cfl, 0, s); });
    ++k;
  }
  if (separate_gate(c))
    for (int d = 0; d < c->D; ++d) {
      traced(c, s, HRM_KERNEL_GATE, [&] {
        launch_gate(c->N, c->D, d, c->P32, c->R32, c->dg, c->blob, gate_logit_threshold(c), c->gate[d],
                    &c->st->waits, c->gate_blocks, s);
      });
      ++k;
    }
  // the sweeps: independent (each reads the primitives and writes its own flux
  // planes), so directions d > 0 run on their own streams beside direction 0
  const bool fork = c->D > 1 && c->par[1];
  traced(c, s, HRM_KERNEL_SWEEPS, [&] {
    if (fork) {
      cudaEventRecord(c->ev_fork, s);
      for (int d = 1; d < c->D; ++d) cudaStreamWaitEvent(c->par[d], c->ev_fork, 0);
    }
    for (int d = 0; d < c->D; ++d) {
      const cudaStream_t sd = (fork && d > 0) ? c->par[d] : s;
      GateArgs ga = gate_of(c, d);
      if (ga.defer_list) {  // the deferred midpoints run beside the next sweep
        ga.side = c->side[d];
        ga.ev_fast = c->ev_fast[d];
        ga.ev_fix = c->ev_fix[d];
      }
      traced(c, sd, HRM_KERNEL_FACE_X + d, [&] {
        c->fk->face[d](c->params.precision, Wsrc, c->V, c->AUX, c->P32, c->F[d], c->dg, c->fl, c->dp, c->st, ga,
                       sd);
      });
      k += sweep_kernels(c);
    }
    if (fork)
      for (int d = 1; d < c->D; ++d) {
        cudaEventRecord(c->ev_join[d], c->par[d]);
        cudaStreamWaitEvent(s, c->ev_join[d], 0);
      }
  });
  if (defer_sweep(c))
    for (int d = 0; d < c->D; ++d) cudaStreamWaitEvent(s, c->ev_fix[d], 0);
  traced(c, s, HRM_KERNEL_UPDATE, [&] {
    if (fuse_next)
      launch_update32p(c->N, c->D, c->Wn, Wsrc, Wout, c->F[0], c->F[1], c->F[2], c->dg, c->fl, c->st, a, b, relax,
                       count, c->P32, r32_target(c), s, tau_next ? 1 : 0);
    else
      c->fk->update(0, c->params.precision == HRM_FP32, c->Wn, Wsrc, Wout, c->F[0], c->F[1], c->F[2], c->dg,
                    c->fl, c->st, a, b, relax, count, same_out ? same : nullptr, s);
  });
  ++k;
  return k;
}

// Kernels of one full step (Sec. 4.4): SSP-RK3 in Shu-Osher form, SSP-RK2 or
// forward Euler, relaxation after every stage (or after the step).
int enqueue_step(hrm_ctx* c, cudaStream_t s) {
  const int rs = c->params.relax_mode == HRM_RELAX_STAGE;
  const int rf = c->params.relax_mode != HRM_RELAX_OFF;
  const int ck = c->params.check ? 1 : 0;  // admissibility counters, read only with params.check
  const bool fp32 = c->params.precision == HRM_FP32;  // stages after the first take fused planes
  const bool fl = fuse_last(c);  // the last stage: the next step's planes and CFL maxima too
  int k = 0;
  switch (c->params.integrator) {
    case HRM_EULER:
      k += enqueue_stage(c, s, c->Wn, c->Wn, 0.0, 1.0, rf, ck, true, false, fl, fl);
      break;
    case HRM_RK2:
      k += enqueue_stage(c, s, c->Wn, c->Ws, 0.0, 1.0, rs, 0, true, false, fp32, false, false, true);
      k += enqueue_stage(c, s, c->Ws, c->Wn, 0.5, 0.5, rf, ck, false, fp32, fl, fl, true, false);
      break;
    default:
      k += enqueue_stage(c, s, c->Wn, c->Ws, 0.0, 1.0, rs, 0, true, false, fp32, false, false, true);
      k += enqueue_stage(c, s, c->Ws, c->Ws, 0.75, 0.25, rs, 0, false, fp32, fp32, false, true, true);
      k += enqueue_stage(c, s, c->Ws, c->Wn, 1.0 / 3.0, 2.0 / 3.0, rf, ck, false, fp32, fl, fl, true, false);
      break;
  }
  return k;
}

// The persistent step applies to the precision form in 2D with PP-WCNS-IS,
// SSP-RK3, the five-equation CFL speed, no Dirichlet sides and no learned gate.
bool persistent_eligible(const hrm_ctx* c) {
  const hrm_params& p = c->params;
  return c->step_path == 1 && !c->persist_refused && p.precision == HRM_FP32 && c->D == 2 && c->nint == c->nc &&
         !p.learned && p.scheme == HRM_SCHEME_WCNS && p.integrator == HRM_RK3 && !p.cfl_sound &&
         (c->N == 2 || c->N == 3);
}

// Device tables of the persistent step: this context as one instance, its
// cells in items of 1024, its midpoints of both directions in tiles of 128.
hrm_status setup_persistent(hrm_ctx* c) {
  if (c->p_inst) return HRM_OK;
  BatchInst I;
  std::memset(&I, 0, sizeof I);
  I.g = c->dg;
  I.f = c->fl;
  I.N = c->N;
  I.Wn = c->Wn;
  I.Ws = c->Ws;
  I.V = c->V;
  I.AUX = c->AUX;
  for (int d = 0; d < 3; ++d) I.F[d] = c->F[d];
  I.P32 = c->P32;
  I.st = c->st;
  std::vector<WorkItem> cells, tiles;
  constexpr int64_t kCellItem = 1024;
  for (int64_t x = 0; x < c->nint; x += kCellItem) cells.push_back({0, 0, x, std::min<int64_t>(x + kCellItem, c->nint)});
  for (int d = 0; d < 2; ++d) {
    const int64_t nf = (c->dg.n[0] + (d == 0)) * (c->dg.n[1] + (d == 1));
    for (int64_t t = 0; t < nf; t += kBatchFace32Threads)
      tiles.push_back({0, d, t, std::min<int64_t>(t + kBatchFace32Threads, nf)});
  }
  hrm_status s;
  if ((s = cuda_check(c, ctx_malloc(c, &c->p_inst, sizeof I), "alloc instance"))) return s;
  if ((s = cuda_check(c, ctx_malloc(c, &c->p_cells, sizeof(WorkItem) * cells.size()), "alloc items"))) return s;
  if ((s = cuda_check(c, ctx_malloc(c, &c->p_tiles, sizeof(WorkItem) * tiles.size()), "alloc tiles"))) return s;
  if ((s = cuda_check(c, ctx_malloc(c, &c->p_sync, sizeof(GridSync)), "alloc grid sync"))) return s;
  if ((s = cuda_check(c, cudaMemcpyAsync(c->p_inst, &I, sizeof I, cudaMemcpyHostToDevice, c->stream), "copy instance")))
    return s;
  if ((s = cuda_check(c, cudaMemcpyAsync(c->p_cells, cells.data(), sizeof(WorkItem) * cells.size(),
                                         cudaMemcpyHostToDevice, c->stream), "copy items")))
    return s;
  if ((s = cuda_check(c, cudaMemcpyAsync(c->p_tiles, tiles.data(), sizeof(WorkItem) * tiles.size(),
                                         cudaMemcpyHostToDevice, c->stream), "copy tiles")))
    return s;
  if ((s = cuda_check(c, cudaMemsetAsync(c->p_sync, 0, sizeof(GridSync), c->stream), "clear grid sync"))) return s;
  if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "persistent set-up"))) return s;
  c->p_ncell = (int)cells.size();
  c->p_ntiles = (int)tiles.size();
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->p_grid = sms * batch_stage32_fit();
  return c->p_grid > 0 ? HRM_OK : fail(c, HRM_E_CUDA, "persistent stage kernel: no resident block fits an SM");
}

// The three stage launches of one persistent step (SSP-RK3, Shu-Osher form).
hrm_status enqueue_persistent_step(hrm_ctx* c, cudaStream_t s) {
  const int rs = c->params.relax_mode == HRM_RELAX_STAGE;
  const int rf = c->params.relax_mode != HRM_RELAX_OFF;
  for (int k = 0; k < 3; ++k) {
    StageArgs A{};
    A.insts = c->p_inst;
    A.cells = c->p_cells;
    A.tiles = c->p_tiles;
    A.ncell_items = c->p_ncell;
    A.ntiles = c->p_ntiles;
    A.ninst = 1;
    A.src = k == 0 ? 0 : 1;
    A.dst = k == 2 ? 0 : 1;
    A.a = k == 0 ? 0.0 : (k == 1 ? 0.75 : 1.0 / 3.0);
    A.b = k == 0 ? 1.0 : (k == 1 ? 0.25 : 2.0 / 3.0);
    A.relax = k == 2 ? rf : rs;
    A.first = k == 0;
    A.prim = k == 0;
    A.fuse_next = k < 2;
    A.cfl = c->params.cfl;
    A.pr = c->dp;
    A.sync = c->p_sync;
    A.limit_ns = 2000000000ull;
    A.stage = k;
    A.update = 1;
    hrm_status st;
    if ((st = cuda_check(c, cudaMemsetAsync(c->p_sync, 0, kResetWords * sizeof(unsigned int), s), "reset queues")))
      return st;
    if ((st = cuda_check(c, batch_stage32_launch(c->p_grid, A, s), "persistent stage launch"))) return st;
  }
  return HRM_OK;
}

// Capture the persistent step; false when the capture or instantiation was
// refused (the per-phase graph is used from then on).
bool build_persistent_graph(hrm_ctx* c) {
  if (setup_persistent(c)) return false;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const hrm_status se = enqueue_persistent_step(c, c->cap);
  const cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
  if (se || ee != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  const cudaError_t e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->gexec = nullptr;
    return false;
  }
  c->graph_kernels = 3;
  c->persist = true;
  return true;
}

hrm_status build_graph(hrm_ctx* c) {
  drop_graph(c);
  c->nprof = 0;
  c->persist = false;
  if (persistent_eligible(c)) {
    if (build_persistent_graph(c)) return HRM_OK;
    c->persist_refused = true;
    c->err.clear();
  }
  cudaGraph_t g = nullptr;
  hrm_status s = cuda_check(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (s) return s;
  const int k = enqueue_step(c, c->cap);
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if ((s = cuda_check(c, e, "end capture"))) return s;
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if ((s = cuda_check(c, e, "graph instantiate"))) return s;
  c->graph_kernels = k;
  return HRM_OK;
}

// Copy `planes` planes of `cells` doubles between plane strides (in cells).
hrm_status copy_planes(hrm_ctx* c, double* dst, int64_t dpitch, const double* src, int64_t spitch, int64_t cells,
                       int planes, cudaMemcpyKind kind, const char* what) {
  if (dpitch == cells && spitch == cells)
    return cuda_check(c, cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)cells * planes, kind, c->stream), what);
  for (int m = 0; m < planes; ++m)  // one copy per plane (no pitch limit)
    if (hrm_status s = cuda_check(c,
                                  cudaMemcpyAsync(dst + (size_t)m * dpitch, src + (size_t)m * spitch,
                                                  sizeof(double) * (size_t)cells, kind, c->stream),
                                  what))
      return s;
  return HRM_OK;
}

hrm_status check_boundaries(hrm_ctx* c) {
  const int missing = c->bnd_need & ~c->bnd_set;
  if (!missing) return HRM_OK;
  for (int b = 0; b < 6; ++b)
    if (missing >> b & 1) return fail(c, HRM_E_INVAL, "Dirichlet side %d has no boundary state (hrm_set_boundary)", b);
  return HRM_OK;
}

// With params.check, a state set by hrm_set / hrm_set_primitive must be
// admissible (Sec. 2); the state stays set either way.
hrm_status check_initial(hrm_ctx* c) {
  if (!c->params.check) return HRM_OK;
  int64_t n[4];
  if (hrm_status s = hrm_admissibility(c, n)) return s;
  if (n[0] | n[1] | n[2] | n[3])
    return fail(c, HRM_E_INVAL,
                "non-admissible initial state: %lld negative partial density, %lld volume fraction out of "
                "[0,1], %lld rho c^2 <= 0, %lld rho e~ <= 0",
                (long long)n[0], (long long)n[1], (long long)n[2], (long long)n[3]);
  return HRM_OK;
}

void reset_step_state(hrm_ctx* c) {
  StepState z{};
  z.cfl = c->params.cfl;
  cudaMemcpyAsync(c->st, &z, sizeof z, cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  c->wn_relaxed = false;
  c->wn_relaxed_dev = 0;
  c->planes_tau = false;
  c->planes_tau_dev = 0;
}

// The host flags of W^n as the next kernels on the stream must see them.
void sync_flag(hrm_ctx* c, bool v, int& dev, int* target) {
  if ((v ? 1 : 0) == dev) return;
  cudaMemsetAsync(target, v ? 1 : 0, sizeof(int), c->stream);  // bytes 0x01: nonzero
  dev = v ? 1 : 0;
}
void sync_relaxed(hrm_ctx* c) {
  sync_flag(c, c->wn_relaxed, c->wn_relaxed_dev, &c->st->wn_relaxed);
  sync_flag(c, c->planes_tau, c->planes_tau_dev, &c->st->planes_tau);
}

// Every write of the state, and every call that runs a primitive pass or
// consumes the CFL maxima outside a step, leaves the planes and maxima to the
// next step's primitive pass: the maxima the last stage accumulated are
// discarded and the device flag cleared at once (stream order).
void planes_stale(hrm_ctx* c) {
  if (c->planes_tau) cudaMemsetAsync(c->st->tau_bits, 0, sizeof c->st->tau_bits, c->stream);
  c->planes_tau = false;
  sync_flag(c, false, c->planes_tau_dev, &c->st->planes_tau);
}


// After a full step: W^n came out of the form's relaxation when the step
// relaxed at its last stage.
bool step_leaves_relaxed(const hrm_ctx* c) { return c->params.relax_mode != HRM_RELAX_OFF; }

}  // namespace

extern "C" {

hrm_status hrm_set_allocator(hrm_alloc_fn alloc, hrm_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return HRM_E_INVAL;
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return HRM_OK;
}

void hrm_params_default(hrm_params* p) {
  std::memset(p, 0, sizeof *p);
  p->cfl = 0.5;
  p->limiters = 1;
  p->blend = 1;
  p->relax_mode = HRM_RELAX_STAGE;
  p->scheme = HRM_SCHEME_WCNS;
  p->integrator = HRM_RK3;
  p->precision = HRM_FP64;
  p->learned = 0;
  p->check = 1;
  p->eps_ar = 1.0e-10;
  p->eps_a = 1.0e-10;
  p->eps_rhoe = 1.0e-8;
  p->hs_ar = 1.0e-11;
  p->hs_a = 1.0e-11;
  p->hs_rc2 = 1.0e-9;
  p->hs_rhoe = 1.0e-9;
  p->weno_eps = 1.0e-15;
  p->Cs = 1.0e12;
  p->q_sensor = 2.0;
  p->learned_threshold = 0.5;
  p->screen = 1;
}

const char* hrm_last_error(const hrm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

hrm_status hrm_create(hrm_ctx** out, const hrm_grid* grid, int32_t N, const double* gamma, const double* p_inf,
                      const double* c_v, const double* q, const hrm_params* params, void* cuda_stream) {
  if (!out) return HRM_E_INVAL;
  *out = nullptr;
  hrm_ctx* c = new (std::nothrow) hrm_ctx();
  if (!c) return HRM_E_NOMEM;
  auto bail = [&](hrm_status s) {
    g_create_error = c->err;  // reachable through hrm_last_error(NULL)
    hrm_destroy(c);
    return s;
  };
  if (!grid || !gamma || !p_inf || !c_v) return bail(fail(c, HRM_E_INVAL, "null argument"));
  if (N < 2 || N > 3) return bail(fail(c, HRM_E_INVAL, "nspecies %d outside 2..3", N));
  const int D = grid->ndim;
  if (D < 1 || D > 3) return bail(fail(c, HRM_E_INVAL, "ndim %d outside 1..3", D));
  int liq = -1;
  for (int k = 0; k < N; ++k) {
    if (!(gamma[k] > 1.0)) return bail(fail(c, HRM_E_INVAL, "gamma[%d] must exceed 1", k));
    if (!(c_v[k] > 0.0)) return bail(fail(c, HRM_E_INVAL, "c_v[%d] must be positive", k));
    if (p_inf[k] < 0.0) return bail(fail(c, HRM_E_INVAL, "p_inf[%d] must be non-negative", k));
    if (p_inf[k] > 0.0) {
      if (liq >= 0) return bail(fail(c, HRM_E_INVAL, "more than one stiffened gas (Sec. 4.2 allows one)"));
      liq = k;
    }
  }
  c->N = N;
  c->D = D;
  c->M = 2 * N + D;
  c->grid = *grid;
  c->nc = 1;
  for (int d = 0; d < 3; ++d) {
    const int64_t n = d < D ? grid->n[d] : 1;
    if (n < 1) return bail(fail(c, HRM_E_INVAL, "n[%d] must be positive", d));
    c->dg.n[d] = n;
    c->nc *= n;
    if (d < D) {
      if (!(grid->hi[d] > grid->lo[d])) return bail(fail(c, HRM_E_INVAL, "empty extent in direction %d", d));
      c->dg.dx[d] = (grid->hi[d] - grid->lo[d]) / (double)n;
      c->dg.inv_dx[d] = 1.0 / c->dg.dx[d];
      for (int side = 0; side < 2; ++side) {
        const int b = grid->bc[2 * d + side];
        if (b != HRM_BC_TRANSMISSIVE && b != HRM_BC_PERIODIC && b != HRM_BC_DIRICHLET)
          return bail(fail(c, HRM_E_INVAL, "unknown boundary condition %d", b));
        c->dg.bc[2 * d + side] = b;
        if (b == HRM_BC_DIRICHLET) c->bnd_need |= 1 << (2 * d + side);
      }
      if ((grid->bc[2 * d] == HRM_BC_PERIODIC) != (grid->bc[2 * d + 1] == HRM_BC_PERIODIC))
        return bail(fail(c, HRM_E_INVAL, "periodic boundaries must pair in direction %d", d));
      if (grid->bc[2 * d] == HRM_BC_PERIODIC && n < 3)
        return bail(fail(c, HRM_E_INVAL, "periodic direction %d needs at least 3 cells", d));
    } else {
      c->dg.dx[d] = 1.0;
      c->dg.inv_dx[d] = 1.0;
    }
  }
  // Dirichlet slices after the interior cells of every plane
  c->nint = c->nc;
  c->dg.nint = c->nint;
  for (int b = 0; b < 2 * D; ++b)
    if (c->bnd_need >> b & 1) {
      c->dg.goff[b] = c->nc;
      c->nc += c->nint / c->dg.n[b / 2];
    }
  c->dg.ncells = c->nc;
  c->fl.liq = liq < 0 ? 0 : liq;
  for (int k = 0; k < N; ++k) {
    c->fl.inv_gm1[k] = 1.0 / (gamma[k] - 1.0);
    c->fl.gpinf_gm1[k] = gamma[k] * p_inf[k] / (gamma[k] - 1.0);
    c->fl.cv[k] = c_v[k];
    c->fl.cp[k] = gamma[k] * c_v[k];
    c->fl.Rg[k] = c->fl.cp[k] - c_v[k];
    c->fl.q[k] = q ? q[k] : 0.0;
    c->fl.pinf[k] = p_inf[k];
    c->fl.gamma[k] = gamma[k];
  }
  fill_fluid_f(c->fl);
  if (params)
    c->params = *params;
  else
    hrm_params_default(&c->params);
  if (hrm_status s = check_params(c, &c->params)) return bail(s);
  fill_dev_params(c);
  c->ck = cell_kernels(N, D);
  c->fk = face_kernels(N, D);
  if (!c->ck || !c->fk) return bail(fail(c, HRM_E_INVAL, "no kernels for N=%d D=%d", N, D));
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = g_alloc;
  c->dealloc = g_free;
  c->alloc_user = g_alloc_user;
  hrm_status s;
  if ((s = cuda_check(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "stream create")))
    return bail(s);
  const size_t plane = sizeof(double) * (size_t)c->nc;
  const int M = c->M;
  if ((s = cuda_check(c, ctx_malloc(c, &c->Wn, plane * M), "alloc W"))) return bail(s);
  if ((s = cuda_check(c, ctx_malloc(c, &c->Ws, plane * M), "alloc Ws"))) return bail(s);
  if ((s = cuda_check(c, ctx_malloc(c, &c->V, plane * M), "alloc V"))) return bail(s);
  if ((s = cuda_check(c, ctx_malloc(c, &c->AUX, plane * 3), "alloc aux"))) return bail(s);
  if ((s = cuda_check(c, ctx_malloc(c, &c->P32, sizeof(float) * (size_t)c->nc * (M + D + 4 + N - 1)), "alloc fp32 planes")))
    return bail(s);
  if ((s = cuda_check(c, ctx_malloc(c, &c->R32, sizeof(float) * (size_t)c->nc * (D + 2)), "alloc fp32 residues")))
    return bail(s);
  for (int d = 0; d < D; ++d) {
    size_t nf = 1;
    for (int e = 0; e < 3; ++e) nf *= (size_t)(c->dg.n[e] + (e == d));
    if ((s = cuda_check(c, ctx_malloc(c, &c->F[d], sizeof(double) * nf * (M + N - 1)), "alloc faces"))) return bail(s);
    if ((int64_t)nf > c->defer_cap) c->defer_cap = (int64_t)nf;
  }
  if ((s = cuda_check(c, ctx_malloc(c, &c->same, (size_t)c->nc), "alloc unchanged-cell flags"))) return bail(s);
  // worklist of the precision form's deferred midpoints (32-bit entries; none
  // beyond 2^32 - 1 midpoints, where the sweep keeps its fallbacks inline)
  if (c->defer_cap < (int64_t)0xffffffffll) {
    if ((s = cuda_check(c, ctx_malloc(c, &c->defer, sizeof(uint32_t) * (size_t)D * (size_t)(c->defer_cap + 1)),
                        "alloc worklist")))
      return bail(s);
    for (int d = 0; d < D; ++d) {
      if ((s = cuda_check(c, cudaStreamCreateWithFlags(&c->side[d], cudaStreamNonBlocking), "side stream")))
        return bail(s);
      if ((s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fast[d], cudaEventDisableTiming), "event")))
        return bail(s);
      if ((s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fix[d], cudaEventDisableTiming), "event")))
        return bail(s);
    }
  } else {
    c->defer_cap = 0;
  }
  if (D > 1) {
    if ((s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event"))) return bail(s);
    for (int d = 1; d < D; ++d) {
      if ((s = cuda_check(c, cudaStreamCreateWithFlags(&c->par[d], cudaStreamNonBlocking), "sweep stream")))
        return bail(s);
      if ((s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_join[d], cudaEventDisableTiming), "event")))
        return bail(s);
    }
  }
  if ((s = cuda_check(c, ctx_malloc(c, &c->st, sizeof(StepState)), "alloc step state"))) return bail(s);
#ifdef HRM_BOUNDS_CHECK
  if ((s = cuda_check(c, ctx_malloc(c, &c->dg.oob, sizeof(unsigned long long)), "alloc bounds counter")))
    return bail(s);
  cudaMemsetAsync(c->dg.oob, 0, sizeof(unsigned long long), c->stream);
#endif
  cudaMemsetAsync(c->Wn, 0, plane * M, c->stream);
  reset_step_state(c);
  if ((s = cuda_check(c, cudaGetLastError(), "init"))) return bail(s);
  *out = c;
  return HRM_OK;
}

void hrm_destroy(hrm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  ctx_free(c, c->Wn);
  ctx_free(c, c->Ws);
  ctx_free(c, c->same);
  ctx_free(c, c->defer);
  ctx_free(c, c->V);
  ctx_free(c, c->AUX);
  ctx_free(c, c->P32);
  ctx_free(c, c->R32);
  for (int d = 0; d < 3; ++d) ctx_free(c, c->F[d]);
  ctx_free(c, c->st);
  ctx_free(c, c->dg.oob);
  ctx_free(c, c->blob);
  for (int d = 0; d < 3; ++d) ctx_free(c, c->gate[d]);
  ctx_free(c, c->p_inst);
  ctx_free(c, c->p_cells);
  ctx_free(c, c->p_tiles);
  ctx_free(c, c->p_sync);
  for (int i = 0; i < 2 * kMaxProf; ++i)
    if (c->prof_ev[i]) cudaEventDestroy(c->prof_ev[i]);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (int d = 0; d < 3; ++d) {
    if (c->par[d]) cudaStreamDestroy(c->par[d]);
    if (c->ev_join[d]) cudaEventDestroy(c->ev_join[d]);
    if (c->side[d]) cudaStreamDestroy(c->side[d]);
    if (c->ev_fast[d]) cudaEventDestroy(c->ev_fast[d]);
    if (c->ev_fix[d]) cudaEventDestroy(c->ev_fix[d]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

hrm_status hrm_set_step_path(hrm_ctx* c, int32_t path) {
  if (!c || (path != 0 && path != 1)) return c ? fail(c, HRM_E_INVAL, "step path must be 0 or 1") : HRM_E_INVAL;
  if (path != c->step_path) {
    drop_graph(c);
    planes_stale(c);
  }
  c->step_path = path;
  return HRM_OK;
}

int32_t hrm_step_launches(const hrm_ctx* c) {
  if (!c) return 0;
  return c->gexec ? (int32_t)c->graph_kernels : 0;
}

hrm_status hrm_set_profiling(hrm_ctx* c, int32_t on) {
  if (!c) return HRM_E_INVAL;
  if (on && !c->prof_ev[0]) {
    for (int i = 0; i < 2 * kMaxProf; ++i) {
      hrm_status s = cuda_check(c, cudaEventCreate(&c->prof_ev[i]), "event create");
      if (s) return s;
    }
  }
  if ((on != 0) != (c->profiling != 0)) drop_graph(c);
  c->profiling = on != 0;
  return HRM_OK;
}

int32_t hrm_profile_read(hrm_ctx* c, int32_t max, float* ms, int32_t* kind) {
  if (!c || !c->profiling || !c->gexec) return 0;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return 0;
  if (c->persist) {
    // phase brackets of the three stage launches from their %globaltimer stamps
    unsigned long long st[3][5];
    if (cudaMemcpy(st, c->p_sync->stamp, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int n = 0;
    auto put = [&](int k, unsigned long long a, unsigned long long b) {
      if (n >= max) return;
      if (ms) ms[n] = b > a ? (float)((double)(b - a) * 1e-6) : 0.f;
      if (kind) kind[n] = k;
      ++n;
    };
    for (int k = 0; k < 3; ++k) {
      if (k == 0) {
        put(HRM_KERNEL_PRIM, st[k][0], st[k][1]);
        put(HRM_KERNEL_FINALIZE, st[k][1], st[k][2]);
      }
      // both directions' midpoints run in one phase
      put(HRM_KERNEL_SWEEPS, st[k][2], st[k][3]);
      put(HRM_KERNEL_FACE_X, st[k][2], st[k][3]);
      put(HRM_KERNEL_FACE_X + 1, st[k][2], st[k][3]);
      put(HRM_KERNEL_UPDATE, st[k][3], st[k][4]);
    }
    return n;
  }
  const int n = c->nprof < max ? c->nprof : max;
  for (int i = 0; i < n; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();  // leave no sticky error for the next call
      return 0;
    }
    if (ms) ms[i] = t;
    if (kind) kind[i] = c->prof_kind[i];
  }
  return n;
}

hrm_status hrm_set_params(hrm_ctx* c, const hrm_params* p) {
  if (!c || !p) return HRM_E_INVAL;
  if (hrm_status s = check_params(c, p)) return s;
  c->params = *p;
  fill_dev_params(c);
  drop_graph(c);
  c->wn_relaxed = false;
  planes_stale(c);
  StepState* st = c->st;
  double cfl = p->cfl;
  cudaMemcpyAsync(&st->cfl, &cfl, sizeof cfl, cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  return last_launch(c, "set params");
}

hrm_status hrm_set(hrm_ctx* c, const double* W, int32_t on_device) {
  Range range("hrm_set");
  if (!c || !W) return HRM_E_INVAL;
  hrm_status s = copy_planes(c, c->Wn, c->nc, W, c->nint, c->nint, c->M,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, "copy W");
  if (s) return s;
  reset_step_state(c);
  if ((s = last_launch(c, "set"))) return s;
  return check_initial(c);
}

hrm_status hrm_set_primitive(hrm_ctx* c, const double* prim, int32_t on_device) {
  Range range("hrm_set_primitive");
  if (!c || !prim) return HRM_E_INVAL;
  hrm_status s = copy_planes(c, c->V, c->nc, prim, c->nint, c->nint, c->N + c->D + 1,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, "copy primitives");
  if (s) return s;
  c->ck->ic(c->V, c->Wn, c->dg, c->fl, 0, c->nint, c->stream);
  ++c->launches;
  if ((s = last_launch(c, "initial state"))) return s;
  reset_step_state(c);
  if ((s = last_launch(c, "set primitive"))) return s;
  return check_initial(c);
}

hrm_status hrm_set_boundary(hrm_ctx* c, int32_t side, const double* values, int32_t primitive,
                            int32_t on_device) {
  Range range("hrm_set_boundary");
  if (!c || !values) return HRM_E_INVAL;
  planes_stale(c);
  if (side < 0 || side >= 2 * c->D || c->dg.bc[side] != HRM_BC_DIRICHLET)
    return fail(c, HRM_E_INVAL, "side %d is not a Dirichlet side", side);
  const int64_t off = c->dg.goff[side], ns = c->nint / c->dg.n[side / 2];
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  hrm_status s;
  if (primitive) {
    if ((s = copy_planes(c, c->V + off, c->nc, values, ns, ns, c->N + c->D + 1, k, "copy boundary primitives")))
      return s;
    c->ck->ic(c->V, c->Wn, c->dg, c->fl, off, off + ns, c->stream);
    ++c->launches;
    if ((s = last_launch(c, "boundary state"))) return s;
  } else if ((s = copy_planes(c, c->Wn + off, c->nc, values, ns, ns, c->M, k, "copy boundary W"))) {
    return s;
  }
  // the RK stage state reads the same slice
  if ((s = copy_planes(c, c->Ws + off, c->nc, c->Wn + off, c->nc, ns, c->M, cudaMemcpyDeviceToDevice,
                       "copy boundary to stage state")))
    return s;
  c->bnd_set |= 1 << side;
  if (!on_device) return cuda_check(c, cudaStreamSynchronize(c->stream), "boundary sync");
  return HRM_OK;
}

hrm_status hrm_dt(hrm_ctx* c, double cfl, double* dt_out, double* tau_out) {
  Range range("hrm_dt");
  if (!c || !(cfl > 0.0)) return c ? fail(c, HRM_E_INVAL, "cfl must be positive") : HRM_E_INVAL;
  planes_stale(c);
  if (hrm_status s = check_boundaries(c)) return s;
  c->ck->prim(c->Wn, c->V, c->AUX, nullptr, nullptr, c->dg, c->fl, c->st, tau_mode(c), nullptr, c->stream);
  launch_finalize(c->st, c->dg, c->D, cfl, 1, c->stream);
  c->launches += 2;
  StepState h;
  hrm_status s = cuda_check(c, cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream), "read dt");
  if (s) return s;
  if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "dt sync"))) return s;
  if (dt_out) *dt_out = h.dt;
  if (tau_out)
    for (int d = 0; d < c->D; ++d) tau_out[d] = h.tau[d];
  return HRM_OK;
}

hrm_status hrm_step(hrm_ctx* c, double dt, int32_t nsteps) {
  Range range("hrm_step");
  if (!c) return HRM_E_INVAL;
  if (nsteps < 0) return fail(c, HRM_E_INVAL, "nsteps must be non-negative");
  if (nsteps == 0) return HRM_OK;
  hrm_status s;
  if ((s = check_boundaries(c))) return s;
  if (!c->gexec && (s = build_graph(c))) return s;
  launch_set_dt(c->st, dt > 0.0 ? dt : 0.0, c->stream);
  ++c->launches;
  // admissibility counters and the tensor-core wait counter that follows them
  if (c->params.check) cudaMemsetAsync(&c->st->counts, 0, 5 * sizeof(unsigned long long), c->stream);
  for (int i = 0; i < nsteps; ++i) {
    sync_relaxed(c);
    if ((s = cuda_check(c, cudaGraphLaunch(c->gexec, c->stream), "graph launch"))) return s;
    c->launches += c->graph_kernels;
    c->wn_relaxed = step_leaves_relaxed(c);
    c->planes_tau = fuse_last(c) && !c->persist;
  }
  if (!c->params.check) return last_launch(c, "step");
  if (c->persist) {
    // the persistent step counts nothing itself: the final state's admissibility,
    // and the grid-barrier waits that ran out
    c->ck->admiss(c->Wn, c->dg, c->fl, c->st, c->stream);
    ++c->launches;
    unsigned int expired = 0;
    if ((s = cuda_check(c, cudaMemcpyAsync(&expired, &c->p_sync->expired, sizeof expired, cudaMemcpyDeviceToHost,
                                           c->stream), "read barrier state")))
      return s;
    if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "step sync"))) return s;
    if (expired != c->p_expired_seen) {
      const unsigned int n = expired - c->p_expired_seen;
      c->p_expired_seen = expired;
      return fail(c, HRM_E_TIMEOUT, "%u grid-barrier waits of the persistent step ran out", n);
    }
  }
  unsigned long long cnt[5];
  static_assert(offsetof(StepState, waits) == offsetof(StepState, counts) + 4 * sizeof(unsigned long long),
                "wait counter follows the admissibility counters");
  if ((s = cuda_check(c, cudaMemcpyAsync(cnt, c->st->counts, sizeof cnt, cudaMemcpyDeviceToHost, c->stream),
                      "read counters")))
    return s;
  if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "step sync"))) return s;
  if (cnt[4])
    return fail(c, HRM_E_TIMEOUT, "%llu tensor-core waits of the learned gate ran out", cnt[4]);
  if (cnt[0] | cnt[1] | cnt[2] | cnt[3])
    return fail(c, HRM_E_ADMISSIBILITY,
                "non-admissible cells: %llu negative partial density, %llu volume fraction out of [0,1], "
                "%llu rho c^2 <= 0, %llu rho e~ <= 0",
                cnt[0], cnt[1], cnt[2], cnt[3]);
  return HRM_OK;
}

// ---------------------------------------------------------------- stepwise stages (domain decomposition)

hrm_status hrm_step_tau(hrm_ctx* c, double* tau) {
  Range range("hrm_step_tau");
  if (!c || !tau) return c ? fail(c, HRM_E_INVAL, "null tau") : HRM_E_INVAL;
  planes_stale(c);
  hrm_status s;
  if ((s = check_boundaries(c))) return s;
  // the primitive kernel of a step's first stage, with its CFL maxima
  if (c->params.precision == HRM_FP32)
    launch_prim32(c->N, c->D, c->Wn, c->P32, r32_target(c), c->dg, c->fl, c->st, tau_mode(c), c->stream);
  else
    c->ck->prim(c->Wn, c->V, c->AUX, p32_target(c), r32_target(c), c->dg, c->fl, c->st, tau_mode(c), nullptr,
                c->stream);
  ++c->launches;
  unsigned long long bits[3] = {0ull, 0ull, 0ull};
  if ((s = cuda_check(c, cudaMemcpyAsync(bits, c->st->tau_bits, sizeof bits, cudaMemcpyDeviceToHost, c->stream),
                      "read tau")))
    return s;
  if ((s = cuda_check(c, cudaMemsetAsync(c->st->tau_bits, 0, sizeof bits, c->stream), "clear tau"))) return s;
  if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "tau sync"))) return s;
  for (int d = 0; d < c->D; ++d) std::memcpy(&tau[d], &bits[d], sizeof(double));
  return HRM_OK;
}

hrm_status hrm_begin_step(hrm_ctx* c, const double* tau, double dt) {
  Range range("hrm_begin_step");
  if (!c || !tau) return c ? fail(c, HRM_E_INVAL, "null tau") : HRM_E_INVAL;
  planes_stale(c);
  unsigned long long bits[3] = {0ull, 0ull, 0ull};
  double sum = 0.0;
  for (int d = 0; d < c->D; ++d) {
    if (!(tau[d] >= 0.0)) return fail(c, HRM_E_INVAL, "tau[%d] must be a non-negative number", d);
    std::memcpy(&bits[d], &tau[d], sizeof(double));
    sum += tau[d];
  }
  if (!(dt > 0.0) && !(sum > 0.0)) return fail(c, HRM_E_INVAL, "no step: dt <= 0 and all tau_d are 0");
  hrm_status s;
  if ((s = cuda_check(c, cudaMemcpyAsync(c->st->tau_bits, bits, sizeof bits, cudaMemcpyHostToDevice, c->stream),
                      "set tau")))
    return s;
  launch_set_dt(c->st, dt > 0.0 ? dt : 0.0, c->stream);
  launch_finalize(c->st, c->dg, c->D, c->params.cfl, 0, c->stream);
  c->launches += 2;
  if ((s = last_launch(c, "begin step"))) return s;
  // host values: the copy above reads the caller's array
  return cuda_check(c, cudaStreamSynchronize(c->stream), "begin step sync");
}

int32_t hrm_stages(const hrm_ctx* c) {
  if (!c) return 0;
  return c->params.integrator == HRM_EULER ? 1 : (c->params.integrator == HRM_RK2 ? 2 : 3);
}

hrm_status hrm_stage(hrm_ctx* c, int32_t stage) {
  Range range("hrm_stage");
  if (!c) return HRM_E_INVAL;
  planes_stale(c);
  const int ns = hrm_stages(c);
  if (stage < 0 || stage >= ns) return fail(c, HRM_E_INVAL, "stage %d outside 0..%d", stage, ns - 1);
  hrm_status s;
  if ((s = check_boundaries(c))) return s;
  const int rs = c->params.relax_mode == HRM_RELAX_STAGE;
  const int rf = c->params.relax_mode != HRM_RELAX_OFF;
  const bool last = stage == ns - 1;
  const double* src = stage == 0 ? c->Wn : c->Ws;
  double* dst = last ? c->Wn : c->Ws;
  double a = 0.0, b = 1.0;
  if (c->params.integrator == HRM_RK2 && stage == 1) a = b = 0.5;
  if (c->params.integrator == HRM_RK3 && stage == 1) {
    a = 0.75;
    b = 0.25;
  }
  if (c->params.integrator == HRM_RK3 && stage == 2) {
    a = 1.0 / 3.0;
    b = 2.0 / 3.0;
  }
  const int prof = c->profiling;
  c->profiling = 0;  // event brackets belong to the captured step graph
  sync_relaxed(c);
  c->launches += enqueue_stage(c, c->stream, src, dst, a, b, last ? rf : rs, 0, false);
  c->profiling = prof;
  if (last) c->wn_relaxed = step_leaves_relaxed(c);
  return last_launch(c, "stage");
}

hrm_status hrm_layers(hrm_ctx* c, int32_t stage, int32_t set, int64_t first, int64_t count, double* buf,
                      int32_t on_device) {
  Range range("hrm_layers");
  if (!c || (!buf && count > 0)) return c ? fail(c, HRM_E_INVAL, "null buffer") : HRM_E_INVAL;
  if (stage < 0 || stage >= hrm_stages(c)) return fail(c, HRM_E_INVAL, "stage %d out of range", stage);
  const int ds = c->D - 1;  // slowest direction
  int64_t layer = 1;
  for (int d = 0; d < ds; ++d) layer *= c->dg.n[d];
  if (first < 0 || count < 0 || first + count > c->dg.n[ds])
    return fail(c, HRM_E_INVAL, "layers %lld..%lld outside 0..%lld", (long long)first, (long long)(first + count),
                (long long)c->dg.n[ds]);
  if (count == 0) return HRM_OK;
  double* state = stage == 0 ? c->Wn : c->Ws;
  const int64_t cells = count * layer, off = first * layer;
  hrm_status s;
  if (set) {
    c->wn_relaxed = false;  // the written cells need not be relaxation output
    planes_stale(c);
  }
  if (set)
    s = copy_planes(c, state + off, c->nc, buf, cells, cells, c->M,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, "set layers");
  else
    s = copy_planes(c, buf, cells, state + off, c->nc, cells, c->M,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, "get layers");
  if (s) return s;
  if (!on_device) return cuda_check(c, cudaStreamSynchronize(c->stream), "layers sync");
  return HRM_OK;
}

hrm_status hrm_relax(hrm_ctx* c) {
  Range range("hrm_relax");
  if (!c) return HRM_E_INVAL;
  c->ck->relax(c->Wn, c->dg, c->fl, c->stream);
  ++c->launches;
  c->wn_relaxed = false;  // (not tracked: in the precision form this is not relax_fast)
  planes_stale(c);
  return last_launch(c, "relax");
}

hrm_status hrm_rhs(hrm_ctx* c, const double* lam, double* rhs) {
  Range range("hrm_rhs");
  if (!c || !lam || !rhs) return HRM_E_INVAL;
  planes_stale(c);
  double l3[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < c->D; ++d) l3[d] = lam[d];
  hrm_status s;
  if ((s = check_boundaries(c))) return s;
  if ((s = cuda_check(c, cudaMemcpyAsync(c->st->lam, l3, sizeof l3, cudaMemcpyHostToDevice, c->stream),
                      "copy lambda")))
    return s;
  // with Dirichlet slices the planes are staged at the stored stride
  double* out = c->nint == c->nc ? rhs : c->Ws;
  if (c->params.precision == HRM_FP32)
    launch_prim32(c->N, c->D, c->Wn, c->P32, r32_target(c), c->dg, c->fl, c->st, 0, c->stream);
  else
    c->ck->prim(c->Wn, c->V, c->AUX, p32_target(c), r32_target(c), c->dg, c->fl, c->st, 0, nullptr, c->stream);
  for (int d = 0; d < c->D; ++d) {
    if (separate_gate(c)) {
      launch_gate(c->N, c->D, d, c->P32, c->R32, c->dg, c->blob, gate_logit_threshold(c), c->gate[d],
                  &c->st->waits, c->gate_blocks, c->stream);
      ++c->launches;
    }
    c->fk->face[d](c->params.precision, c->Wn, c->V, c->AUX, c->P32, c->F[d], c->dg, c->fl, c->dp, c->st,
                   gate_of(c, d), c->stream);
  }
  c->fk->update(1, 0, c->Wn, c->Wn, out, c->F[0], c->F[1], c->F[2], c->dg, c->fl, c->st, 0.0, 1.0, 0, 0,
                nullptr, c->stream);
  c->launches += 2 + c->D * sweep_kernels(c);
  if ((s = last_launch(c, "rhs"))) return s;
  // (the update writes interior cells only: the stage state's slices stay)
  if (out != rhs &&
      (s = copy_planes(c, rhs, c->nint, out, c->nc, c->nint, c->M, cudaMemcpyDeviceToDevice, "copy rhs")))
    return s;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "rhs sync");
}

hrm_status hrm_get(hrm_ctx* c, int32_t field, double* dst, int32_t on_device) {
  Range range("hrm_get");
  if (!c || !dst) return HRM_E_INVAL;
  int planes;
  const double* src;
  switch (field) {
    case HRM_FIELD_W:
      planes = c->M;
      src = c->Wn;
      break;
    case HRM_FIELD_V:
      planes = c->M;
      break;
    case HRM_FIELD_C5:
    case HRM_FIELD_C4:
      planes = 1;
      break;
    case HRM_FIELD_PT:
      planes = 2;
      break;
    case HRM_FIELD_PSI_GAMMA:
      planes = c->N + 1;
      break;
    case HRM_FIELD_ALPHA:
    case HRM_FIELD_Y:
      planes = c->N;
      break;
    case HRM_FIELD_SCHLIEREN:
      planes = 1;
      break;
    default:
      return fail(c, HRM_E_INVAL, "unknown field %d", field);
  }
  if (field != HRM_FIELD_W) {
    c->ck->fields(c->Wn, c->Ws, field, c->dg, c->fl, c->stream);
    ++c->launches;
    src = c->Ws;
  }
  hrm_status s = copy_planes(c, dst, c->nint, src, c->nc, c->nint, planes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, "copy field");
  if (s) return s;
  if (!on_device) return cuda_check(c, cudaStreamSynchronize(c->stream), "get sync");
  return last_launch(c, "get");
}

hrm_status hrm_time(hrm_ctx* c, double* t, int64_t* steps) {
  if (!c) return HRM_E_INVAL;
  StepState h;
  hrm_status s = cuda_check(c, cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream), "read time");
  if (s) return s;
  if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "time sync"))) return s;
  if (t) *t = h.t;
  if (steps) *steps = h.steps;
  return HRM_OK;
}

int64_t hrm_bounds_violations(hrm_ctx* c) {
  if (!c || !c->dg.oob) return -1;
  unsigned long long n = 0;
  if (cudaMemcpyAsync(&n, c->dg.oob, sizeof n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return -1;
  return (int64_t)n;
}

hrm_status hrm_set_time(hrm_ctx* c, double t, int64_t steps) {
  if (!c || steps < 0) return HRM_E_INVAL;
  const long long n = steps;
  hrm_status s;
  if ((s = cuda_check(c, cudaMemcpyAsync(&c->st->t, &t, sizeof t, cudaMemcpyHostToDevice, c->stream), "set time")))
    return s;
  if ((s = cuda_check(c, cudaMemcpyAsync(&c->st->steps, &n, sizeof n, cudaMemcpyHostToDevice, c->stream),
                      "set steps")))
    return s;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "set time sync");
}

hrm_status hrm_admissibility(hrm_ctx* c, int64_t counts[4]) {
  if (!c || !counts) return HRM_E_INVAL;
  cudaMemsetAsync(&c->st->counts, 0, sizeof(c->st->counts), c->stream);
  c->ck->admiss(c->Wn, c->dg, c->fl, c->st, c->stream);
  ++c->launches;
  unsigned long long h[4];
  hrm_status s = cuda_check(c, cudaMemcpyAsync(h, c->st->counts, sizeof h, cudaMemcpyDeviceToHost, c->stream),
                            "read counters");
  if (s) return s;
  if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "admissibility sync"))) return s;
  for (int i = 0; i < 4; ++i) counts[i] = (int64_t)h[i];
  return HRM_OK;
}

int64_t hrm_kernel_launches(const hrm_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"

namespace {
size_t gate_bytes(const hrm_ctx* c, int d) { return (size_t)face_total(c->dg, d); }

hrm_status ensure_gates(hrm_ctx* c) {
  for (int d = 0; d < c->D; ++d) {
    if (c->gate[d]) continue;
    hrm_status s = cuda_check(c, ctx_malloc(c, &c->gate[d], gate_bytes(c, d)), "alloc gate");
    if (s) return s;
    cudaMemsetAsync(c->gate[d], 0, gate_bytes(c, d), c->stream);
  }
  return HRM_OK;
}
}  // namespace

extern "C" {

hrm_status hrm_set_detector(hrm_ctx* c, const hrm_detector* det) {
  if (!c || !det || !detector_blob(det)) return c ? fail(c, HRM_E_INVAL, "null detector") : HRM_E_INVAL;
  hrm_status s;
  if (!c->blob && (s = cuda_check(c, ctx_malloc(c, &c->blob, sizeof(mlp::GateBlob)), "alloc gate weights")))
    return s;
  if ((s = ensure_gates(c))) return s;
  // the detector's weights are final once its own stream has drained
  if ((s = cuda_check(c, cudaDeviceSynchronize(), "detector sync"))) return s;
  if ((s = cuda_check(c,
                      cudaMemcpyAsync(c->blob, detector_blob(det), sizeof(mlp::GateBlob), cudaMemcpyDeviceToDevice,
                                      c->stream),
                      "copy gate weights")))
    return s;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->gate_blocks = (sms > 0 ? sms : 1) * 8;
  drop_graph(c);
  return cuda_check(c, cudaStreamSynchronize(c->stream), "set detector");
}

hrm_status hrm_set_gate(hrm_ctx* c, int32_t dir, const uint8_t* gate) {
  if (!c || !gate) return HRM_E_INVAL;
  if (dir < 0 || dir >= c->D) return fail(c, HRM_E_INVAL, "direction %d outside 0..%d", dir, c->D - 1);
  hrm_status s;
  if ((s = ensure_gates(c))) return s;
  if ((s = cuda_check(c, cudaMemcpyAsync(c->gate[dir], gate, gate_bytes(c, dir), cudaMemcpyHostToDevice, c->stream),
                      "copy gate")))
    return s;
  c->gate_set[dir] = 1;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "set gate");
}

hrm_status hrm_get_gate(hrm_ctx* c, int32_t dir, uint8_t* gate) {
  if (!c || !gate) return HRM_E_INVAL;
  if (dir < 0 || dir >= c->D) return fail(c, HRM_E_INVAL, "direction %d outside 0..%d", dir, c->D - 1);
  if (!c->gate[dir]) return fail(c, HRM_E_INVAL, "no gate on this context");
  hrm_status s = cuda_check(
      c, cudaMemcpyAsync(gate, c->gate[dir], gate_bytes(c, dir), cudaMemcpyDeviceToHost, c->stream), "read gate");
  if (s) return s;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "get gate");
}

}  // extern "C"

namespace hrm {
void set_thread_error(const char* msg) { g_create_error = msg; }

hrm_status ctx_view(hrm_ctx* c, CtxView* v) {
  if (!c || !v) return HRM_E_INVAL;
  v->N = c->N;
  v->D = c->D;
  v->M = c->M;
  v->nc = c->nc;
  v->dg = c->dg;
  v->fl = c->fl;
  v->dp = c->dp;
  v->Wn = c->Wn;
  v->V = c->V;
  v->AUX = c->AUX;
  v->P32 = c->P32;
  v->R32 = c->R32;
  v->st = c->st;
  v->ck = c->ck;
  v->stream = c->stream;
  return HRM_OK;
}

void ctx_add_launches(hrm_ctx* c, int64_t n) {
  if (c) c->launches += n;
}

const FaceKernels* face_kernels(int N, int D) {
  if (D == 1) return face_kernels_d1(N);
  if (D == 2) return face_kernels_d2(N);
  if (D == 3) return face_kernels_d3(N);
  return nullptr;
}
}  // namespace hrm

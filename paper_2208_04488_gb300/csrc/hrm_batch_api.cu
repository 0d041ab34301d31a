// C ABI of the batched form (include/hrm.h, hrm_batch_*): many independent 2D
// problems of uneven size advanced together, one persistent cooperative launch
// per RK stage and one captured CUDA graph per step; the launch shape picked by
// an autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/hrm.h"
#include "hrm_batch.cuh"
#include "hrm_launch.h"

using namespace hrm;

namespace {

struct Shape {
  int cell_tile = 4096;   // cells per work item of the per-cell phases
  int blocks_per_sm = 0;  // persistent grid = SMs x blocks_per_sm (0: all that fit)
};

// Time limit of one grid-barrier wait of the persistent kernel: far above any
// phase's duration, so that only a barrier that cannot complete runs out.
constexpr uint64_t kBarrierLimitNs = 2000000000ull;

}  // namespace

struct hrm_batch {
  int ninst = 0, D = 2;
  hrm_params params{};
  DevParams dp{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<BatchInst> host;   // per-instance description (device pointers)
  std::vector<int> N;
  BatchInst* d_insts = nullptr;
  WorkItem* d_cells = nullptr;   // cell work items, grouped by species count
  int ncell_items = 0;
  WorkItem* d_tiles = nullptr;   // 128-midpoint tiles, grouped by species count and direction (in pad)
  int ntiles = 0;
  GridSync* sync = nullptr;      // queues and barrier of the persistent launches
  unsigned int expired_seen = 0; // barrier waits that ran out, as last reported
  Shape shape;
  int sms = 0;
  int fit = 0;                   // resident blocks per SM of the persistent kernel
  bool direct = false;           // launches not captured into a graph (capture refused)
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_kernels = 0;
  int64_t launches = 0;
  int64_t total_cells = 0;
  // per instance: W^n came out of the form's relaxation (StepState::wn_relaxed;
  // the updates take the relaxation's result from W^n for unchanged cells only
  // then), and the value last written to the device
  std::vector<char> relaxed, relaxed_dev;
  std::string err;
};

namespace {

thread_local std::string g_batch_create_error = "null batch";

hrm_status bfail(hrm_batch* b, hrm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return s;
}

hrm_status bcuda(hrm_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HRM_OK;
  return bfail(b, e == cudaErrorMemoryAllocation ? HRM_E_NOMEM : HRM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void drop_graph(hrm_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_kernels = 0;
}

// Work items: every instance's cells in chunks of cell_tile, grouped by species
// count; tiles of 128 midpoints of every instance and direction, grouped by
// species count and direction (the direction in WorkItem::pad). No item spans
// two instances.
hrm_status build_items(hrm_batch* b) {
  std::vector<WorkItem> cells, tiles;
  for (int gN = 2; gN <= 3; ++gN)
    for (int i = 0; i < b->ninst; ++i) {
      if (b->N[i] != gN) continue;
      const DevGrid& g = b->host[i].g;
      for (int64_t c = 0; c < g.ncells; c += b->shape.cell_tile)
        cells.push_back({i, 0, c, std::min<int64_t>(c + b->shape.cell_tile, g.ncells)});
    }
  for (int gN = 2; gN <= 3; ++gN)
    for (int d = 0; d < 2; ++d)
      for (int i = 0; i < b->ninst; ++i) {
        if (b->N[i] != gN) continue;
        const DevGrid& g = b->host[i].g;
        const int64_t nf = (g.n[0] + (d == 0)) * (g.n[1] + (d == 1)) * g.n[2];
        for (int64_t t = 0; t < nf; t += kBatchFace32Threads)
          tiles.push_back({i, d, t, std::min<int64_t>(t + kBatchFace32Threads, nf)});
      }
  cudaFree(b->d_cells);
  cudaFree(b->d_tiles);
  b->d_cells = nullptr;
  b->d_tiles = nullptr;
  hrm_status s;
  if ((s = bcuda(b, cudaMalloc(&b->d_cells, sizeof(WorkItem) * cells.size()), "alloc work items"))) return s;
  if ((s = bcuda(b, cudaMalloc(&b->d_tiles, sizeof(WorkItem) * tiles.size()), "alloc tiles"))) return s;
  if ((s = bcuda(b, cudaMemcpy(b->d_cells, cells.data(), sizeof(WorkItem) * cells.size(), cudaMemcpyHostToDevice),
                 "copy work items")))
    return s;
  if ((s = bcuda(b, cudaMemcpy(b->d_tiles, tiles.data(), sizeof(WorkItem) * tiles.size(), cudaMemcpyHostToDevice),
                 "copy tiles")))
    return s;
  b->ncell_items = (int)cells.size();
  b->ntiles = (int)tiles.size();
  drop_graph(b);
  return HRM_OK;
}

int grid_blocks(const hrm_batch* b) {
  const int per_sm = b->shape.blocks_per_sm > 0 ? std::min(b->shape.blocks_per_sm, b->fit) : b->fit;
  return b->sms * per_sm;
}

// One RK stage: reset the phase queues and the barrier count, then the
// persistent launch (SSP-RK3 in Shu-Osher form; src/dst 0 = W^n, 1 = stage state).
hrm_status enqueue_stage(hrm_batch* b, cudaStream_t s, int stage) {
  const bool fp32 = b->params.precision == HRM_FP32;
  const int rs = b->params.relax_mode == HRM_RELAX_STAGE;
  const int rf = b->params.relax_mode != HRM_RELAX_OFF;
  StageArgs A{};
  A.insts = b->d_insts;
  A.cells = b->d_cells;
  A.tiles = b->d_tiles;
  A.ncell_items = b->ncell_items;
  A.ntiles = b->ntiles;
  A.ninst = b->ninst;
  A.src = stage == 0 ? 0 : 1;
  A.dst = stage == 2 ? 0 : 1;
  A.a = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
  A.b = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
  A.relax = stage == 2 ? rf : rs;
  A.first = stage == 0;
  // precision form: the updates of stages 1 and 2 write the next stage's FP32 planes
  A.prim = (!fp32 || stage == 0) ? 1 : 0;
  A.fuse_next = fp32 && stage < 2 ? 1 : 0;
  A.cfl = b->params.cfl;
  A.pr = b->dp;
  A.sync = b->sync;
  A.limit_ns = kBarrierLimitNs;
  A.stage = stage;
  A.update = 1;
  hrm_status st;
  if ((st = bcuda(b, cudaMemsetAsync(b->sync, 0, kResetWords * sizeof(unsigned int), s), "reset queues"))) return st;
  const cudaError_t e = fp32 ? batch_stage32_launch(grid_blocks(b), A, s) : batch_stage64_launch(grid_blocks(b), A, s);
  return bcuda(b, e, "persistent stage launch");
}

hrm_status enqueue_step(hrm_batch* b, cudaStream_t s) {
  for (int k = 0; k < 3; ++k)
    if (hrm_status st = enqueue_stage(b, s, k)) return st;
  return HRM_OK;
}

// One graph per step with the three stage launches; where capturing a
// cooperative launch is refused, the stages are launched directly.
hrm_status build_graph(hrm_batch* b) {
  drop_graph(b);
  b->graph_kernels = 3;
  if (b->direct) return HRM_OK;
  cudaGraph_t g = nullptr;
  hrm_status s = bcuda(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (s) return s;
  const hrm_status se = enqueue_step(b, b->cap);
  const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (se || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    b->direct = true;
    return HRM_OK;
  }
  cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->gexec = nullptr;
    b->direct = true;
  }
  return HRM_OK;
}

hrm_status launch_step(hrm_batch* b) {
  if (b->direct) return enqueue_step(b, b->stream);
  return bcuda(b, cudaGraphLaunch(b->gexec, b->stream), "graph launch");
}

void reset_instance(hrm_batch* b, int i) {
  StepState z{};
  z.cfl = b->params.cfl;
  cudaMemcpyAsync(b->host[i].st, &z, sizeof z, cudaMemcpyHostToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  if ((int)b->relaxed.size() > i) b->relaxed[i] = b->relaxed_dev[i] = 0;
}

// The relaxed-state flags as the next step's kernels must see them.
void sync_relaxed(hrm_batch* b) {
  for (int i = 0; i < b->ninst; ++i)
    if (b->relaxed[i] != b->relaxed_dev[i]) {
      cudaMemsetAsync(&b->host[i].st->wn_relaxed, b->relaxed[i] ? 1 : 0, sizeof(int), b->stream);
      b->relaxed_dev[i] = b->relaxed[i];
    }
}

}  // namespace

extern "C" {

const char* hrm_batch_last_error(const hrm_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void hrm_batch_destroy(hrm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& I : b->host) {
    cudaFree(I.Wn);
    cudaFree(I.Ws);
    cudaFree(I.V);
    cudaFree(I.AUX);
    cudaFree(I.P32);
    for (int d = 0; d < 3; ++d) cudaFree(I.F[d]);
    cudaFree(I.st);
  }
  cudaFree(b->d_insts);
  cudaFree(b->d_cells);
  cudaFree(b->d_tiles);
  cudaFree(b->sync);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

hrm_status hrm_batch_create(hrm_batch** out, int32_t ninst, const hrm_instance* inst, const hrm_params* params,
                            void* cuda_stream) {
  if (!out) return HRM_E_INVAL;
  *out = nullptr;
  hrm_batch* b = new (std::nothrow) hrm_batch();
  if (!b) return HRM_E_NOMEM;
  auto bail = [&](hrm_status s) {
    g_batch_create_error = b->err;
    hrm_batch_destroy(b);
    return s;
  };
  if (!inst || ninst < 1) return bail(bfail(b, HRM_E_INVAL, "need at least one instance"));
  if (params)
    b->params = *params;
  else
    hrm_params_default(&b->params);
  const hrm_params& p = b->params;
  if (!(p.weno_eps > 0.0 && p.weno_eps <= 1e50)) return bail(bfail(b, HRM_E_INVAL, "weno_eps must lie in (0, 1e50]"));
  if (p.cfl <= 0.0 || (p.limiters && p.cfl > 0.5))
    return bail(bfail(b, HRM_E_INVAL, "cfl must be in (0, 0.5] with the limiters on (Sec. 4.1.2)"));
  if (p.scheme != HRM_SCHEME_WCNS || p.integrator != HRM_RK3 || p.learned || p.precision < 0 || p.precision > 1 ||
      p.relax_mode < 0 || p.relax_mode > 2 || p.cfl_sound != 0)
    return bail(bfail(b, HRM_E_INVAL,
                      "batched form: PP-WCNS-IS with SSP-RK3, FP64 or FP32 precision, five-equation CFL speed only"));
  b->dp.limiters = p.limiters;
  b->dp.blend = p.blend;
  b->dp.scheme = p.scheme;
  b->dp.qexp = (int)p.q_sensor;
  b->dp.eps_ar = p.eps_ar;
  b->dp.eps_a = p.eps_a;
  b->dp.eps_rhoe = p.eps_rhoe;
  b->dp.hs_ar = p.hs_ar;
  b->dp.hs_a = p.hs_a;
  b->dp.hs_rc2 = p.hs_rc2;
  b->dp.hs_rhoe = p.hs_rhoe;
  b->dp.weno_eps = p.weno_eps;
  b->dp.Cs = p.Cs;
  fill_screen(b->dp, p.screen);
  b->ninst = ninst;
  b->stream = (cudaStream_t)cuda_stream;
  hrm_status s;
  if ((s = bcuda(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "stream create"))) return bail(s);
  int dev = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return bail(bfail(b, HRM_E_CUDA, "the device does not support cooperative launches"));
  b->fit = p.precision == HRM_FP32 ? batch_stage32_fit() : batch_stage64_fit();
  if (b->fit < 1) return bail(bfail(b, HRM_E_CUDA, "persistent stage kernel: no resident block fits an SM"));
  if ((s = bcuda(b, cudaMalloc(&b->sync, sizeof(GridSync)), "alloc grid sync"))) return bail(s);
  if ((s = bcuda(b, cudaMemset(b->sync, 0, sizeof(GridSync)), "clear grid sync"))) return bail(s);
  b->host.resize(ninst);
  b->N.resize(ninst);
  b->relaxed.assign(ninst, 0);
  b->relaxed_dev.assign(ninst, 0);
  for (int i = 0; i < ninst; ++i) {
    const hrm_instance& in = inst[i];
    BatchInst& I = b->host[i];
    std::memset(&I, 0, sizeof I);
    const int N = in.nspecies;
    if (N < 2 || N > 3) return bail(bfail(b, HRM_E_INVAL, "instance %d: nspecies outside 2..3", i));
    if (in.grid.ndim != 2) return bail(bfail(b, HRM_E_INVAL, "instance %d: the batched form is 2D", i));
    int liq = -1;
    for (int k = 0; k < N; ++k) {
      if (!(in.gamma[k] > 1.0) || !(in.c_v[k] > 0.0) || in.p_inf[k] < 0.0)
        return bail(bfail(b, HRM_E_INVAL, "instance %d: invalid species table", i));
      if (in.p_inf[k] > 0.0) {
        if (liq >= 0) return bail(bfail(b, HRM_E_INVAL, "instance %d: more than one stiffened gas", i));
        liq = k;
      }
      I.f.inv_gm1[k] = 1.0 / (in.gamma[k] - 1.0);
      I.f.gpinf_gm1[k] = in.gamma[k] * in.p_inf[k] / (in.gamma[k] - 1.0);
      I.f.cv[k] = in.c_v[k];
      I.f.cp[k] = in.gamma[k] * in.c_v[k];
      I.f.Rg[k] = I.f.cp[k] - in.c_v[k];
      I.f.q[k] = in.q[k];
      I.f.pinf[k] = in.p_inf[k];
      I.f.gamma[k] = in.gamma[k];
    }
    I.f.liq = liq < 0 ? 0 : liq;
    fill_fluid_f(I.f);
    I.N = N;
    b->N[i] = N;
    I.g.oob = nullptr;
    I.g.ncells = 1;
    for (int d = 0; d < 3; ++d) {
      const int64_t n = d < 2 ? in.grid.n[d] : 1;
      if (n < 1) return bail(bfail(b, HRM_E_INVAL, "instance %d: empty grid", i));
      I.g.n[d] = n;
      I.g.ncells *= n;
      if (d < 2) {
        if (!(in.grid.hi[d] > in.grid.lo[d])) return bail(bfail(b, HRM_E_INVAL, "instance %d: empty extent", i));
        I.g.dx[d] = (in.grid.hi[d] - in.grid.lo[d]) / (double)n;
        I.g.inv_dx[d] = 1.0 / I.g.dx[d];
        for (int side = 0; side < 2; ++side) {
          const int bc = in.grid.bc[2 * d + side];
          if (bc != HRM_BC_TRANSMISSIVE && bc != HRM_BC_PERIODIC)
            return bail(bfail(b, HRM_E_INVAL, "instance %d: unknown boundary condition", i));
          I.g.bc[2 * d + side] = bc;
        }
        if ((I.g.bc[2 * d] == HRM_BC_PERIODIC) != (I.g.bc[2 * d + 1] == HRM_BC_PERIODIC) ||
            (I.g.bc[2 * d] == HRM_BC_PERIODIC && n < 3))
          return bail(bfail(b, HRM_E_INVAL, "instance %d: invalid periodic direction", i));
      } else {
        I.g.dx[d] = 1.0;
        I.g.inv_dx[d] = 1.0;
      }
    }
    I.g.nint = I.g.ncells;
    const int M = 2 * N + 2;
    const size_t plane = sizeof(double) * (size_t)I.g.ncells;
    b->total_cells += I.g.ncells;
    if ((s = bcuda(b, cudaMalloc(&I.Wn, plane * M), "alloc W"))) return bail(s);
    if ((s = bcuda(b, cudaMalloc(&I.Ws, plane * M), "alloc Ws"))) return bail(s);
    if ((s = bcuda(b, cudaMalloc(&I.V, plane * M), "alloc V"))) return bail(s);
    if ((s = bcuda(b, cudaMalloc(&I.AUX, plane * 3), "alloc aux"))) return bail(s);
    if ((s = bcuda(b, cudaMalloc(&I.P32, sizeof(float) * (size_t)I.g.ncells * (M + 2 + 4 + N - 1)), "alloc P32")))
      return bail(s);
    for (int d = 0; d < 2; ++d) {
      const size_t nf = (size_t)((I.g.n[0] + (d == 0)) * (I.g.n[1] + (d == 1)));
      if ((s = bcuda(b, cudaMalloc(&I.F[d], sizeof(double) * nf * (M + N - 1)), "alloc faces"))) return bail(s);
    }
    if ((s = bcuda(b, cudaMalloc(&I.st, sizeof(StepState)), "alloc step state"))) return bail(s);
    cudaMemsetAsync(I.Wn, 0, plane * M, b->stream);
    reset_instance(b, i);
  }
  if ((s = bcuda(b, cudaMalloc(&b->d_insts, sizeof(BatchInst) * ninst), "alloc instances"))) return bail(s);
  if ((s = bcuda(b, cudaMemcpy(b->d_insts, b->host.data(), sizeof(BatchInst) * ninst, cudaMemcpyHostToDevice),
                 "copy instances")))
    return bail(s);
  if ((s = build_items(b))) return bail(s);
  *out = b;
  return HRM_OK;
}

static hrm_status check_inst(hrm_batch* b, int32_t i) {
  if (!b) return HRM_E_INVAL;
  if (i < 0 || i >= b->ninst) return bfail(b, HRM_E_INVAL, "instance %d out of range", i);
  return HRM_OK;
}

hrm_status hrm_batch_set_primitive(hrm_batch* b, int32_t i, const double* prim, int32_t on_device) {
  if (hrm_status s = check_inst(b, i)) return s;
  if (!prim) return bfail(b, HRM_E_INVAL, "null primitives");
  BatchInst& I = b->host[i];
  const int N = b->N[i];
  const size_t bytes = sizeof(double) * (size_t)I.g.ncells * (N + 2 + 1);
  hrm_status s = bcuda(b, cudaMemcpyAsync(I.V, prim, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                          b->stream), "copy primitives");
  if (s) return s;
  cell_kernels(N, 2)->ic(I.V, I.Wn, I.g, I.f, 0, I.g.nint, b->stream);
  ++b->launches;
  reset_instance(b, i);
  return bcuda(b, cudaGetLastError(), "initial state");
}

hrm_status hrm_batch_set(hrm_batch* b, int32_t i, const double* W, int32_t on_device) {
  if (hrm_status s = check_inst(b, i)) return s;
  if (!W) return bfail(b, HRM_E_INVAL, "null state");
  BatchInst& I = b->host[i];
  const size_t bytes = sizeof(double) * (size_t)I.g.ncells * (2 * b->N[i] + 2);
  hrm_status s = bcuda(b, cudaMemcpyAsync(I.Wn, W, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                          b->stream), "copy state");
  if (s) return s;
  reset_instance(b, i);
  return HRM_OK;
}

hrm_status hrm_batch_get(hrm_batch* b, int32_t i, double* dst, int32_t on_device) {
  if (hrm_status s = check_inst(b, i)) return s;
  if (!dst) return bfail(b, HRM_E_INVAL, "null destination");
  BatchInst& I = b->host[i];
  const size_t bytes = sizeof(double) * (size_t)I.g.ncells * (2 * b->N[i] + 2);
  hrm_status s = bcuda(b, cudaMemcpyAsync(dst, I.Wn, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                          b->stream), "copy state");
  if (s) return s;
  if (!on_device) return bcuda(b, cudaStreamSynchronize(b->stream), "get sync");
  return HRM_OK;
}

hrm_status hrm_batch_step(hrm_batch* b, int32_t nsteps) {
  if (!b) return HRM_E_INVAL;
  if (nsteps < 0) return bfail(b, HRM_E_INVAL, "nsteps must be non-negative");
  if (nsteps == 0) return HRM_OK;
  hrm_status s;
  if (!b->gexec && !b->direct && (s = build_graph(b))) return s;
  const char after = b->params.relax_mode != HRM_RELAX_OFF;
  for (int i = 0; i < nsteps; ++i) {
    sync_relaxed(b);
    if ((s = launch_step(b))) return s;
    b->launches += b->graph_kernels;
    std::fill(b->relaxed.begin(), b->relaxed.end(), after);
  }
  if (!b->params.check) return bcuda(b, cudaGetLastError(), "batch step");
  unsigned int expired = 0;
  if ((s = bcuda(b, cudaMemcpyAsync(&expired, &b->sync->expired, sizeof expired, cudaMemcpyDeviceToHost, b->stream),
                 "read barrier state")))
    return s;
  if ((s = bcuda(b, cudaStreamSynchronize(b->stream), "batch step sync"))) return s;
  if (expired != b->expired_seen) {
    const unsigned int n = expired - b->expired_seen;
    b->expired_seen = expired;
    return bfail(b, HRM_E_TIMEOUT, "%u grid-barrier waits of the persistent stage kernel ran out", n);
  }
  int64_t c[4];
  if ((s = hrm_batch_admissibility(b, c))) return s;
  if (c[0] | c[1] | c[2] | c[3])
    return bfail(b, HRM_E_ADMISSIBILITY, "non-admissible cells: %lld %lld %lld %lld", (long long)c[0],
                 (long long)c[1], (long long)c[2], (long long)c[3]);
  return HRM_OK;
}

hrm_status hrm_batch_time(hrm_batch* b, int32_t i, double* t, int64_t* steps) {
  if (hrm_status s = check_inst(b, i)) return s;
  StepState h;
  hrm_status s = bcuda(b, cudaMemcpyAsync(&h, b->host[i].st, sizeof h, cudaMemcpyDeviceToHost, b->stream), "time");
  if (s) return s;
  if ((s = bcuda(b, cudaStreamSynchronize(b->stream), "time sync"))) return s;
  if (t) *t = h.t;
  if (steps) *steps = h.steps;
  return HRM_OK;
}

hrm_status hrm_batch_admissibility(hrm_batch* b, int64_t counts[4]) {
  if (!b || !counts) return HRM_E_INVAL;
  for (int k = 0; k < 4; ++k) counts[k] = 0;
  for (int i = 0; i < b->ninst; ++i) {
    BatchInst& I = b->host[i];
    cudaMemsetAsync(&I.st->counts, 0, sizeof(I.st->counts), b->stream);
    cell_kernels(b->N[i], 2)->admiss(I.Wn, I.g, I.f, I.st, b->stream);
    ++b->launches;
    unsigned long long h[4];
    hrm_status s = bcuda(b, cudaMemcpyAsync(h, I.st->counts, sizeof h, cudaMemcpyDeviceToHost, b->stream), "counters");
    if (s) return s;
    if ((s = bcuda(b, cudaStreamSynchronize(b->stream), "counters sync"))) return s;
    for (int k = 0; k < 4; ++k) counts[k] += (int64_t)h[k];
  }
  return HRM_OK;
}

hrm_status hrm_batch_set_launch(hrm_batch* b, int32_t face_threads, int32_t face_tile, int32_t cell_tile,
                                int32_t blocks_per_sm) {
  if (!b) return HRM_E_INVAL;
  (void)face_threads;
  (void)face_tile;
  if (cell_tile < 256 || blocks_per_sm < 0 || blocks_per_sm > 32) return bfail(b, HRM_E_INVAL, "invalid launch shape");
  b->shape.cell_tile = cell_tile;
  b->shape.blocks_per_sm = blocks_per_sm;
  return build_items(b);
}

hrm_status hrm_batch_tune(hrm_batch* b, int32_t steps_per_trial, int32_t* best) {
  if (!b || steps_per_trial < 1) return HRM_E_INVAL;
  // save the states: tuning advances them
  std::vector<double*> saved(b->ninst, nullptr);
  std::vector<StepState> saved_st(b->ninst);
  hrm_status s = HRM_OK;
  for (int i = 0; i < b->ninst && !s; ++i) {
    const size_t bytes = sizeof(double) * (size_t)b->host[i].g.ncells * (2 * b->N[i] + 2);
    s = bcuda(b, cudaMalloc(&saved[i], bytes), "alloc tuning copy");
    if (!s) s = bcuda(b, cudaMemcpyAsync(saved[i], b->host[i].Wn, bytes, cudaMemcpyDeviceToDevice, b->stream), "save");
    if (!s) s = bcuda(b, cudaMemcpyAsync(&saved_st[i], b->host[i].st, sizeof(StepState), cudaMemcpyDeviceToHost,
                                         b->stream), "save step state");
  }
  if (!s) s = bcuda(b, cudaStreamSynchronize(b->stream), "save sync");
  const int tiles[] = {1024, 4096, 16384};  // cells per work item
  float best_ms = 1e30f;
  Shape best_shape = b->shape;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int tl : tiles)
    for (int bp = 1; bp <= b->fit; ++bp) {
      if (s) break;
      if ((s = hrm_batch_set_launch(b, kBatchFace32Threads, kBatchFace32Threads, tl, bp))) break;
      if ((s = build_graph(b))) break;
      if ((s = launch_step(b))) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < steps_per_trial && !s; ++k) s = launch_step(b);
      cudaEventRecord(e1, b->stream);
      if (s || (s = bcuda(b, cudaEventSynchronize(e1), "tuning trial"))) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      b->launches += b->graph_kernels * (steps_per_trial + 1);
      if (ms < best_ms) {
        best_ms = ms;
        best_shape = b->shape;
      }
      // restore the states for the next trial
      for (int i = 0; i < b->ninst; ++i) {
        const size_t bytes = sizeof(double) * (size_t)b->host[i].g.ncells * (2 * b->N[i] + 2);
        cudaMemcpyAsync(b->host[i].Wn, saved[i], bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(b->host[i].st, &saved_st[i], sizeof(StepState), cudaMemcpyHostToDevice, b->stream);
      }
      cudaStreamSynchronize(b->stream);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (double* p : saved) cudaFree(p);
  if (s) return s;
  b->shape = best_shape;
  if ((s = build_items(b))) return s;
  if (best) {
    best[0] = kBatchFace32Threads;
    best[1] = kBatchFace32Threads;
    best[2] = best_shape.cell_tile;
    best[3] = best_shape.blocks_per_sm;
  }
  return HRM_OK;
}

int64_t hrm_batch_kernel_launches(const hrm_batch* b) { return b ? b->launches : 0; }

int64_t hrm_batch_total_cells(const hrm_batch* b) { return b ? b->total_cells : 0; }

}  // extern "C"

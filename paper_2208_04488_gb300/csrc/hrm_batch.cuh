// Batched form: many independent problems of uneven size advanced together,
// one persistent launch per RK stage for all of them. Blocks take work items
// (instance, element range) from queues; every item lies inside one instance,
// so the per-element bodies are exactly those of the single-instance kernels
// and a batched instance reproduces its own context bit for bit.
#pragma once

#include "hrm_cell.cuh"
#include "hrm_face32.cuh"
#include "hrm_sync.cuh"

namespace hrm {

// Device-side description of one instance.
struct BatchInst {
  DevGrid g;
  DevFluid f;
  int32_t N;
  int32_t pad;
  double* Wn;
  double* Ws;
  double* V;
  double* AUX;
  double* F[3];
  float* P32;
  StepState* st;
};

// A contiguous range [begin, end) of cells or faces of one instance.
struct WorkItem {
  int32_t inst;
  int32_t pad;
  int64_t begin;
  int64_t end;
};

__device__ __forceinline__ const double* pick(const BatchInst& I, int sel) { return sel == 0 ? I.Wn : I.Ws; }
__device__ __forceinline__ double* pick_mut(const BatchInst& I, int sel) { return sel == 0 ? I.Wn : I.Ws; }

constexpr int kBatchFace32Threads = 128;  // threads of the persistent kernel: one per midpoint of a tile

// ---------------------------------------------------------------- persistent stage kernel
// One launch per RK stage for every instance: the primitive phase, at the first
// stage the step scalars of every instance, the midpoint phase over
// 128-midpoint tiles of both directions, the update phase -- separated by the
// bounded grid barrier of hrm_sync.cuh. Blocks take work items from one queue
// per phase; the cell items are grouped by species count and the tiles by
// species count and direction, so that neighbouring items run the same code.
// Every element goes through the single-context body, so an instance
// reproduces its own context bit for bit (FP64), and the precision form's
// rounding is the single context's too (its units are built without FMA
// contraction). All data written in one phase and read in a later one is
// reached through the instance table, never through a read-only kernel
// argument.

struct StageArgs {
  const BatchInst* insts;
  const WorkItem* cells;  // cell work items
  const WorkItem* tiles;  // 128-midpoint tiles, the direction in WorkItem::pad
  int ncell_items, ntiles, ninst;
  int src, dst;           // 0: W^n, 1: the stage state
  double a, b;            // W_dst = a W^n + b (W_src + dt RHS)
  int relax;
  int prim;               // 1: primitive phase (0: the previous stage's update wrote the FP32 planes)
  int first;              // 1: CFL maxima in the primitive phase, then the step scalars
  int fuse_next;          // precision form: the update writes the next stage's FP32 planes
  double cfl;
  DevParams pr;
  GridSync* sync;
  uint64_t limit_ns;      // time limit of one barrier wait
  int stage;              // 0..2: slot of the phase stamps
  int update;             // 1: the update phase runs in this launch (0: the caller runs it after)
};

// Step scalars of instance I from its CFL maxima (as k_finalize: a requested
// step dt_req > 0 is taken as it is).
template <int D>
__device__ __forceinline__ void batch_finalize_inst(const BatchInst& I, double cfl) {
  StepState* st = I.st;
  double tau[3] = {0.0, 0.0, 0.0}, sum = 0.0;
  for (int d = 0; d < D; ++d) {
    tau[d] = __longlong_as_double((long long)st->tau_bits[d]);
    sum = sum + tau[d];
    st->tau_bits[d] = 0ull;
  }
  const double dt = st->dt_req > 0.0 ? st->dt_req : cfl / sum;
  for (int d = 0; d < D; ++d) {
    const double sigma = tau[d] / sum;
    st->lam[d] = dt / (sigma * I.g.dx[d]);
    st->tau[d] = tau[d];
  }
  st->dt = dt;
  st->t = st->t + dt;
  st->steps = st->steps + 1;
}

// The full precision-form midpoint (FP64 limiters where a screen fails), out
// of line: rarely taken, and kept out of the persistent kernel's hot code.
template <int N, int D, int DIR>
__device__ __noinline__ void face32_full(int64_t t, const Nodes6& nd, const BatchInst& I, int src,
                                         const DevParams& pr, float* xs) {
  face32_body<N, D, DIR, false, true>(t, nd, pick(I, src), nullptr, nullptr, I.P32, I.F[DIR], I.g, I.f, pr,
                                      I.st->lam[DIR], false, xs);
}

template <int N, int D, int DIR, bool FP32>
__device__ __forceinline__ void stage_face(const BatchInst& I, int64_t t, int src, const DevParams& pr, float* xs) {
  Nodes6 nd;
  if (!face_nodes<DIR>(I.g, t, nd)) return;
  if constexpr (FP32) {
    if (!face32_body<N, D, DIR, true, true>(t, nd, pick(I, src), nullptr, nullptr, I.P32, I.F[DIR], I.g, I.f, pr,
                                            I.st->lam[DIR], false, xs))
      face32_full<N, D, DIR>(t, nd, I, src, pr, xs);
  } else {
    face_body<double, N, D, DIR>(t, nd, pick(I, src), I.V, I.AUX, I.F[DIR], I.g, I.f, pr, I.st->lam[DIR]);
  }
}

template <int N, int D, bool FP32>
__device__ __forceinline__ void stage_prim(const BatchInst& I, const WorkItem& w, int src, int tau) {
  double s[D];
#pragma unroll
  for (int d = 0; d < D; ++d) s[d] = 0.0;
  const double* W = pick(I, src);
  for (int64_t c = w.begin + threadIdx.x; c < w.end; c += blockDim.x) {
    double sc[D];
    if constexpr (FP32)
      prim32_body<N, D>(c, W, I.P32, nullptr, I.g, I.f, sc);
    else
      prim_body<N, D>(c, W, I.V, I.AUX, nullptr, nullptr, I.g, I.f, sc);
#pragma unroll
    for (int d = 0; d < D; ++d) s[d] = (sc[d] != sc[d]) ? sc[d] : (sc[d] > s[d] ? sc[d] : s[d]);
  }
  if (tau) block_tau_max<D>(s, I.st->tau_bits);
}

template <int N, int D, bool FP32>
__device__ __forceinline__ void stage_update(const BatchInst& I, const WorkItem& w, const StageArgs& A) {
  const double* Wsrc = pick(I, A.src);
  double* Wout = pick_mut(I, A.dst);
  const double dt = I.st->dt;
  for (int64_t c = w.begin + threadIdx.x; c < w.end; c += blockDim.x) {
    if constexpr (FP32) {
      if (A.fuse_next) {
        // as k_update32p: combination, relaxation, store, next stage's FP32 planes
        update32p_cell<N, D>(c, I.Wn, Wsrc, Wout, I.F[0], I.F[1], I.F[2], I.g, I.f, I.st, A.a, A.b, A.relax, 0,
                             I.P32, nullptr);
        continue;
      }
    }
    update_body<N, D, 0, FP32>(c, I.Wn, Wsrc, Wout, I.F[0], I.F[1], I.F[2], I.g, I.f, I.st, dt, A.a, A.b, A.relax,
                               0);
  }
}

template <int D, bool FP32>
__device__ __forceinline__ void batch_stage(const StageArgs& A) {
  __shared__ float xs[2 * Lay<3, D>::M * kBatchFace32Threads];  // the FP32 bodies' column (largest N)
  const unsigned int nb = gridDim.x;
  const bool stamper = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long* stamp = A.sync->stamp[A.stage];
  if (stamper) stamp[0] = tc::global_ns();
  if (A.prim) {
    for (int it = next_item(A.sync, 0); it < A.ncell_items; it = next_item(A.sync, 0)) {
      const WorkItem w = A.cells[it];
      const BatchInst& I = A.insts[w.inst];
      if (I.N == 2)
        stage_prim<2, D, FP32>(I, w, A.src, A.first);
      else
        stage_prim<3, D, FP32>(I, w, A.src, A.first);
    }
    if (!grid_barrier(A.sync, nb, A.limit_ns)) return;
  }
  if (stamper) stamp[1] = tc::global_ns();
  if (A.first) {
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < A.ninst; i += blockDim.x) batch_finalize_inst<D>(A.insts[i], A.cfl);
    if (!grid_barrier(A.sync, nb, A.limit_ns)) return;
  }
  if (stamper) stamp[2] = tc::global_ns();
  for (int it = next_item(A.sync, 1); it < A.ntiles; it = next_item(A.sync, 1)) {
    const WorkItem w = A.tiles[it];
    const BatchInst& I = A.insts[w.inst];
    const int64_t t = w.begin + threadIdx.x;
    if (t >= w.end) continue;
    const int key = I.N * 2 + w.pad;
    if (key == 4)
      stage_face<2, D, 0, FP32>(I, t, A.src, A.pr, xs);
    else if (key == 5)
      stage_face<2, D, 1, FP32>(I, t, A.src, A.pr, xs);
    else if (key == 6)
      stage_face<3, D, 0, FP32>(I, t, A.src, A.pr, xs);
    else
      stage_face<3, D, 1, FP32>(I, t, A.src, A.pr, xs);
  }
  if (A.update) {
    if (!grid_barrier(A.sync, nb, A.limit_ns)) return;
    if (stamper) stamp[3] = tc::global_ns();
    for (int it = next_item(A.sync, 2); it < A.ncell_items; it = next_item(A.sync, 2)) {
      const WorkItem w = A.cells[it];
      const BatchInst& I = A.insts[w.inst];
      if (I.N == 2)
        stage_update<2, D, FP32>(I, w, A);
      else
        stage_update<3, D, FP32>(I, w, A);
    }
  }
  // the last block to finish stamps the end of the launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&A.sync->done, 1u) == nb - 1u) stamp[4] = tc::global_ns();
  }
}

// Persistent stage launchers for D = 2 (FP64: hrm_batch64_d2.cu, precision
// form: hrm_batch32_d2.cu): a cooperative launch of `grid` blocks of
// kBatchFace32Threads threads; *_fit: the most blocks per SM that can be
// resident at once.
int batch_stage64_fit();
int batch_stage32_fit();
cudaError_t batch_stage64_launch(int grid, const StageArgs& A, cudaStream_t s);
cudaError_t batch_stage32_launch(int grid, const StageArgs& A, cudaStream_t s);

}  // namespace hrm

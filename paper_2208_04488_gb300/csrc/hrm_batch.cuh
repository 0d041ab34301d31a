// Batched form: many independent problems of uneven size advanced together,
// one persistent launch per phase for all of them. Blocks loop over a table of
// work items (instance, element range); every item lies inside one instance,
// so the per-element bodies are exactly those of the single-instance kernels
// and a batched instance reproduces its own context bit for bit.
#pragma once

#include "hrm_cell.cuh"
#include "hrm_face32.cuh"

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

constexpr int kBatchMaxThreads = 256;

__device__ __forceinline__ const double* pick(const BatchInst& I, int sel) { return sel == 0 ? I.Wn : I.Ws; }
__device__ __forceinline__ double* pick_mut(const BatchInst& I, int sel) { return sel == 0 ? I.Wn : I.Ws; }

// Each kernel is instantiated per species count N and runs over the work items
// of the instances with that N (the item lists are grouped by N), so that its
// body is one specialisation and its register count that of the single-context
// kernel.

// Primitives of every cell of the instances (+ per-instance CFL maxima).
template <int D, int N>
__global__ void __launch_bounds__(kBatchMaxThreads)
    k_batch_prim(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ items, int nitems, int src,
                 int fp32, int tau) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BatchInst& I = insts[w.inst];
    double s[D];
#pragma unroll
    for (int d = 0; d < D; ++d) s[d] = 0.0;
    const double* W = pick(I, src);
    float* P32 = fp32 ? I.P32 : nullptr;
    for (int64_t c = w.begin + threadIdx.x; c < w.end; c += blockDim.x) {
      double sc[D];
      prim_body<N, D>(c, W, I.V, I.AUX, P32, nullptr, I.g, I.f, sc);
#pragma unroll
      for (int d = 0; d < D; ++d) s[d] = (sc[d] != sc[d]) ? sc[d] : (sc[d] > s[d] ? sc[d] : s[d]);
    }
    if (tau) block_tau_max<D>(s, I.st->tau_bits);
  }
}

// FP32 planes (and CFL maxima) of the instances for the precision form.
template <int D, int N>
__global__ void __launch_bounds__(kBatchMaxThreads)
    k_batch_prim32(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ items, int nitems, int src,
                   int tau) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BatchInst& I = insts[w.inst];
    double s[D];
#pragma unroll
    for (int d = 0; d < D; ++d) s[d] = 0.0;
    const double* W = pick(I, src);
    for (int64_t c = w.begin + threadIdx.x; c < w.end; c += blockDim.x) {
      double sc[D];
      prim32_body<N, D>(c, W, I.P32, nullptr, I.g, I.f, sc);
#pragma unroll
      for (int d = 0; d < D; ++d) s[d] = (sc[d] != sc[d]) ? sc[d] : (sc[d] > s[d] ? sc[d] : s[d]);
    }
    if (tau) block_tau_max<D>(s, I.st->tau_bits);
  }
}

// Midpoints of direction DIR of the instances: FP64 (bit-exact; up to 256
// threads per block) or the precision form (at most 128 threads, three blocks
// per SM, as the single-context sweep).
constexpr int kBatchFace32Threads = 128;

template <int D, int DIR, int N>
__device__ __forceinline__ void batch_face_items(const BatchInst* __restrict__ insts,
                                                 const WorkItem* __restrict__ items, int nitems, int src,
                                                 const DevParams& pr, bool fp32) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BatchInst& I = insts[w.inst];
    const double* W = pick(I, src);
    const double lam = I.st->lam[DIR];
    for (int64_t t = w.begin + threadIdx.x; t < w.end; t += blockDim.x) {
      Nodes6 nd;
      if (!face_nodes<DIR>(I.g, t, nd)) continue;
      if (fp32)
        face32_body<N, D, DIR>(t, nd, W, I.V, I.AUX, I.P32, I.F[DIR], I.g, I.f, pr, lam);
      else
        face_body<double, N, D, DIR>(t, nd, W, I.V, I.AUX, I.F[DIR], I.g, I.f, pr, lam);
    }
  }
}

template <int D, int DIR, int N>
__global__ void __launch_bounds__(kBatchMaxThreads)
    k_batch_face64(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ items, int nitems, int src,
                   DevParams pr) {
  batch_face_items<D, DIR, N>(insts, items, nitems, src, pr, false);
}

template <int D, int DIR, int N>
__global__ void __launch_bounds__(kBatchFace32Threads, 3)
    k_batch_face32(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ items, int nitems, int src,
                   DevParams pr) {
  batch_face_items<D, DIR, N>(insts, items, nitems, src, pr, true);
}

// The precision form's screened sweep over tiles of 128 midpoints of the
// instances (one block per tile, one launch for all instances of a species
// count), the body as k_face32_fast's: midpoints whose screens fail are
// appended to `list` as (instance << 40 | midpoint) for k_batch_face32_fix.
// *count must be 0 at launch; list holds one entry per midpoint of the tiles.
// Six blocks per SM, as the single-context sweep (1.6 % shorter batched step
// than five; the same results).
template <int D, int DIR, int N>
__global__ void __launch_bounds__(kBatchFace32Threads, 6)
    k_batch_face32_tiles(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ tiles, int src,
                         DevParams pr, unsigned long long* __restrict__ list, uint32_t* __restrict__ count) {
  const WorkItem w = tiles[blockIdx.x];
  const BatchInst& I = insts[w.inst];
  const int64_t t = w.begin + threadIdx.x;
  Nodes6 nd;
  bool need = false;
  if (t < w.end && face_nodes<DIR>(I.g, t, nd))
    need = !face32_body<N, D, DIR, true>(t, nd, pick(I, src), I.V, I.AUX, I.P32, I.F[DIR], I.g, I.f, pr,
                                         I.st->lam[DIR]);
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (need)
    list[base + __popc(m & ((1u << lane) - 1u))] = ((unsigned long long)w.inst << 40) | (unsigned long long)t;
}

// FP64 midpoints over the same 128-midpoint tiles (one block per tile; the
// per-midpoint body is the single-context FP64 sweep's, bit for bit).
template <int D, int DIR, int N>
__global__ void __launch_bounds__(kBatchFace32Threads)
    k_batch_face64_tiles(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ tiles, int src,
                         DevParams pr) {
  const WorkItem w = tiles[blockIdx.x];
  const BatchInst& I = insts[w.inst];
  const int64_t t = w.begin + threadIdx.x;
  Nodes6 nd;
  if (t < w.end && face_nodes<DIR>(I.g, t, nd))
    face_body<double, N, D, DIR>(t, nd, pick(I, src), I.V, I.AUX, I.F[DIR], I.g, I.f, pr, I.st->lam[DIR]);
}

// The deferred midpoints of k_batch_face32_tiles with the full body, spread
// lane-major over one-warp blocks (each is a long FP64 chain).
template <int D, int DIR, int N>
__global__ void __launch_bounds__(kBatchFace32Threads, 2)
    k_batch_face32_fix(const BatchInst* __restrict__ insts, int src, DevParams pr,
                       const unsigned long long* __restrict__ list, const uint32_t* __restrict__ count) {
  const int64_t n = *count;
  for (int64_t r = threadIdx.x;; r += blockDim.x) {
    const int64_t i = r * gridDim.x + blockIdx.x;
    if (i >= n) break;
    const unsigned long long e = list[i];
    const BatchInst& I = insts[(int)(e >> 40)];
    const int64_t t = (int64_t)(e & ((1ull << 40) - 1ull));
    Nodes6 nd;
    if (!face_nodes<DIR>(I.g, t, nd)) continue;
    face32_body<N, D, DIR>(t, nd, pick(I, src), I.V, I.AUX, I.P32, I.F[DIR], I.g, I.f, pr, I.st->lam[DIR]);
  }
}

// Flux difference, SSP-RK combination and relaxation of every cell of the instances.
template <int D, bool FAST, int N>
__global__ void __launch_bounds__(kBatchMaxThreads)
    k_batch_update(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ items, int nitems, int src,
                   int dst, double a, double b, int relax, int count) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BatchInst& I = insts[w.inst];
    const double* Wsrc = pick(I, src);
    double* Wout = pick_mut(I, dst);
    const double dt = I.st->dt;
    for (int64_t c = w.begin + threadIdx.x; c < w.end; c += blockDim.x)
      update_body<N, D, 0, FAST>(c, I.Wn, Wsrc, Wout, I.F[0], I.F[1], I.F[2], I.g, I.f, I.st, dt, a, b, relax,
                                 count);
  }
}

// Host launchers (instantiated for D = 2 in hrm_batch64_d2.cu / hrm_batch32_d2.cu).
struct BatchLaunch {
  int grid;      // persistent blocks
  int threads;   // threads per block
};

void batch_prim_d2(int N, const BatchLaunch&, const BatchInst*, const WorkItem*, int nitems, int src, int tau,
                   cudaStream_t);
void batch_prim32_d2(int N, const BatchLaunch&, const BatchInst*, const WorkItem*, int nitems, int src, int tau,
                     cudaStream_t);
void batch_finalize(const BatchInst*, int ninst, int D, double cfl, cudaStream_t);
void batch_face64_d2(int N, int dir, const BatchLaunch&, const BatchInst*, const WorkItem*, int nitems, int src,
                     const DevParams&, cudaStream_t);
void batch_face32_d2(int N, int dir, const BatchLaunch&, const BatchInst*, const WorkItem*, int nitems, int src,
                     const DevParams&, cudaStream_t);
// The FP64 sweep over ntiles 128-midpoint tiles.
void batch_face64_tiles_d2(int N, int dir, const BatchInst*, const WorkItem* tiles, int ntiles, int src,
                           const DevParams&, cudaStream_t);
// The screened sweep over ntiles 128-midpoint tiles and the fix-up of its
// deferred midpoints (after a reset of *count).
void batch_face32_tiles_d2(int N, int dir, const BatchInst*, const WorkItem* tiles, int ntiles, int src,
                           const DevParams&, unsigned long long* list, uint32_t* count, cudaStream_t);
void batch_update64_d2(int N, const BatchLaunch&, const BatchInst*, const WorkItem*, int nitems, int src, int dst,
                       double a, double b, int relax, int count, cudaStream_t);
void batch_update32_d2(int N, const BatchLaunch&, const BatchInst*, const WorkItem*, int nitems, int src, int dst,
                       double a, double b, int relax, int count, cudaStream_t);

}  // namespace hrm

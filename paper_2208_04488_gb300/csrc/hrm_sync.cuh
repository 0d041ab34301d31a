// Grid-wide synchronisation of the batched form's persistent stage kernel:
// phase work queues and a bounded grid barrier. Its blocks must all be resident
// at once (a cooperative launch of at most the occupancy-derived grid); a
// barrier whose wait runs out -- 2^26 polls or the caller's time limit of
// %globaltimer -- counts itself in `expired` and makes the block leave the
// kernel, so a barrier that cannot complete ends the launch instead of
// hanging it; the host turns the count into HRM_E_TIMEOUT.
#pragma once

#include <cstdint>

#include "hrm_tc.cuh"

namespace hrm {

// Device state of one persistent launch; the first kResetWords words (`queue`,
// `arrived`, `done`) must be 0 at launch (a memset node before each launch),
// `generation` may hold anything. `stamp` receives %globaltimer at the phase
// boundaries of each stage's launch (profiling).
struct GridSync {
  unsigned int queue[4];    // next work item of each phase
  unsigned int arrived;     // blocks at the current barrier
  unsigned int done;        // blocks that finished the launch
  unsigned int generation;  // completed barriers
  unsigned int expired;     // barrier waits that ran out (accumulates over launches)
  unsigned long long stamp[3][5];  // per stage: start, after prim, after finalize, after midpoints, end
};
constexpr int kResetWords = 6;

// Barrier of all `nblocks` blocks of the grid: every thread's earlier global
// writes are visible to every thread after it (fence, arrival count, release by
// the last block's generation increment, fence; the scheme of a cooperative
// grid sync). Returns false in every thread of a block whose wait ran out.
__device__ __forceinline__ bool grid_barrier(GridSync* s, unsigned int nblocks, uint64_t limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* gen = &s->generation;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(&s->arrived, 1u) == nblocks - 1u) {
      atomicExch(&s->arrived, 0u);
      __threadfence();
      atomicAdd(&s->generation, 1u);
    } else {
      const uint64_t t0 = tc::global_ns();
      for (uint32_t it = 0; *gen == g; ++it) {
        if (it >= (1u << 26) || ((it & 63u) == 63u && tc::global_ns() - t0 > limit_ns)) {
          ok = 0;
          atomicAdd(&s->expired, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Next item of phase q for the whole block (thread 0 takes it from the queue).
__device__ __forceinline__ int next_item(GridSync* s, int q) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = (int)atomicAdd(&s->queue[q], 1u);
  __syncthreads();
  return s_item;
}

}  // namespace hrm

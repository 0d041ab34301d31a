// hrm_dt_noalloc: the CFL time step of a state without any device allocation.
//
// For callers that may not allocate device memory: an application whose memory
// is already owned by its own pool (a caching allocator that holds the free
// device memory, or a fixed budget per solver), or code that runs where
// cudaMalloc is not allowed (for example inside a region being captured into a
// CUDA graph). The caller passes the state and the output buffer; the only
// scratch is the file-scope array below, which exists once per device for the
// lifetime of the process.
//
// Built without FMA contraction and with the same per-cell primitive code as
// the context path, so it returns the same dt as hrm_dt bit for bit.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/hrm.h"
#include "hrm_cell.cuh"

// One partial maximum per block of 2048 cells and direction (bit patterns of
// non-negative doubles): 65536 x 3 x 8 bytes = 1.5 MiB per device, held from
// module load until the process exits. Every call writes the entries
// [0, nblocks) before it reads them, so nothing needs clearing between calls;
// two calls that overlap on the GPU write the same entries and race.
static __device__ __align__(256) unsigned long long g_dt_partials[65536 * 3];

namespace {

using namespace hrm;

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;  // 2048
constexpr int kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
unsigned long long* g_partials_addr[kMaxDevices] = {};

template <int N, int D>
__global__ void __launch_bounds__(kThreads)
    k_dt_partials(const double* __restrict__ W, DevGrid g, DevFluid f, unsigned long long* partials) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock;
  double mx[D];
#pragma unroll
  for (int d = 0; d < D; ++d) mx[d] = 0.0;
  for (int i = 0; i < kCellsPerThread; ++i) {
    const int64_t c = base + (int64_t)i * kThreads + threadIdx.x;
    if (c >= nc) break;
    double w[M], v[M], rho, cs, rc2;
#pragma unroll
    for (int m = 0; m < M; ++m) w[m] = W[m * nc + c];
    cell_prim<N, D>(w, f, v, rho, cs, rc2);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double s = (fabs(v[L::MOM + d]) + cs) / g.dx[d];
      mx[d] = (s != s) ? s : (s > mx[d] ? s : mx[d]);  // NaN propagates as the largest value
    }
  }
  __shared__ unsigned long long red[D][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    unsigned long long b = dbits(mx[d]);
    if (mx[d] != mx[d]) b = 0x7ff8000000000000ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
      b = x > b ? x : b;
    }
    if (lane == 0) red[d][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x < D) {
    unsigned long long b = 0;
    for (int w = 0; w < kThreads / 32; ++w) b = red[threadIdx.x][w] > b ? red[threadIdx.x][w] : b;
    partials[(int64_t)blockIdx.x * 3 + threadIdx.x] = b;
  }
}

// One block: tau_d = max over the partials, dt = cfl / sum_d tau_d (Sec. 4.1.2).
__global__ void __launch_bounds__(kThreads)
    k_dt_final(const unsigned long long* partials, int nblocks, int D, double cfl, double* out) {
  __shared__ unsigned long long red[3][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = 0; d < D; ++d) {
    unsigned long long b = 0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
      const unsigned long long x = partials[(int64_t)i * 3 + d];
      b = x > b ? x : b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
      b = x > b ? x : b;
    }
    if (lane == 0) red[d][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tau[3] = {0.0, 0.0, 0.0}, sum = 0.0;
    for (int d = 0; d < D; ++d) {
      unsigned long long b = 0;
      for (int w = 0; w < kThreads / 32; ++w) b = red[d][w] > b ? red[d][w] : b;
      tau[d] = __longlong_as_double((long long)b);
      sum = sum + tau[d];
    }
    out[0] = cfl / sum;
    for (int d = 0; d < D; ++d) out[1 + d] = tau[d];
  }
}

template <int N, int D>
void launch(const double* W, const DevGrid& g, const DevFluid& f, unsigned long long* partials, int nblocks,
            double cfl, double* out, cudaStream_t s) {
  k_dt_partials<N, D><<<nblocks, kThreads, 0, s>>>(W, g, f, partials);
  k_dt_final<<<1, kThreads, 0, s>>>(partials, nblocks, D, cfl, out);
}

// Device address of the scratch array for the current device; looked up once
// per device (cudaGetSymbolAddress allocates nothing).
hrm_status partials_address(unsigned long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HRM_E_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dt_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return HRM_E_CUDA;
    }
    g_partials_addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_partials_addr[dev];
  return HRM_OK;
}

}  // namespace

namespace hrm {
void set_thread_error(const char* msg);
}

extern "C" hrm_status hrm_dt_noalloc(int32_t nspecies, int32_t ndim, const int64_t* n, const double* dx,
                                     const double* gamma, const double* p_inf, const double* c_v,
                                     const double* q, const double* W_device, double cfl, double* out_device,
                                     void* stream) {
  auto inval = [](const char* m) {
    hrm::set_thread_error(m);
    return HRM_E_INVAL;
  };
  if (!n || !dx || !gamma || !p_inf || !c_v || !W_device || !out_device) return inval("null argument");
  if (nspecies < 2 || nspecies > 3) return inval("nspecies outside 2..3");
  if (ndim < 1 || ndim > 3) return inval("ndim outside 1..3");
  if (!(cfl > 0.0)) return inval("cfl must be positive");
  DevGrid g;
  std::memset(&g, 0, sizeof g);
  g.ncells = 1;
  for (int d = 0; d < 3; ++d) {
    const int64_t nd = d < ndim ? n[d] : 1;
    if (nd < 1) return inval("cell counts must be positive");
    if (d < ndim && !(dx[d] > 0.0)) return inval("dx must be positive");
    g.n[d] = nd;
    g.dx[d] = d < ndim ? dx[d] : 1.0;
    g.inv_dx[d] = 1.0 / g.dx[d];
    if (g.ncells > (int64_t)kMaxBlocks * kCellsPerBlock / nd) {
      return inval("hrm_dt_noalloc: more than 65536 x 2048 = 134217728 cells (its fixed scratch holds one "
                   "partial maximum per 2048 cells); use hrm_dt");
    }
    g.ncells *= nd;
  }
  g.nint = g.ncells;
  DevFluid f;
  std::memset(&f, 0, sizeof f);
  int liq = -1;
  for (int k = 0; k < nspecies; ++k) {
    if (!(gamma[k] > 1.0) || !(c_v[k] > 0.0) || p_inf[k] < 0.0) return inval("invalid species table");
    if (p_inf[k] > 0.0) {
      if (liq >= 0) return inval("more than one stiffened gas");
      liq = k;
    }
    f.inv_gm1[k] = 1.0 / (gamma[k] - 1.0);
    f.gpinf_gm1[k] = gamma[k] * p_inf[k] / (gamma[k] - 1.0);
    f.cv[k] = c_v[k];
    f.cp[k] = gamma[k] * c_v[k];
    f.Rg[k] = f.cp[k] - c_v[k];
    f.q[k] = q ? q[k] : 0.0;
    f.pinf[k] = p_inf[k];
    f.gamma[k] = gamma[k];
  }
  f.liq = liq < 0 ? 0 : liq;
  fill_fluid_f(f);
  // An error pending from earlier work belongs to its owner: report it without
  // clearing it, and launch nothing, so the check after the launches sees only
  // errors of this call.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    hrm::set_thread_error("hrm_dt_noalloc: a CUDA error from earlier work is pending; nothing launched");
    return HRM_E_CUDA;
  }
  unsigned long long* partials = nullptr;
  if (partials_address(&partials) != HRM_OK) {
    hrm::set_thread_error("hrm_dt_noalloc: scratch address lookup failed");
    return HRM_E_CUDA;
  }
  const int nblocks = (int)((g.ncells + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = (cudaStream_t)stream;
  const int key = nspecies * 10 + ndim;
  switch (key) {
    case 21: launch<2, 1>(W_device, g, f, partials, nblocks, cfl, out_device, s); break;
    case 22: launch<2, 2>(W_device, g, f, partials, nblocks, cfl, out_device, s); break;
    case 23: launch<2, 3>(W_device, g, f, partials, nblocks, cfl, out_device, s); break;
    case 31: launch<3, 1>(W_device, g, f, partials, nblocks, cfl, out_device, s); break;
    case 32: launch<3, 2>(W_device, g, f, partials, nblocks, cfl, out_device, s); break;
    default: launch<3, 3>(W_device, g, f, partials, nblocks, cfl, out_device, s); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    hrm::set_thread_error(cudaGetErrorString(e));
    return HRM_E_CUDA;
  }
  return HRM_OK;
}

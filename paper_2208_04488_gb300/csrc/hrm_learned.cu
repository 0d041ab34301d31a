// Learned smoothness detector: inference (the gate kernel, tensor cores) and
// training (forward, back-propagation and Adam kernels in FP32) of the
// 30 -> 32 -> 32 -> 1 perceptron, and the hrm_detector C ABI.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>

#include "hrm_learned.h"

using namespace hrm;
using namespace hrm::mlp;

namespace {

constexpr int kParamsPad = 2084;  // per-block gradient row (16-byte multiple)
constexpr int kGateThreads = 128;
constexpr int kTrainThreads = 128;
constexpr int kS = 33;  // shared row stride of the per-sample training arrays
constexpr size_t kTrainSmem = sizeof(float) * (kParamsPad + 5 * kTrainThreads * kS + kTrainThreads);

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// ---------------------------------------------------------------- inference

// The inference weights from the FP32 parameters: W1 and W2 transposed into
// bf16 K-major operand tiles (tc::tile_offset), the rest in FP32.
__global__ void k_pack_blob(const float* __restrict__ th, GateBlob* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kHid * 32) {
    const int n = i / 32, k = i % 32;
    const int e = tc::tile_offset(n, k) / 2;
    b->w1[e] = __float2bfloat16_rn(k < kIn ? th[oW1 + k * kHid + n] : 0.f);
    b->w2[e] = __float2bfloat16_rn(th[oW2 + k * kHid + n]);
  }
  if (i < kHid) {
    b->b1[i] = th[oB1 + i];
    b->b2[i] = th[oB2 + i];
    b->w3[i] = th[oW3 + i];
  }
  if (i < 31) b->pad[i] = 0.f;
  if (i == 0) b->b3 = th[oB3];
}

// Gate byte of every midpoint of direction DIR: 1 where the logit exceeds zthr.
// Persistent CTAs of 128 threads, one midpoint per thread and tile of 128.
template <int N, int D, int DIR>
__global__ void __launch_bounds__(kGateThreads)
    k_gate(const float* __restrict__ P32, const float* __restrict__ R32, DevGrid g, const GateBlob* __restrict__ blob,
           float zthr, uint8_t* __restrict__ gate, unsigned long long* __restrict__ waits) {
  static_assert(kGateThreads == tc::kRows, "one midpoint per MMA row");
  __shared__ NetTile S;
  const uint32_t tmem = net_begin(S, blob);
  uint32_t phase = 0;
  const float z0 = net_zero_logit(S, tmem, phase, waits);
  const int64_t nf = face_total(g, DIR);
  // the trip count is the same for every thread of the CTA (all take part in the MMAs)
  for (int64_t base = (int64_t)blockIdx.x * kGateThreads; base < nf; base += (int64_t)gridDim.x * kGateThreads) {
    const int64_t t = base + threadIdx.x;
    Nodes6 nd;
    const bool ok = face_nodes<DIR>(g, t, nd);
    float x[kIn];
    if (ok) {
      stencil_features<N, D, DIR>(nd, P32, R32, g.ncells, x);
    } else {
#pragma unroll
      for (int k = 0; k < kIn; ++k) x[k] = 0.f;
    }
    const float z = net_logit_or_zero(S, x, z0, tmem, phase, waits);
    if (ok) gate[t] = z > zthr ? 1 : 0;
  }
  net_end(tmem);
}

// Shared-memory halo tile of the gate kernel's TMA path: for each of the ten
// (quantity, value | residue) FP32 planes, the six nodes of 128 consecutive y
// (or z) midpoints as 6 rows of 128 cells, or for 128 consecutive x midpoints
// one row of 136 cells starting 4 cells left of the first (a 16-byte-aligned
// start); slots 128-byte aligned.
template <int DIR>
struct Halo {
  static constexpr int kW = DIR == 0 ? 136 : 128;  // box width (cells along x)
  static constexpr int kH = DIR == 0 ? 1 : 6;      // box height (rows along the sweep direction)
  static constexpr int kSlot = (kW * kH + 31) / 32 * 32;
  static constexpr size_t kBytes = sizeof(float) * 2 * kQuant * kSlot;
};

// The gate kernel with its stencil inputs staged by TMA: per tile of 128
// midpoints along x (one row of the midpoint grid), one thread loads the halo
// boxes of the stencil planes from the 4-D tensor maps (x, y, z, plane) of P32
// and R32 into shared memory, completing on an mbarrier (bounded wait).
// Midpoints whose six nodes are all interior cells read their features from
// the tile; the others (boundary mappings, Dirichlet slices) read the planes
// directly. Both go through features_from, so the features are the same.
template <int N, int D, int DIR>
__global__ void __launch_bounds__(kGateThreads)
    k_gate_tma(const __grid_constant__ CUtensorMap tP, const __grid_constant__ CUtensorMap tR,
               const float* __restrict__ P32, const float* __restrict__ R32, DevGrid g,
               const GateBlob* __restrict__ blob, float zthr, uint8_t* __restrict__ gate,
               unsigned long long* __restrict__ waits) {
  static_assert(kGateThreads == tc::kRows, "one midpoint per MMA row");
  using H = Halo<DIR>;
  extern __shared__ __align__(128) float halo_raw[];
  // TMA destinations 128-byte aligned (the launch adds 128 bytes for this)
  float* halo = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(halo_raw) + 127) & ~uintptr_t(127));
  __shared__ NetTile S;
  __shared__ unsigned long long tbar;
  const uint32_t tmem = net_begin(S, blob);
  if (threadIdx.x == 0) tc::bar_init(tc::smem_u32(&tbar));
  __syncthreads();
  uint32_t phase = 0, tphase = 0;
  const float z0 = net_zero_logit(S, tmem, phase, waits);
  const int64_t n0 = g.n[0], nd_ = g.n[DIR];
  const int64_t f0 = n0 + (DIR == 0), f1 = g.n[1] + (DIR == 1), f2 = g.n[2] + (DIR == 2);
  const int64_t tpr = (f0 + kGateThreads - 1) / kGateThreads;  // tiles per row of the midpoint grid
  const int64_t ntiles = tpr * f1 * f2;
  const int i = threadIdx.x;
  // the trip count is the same for every thread of the CTA (all take part in the MMAs)
  for (int64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const int64_t r = T / tpr, x0 = (T % tpr) * kGateThreads;
    const int64_t i1 = r % f1, i2 = r / f1, i0 = x0 + i;
    const bool ok = i0 < f0;
    const int64_t t = r * f0 + i0;
    const int64_t fp = DIR == 0 ? i0 : (DIR == 1 ? i1 : i2);
    const bool inner = ok && fp >= 3 && fp <= nd_ - 3;  // nodes fp-3 .. fp+2 all interior
    // some midpoint of the tile reads the halo (the same for the whole CTA)
    const bool any = DIR == 0 ? (x0 <= n0 - 3 && x0 + kGateThreads - 1 >= 3) : (fp >= 3 && fp <= nd_ - 3);
    if (any) {
      const uint32_t bar = tc::smem_u32(&tbar);
      if (threadIdx.x == 0) {
        constexpr uint32_t kLoads = N < 3 ? 2 * kQuant - 2 : 2 * kQuant;
        tc::bar_expect(bar, kLoads * (uint32_t)(sizeof(float) * H::kW * H::kH));
        const int c0 = (int)(DIR == 0 ? x0 - 4 : x0);
        const int c1 = (int)(DIR == 1 ? i1 - 3 : i1);
        const int c2 = (int)(DIR == 2 ? i2 - 3 : i2);
#pragma unroll
        for (int q = 0; q < kQuant; ++q) {
          if (q == 1 && N < 3) continue;
          tc::tma_load_4d(tc::smem_u32(halo + (2 * q) * H::kSlot), &tP, c0, c1, c2, val_plane<N, D, DIR>(q), bar);
          tc::tma_load_4d(tc::smem_u32(halo + (2 * q + 1) * H::kSlot), q < 2 ? &tP : &tR, c0, c1, c2,
                          res_plane<N, D, DIR>(q), bar);
        }
      }
      if (!tc::bar_wait(bar, tphase) && waits) atomicAdd(waits, 1ull);
      tphase ^= 1u;
    }
    float x[kIn];
    if (inner) {
      auto at = [&](int sl, int j) -> float {
        return DIR == 0 ? halo[sl * H::kSlot + i + 1 + j] : halo[sl * H::kSlot + j * H::kW + i];
      };
      features_from<N>([&](int q, int j) { return at(2 * q, j); }, [&](int q, int j) { return at(2 * q + 1, j); },
                       x);
    } else if (ok) {
      Nodes6 nd;
      face_nodes<DIR>(g, t, nd);
      stencil_features<N, D, DIR>(nd, P32, R32, g.ncells, x);
    } else {
#pragma unroll
      for (int k = 0; k < kIn; ++k) x[k] = 0.f;
    }
    const float z = net_logit_or_zero(S, x, z0, tmem, phase, waits);
    if (ok) gate[t] = z > zthr ? 1 : 0;
  }
  net_end(tmem);
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// 4-D tensor map (x, y, z, plane) of `planes` FP32 planes of g.ncells cells
// (interior cells x fastest, then any boundary slices), box of the halo of DIR.
// False where TMA cannot address it: row or plane strides not multiples of 16
// bytes, or the address not 16-byte aligned.
template <int DIR>
bool halo_map(CUtensorMap* m, const float* base, const DevGrid& g, int planes) {
  const auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) || g.n[0] % 4 != 0 || g.ncells % 4 != 0) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], (cuuint64_t)planes};
  const cuuint64_t strides[3] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)(g.n[0] * g.n[1]) * 4, (cuuint64_t)g.ncells * 4};
  const cuuint32_t box[4] = {(cuuint32_t)Halo<DIR>::kW, DIR == 1 ? 6u : 1u, DIR == 2 ? 6u : 1u, 1u};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N, int D, int DIR>
void gate_dir(const float* P32, const float* R32, const DevGrid& g, const GateBlob* blob, float zthr, uint8_t* gate,
              unsigned long long* waits, int max_blocks, cudaStream_t s) {
  CUtensorMap tP, tR;
  if (halo_map<DIR>(&tP, P32, g, P32Lay<N, D>::PLANES) && halo_map<DIR>(&tR, R32, g, D + 2)) {
    const int64_t f0 = g.n[0] + (DIR == 0);
    const int64_t nt = (f0 + kGateThreads - 1) / kGateThreads * (face_total(g, DIR) / f0);
    const int64_t nb = nt < max_blocks ? (nt > 0 ? nt : 1) : max_blocks;
    k_gate_tma<N, D, DIR><<<(unsigned)nb, kGateThreads, Halo<DIR>::kBytes + 128, s>>>(tP, tR, P32, R32, g, blob, zthr,
                                                                                gate, waits);
    return;
  }
  const int64_t nf = face_total(g, DIR);
  int64_t nb = (nf + kGateThreads - 1) / kGateThreads;
  if (nb > max_blocks) nb = max_blocks;
  if (nb < 1) nb = 1;
  k_gate<N, D, DIR><<<(unsigned)nb, kGateThreads, 0, s>>>(P32, R32, g, blob, zthr, gate, waits);
}

template <int N, int D>
void gate_nd(int dir, const float* P32, const float* R32, const DevGrid& g, const GateBlob* blob, float zthr,
             uint8_t* gate, unsigned long long* waits, int max_blocks, cudaStream_t s) {
  if (dir == 0) gate_dir<N, D, 0>(P32, R32, g, blob, zthr, gate, waits, max_blocks, s);
  if constexpr (D > 1)
    if (dir == 1) gate_dir<N, D, 1>(P32, R32, g, blob, zthr, gate, waits, max_blocks, s);
  if constexpr (D > 2)
    if (dir == 2) gate_dir<N, D, 2>(P32, R32, g, blob, zthr, gate, waits, max_blocks, s);
}

// Logits of dataset rows [first, first + n): bf16 tensor-core path (as the
// gate) or the FP32 training arithmetic.
__global__ void __launch_bounds__(kGateThreads)
    k_logits_bf16(const GateBlob* __restrict__ blob, const float* __restrict__ X, int64_t first, int64_t n,
                  float* __restrict__ z, unsigned long long* __restrict__ waits) {
  __shared__ NetTile S;
  const uint32_t tmem = net_begin(S, blob);
  const int64_t i = (int64_t)blockIdx.x * kGateThreads + threadIdx.x;
  float x[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x[k] = i < n ? X[(first + i) * 32 + k] : 0.f;
  uint32_t phase = 0;
  const float v = net_logit(S, x, tmem, phase, waits);
  net_end(tmem);
  if (i < n) z[i] = v;
}

__device__ __forceinline__ float forward_fp32(const float* th, const float (&x)[kIn], float (&a1)[kHid],
                                              float (&a2)[kHid]) {
#pragma unroll
  for (int n = 0; n < kHid; ++n) a1[n] = th[oB1 + n];
#pragma unroll
  for (int k = 0; k < kIn; ++k) {
    const float xk = x[k];
#pragma unroll
    for (int n = 0; n < kHid; ++n) a1[n] += xk * th[oW1 + k * kHid + n];
  }
#pragma unroll
  for (int n = 0; n < kHid; ++n) a2[n] = th[oB2 + n];
#pragma unroll
  for (int k = 0; k < kHid; ++k) {
    const float hk = fmaxf(a1[k], 0.f);
#pragma unroll
    for (int n = 0; n < kHid; ++n) a2[n] += hk * th[oW2 + k * kHid + n];
  }
  float z = th[oB3];
#pragma unroll
  for (int n = 0; n < kHid; ++n) z += fmaxf(a2[n], 0.f) * th[oW3 + n];
  return z;
}

__global__ void __launch_bounds__(kTrainThreads)
    k_logits_fp32(const float* __restrict__ theta, const float* __restrict__ X, int64_t first, int64_t n,
                  float* __restrict__ z) {
  __shared__ float th[kParamsPad];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kTrainThreads + threadIdx.x;
  if (i >= n) return;
  float x[kIn], a1[kHid], a2[kHid];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x[k] = X[(first + i) * 32 + k];
  z[i] = forward_fp32(th, x, a1, a2);
}

// Confusion counts at logit threshold zthr (positive = smooth = gate on):
// [0] TP, [1] FP (gated where WENO is not smooth), [2] TN, [3] FN; and the
// summed cross-entropy.
__global__ void k_confusion(const float* __restrict__ z, const float* __restrict__ y, int64_t n, float zthr,
                            unsigned long long* __restrict__ counts, double* __restrict__ loss) {
  __shared__ unsigned long long c[4];
  __shared__ double ls;
  if (threadIdx.x < 4) c[threadIdx.x] = 0;
  if (threadIdx.x == 0) ls = 0.0;
  __syncthreads();
  unsigned long long lc[4] = {0, 0, 0, 0};
  double l = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool pos = z[i] > zthr, lab = y[i] > 0.5f;
    lc[pos ? (lab ? 0 : 1) : (lab ? 3 : 2)]++;
    const float zz = z[i];
    l += (double)(fmaxf(zz, 0.f) + log1pf(expf(-fabsf(zz))) - y[i] * zz);
  }
  for (int k = 0; k < 4; ++k) atomicAdd(&c[k], lc[k]);
  atomicAdd(&ls, l);
  __syncthreads();
  if (threadIdx.x < 4) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
  if (threadIdx.x == 0) atomicAdd(loss, ls);
}

// ---------------------------------------------------------------- training

// Forward and back-propagation of one sample per thread; per-block gradient
// (sum over the block's samples) into partials[blockIdx.x][kParamsPad] and the
// summed loss into loss_parts[blockIdx.x]. Sample s of the batch is row
// first + s, or, with draw, row splitmix64(seed + s) mod n.
__global__ void __launch_bounds__(kTrainThreads)
    k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ X, const float* __restrict__ y,
               int64_t n, int64_t first, int64_t count, int draw, uint64_t seed, float* __restrict__ partials,
               float* __restrict__ loss_parts) {
  extern __shared__ float sm[];
  float* th = sm;
  float* xs = th + kParamsPad;
  float* h1s = xs + kTrainThreads * kS;
  float* dh1s = h1s + kTrainThreads * kS;
  float* h2s = dh1s + kTrainThreads * kS;
  float* dh2s = h2s + kTrainThreads * kS;
  float* dzs = dh2s + kTrainThreads * kS;
  const int tid = threadIdx.x;
  for (int i = tid; i < kParams; i += kTrainThreads) th[i] = theta[i];
  const int64_t s = (int64_t)blockIdx.x * kTrainThreads + tid;
  const bool valid = s < count && n > 0;
  int64_t row = 0;
  if (valid) row = draw ? (int64_t)(splitmix64(seed + (uint64_t)s) % (uint64_t)n) : first + s;
  float* xr = xs + tid * kS;
  float* h1r = h1s + tid * kS;
  float* dh1r = dh1s + tid * kS;
  float* h2r = h2s + tid * kS;
  float* dh2r = dh2s + tid * kS;
  const float yy = valid ? y[row] : 0.f;
  // first layer (inputs kept in shared memory for the weight gradient)
  float h[kHid];
  {
    float x[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) {
      x[k] = valid ? X[row * 32 + k] : 0.f;
      xr[k] = x[k];
    }
    __syncthreads();  // th complete
#pragma unroll
    for (int n = 0; n < kHid; ++n) h[n] = th[oB1 + n];
  }
  // outer loops not unrolled (operands re-read from this thread's shared row):
  // a full unroll hoists the weight loads past the register file
#pragma unroll 1
  for (int k = 0; k < kIn; ++k) {
    const float xk = xr[k];
#pragma unroll
    for (int n = 0; n < kHid; ++n) h[n] += xk * th[oW1 + k * kHid + n];
  }
  uint32_t mask1 = 0;  // a1 > 0
#pragma unroll
  for (int n = 0; n < kHid; ++n) {
    mask1 |= (h[n] > 0.f ? 1u : 0u) << n;
    h[n] = fmaxf(h[n], 0.f);
    h1r[n] = h[n];
  }
  // second layer and output
  float a2[kHid];
#pragma unroll
  for (int n = 0; n < kHid; ++n) a2[n] = th[oB2 + n];
#pragma unroll 1
  for (int k = 0; k < kHid; ++k) {
    const float hk = h1r[k];
#pragma unroll
    for (int n = 0; n < kHid; ++n) a2[n] += hk * th[oW2 + k * kHid + n];
  }
  float z = th[oB3];
#pragma unroll
  for (int n = 0; n < kHid; ++n) z += fmaxf(a2[n], 0.f) * th[oW3 + n];
  const float p = 1.f / (1.f + expf(-z));
  const float dz = valid ? p - yy : 0.f;
  float lsum = valid ? fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - yy * z : 0.f;
  // dL/da2 = dz w3 (a2 > 0);  dL/da1 = (W2 dL/da2) (a1 > 0)
#pragma unroll
  for (int m = 0; m < kHid; ++m) {
    h2r[m] = fmaxf(a2[m], 0.f);
    a2[m] = a2[m] > 0.f ? dz * th[oW3 + m] : 0.f;  // now dL/da2
    dh2r[m] = a2[m];
  }
#pragma unroll 1
  for (int k = 0; k < kHid; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < kHid; ++m) acc += th[oW2 + k * kHid + m] * a2[m];
    dh1r[k] = ((mask1 >> k) & 1u) ? acc : 0.f;
  }
  dzs[tid] = dz;
  __syncthreads();
  for (int e = tid; e < kParams; e += kTrainThreads) {
    float acc = 0.f;
    if (e < oB1) {
      const int k = e / kHid, m = e % kHid;
      for (int q = 0; q < kTrainThreads; ++q) acc += xs[q * kS + k] * dh1s[q * kS + m];
    } else if (e < oW2) {
      const int m = e - oB1;
      for (int q = 0; q < kTrainThreads; ++q) acc += dh1s[q * kS + m];
    } else if (e < oB2) {
      const int k = (e - oW2) / kHid, m = (e - oW2) % kHid;
      for (int q = 0; q < kTrainThreads; ++q) acc += h1s[q * kS + k] * dh2s[q * kS + m];
    } else if (e < oW3) {
      const int m = e - oB2;
      for (int q = 0; q < kTrainThreads; ++q) acc += dh2s[q * kS + m];
    } else if (e < oB3) {
      const int m = e - oW3;
      for (int q = 0; q < kTrainThreads; ++q) acc += dzs[q] * h2s[q * kS + m];
    } else {
      for (int q = 0; q < kTrainThreads; ++q) acc += dzs[q];
    }
    partials[(int64_t)blockIdx.x * kParamsPad + e] = acc;
  }
  // block sum of the loss
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  __shared__ float wl[kTrainThreads / 32];
  if ((tid & 31) == 0) wl[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < kTrainThreads / 32; ++w) t += wl[w];
    loss_parts[blockIdx.x] = t;
  }
}

// Sum of the per-block gradients (block order) times scale.
__device__ __forceinline__ float grad_sum(const float* __restrict__ partials, int nblk, int e, float scale) {
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += partials[(int64_t)b * kParamsPad + e];
  return g * scale;
}

__device__ __forceinline__ void loss_sum(const float* __restrict__ loss_parts, int nblk, float scale,
                                         float* __restrict__ out) {
  float l = 0.f;
  for (int b = 0; b < nblk; ++b) l += loss_parts[b];
  *out = l * scale;
}

__global__ void k_mlp_reduce(const float* __restrict__ partials, const float* __restrict__ loss_parts, int nblk,
                             float scale, float* __restrict__ grad, float* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kParams) grad[e] = grad_sum(partials, nblk, e, scale);
  if (e == 0) loss_sum(loss_parts, nblk, scale, loss);
}

// Adam (Kingma & Ba): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// theta <- theta - lr (m / bc1) / (sqrt(v / bc2) + eps), bc_i = 1 - b_i^t;
// g is the batch-mean gradient.
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ partials, const float* __restrict__ loss_parts, int nblk,
                           float inv_batch, float lr, float b1, float b2, float eps, float bc1, float bc2,
                           float* __restrict__ loss_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kParams) {
    const float g = grad_sum(partials, nblk, e, inv_batch);
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    theta[e] = theta[e] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  }
  if (e == 0 && loss_out) loss_sum(loss_parts, nblk, inv_batch, loss_out);
}

}  // namespace

// ---------------------------------------------------------------- the detector object

struct hrm_detector {
  cudaStream_t stream = nullptr;
  int64_t cap = 0, size = 0;
  uint64_t seed = 0;
  int64_t calls = 0;
  int64_t adam_t = 0;
  float* theta = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* X = nullptr;
  float* y = nullptr;
  float* dev = nullptr;
  float* z = nullptr;           // logits scratch (cap)
  float* partials = nullptr;    // [max_blocks][kParamsPad]
  float* loss_parts = nullptr;  // [max_blocks]
  float* scratch = nullptr;     // kParams + 1 + loss history
  int max_blocks = 0;
  int64_t hist_cap = 0;
  float* hist = nullptr;
  GateBlob* blob = nullptr;
  unsigned long long* waits = nullptr;  // tensor-core waits of the inference that ran out
  int32_t* counts = nullptr;
  int64_t* offsets = nullptr;
  int64_t* total = nullptr;
  int64_t nb_cap = 0;
  unsigned long long* conf = nullptr;
  double* conf_loss = nullptr;
  std::string err;
};

namespace {

hrm_status dfail(hrm_detector* d, hrm_status s, const char* fmt, ...) {
  if (d) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    d->err = buf;
  }
  return s;
}

hrm_status dcheck(hrm_detector* d, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HRM_OK;
  return dfail(d, e == cudaErrorMemoryAllocation ? HRM_E_NOMEM : HRM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Synchronise the detector's stream and report inference waits that ran out
// (the counter is cleared once read).
hrm_status waits_check(hrm_detector* d, const char* what) {
  unsigned long long w = 0;
  hrm_status s;
  if ((s = dcheck(d, cudaMemcpyAsync(&w, d->waits, sizeof w, cudaMemcpyDeviceToHost, d->stream), what))) return s;
  if ((s = dcheck(d, cudaStreamSynchronize(d->stream), what))) return s;
  if (w == 0) return HRM_OK;
  cudaMemsetAsync(d->waits, 0, sizeof w, d->stream);
  return dfail(d, HRM_E_TIMEOUT, "%s: %llu tensor-core waits ran out", what, w);
}

hrm_status pack(hrm_detector* d) {
  k_pack_blob<<<(kHid * 32 + 255) / 256, 256, 0, d->stream>>>(d->theta, d->blob);
  return dcheck(d, cudaGetLastError(), "pack weights");
}

hrm_status ensure_blocks(hrm_detector* d, int nblk) {
  if (nblk <= d->max_blocks) return HRM_OK;
  cudaStreamSynchronize(d->stream);
  cudaFree(d->partials);
  cudaFree(d->loss_parts);
  d->partials = nullptr;
  d->loss_parts = nullptr;
  d->max_blocks = 0;
  hrm_status s;
  if ((s = dcheck(d, cudaMalloc(&d->partials, sizeof(float) * (size_t)nblk * kParamsPad), "alloc partials")))
    return s;
  if ((s = dcheck(d, cudaMalloc(&d->loss_parts, sizeof(float) * (size_t)nblk), "alloc partials"))) return s;
  d->max_blocks = nblk;
  return HRM_OK;
}

bool g_smem_set = false;

hrm_status set_train_smem(hrm_detector* d) {
  if (g_smem_set) return HRM_OK;
  hrm_status s = dcheck(
      d, cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem),
      "shared memory attribute");
  if (!s) g_smem_set = true;
  return s;
}

// Launch the gradient kernel over `count` samples (sequential from `first`, or drawn).
hrm_status launch_grad(hrm_detector* d, int64_t first, int64_t count, int draw, uint64_t seed, int* nblk_out) {
  const int nblk = (int)((count + kTrainThreads - 1) / kTrainThreads);
  hrm_status s;
  if ((s = set_train_smem(d))) return s;
  if ((s = ensure_blocks(d, nblk))) return s;
  k_mlp_grad<<<nblk, kTrainThreads, kTrainSmem, d->stream>>>(d->theta, d->X, d->y, d->size, first, count, draw,
                                                             seed, d->partials, d->loss_parts);
  *nblk_out = nblk;
  return dcheck(d, cudaGetLastError(), "gradient kernel");
}

}  // namespace

namespace hrm {
const GateBlob* detector_blob(const hrm_detector* d) { return d ? d->blob : nullptr; }

void launch_gate(int N, int D, int dir, const float* P32, const float* R32, const DevGrid& g, const GateBlob* blob,
                 float zthr, uint8_t* gate, unsigned long long* waits, int max_blocks, cudaStream_t s) {
  const int key = N * 10 + D;
  switch (key) {
    case 21: gate_nd<2, 1>(dir, P32, R32, g, blob, zthr, gate, waits, max_blocks, s); break;
    case 22: gate_nd<2, 2>(dir, P32, R32, g, blob, zthr, gate, waits, max_blocks, s); break;
    case 23: gate_nd<2, 3>(dir, P32, R32, g, blob, zthr, gate, waits, max_blocks, s); break;
    case 31: gate_nd<3, 1>(dir, P32, R32, g, blob, zthr, gate, waits, max_blocks, s); break;
    case 32: gate_nd<3, 2>(dir, P32, R32, g, blob, zthr, gate, waits, max_blocks, s); break;
    case 33: gate_nd<3, 3>(dir, P32, R32, g, blob, zthr, gate, waits, max_blocks, s); break;
    default: break;
  }
}
}  // namespace hrm

extern "C" {

hrm_status hrm_detector_create(hrm_detector** out, int64_t capacity, uint64_t seed, void* stream) {
  if (!out) return HRM_E_INVAL;
  *out = nullptr;
  if (capacity < 0 || capacity > ((int64_t)1 << 31)) return HRM_E_INVAL;
  hrm_detector* d = new (std::nothrow) hrm_detector();
  if (!d) return HRM_E_NOMEM;
  d->stream = (cudaStream_t)stream;
  d->cap = capacity;
  d->seed = seed;
  hrm_status s = HRM_OK;
  auto bail = [&](hrm_status st) {
    hrm_detector_destroy(d);
    return st;
  };
  const size_t P = sizeof(float) * kParams;
  if ((s = dcheck(d, cudaMalloc(&d->theta, P), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->m, P), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->v, P), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->scratch, sizeof(float) * (kParams + 4)), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->blob, sizeof(GateBlob)), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->waits, sizeof(unsigned long long)), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMemsetAsync(d->waits, 0, sizeof(unsigned long long), d->stream), "clear"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->conf, sizeof(unsigned long long) * 4), "alloc"))) return bail(s);
  if ((s = dcheck(d, cudaMalloc(&d->conf_loss, sizeof(double)), "alloc"))) return bail(s);
  if (capacity > 0) {
    if ((s = dcheck(d, cudaMalloc(&d->X, sizeof(float) * 32 * (size_t)capacity), "alloc samples"))) return bail(s);
    if ((s = dcheck(d, cudaMalloc(&d->y, sizeof(float) * (size_t)capacity), "alloc samples"))) return bail(s);
    if ((s = dcheck(d, cudaMalloc(&d->dev, sizeof(float) * (size_t)capacity), "alloc samples"))) return bail(s);
    if ((s = dcheck(d, cudaMalloc(&d->z, sizeof(float) * (size_t)capacity), "alloc samples"))) return bail(s);
  }
  // He-uniform initial weights (seeded), zero biases
  float th[kParams];
  std::mt19937_64 rng(seed);
  auto uni = [&](float a) { return (float)((double)(rng() >> 11) * 0x1.0p-53 * 2.0 - 1.0) * a; };
  std::memset(th, 0, sizeof th);
  for (int i = 0; i < kIn * kHid; ++i) th[oW1 + i] = uni(std::sqrt(6.f / kIn));
  for (int i = 0; i < kHid * kHid; ++i) th[oW2 + i] = uni(std::sqrt(6.f / kHid));
  for (int i = 0; i < kHid; ++i) th[oW3 + i] = uni(std::sqrt(6.f / kHid));
  if ((s = hrm_detector_set_weights(d, th))) return bail(s);
  *out = d;
  return HRM_OK;
}

void hrm_detector_destroy(hrm_detector* d) {
  if (!d) return;
  if (d->stream) cudaStreamSynchronize(d->stream);
  cudaFree(d->theta);
  cudaFree(d->m);
  cudaFree(d->v);
  cudaFree(d->scratch);
  cudaFree(d->blob);
  cudaFree(d->waits);
  cudaFree(d->conf);
  cudaFree(d->conf_loss);
  cudaFree(d->X);
  cudaFree(d->y);
  cudaFree(d->dev);
  cudaFree(d->z);
  cudaFree(d->partials);
  cudaFree(d->loss_parts);
  cudaFree(d->hist);
  cudaFree(d->counts);
  cudaFree(d->offsets);
  cudaFree(d->total);
  delete d;
}

const char* hrm_detector_last_error(const hrm_detector* d) { return d ? d->err.c_str() : "null detector"; }

hrm_status hrm_detector_set_weights(hrm_detector* d, const float* theta) {
  if (!d || !theta) return HRM_E_INVAL;
  hrm_status s;
  const size_t P = sizeof(float) * kParams;
  if ((s = dcheck(d, cudaMemcpyAsync(d->theta, theta, P, cudaMemcpyHostToDevice, d->stream), "copy weights")))
    return s;
  cudaMemsetAsync(d->m, 0, P, d->stream);
  cudaMemsetAsync(d->v, 0, P, d->stream);
  d->adam_t = 0;
  if ((s = pack(d))) return s;
  return dcheck(d, cudaStreamSynchronize(d->stream), "set weights");
}

hrm_status hrm_detector_get_weights(hrm_detector* d, float* theta) {
  if (!d || !theta) return HRM_E_INVAL;
  hrm_status s = dcheck(
      d, cudaMemcpyAsync(theta, d->theta, sizeof(float) * kParams, cudaMemcpyDeviceToHost, d->stream), "copy weights");
  if (s) return s;
  return dcheck(d, cudaStreamSynchronize(d->stream), "get weights");
}

int64_t hrm_detector_size(const hrm_detector* d) { return d ? d->size : 0; }

hrm_status hrm_detector_clear(hrm_detector* d) {
  if (!d) return HRM_E_INVAL;
  d->size = 0;
  return HRM_OK;
}

hrm_status hrm_detector_add_samples(hrm_detector* d, const float* X, const float* y, int64_t n) {
  if (!d || (n > 0 && (!X || !y)) || n < 0) return HRM_E_INVAL;
  if (d->size + n > d->cap) return dfail(d, HRM_E_INVAL, "%lld samples exceed the capacity", (long long)n);
  if (n == 0) return HRM_OK;
  hrm_status s;
  if ((s = dcheck(d,
                  cudaMemcpy2DAsync(d->X + d->size * 32, 32 * sizeof(float), X, kIn * sizeof(float),
                                    kIn * sizeof(float), (size_t)n, cudaMemcpyHostToDevice, d->stream),
                  "copy samples")))
    return s;
  cudaMemsetAsync(d->dev + d->size, 0, sizeof(float) * n, d->stream);
  if ((s = dcheck(d, cudaMemcpyAsync(d->y + d->size, y, sizeof(float) * n, cudaMemcpyHostToDevice, d->stream),
                  "copy labels")))
    return s;
  // zero the two padding columns
  if ((s = dcheck(d,
                  cudaMemset2DAsync(d->X + d->size * 32 + kIn, 32 * sizeof(float), 0, 2 * sizeof(float), (size_t)n,
                                    d->stream),
                  "pad samples")))
    return s;
  d->size += n;
  return dcheck(d, cudaStreamSynchronize(d->stream), "add samples");
}

hrm_status hrm_detector_samples(hrm_detector* d, int64_t first, int64_t n, float* X, float* y, float* dev) {
  if (!d || first < 0 || n < 0 || first + n > d->size) return HRM_E_INVAL;
  if (n == 0) return HRM_OK;
  hrm_status s = HRM_OK;
  if (X)
    s = dcheck(d,
               cudaMemcpy2DAsync(X, kIn * sizeof(float), d->X + first * 32, 32 * sizeof(float), kIn * sizeof(float),
                                 (size_t)n, cudaMemcpyDeviceToHost, d->stream),
               "read samples");
  if (!s && y)
    s = dcheck(d, cudaMemcpyAsync(y, d->y + first, sizeof(float) * n, cudaMemcpyDeviceToHost, d->stream),
               "read labels");
  if (!s && dev)
    s = dcheck(d, cudaMemcpyAsync(dev, d->dev + first, sizeof(float) * n, cudaMemcpyDeviceToHost, d->stream),
               "read deviations");
  if (s) return s;
  return dcheck(d, cudaStreamSynchronize(d->stream), "read samples");
}

hrm_status hrm_detector_collect(hrm_detector* d, hrm_ctx* ctx, double delta, double keep_rough, double keep_smooth,
                                double keep_flat, int64_t* added) {
  if (!d || !ctx) return HRM_E_INVAL;
  if (!(delta > 0.0) || keep_rough < 0 || keep_smooth < 0 || keep_flat < 0)
    return dfail(d, HRM_E_INVAL, "delta must be positive, keep probabilities non-negative");
  CtxView c;
  hrm_status s;
  if ((s = ctx_view(ctx, &c))) return dfail(d, s, "context not usable");
  cudaStream_t st = c.stream;
  // primitives and FP32 planes of the context's current state
  c.ck->prim(c.Wn, c.V, c.AUX, c.P32, c.R32, c.dg, c.fl, c.st, 0, nullptr, st);
  ctx_add_launches(ctx, 1);
  int64_t before = d->size;
  for (int dir = 0; dir < c.D; ++dir) {
    const int64_t nf = face_total(c.dg, dir);
    const int64_t nb = (nf + kCollectThreads - 1) / kCollectThreads;
    if (nb > d->nb_cap) {
      cudaStreamSynchronize(st);
      cudaFree(d->counts);
      cudaFree(d->offsets);
      cudaFree(d->total);
      d->counts = nullptr;
      d->offsets = nullptr;
      d->total = nullptr;
      d->nb_cap = 0;
      if ((s = dcheck(d, cudaMalloc(&d->counts, sizeof(int32_t) * nb), "alloc"))) return s;
      if ((s = dcheck(d, cudaMalloc(&d->offsets, sizeof(int64_t) * nb), "alloc"))) return s;
      if ((s = dcheck(d, cudaMalloc(&d->total, sizeof(int64_t)), "alloc"))) return s;
      d->nb_cap = nb;
    }
    CollectArgs a;
    a.V = c.V;
    a.AUX = c.AUX;
    a.P32 = c.P32;
    a.R32 = c.R32;
    a.g = c.dg;
    a.eps = c.dp.weno_eps;
    a.delta = delta;
    a.keep_rough = keep_rough;
    a.keep_smooth = keep_smooth;
    a.keep_flat = keep_flat;
    uint64_t h = d->seed ^ ((uint64_t)d->calls << 8) ^ (uint64_t)dir;
    h += 0x9E3779B97F4A7C15ull;
    h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
    a.salt = h ^ (h >> 27);
    a.counts = d->counts;
    a.offsets = d->offsets;
    a.X = d->X;
    a.y = d->y;
    a.dev = d->dev;
    a.cap = d->cap;
    launch_collect(c.N, c.D, dir, 0, a, st);
    launch_scan(d->counts, nb, d->size, d->offsets, d->total, st);
    launch_collect(c.N, c.D, dir, 1, a, st);
    ctx_add_launches(ctx, 3);
    int64_t tot = 0;
    if ((s = dcheck(d, cudaMemcpyAsync(&tot, d->total, sizeof tot, cudaMemcpyDeviceToHost, st), "read count")))
      return s;
    if ((s = dcheck(d, cudaStreamSynchronize(st), "collect"))) return s;
    d->size = d->size + tot < d->cap ? d->size + tot : d->cap;
  }
  ++d->calls;
  if (added) *added = d->size - before;
  return HRM_OK;
}

hrm_status hrm_detector_gradient(hrm_detector* d, int64_t first, int64_t n, float* grad, double* loss) {
  if (!d || first < 0 || n <= 0 || first + n > d->size) return HRM_E_INVAL;
  int nblk = 0;
  hrm_status s;
  if ((s = launch_grad(d, first, n, 0, 0, &nblk))) return s;
  k_mlp_reduce<<<(kParams + 255) / 256, 256, 0, d->stream>>>(d->partials, d->loss_parts, nblk, 1.f, d->scratch,
                                                             d->scratch + kParams);
  float h[kParams + 1];
  if ((s = dcheck(d, cudaMemcpyAsync(h, d->scratch, sizeof h, cudaMemcpyDeviceToHost, d->stream), "read gradient")))
    return s;
  if ((s = dcheck(d, cudaStreamSynchronize(d->stream), "gradient"))) return s;
  if (grad) std::memcpy(grad, h, sizeof(float) * kParams);
  if (loss) *loss = h[kParams];
  return HRM_OK;
}

hrm_status hrm_detector_train(hrm_detector* d, int32_t steps, int32_t batch, double lr, float* loss_per_step) {
  if (!d || steps < 0 || !(lr > 0.0)) return HRM_E_INVAL;
  if (d->size == 0) return dfail(d, HRM_E_INVAL, "no training samples");
  hrm_status s;
  const bool full = batch <= 0 || (int64_t)batch >= d->size;
  const int64_t count = full ? d->size : batch;
  if (steps > d->hist_cap) {
    cudaStreamSynchronize(d->stream);
    cudaFree(d->hist);
    d->hist = nullptr;
    d->hist_cap = 0;
    if ((s = dcheck(d, cudaMalloc(&d->hist, sizeof(float) * (size_t)steps), "alloc history"))) return s;
    d->hist_cap = steps;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int32_t k = 0; k < steps; ++k) {
    int nblk = 0;
    const uint64_t seed = d->seed * 0x2545F4914F6CDD1Dull + (uint64_t)(d->adam_t + 1) * 0x9E3779B97F4A7C15ull;
    if ((s = launch_grad(d, 0, count, full ? 0 : 1, seed, &nblk))) return s;
    ++d->adam_t;
    const double t = (double)d->adam_t;
    const float bc1 = (float)(1.0 - std::pow((double)b1, t));
    const float bc2 = (float)(1.0 - std::pow((double)b2, t));
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, d->stream>>>(d->theta, d->m, d->v, d->partials, d->loss_parts, nblk,
                                                             1.f / (float)count, (float)lr, b1, b2, eps, bc1, bc2,
                                                             d->hist + k);
    if ((s = dcheck(d, cudaGetLastError(), "adam kernel"))) return s;
  }
  if ((s = pack(d))) return s;
  if (loss_per_step && steps > 0)
    if ((s = dcheck(d,
                    cudaMemcpyAsync(loss_per_step, d->hist, sizeof(float) * steps, cudaMemcpyDeviceToHost,
                                    d->stream),
                    "read losses")))
      return s;
  return dcheck(d, cudaStreamSynchronize(d->stream), "train");
}

hrm_status hrm_detector_logits(hrm_detector* d, int64_t first, int64_t n, int32_t bf16, float* z) {
  if (!d || !z || first < 0 || n < 0 || first + n > d->size) return HRM_E_INVAL;
  if (n == 0) return HRM_OK;
  if (bf16)
    k_logits_bf16<<<(unsigned)((n + kGateThreads - 1) / kGateThreads), kGateThreads, 0, d->stream>>>(
        d->blob, d->X, first, n, d->z, d->waits);
  else
    k_logits_fp32<<<(unsigned)((n + kTrainThreads - 1) / kTrainThreads), kTrainThreads, 0, d->stream>>>(
        d->theta, d->X, first, n, d->z);
  hrm_status s;
  if ((s = dcheck(d, cudaGetLastError(), "logits"))) return s;
  if ((s = dcheck(d, cudaMemcpyAsync(z, d->z, sizeof(float) * n, cudaMemcpyDeviceToHost, d->stream), "read logits")))
    return s;
  return waits_check(d, "logits");
}

hrm_status hrm_detector_evaluate(hrm_detector* d, double threshold, int32_t bf16, int64_t counts[4], double* loss) {
  if (!d || !(threshold > 0.0 && threshold < 1.0)) return HRM_E_INVAL;
  const int64_t n = d->size;
  hrm_status s;
  cudaMemsetAsync(d->conf, 0, sizeof(unsigned long long) * 4, d->stream);
  cudaMemsetAsync(d->conf_loss, 0, sizeof(double), d->stream);
  if (n > 0) {
    if (bf16)
      k_logits_bf16<<<(unsigned)((n + kGateThreads - 1) / kGateThreads), kGateThreads, 0, d->stream>>>(
          d->blob, d->X, 0, n, d->z, d->waits);
    else
      k_logits_fp32<<<(unsigned)((n + kTrainThreads - 1) / kTrainThreads), kTrainThreads, 0, d->stream>>>(
          d->theta, d->X, 0, n, d->z);
    const float zthr = (float)std::log(threshold / (1.0 - threshold));
    k_confusion<<<256, 256, 0, d->stream>>>(d->z, d->y, n, zthr, d->conf, d->conf_loss);
  }
  if ((s = dcheck(d, cudaGetLastError(), "evaluate"))) return s;
  unsigned long long h[4];
  double l = 0.0;
  cudaMemcpyAsync(h, d->conf, sizeof h, cudaMemcpyDeviceToHost, d->stream);
  cudaMemcpyAsync(&l, d->conf_loss, sizeof l, cudaMemcpyDeviceToHost, d->stream);
  if ((s = waits_check(d, "evaluate"))) return s;
  if (counts)
    for (int k = 0; k < 4; ++k) counts[k] = (int64_t)h[k];
  if (loss) *loss = n > 0 ? l / (double)n : 0.0;
  return HRM_OK;
}

}  // extern "C"

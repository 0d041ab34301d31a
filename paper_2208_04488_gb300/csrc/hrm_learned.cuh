// Learned smoothness detector: a 30 -> 32 -> 32 -> 1 multilayer perceptron
// (ReLU hidden layers, sigmoid output) that reads the six-node stencil of a
// midpoint and predicts whether full WENO-IS (App. C) would keep every
// nonlinear weight of every characteristic field within delta of its linear
// weight d_k. Where it does, the midpoint is gated: the interpolation uses d_k
// and skips the weight computation; the projection, both limiters, the
// Riemann solves and the flux difference are unchanged.
//
// Inputs, per stencil and per quantity q in (alpha_1, alpha_2, rho, u_n, p),
// the normalised shape (q_j - mean q) / (max q - min q + 1e-30) over the nodes
// i-2 .. i+3, formed on the differences q_j - q_i (zero for an absent
// alpha_2). Inference: bfloat16 inputs and weights on the tensor cores
// (tcgen05.mma, FP32 accumulation in tensor memory), one CTA per 128
// midpoints (hrm_tc.cuh).
#pragma once

#include <cuda_bf16.h>

#include "hrm_face32.cuh"
#include "hrm_tc.cuh"

namespace hrm {
namespace mlp {

constexpr int kIn = 30, kHid = 32;
// FP32 parameter vector: W1[kIn][kHid], b1, W2[kHid][kHid], b2, w3, b3
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kIn * kHid;
constexpr int oW2 = oB1 + kHid;
constexpr int oB2 = oW2 + kHid * kHid;
constexpr int oW3 = oB2 + kHid;
constexpr int oB3 = oW3 + kHid;
constexpr int kParams = oB3 + 1;  // 2081

// Inference weights, prepared once on the device from the FP32 parameters and
// copied into shared memory per CTA: W1 and W2 transposed ([hidden n][input k],
// k >= kIn zero) as bf16 K-major operand tiles for the fifth-generation tensor
// cores in the no-swizzle core-matrix arrangement (element (n, k) at byte
// (n / 8) * 512 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2), then the FP32
// biases, output weights and output bias.
struct __align__(128) GateBlob {
  __nv_bfloat16 w1[kHid * 32];
  __nv_bfloat16 w2[kHid * 32];
  float b1[kHid], b2[kHid], w3[kHid];
  float b3, pad[31];
};
static_assert(sizeof(GateBlob) % 16 == 0, "blob copies in 16-byte words");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Shared memory of one CTA evaluating the network for 128 stencils.
struct __align__(128) NetTile {
  __nv_bfloat16 a[tc::kRows * 32];  // A operand: the features, then the first hidden layer (8 KB)
  GateBlob w;                       // B operands, biases, output weights
  unsigned long long bar;           // MMA completion barrier
  uint32_t tmem;                    // tensor-memory base address written by tcgen05.alloc
};

// Row r of the A operand from 32 FP32 values rounded to bf16: four 16-byte
// stores (eight consecutive rows fill 128 contiguous bytes: no bank conflict).
__device__ __forceinline__ void store_a_row(__nv_bfloat16* a, int r, const float (&x)[32]) {
  char* base = reinterpret_cast<char*>(a) + tc::tile_offset(r, 0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint4 v;
    v.x = pack_bf16(x[8 * c + 0], x[8 * c + 1]);
    v.y = pack_bf16(x[8 * c + 2], x[8 * c + 3]);
    v.z = pack_bf16(x[8 * c + 4], x[8 * c + 5]);
    v.w = pack_bf16(x[8 * c + 6], x[8 * c + 7]);
    *reinterpret_cast<uint4*>(base + c * 128) = v;
  }
}

// CTA set-up (all 128 threads): the weights into shared memory, the completion
// barrier, 32 tensor-memory columns. Returns the tensor-memory base address.
__device__ __forceinline__ uint32_t net_begin(NetTile& S, const GateBlob* __restrict__ blob) {
  const uint4* src = reinterpret_cast<const uint4*>(blob);
  uint4* dst = reinterpret_cast<uint4*>(&S.w);
  for (int i = threadIdx.x; i < (int)(sizeof(GateBlob) / 16); i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) tc::bar_init(tc::smem_u32(&S.bar));
  if (threadIdx.x < 32) tc::tmem_alloc(tc::smem_u32(&S.tmem));
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  return S.tmem;
}

// CTA tear-down (all 128 threads, after their last tensor-memory load): frees
// the tensor memory.
__device__ __forceinline__ void net_end(uint32_t tmem) {
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after();
    tc::tmem_free(tmem);
  }
}

// One hidden layer: every thread has written its row of S.a; one thread issues
// D = A B as two K = 16 slices and commits; all wait (bounded) and read their
// row of D.
__device__ __forceinline__ void net_layer(NetTile& S, const __nv_bfloat16* b, uint32_t tmem, uint32_t& phase,
                                          unsigned long long* waits, float (&d)[32]) {
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  const uint32_t bar = tc::smem_u32(&S.bar);
  if (threadIdx.x == 0) {
    tc::fence_after();
    const uint32_t a0 = tc::smem_u32(S.a), b0 = tc::smem_u32(b);
#pragma unroll
    for (uint32_t j = 0; j < 2; ++j)
      tc::mma_bf16(tmem, tc::smem_desc(a0 + 256 * j, 128, 512), tc::smem_desc(b0 + 256 * j, 128, 512), j);
    tc::mma_commit(bar);
  }
  if (!tc::bar_wait(bar, phase) && waits) atomicAdd(waits, 1ull);
  phase ^= 1u;
  tc::fence_after();
  // warp w reads tensor-memory lanes 32 w .. 32 w + 31: its own rows
  tc::tmem_ld32(tmem + ((uint32_t)(threadIdx.x & ~31) << 16), d);
}

// Logit of this thread's stencil from its features (all 128 threads call it).
__device__ __forceinline__ float net_logit(NetTile& S, const float (&x)[kIn], uint32_t tmem, uint32_t& phase,
                                           unsigned long long* waits) {
  const int r = threadIdx.x;
  float v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = k < kIn ? x[k] : 0.f;
  store_a_row(S.a, r, v);
  float d[32];
  net_layer(S, S.w.w1, tmem, phase, waits, d);
#pragma unroll
  for (int n = 0; n < kHid; ++n) v[n] = fmaxf(d[n] + S.w.b1[n], 0.f);
  store_a_row(S.a, r, v);
  net_layer(S, S.w.w2, tmem, phase, waits, d);
  float z = 0.f;
#pragma unroll
  for (int n = 0; n < kHid; ++n) z += fmaxf(d[n] + S.w.b2[n], 0.f) * S.w.w3[n];
  return z + S.w.b3;
}

// Logit of every thread's row, skipping the network for a tile of uniform
// stencils: a uniform stencil has exactly zero features, and an MMA row depends
// only on its own A row, so its logit is the zero-feature logit z0 the CTA
// computed once through the same path. CTA-wide (the same trip count for all).
__device__ __forceinline__ float net_logit_or_zero(NetTile& S, const float (&x)[kIn], float z0, uint32_t tmem,
                                                   uint32_t& phase, unsigned long long* waits) {
  int nz = 0;
#pragma unroll
  for (int k = 0; k < kIn; ++k) nz |= x[k] != 0.f;
  if (!__syncthreads_or(nz)) return z0;
  return net_logit(S, x, tmem, phase, waits);
}

// The zero-feature logit (every row zero), once per CTA.
__device__ __forceinline__ float net_zero_logit(NetTile& S, uint32_t tmem, uint32_t& phase,
                                                unsigned long long* waits) {
  float x0[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x0[k] = 0.f;
  return net_logit(S, x0, tmem, phase, waits);
}

// ---------------------------------------------------------------- one warp, 32 stencils
// The same network for the 32 stencils of one warp with warp-level MMA
// (mma.sync m16n8k16, bf16 inputs, FP32 accumulation): what the precision
// form's midpoint sweep runs in place of the gate kernel, only in warps that
// hold a non-uniform stencil. The B operands are read from the blob's tcgen05
// arrangement in global memory (L1-resident): B fragment word (n, k..k+1), k
// even, is one 32-bit word there.
__device__ __forceinline__ uint32_t blob_word(const __nv_bfloat16* w, int n, int k) {
  const char* p = reinterpret_cast<const char*>(w) + (n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
  return __ldg(reinterpret_cast<const unsigned int*>(p));
}

// D = A B + D: A 16x16 bf16 row-major fragments, B 16x8 bf16 column-major, D FP32.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Row stride (bf16) of a warp's feature tile in shared memory: 80 bytes, so
// that the eight rows a fragment load touches fall in distinct banks.
constexpr int kWarpRow = 40;

// Lane r writes its features as row r of the warp's tile X (bf16, columns
// kIn..31 zero).
__device__ __forceinline__ void warp_store_row(__nv_bfloat16 (*X)[kWarpRow], int r, const float (&x)[kIn]) {
  uint32_t* row = reinterpret_cast<uint32_t*>(X[r]);
#pragma unroll
  for (int k = 0; k < 16; ++k) row[k] = pack_bf16(2 * k < kIn ? x[2 * k] : 0.f, 2 * k + 1 < kIn ? x[2 * k + 1] : 0.f);
}

// Logit of the stencil in row `lane` of X. All 32 lanes call it, after every
// lane stored its row (and a __syncwarp). Fragment layout of m16n8k16: lane 4 g
// + q holds A rows g, g + 8 at columns 2q, 2q + 1 (and + 8), B column g at
// rows 2q, 2q + 1 (and + 8), and D rows g, g + 8 at columns 2q, 2q + 1, so the
// D tiles of one layer (bias, ReLU, bf16) are the A fragments of the next.
__device__ __forceinline__ float warp_logit(const GateBlob& W, const __nv_bfloat16 (*X)[kWarpRow], int lane) {
  const int g = lane >> 2, q = lane & 3;
  auto ld32 = [](const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); };
  float zr[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    float c1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) c1[nt][0] = c1[nt][1] = c1[nt][2] = c1[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      uint32_t a[4];
      a[0] = ld32(&X[16 * mt + g][16 * kt + 2 * q]);
      a[1] = ld32(&X[16 * mt + g + 8][16 * kt + 2 * q]);
      a[2] = ld32(&X[16 * mt + g][16 * kt + 2 * q + 8]);
      a[3] = ld32(&X[16 * mt + g + 8][16 * kt + 2 * q + 8]);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        mma_bf16(c1[nt], a, blob_word(W.w1, 8 * nt + g, 16 * kt + 2 * q),
                 blob_word(W.w1, 8 * nt + g, 16 * kt + 2 * q + 8));
    }
    uint32_t h[2][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = 8 * nt + 2 * q;
      const float b0 = __ldg(&W.b1[col]), b1 = __ldg(&W.b1[col + 1]);
      h[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(fmaxf(c1[nt][0] + b0, 0.f), fmaxf(c1[nt][1] + b1, 0.f));
      h[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(fmaxf(c1[nt][2] + b0, 0.f), fmaxf(c1[nt][3] + b1, 0.f));
    }
    float c2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) c2[nt][0] = c2[nt][1] = c2[nt][2] = c2[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        mma_bf16(c2[nt], h[kt], blob_word(W.w2, 8 * nt + g, 16 * kt + 2 * q),
                 blob_word(W.w2, 8 * nt + g, 16 * kt + 2 * q + 8));
    // output layer in FP32: this lane's columns, then the sum over the quad
    float sg = 0.f, sg8 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = 8 * nt + 2 * q;
      const float b0 = __ldg(&W.b2[col]), b1 = __ldg(&W.b2[col + 1]);
      const float w0 = __ldg(&W.w3[col]), w1 = __ldg(&W.w3[col + 1]);
      sg += fmaxf(c2[nt][0] + b0, 0.f) * w0 + fmaxf(c2[nt][1] + b1, 0.f) * w1;
      sg8 += fmaxf(c2[nt][2] + b0, 0.f) * w0 + fmaxf(c2[nt][3] + b1, 0.f) * w1;
    }
    sg += __shfl_xor_sync(0xffffffffu, sg, 1);
    sg += __shfl_xor_sync(0xffffffffu, sg, 2);
    sg8 += __shfl_xor_sync(0xffffffffu, sg8, 1);
    sg8 += __shfl_xor_sync(0xffffffffu, sg8, 2);
    const float b3 = __ldg(&W.b3);
    zr[mt][0] = sg + b3;
    zr[mt][1] = sg8 + b3;
  }
  // row r = 16 mt + 8 half + g' is held by lanes 4 g' .. 4 g' + 3
  const int src = 4 * (lane & 7);
  const float v00 = __shfl_sync(0xffffffffu, zr[0][0], src);
  const float v01 = __shfl_sync(0xffffffffu, zr[0][1], src);
  const float v10 = __shfl_sync(0xffffffffu, zr[1][0], src);
  const float v11 = __shfl_sync(0xffffffffu, zr[1][1], src);
  const int half = (lane >> 3) & 1;
  return (lane >> 4) ? (half ? v11 : v10) : (half ? v01 : v00);
}

// Normalise six differences (d[2] = 0) into x[0..5].
__device__ __forceinline__ void normalise6(const float (&d)[6], float* x) {
  float s = 0.f, lo = 0.f, hi = 0.f;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    s += d[j];
    lo = fminf(lo, d[j]);
    hi = fmaxf(hi, d[j]);
  }
  const float mean = s * (1.f / 6.f);
  const float inv = 1.f / ((hi - lo) + 1e-30f);
#pragma unroll
  for (int j = 0; j < 6; ++j) x[j] = (d[j] - mean) * inv;
}

// Stencil quantities of the features: 0, 1 = alpha_1, alpha_2 (the second
// absent for N = 2), 2 = rho, 3 = u_DIR, 4 = p.
constexpr int kQuant = 5;

// The 30 normalised features from a node loader: val(s, j) and res(s, j) are
// the FP32 value and its FP32 rounding residue of quantity s at stencil node j
// (i-2 .. i+3). Every difference q_j - q_i is formed from both, so that
// variations far below FP32 resolution keep their shape.
template <int N, typename Val, typename Res>
__device__ __forceinline__ void features_from(Val val, Res res, float (&x)[kIn]) {
  float d[6];
#pragma unroll
  for (int s = 0; s < kQuant; ++s) {
    if (s == 1 && N < 3) {
#pragma unroll
      for (int j = 0; j < 6; ++j) x[6 + j] = 0.f;
      continue;
    }
    const float c2 = val(s, 2), r2 = res(s, 2);
#pragma unroll
    for (int j = 0; j < 6; ++j) d[j] = (val(s, j) - c2) + (res(s, j) - r2);
    normalise6(d, x + 6 * s);
  }
}

// FP32 planes holding quantity s (values in P32; residues of the volume
// fractions in P32, those of rho, u_DIR and p in R32).
template <int N, int D, int DIR>
__host__ __device__ constexpr int val_plane(int s) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  return s < 2 ? L::AL + s : (s == 2 ? Q::RHO : (s == 3 ? L::MOM + DIR : L::EN));
}
template <int N, int D, int DIR>
__host__ __device__ constexpr int res_plane(int s) {
  using Q = P32Lay<N, D>;
  return s < 2 ? Q::ALO + s : (s == 2 ? 0 : (s == 3 ? 1 + DIR : 1 + D));
}

// The features of a midpoint read straight from the FP32 planes at its six
// nodes (nd: cell indices after the boundary mapping).
template <int N, int D, int DIR>
__device__ __forceinline__ void stencil_features(const Nodes6& nd, const float* __restrict__ P32,
                                                 const float* __restrict__ R32, int64_t nc, float (&x)[kIn]) {
  auto val = [&](int s, int j) -> float { return P32[(int64_t)val_plane<N, D, DIR>(s) * nc + nd.c[j]]; };
  auto res = [&](int s, int j) -> float {
    return (s < 2 ? P32 : R32)[(int64_t)res_plane<N, D, DIR>(s) * nc + nd.c[j]];
  };
  features_from<N>(val, res, x);
}

}  // namespace mlp

}  // namespace hrm

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
// (mma.sync m16n8k16, FP32 accumulation), one warp per 32 midpoints.
#pragma once

#include <cuda_bf16.h>

#include "hrm_face32.cuh"

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
constexpr int kRow = 40;          // bf16 row stride of the operand tiles (80 B: conflict-free fragments)

// Inference weights in the layout the fragments read (prepared once on the
// device from the FP32 parameters; copied into shared memory per block).
struct __align__(16) GateBlob {
  __nv_bfloat16 w1t[kHid][kRow];  // [hidden n][input k]; k >= kIn zero
  __nv_bfloat16 w2t[kHid][kRow];  // [hidden n][hidden k]
  float b1[kHid], b2[kHid], w3[kHid];
  float b3, pad[3];
};
static_assert(sizeof(GateBlob) % 16 == 0, "blob copies in 16-byte words");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D = A B + D, A 16x16 bf16 (row-major fragments), B 16x8 bf16 (column-major), FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Logit of the stencil whose features lane r of the warp wrote into row r of X
// (bf16, kRow stride; columns kIn..31 zero). All 32 lanes must call it.
// Fragment layout of m16n8k16: lane = 4 g + q holds A rows g, g+8 at columns
// 2q, 2q+1 (+8), B column g at rows 2q, 2q+1 (+8), C rows g, g+8 at columns
// 2q, 2q+1. The C tiles of one layer are the A fragments of the next.
__device__ __forceinline__ float warp_logit(const GateBlob& W, const __nv_bfloat16 (*X)[kRow], int lane) {
  const int g = lane >> 2, q = lane & 3;
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
        mma_bf16(c1[nt], a, ld32(&W.w1t[8 * nt + g][16 * kt + 2 * q]), ld32(&W.w1t[8 * nt + g][16 * kt + 2 * q + 8]));
    }
    // bias + ReLU, rounded to bf16: the A fragments of the second layer
    uint32_t h[2][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = 8 * nt + 2 * q;
      const float b0 = W.b1[col], b1 = W.b1[col + 1];
      const uint32_t rg = pack_bf16(fmaxf(c1[nt][0] + b0, 0.f), fmaxf(c1[nt][1] + b1, 0.f));
      const uint32_t rg8 = pack_bf16(fmaxf(c1[nt][2] + b0, 0.f), fmaxf(c1[nt][3] + b1, 0.f));
      h[nt >> 1][(nt & 1) * 2 + 0] = rg;
      h[nt >> 1][(nt & 1) * 2 + 1] = rg8;
    }
    float c2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) c2[nt][0] = c2[nt][1] = c2[nt][2] = c2[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        mma_bf16(c2[nt], h[kt], ld32(&W.w2t[8 * nt + g][16 * kt + 2 * q]),
                 ld32(&W.w2t[8 * nt + g][16 * kt + 2 * q + 8]));
    // output layer in FP32: partial dot products over this lane's columns, then the quad
    float sg = 0.f, sg8 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = 8 * nt + 2 * q;
      const float b0 = W.b2[col], b1 = W.b2[col + 1], w0 = W.w3[col], w1 = W.w3[col + 1];
      sg += fmaxf(c2[nt][0] + b0, 0.f) * w0 + fmaxf(c2[nt][1] + b1, 0.f) * w1;
      sg8 += fmaxf(c2[nt][2] + b0, 0.f) * w0 + fmaxf(c2[nt][3] + b1, 0.f) * w1;
    }
    sg += __shfl_xor_sync(0xffffffffu, sg, 1);
    sg += __shfl_xor_sync(0xffffffffu, sg, 2);
    sg8 += __shfl_xor_sync(0xffffffffu, sg8, 1);
    sg8 += __shfl_xor_sync(0xffffffffu, sg8, 2);
    zr[mt][0] = sg + W.b3;
    zr[mt][1] = sg8 + W.b3;
  }
  // row r = 16 mt + 8 half + g' lives in lanes 4 g'
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

// The 30 normalised features of a midpoint from the FP32 planes of the
// precision form: every difference q_j - q_i is formed from the FP32 value
// and its rounding residue (the volume fractions' from P32, those of rho,
// u_DIR and p from R32), so that variations far below FP32 resolution keep
// their shape.
template <int N, int D, int DIR>
__device__ __forceinline__ void stencil_features(const Nodes6& nd, const float* __restrict__ P32,
                                                 const float* __restrict__ R32, int64_t nc, float (&x)[kIn]) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  auto ld = [&](int plane, int j) -> float { return P32[(int64_t)plane * nc + nd.c[j]]; };
  float d[6];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (k < N - 1) {
      const float h2 = ld(L::AL + k, 2), l2 = ld(Q::ALO + k, 2);
#pragma unroll
      for (int j = 0; j < 6; ++j) d[j] = (ld(L::AL + k, j) - h2) + (ld(Q::ALO + k, j) - l2);
      normalise6(d, x + 6 * k);
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) x[6 * k + j] = 0.f;
    }
  }
  const int planes[3] = {Q::RHO, L::MOM + DIR, L::EN};
  const int rplanes[3] = {0, 1 + DIR, 1 + D};
  auto lr = [&](int plane, int j) -> float { return R32[(int64_t)plane * nc + nd.c[j]]; };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float c2 = ld(planes[a], 2), r2 = lr(rplanes[a], 2);
#pragma unroll
    for (int j = 0; j < 6; ++j) d[j] = (ld(planes[a], j) - c2) + (lr(rplanes[a], j) - r2);
    normalise6(d, x + 12 + 6 * a);
  }
}

// Write one lane's features as a bf16 row (columns kIn..31 zero).
__device__ __forceinline__ void store_row(__nv_bfloat16* row, const float (&x)[kIn]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(row);
#pragma unroll
  for (int k = 0; k < kIn / 2; ++k) r[k] = pack_bf16(x[2 * k], x[2 * k + 1]);
  r[kIn / 2] = 0u;
}

}  // namespace mlp

// Precision-form midpoint sweep with the detector evaluated in the same
// kernel: each warp forms its 32 stencils' features, runs the network on the
// tensor cores, records the decisions in gate_out and then computes its
// midpoints with the linear weights where gated. All lanes take part in the
// network even past the last midpoint. DEFER: as k_face32_fast, midpoints whose
// screens fail go to `list` (k_face32_fix then reads their gate bytes).
template <int N, int D, int DIR, bool DEFER = false>
__global__ void __launch_bounds__(kFaceThreads, DEFER ? 4 : 3)
    k_face32_learned(const double* __restrict__ W, const float* __restrict__ P32, const float* __restrict__ R32,
                     double* __restrict__ out, DevGrid g, DevFluid f, DevParams pr, const StepState* __restrict__ st,
                     const mlp::GateBlob* __restrict__ blob, float zthr, uint8_t* __restrict__ gate_out,
                     uint32_t* __restrict__ list = nullptr, uint32_t* __restrict__ count = nullptr) {
  __shared__ __align__(16) mlp::GateBlob Wb;
  __shared__ __align__(16) __nv_bfloat16 X[kFaceThreads / 32][32][mlp::kRow];
  {
    const uint4* src = reinterpret_cast<const uint4*>(blob);
    uint4* dst = reinterpret_cast<uint4*>(&Wb);
    for (int i = threadIdx.x; i < (int)(sizeof(mlp::GateBlob) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Nodes6 nd;
  const bool ok = face_nodes<DIR>(g, t, nd);
  bool lin;
  {
    float x[mlp::kIn];
    if (ok) {
      mlp::stencil_features<N, D, DIR>(nd, P32, R32, g.ncells, x);
    } else {
#pragma unroll
      for (int k = 0; k < mlp::kIn; ++k) x[k] = 0.f;
    }
    mlp::store_row(X[warp][lane], x);
    __syncwarp();
    lin = mlp::warp_logit(Wb, X[warp], lane) > zthr;
  }
  if constexpr (!DEFER) {
    if (!ok) return;
    gate_out[t] = lin ? 1 : 0;
    face32_body<N, D, DIR>(t, nd, W, nullptr, nullptr, P32, out, g, f, pr, st->lam[DIR], lin);
  } else {
    bool need = false;
    if (ok) {
      gate_out[t] = lin ? 1 : 0;
      need = !face32_body<N, D, DIR, true>(t, nd, W, nullptr, nullptr, P32, out, g, f, pr, st->lam[DIR], lin);
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (need) list[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)t;
  }
}

}  // namespace hrm

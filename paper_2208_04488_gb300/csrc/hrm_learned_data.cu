// Training data of the learned smoothness detector, collected from states the
// method itself produces: for every midpoint of a direction, the 30 stencil
// features (exactly as the gate computes them) and the label, 1 when every
// WENO-IS weight of every characteristic field and both biases lies within
// delta of its linear weight d_k (App. C, App. D), else 0. Midpoints are kept
// with a probability that depends on their class (rough, smooth, or uniform
// stencil), drawn from a counter-based hash of the midpoint index, and written
// in index order (count pass, scan, write pass), so a collection is
// reproducible.
//
// Built without FMA contraction: the weight deviation is computed with the
// same FP64 operations as the method's interpolation.
#include "hrm_learned.h"

namespace hrm {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Largest weight deviation over both biases and all characteristic fields of
// the midpoint (the projection of the FP64 midpoint kernel).
template <int N, int D, int DIR>
__device__ double stencil_dev(const Nodes6& nd, const double* __restrict__ V, const double* __restrict__ AUX,
                              int64_t nc, double eps) {
  using L = Lay<N, D>;
  const double* Cc = AUX;
  const double* Rr = AUX + nc;
  double p6[6], u6[6], w6[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    p6[j] = V[L::EN * nc + nd.c[j]];
    u6[j] = V[(L::MOM + DIR) * nc + nd.c[j]];
  }
  const double rhob = 0.5 * (Rr[nd.c[2]] + Rr[nd.c[3]]);
  const double cb = 0.5 * (Cc[nd.c[2]] + Cc[nd.c[3]]);
  const double inv_rc = 1.0 / (rhob * cb);
  const double rc2b = rhob * cb * cb;
  double mx = 0.0;
  auto both = [&]() {
    const double l = weno_dev<double>(w6[0], w6[1], w6[2], w6[3], w6[4], eps);
    const double r = weno_dev<double>(w6[5], w6[4], w6[3], w6[2], w6[1], eps);
    if (!(l <= mx)) mx = l;
    if (!(r <= mx)) mx = r;
  };
#pragma unroll
  for (int j = 0; j < 6; ++j) w6[j] = u6[j] - inv_rc * p6[j];
  both();
#pragma unroll
  for (int j = 0; j < 6; ++j) w6[j] = u6[j] + inv_rc * p6[j];
  both();
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = V[k * nc + nd.c[j]];
    const double arb = 0.5 * (w6[2] + w6[3]);
    const double coef = arb / rc2b;
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = w6[j] - coef * p6[j];
    both();
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (d == DIR) continue;
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = V[(L::MOM + d) * nc + nd.c[j]];
    both();
  }
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = V[(L::AL + k) * nc + nd.c[j]];
    both();
  }
  return mx;
}

template <int N, int D, int DIR>
__global__ void __launch_bounds__(kCollectThreads) k_collect(CollectArgs a, int pass) {
  const int64_t t = (int64_t)blockIdx.x * kCollectThreads + threadIdx.x;
  Nodes6 nd;
  const bool in = face_nodes<DIR>(a.g, t, nd);
  bool keep = false;
  float x[mlp::kIn];
  double dv = 0.0;
  if (in) {
    mlp::stencil_features<N, D, DIR>(nd, a.P32, a.R32, a.g.ncells, x);
    dv = stencil_dev<N, D, DIR>(nd, a.V, a.AUX, a.g.ncells, a.eps);
    bool flat = true;
#pragma unroll
    for (int k = 0; k < mlp::kIn; ++k) flat &= x[k] == 0.f;
    const bool smooth = dv < a.delta;
    const double p = !smooth ? a.keep_rough : (flat ? a.keep_flat : a.keep_smooth);
    const double u = (double)(splitmix64(a.salt ^ (uint64_t)t) >> 11) * 0x1.0p-53;
    keep = u < p;
  }
  if (pass == 0) {
    const int n = __syncthreads_count(keep);
    if (threadIdx.x == 0) a.counts[blockIdx.x] = n;
    return;
  }
  __shared__ int wsum[kCollectThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned ball = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) wsum[warp] = __popc(ball);
  __syncthreads();
  if (!keep) return;
  int pre = __popc(ball & ((1u << lane) - 1u));
  for (int w = 0; w < warp; ++w) pre += wsum[w];
  const int64_t pos = a.offsets[blockIdx.x] + pre;
  if (pos >= a.cap) return;
  float4* row = reinterpret_cast<float4*>(a.X + pos * 32);
#pragma unroll
  for (int k = 0; k < 7; ++k) row[k] = make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
  row[7] = make_float4(x[28], x[29], 0.f, 0.f);
  a.y[pos] = dv < a.delta ? 1.f : 0.f;
  a.dev[pos] = (float)dv;
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
    k_scan(const int32_t* __restrict__ counts, int64_t nb, int64_t base, int64_t* __restrict__ offsets,
           int64_t* __restrict__ total) {
  __shared__ int64_t part[kScanThreads];
  const int64_t chunk = (nb + kScanThreads - 1) / kScanThreads;
  const int64_t lo = (int64_t)threadIdx.x * chunk;
  const int64_t hi = lo + chunk < nb ? lo + chunk : nb;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // inclusive scan of the chunk sums (Hillis-Steele)
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = base + part[threadIdx.x] - s;
  for (int64_t i = lo; i < hi; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == kScanThreads - 1) *total = part[kScanThreads - 1];
}

template <int N, int D>
void collect_nd(int dir, int pass, const CollectArgs& a, cudaStream_t s) {
  const int64_t nf = face_total(a.g, dir);
  const unsigned grid = (unsigned)((nf + kCollectThreads - 1) / kCollectThreads);
  if (dir == 0) k_collect<N, D, 0><<<grid, kCollectThreads, 0, s>>>(a, pass);
  if constexpr (D > 1)
    if (dir == 1) k_collect<N, D, 1><<<grid, kCollectThreads, 0, s>>>(a, pass);
  if constexpr (D > 2)
    if (dir == 2) k_collect<N, D, 2><<<grid, kCollectThreads, 0, s>>>(a, pass);
}

}  // namespace

void launch_collect(int N, int D, int dir, int pass, const CollectArgs& a, cudaStream_t s) {
  const int key = N * 10 + D;
  switch (key) {
    case 21: collect_nd<2, 1>(dir, pass, a, s); break;
    case 22: collect_nd<2, 2>(dir, pass, a, s); break;
    case 23: collect_nd<2, 3>(dir, pass, a, s); break;
    case 31: collect_nd<3, 1>(dir, pass, a, s); break;
    case 32: collect_nd<3, 2>(dir, pass, a, s); break;
    case 33: collect_nd<3, 3>(dir, pass, a, s); break;
    default: break;
  }
}

void launch_scan(const int32_t* counts, int64_t nb, int64_t base, int64_t* offsets, int64_t* total, cudaStream_t s) {
  k_scan<<<1, kScanThreads, 0, s>>>(counts, nb, base, offsets, total);
}

}  // namespace hrm

// A cache-friendly processing order for the refinement stage.
//
// Refining row i reads the FP32 rows of its candidates; neighbouring rows of
// the same cluster share most candidates.  Processing the rows cluster by
// cluster lets the warps of one CTA (and the SM's L1) reuse those rows.  The
// order only changes which rows run together, never a result.
//
//   1. every row's best 4 non-self candidates from the similarity lists;
//   2. label propagation: label_i = min(i, labels of those candidates), a few
//      rounds (connected rows converge to a common label);
//   3. counting sort of the rows by label.
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int NB = 4;

__global__ void k_top_nb(const float* __restrict__ part_s, const int32_t* __restrict__ part_i, int P, int K,
                         int64_t n, int32_t* __restrict__ nb, int32_t* __restrict__ label) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float bs[NB];
  int bi[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    bs[k] = -3.0e38f;
    bi[k] = int(i);
  }
  const size_t base = size_t(i) * P * K;
  for (int p = 0; p < P; ++p) {
    for (int e = 0; e < NB + 1 && e < K; ++e) {  // the lists are sorted: the first NB+1 cover self
      const int c = part_i[base + size_t(p) * K + e];
      if (c < 0 || c >= n || c == i) continue;  // empty slot (or a list an aborted stage left unwritten)
      float s = part_s[base + size_t(p) * K + e];
      int ci = c;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (ranks_before(s, ci, bs[k], bi[k])) {
          const float ts = bs[k];
          const int ti = bi[k];
          bs[k] = s;
          bi[k] = ci;
          s = ts;
          ci = ti;
        }
      }
    }
  }
  int m = int(i);
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    nb[i * NB + k] = bi[k];
    m = min(m, bi[k]);
  }
  label[i] = m;
}

// In place: labels only decrease, so reading a neighbour's newer label is fine.
__global__ void k_label_step(const int32_t* __restrict__ nb, int64_t n, int32_t* label) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = label[i];
#pragma unroll
  for (int k = 0; k < NB; ++k) m = min(m, label[nb[i * NB + k]]);
  label[i] = m;
}

__global__ void k_label_count(const int32_t* __restrict__ label, int64_t n, int32_t* __restrict__ cnt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[label[i]], 1);
}

__global__ void k_label_scatter(const int32_t* __restrict__ label, int64_t n, const int32_t* __restrict__ start,
                                int32_t* __restrict__ fill, int32_t* __restrict__ order) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int l = label[i];
  order[start[l] + atomicAdd(&fill[l], 1)] = int32_t(i);
}

}  // namespace

int launch_cluster_order(const Shape& sh, const float* part_s, const int32_t* part_i, int32_t* nb, int32_t* label,
                         int32_t* cnt, int32_t* start, int32_t* fill, int32_t* order, cudaStream_t s) {
  const int T = 256;
  const int64_t n = sh.n;
  const unsigned g = unsigned((n + T - 1) / T);
  k_top_nb<<<g, T, 0, s>>>(part_s, part_i, sh.P, sh.K, n, nb, label);
  for (int r = 0; r < 3; ++r) k_label_step<<<g, T, 0, s>>>(nb, n, label);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * size_t(n), s);
  cudaMemsetAsync(fill, 0, sizeof(int32_t) * size_t(n), s);
  k_label_count<<<g, T, 0, s>>>(label, n, cnt);
  launch_scan32(cnt, n, start, s);
  k_label_scatter<<<g, T, 0, s>>>(label, n, start, fill, order);
  return 7;
}

int cluster_order_nb() { return NB; }

}  // namespace rr

// K3: graph construction (Eq. 8-12) from the exact neighbour lists.
//
//   A_ij = 1 iff j in N(i, k1)                       (Eq. 8)
//   A*   = (A + A^T) / 2, entries 1 (reciprocal) or 1/2 (one-way)   (Eq. 9, 10)
//   h_i^(0) = row i of A* (or of A)                  (Eq. 11, Table 1)
//   message weights e_ij^alpha for j in N(i, k2)     (Eq. 12, 14)
//
// Rows of A^T are gathered by a counting sort of the n*k1 edges (in-degree
// count, exclusive scan, scatter), each out-list and in-list is sorted by
// index, and row i of A* is the sorted union of the two lists: value 1 where
// the column is in both, 1/2 otherwise.  h^(0) is written as CSR (rowptr,
// col ascending, val) and mirrored into the padded-CSR (start, len) form the
// propagation layers use.
//
// The message list of row i folds the residual term of Eq. 13 into the self
// coefficient: entries (j, c_j) for j in N(i, k2) with c_j = e_ij^alpha (sum)
// or e_ij^alpha / k2 (mean), and c_i gets +1; self is appended with c_i = 1
// when it is not in N(i, k2).  Max aggregator: the k2 entries (j, e_ij^alpha)
// are combined by element-wise max, and the residual follows as a last entry
// (i, -1): a negative coefficient means "add with weight 1".
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

__global__ void k3_indeg(const int32_t* __restrict__ knn, int64_t edges, int32_t* __restrict__ indeg) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < edges) atomicAdd(&indeg[knn[e]], 1);
}

__global__ void k3_scatter(const int32_t* __restrict__ knn, int64_t edges, int k1, const int32_t* __restrict__ inptr,
                           int32_t* __restrict__ fill, int32_t* __restrict__ insrc) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= edges) return;
  const int32_t j = knn[e];
  const int32_t pos = inptr[j] + atomicAdd(&fill[j], 1);
  insrc[pos] = int32_t(e / k1);
}

__device__ __forceinline__ int lower_bound(const int32_t* a, int m, int32_t v) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One warp per row: sort the out-list and the in-list by index (rank by
// counting; the values of each list are distinct), count |out n in|.
__global__ void k3_sort_count(const int32_t* __restrict__ knn, int64_t n, int k1, const int32_t* __restrict__ inptr,
                              const int32_t* __restrict__ insrc, int32_t* __restrict__ out_sorted,
                              int32_t* __restrict__ in_sorted, int32_t* __restrict__ rowcnt, int feature) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int32_t* o = knn + i * k1;
  for (int r = lane; r < k1; r += kWarp) {
    const int32_t v = o[r];
    int rank = 0;
    for (int q = 0; q < k1; ++q) rank += o[q] < v;
    out_sorted[i * k1 + rank] = v;
  }
  const int32_t a = inptr[i], m = inptr[i + 1] - a;
  for (int r = lane; r < m; r += kWarp) {
    const int32_t v = insrc[a + r];
    int rank = 0;
    for (int q = 0; q < m; ++q) rank += insrc[a + q] < v;
    in_sorted[a + rank] = v;
  }
  __syncwarp();
  int both = 0;
  for (int r = lane; r < k1; r += kWarp) {
    const int32_t v = out_sorted[i * k1 + r];
    const int p = lower_bound(in_sorted + a, m, v);
    both += (p < m && in_sorted[a + p] == v);
  }
  both = warp_sum(both);
  if (lane == 0) rowcnt[i] = feature == RERANK_FEAT_A ? k1 : k1 + m - both;
}

// One thread per row: merge the two sorted lists into row i of A* (or copy A).
__global__ void k3_fill(const int32_t* __restrict__ out_sorted, const int32_t* __restrict__ in_sorted,
                        const int32_t* __restrict__ inptr, const int32_t* __restrict__ h0ptr, int64_t n, int k1,
                        int feature, int32_t* __restrict__ col, float* __restrict__ val,
                        int64_t* __restrict__ start, int32_t* __restrict__ len, long long* __restrict__ nnz0) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t* o = out_sorted + i * k1;
  int32_t pos = h0ptr[i];
  if (feature == RERANK_FEAT_A) {
    for (int p = 0; p < k1; ++p) {
      col[pos + p] = o[p];
      val[pos + p] = 1.0f;
    }
    pos += k1;
  } else {
    const int32_t* in = in_sorted + inptr[i];
    const int m = inptr[i + 1] - inptr[i];
    int p = 0, q = 0;
    while (p < k1 || q < m) {
      const int32_t vo = p < k1 ? o[p] : kInvalidIdx;
      const int32_t vi = q < m ? in[q] : kInvalidIdx;
      if (vo == vi) {
        col[pos] = vo;
        val[pos] = 1.0f;
        ++p;
        ++q;
      } else if (vo < vi) {
        col[pos] = vo;
        val[pos] = 0.5f;
        ++p;
      } else {
        col[pos] = vi;
        val[pos] = 0.5f;
        ++q;
      }
      ++pos;
    }
  }
  start[i] = h0ptr[i];
  len[i] = pos - h0ptr[i];
  if (i == n - 1) {
    start[n] = pos;
    if (nnz0) *nnz0 = pos;  // nnz of h^(0)
  }
}

__global__ void k3_edges(const int32_t* __restrict__ knn, const float* __restrict__ score, int64_t n, int k1, int k2,
                         float alpha, int aggregator, int32_t* __restrict__ nbr, float* __restrict__ nbr_w,
                         int32_t* __restrict__ nbr_n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cnt = 0;
  bool self = false;
  const bool agg_max = aggregator == RERANK_AGG_MAX;
  for (int r = 0; r < k2; ++r) {
    const int32_t j = knn[i * k1 + r];
    const float e = score[i * k1 + r];
    float w = alpha == 2.0f ? e * e : (alpha == 0.0f ? 1.0f : powf(e, alpha));
    if (aggregator == RERANK_AGG_MEAN) w = w / float(k2);
    if (j == i && !agg_max) {
      w += 1.0f;
      self = true;
    }
    nbr[i * (k2 + 1) + cnt] = j;
    nbr_w[i * (k2 + 1) + cnt] = w;
    ++cnt;
  }
  if (!self) {
    // The residual h_i of Eq. 13.  With the max aggregator it is its own last
    // message, marked by a negative weight: added after the element-wise max
    // of the k2 weighted neighbour rows.
    nbr[i * (k2 + 1) + cnt] = int32_t(i);
    nbr_w[i * (k2 + 1) + cnt] = agg_max ? -1.0f : 1.0f;
    ++cnt;
  }
  nbr_n[i] = cnt;
}

}  // namespace

int launch_graph(const Shape& sh, const Buffers& b, float alpha, int aggregator, int feature, long long* status,
                  cudaStream_t s) {
  const int64_t n = sh.n, edges = n * sh.k1;
  const int T = 256;
  cudaMemsetAsync(b.indeg, 0, sizeof(int32_t) * n, s);
  cudaMemsetAsync(b.fill, 0, sizeof(int32_t) * n, s);
  k3_indeg<<<unsigned((edges + T - 1) / T), T, 0, s>>>(b.knn_idx, edges, b.indeg);
  launch_scan32(b.indeg, n, b.inptr, s);
  k3_scatter<<<unsigned((edges + T - 1) / T), T, 0, s>>>(b.knn_idx, edges, sh.k1, b.inptr, b.fill, b.insrc);
  k3_sort_count<<<unsigned((n * kWarp + T - 1) / T), T, 0, s>>>(b.knn_idx, n, sh.k1, b.inptr, b.insrc, b.out_sorted,
                                                               b.in_sorted, b.rowcnt, feature);
  launch_scan32(b.rowcnt, n, b.h0ptr, s);
  k3_fill<<<unsigned((n + T - 1) / T), T, 0, s>>>(b.out_sorted, b.in_sorted, b.inptr, b.h0ptr, n, sh.k1, feature,
                                                  b.col[2], b.val[2], b.start[2], b.len[2],
                                                  status ? status + kStNnz0 : nullptr);
  k3_edges<<<unsigned((n + T - 1) / T), T, 0, s>>>(b.knn_idx, b.knn_score, n, sh.k1, sh.k2, alpha, aggregator, b.nbr,
                                                   b.nbr_w, b.nbr_n);
  return 7;
}

}  // namespace rr

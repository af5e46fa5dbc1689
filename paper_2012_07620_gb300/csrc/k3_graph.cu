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
#include <algorithm>

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

// ---- incremental graph of a serving request (A* features) ----
// Union rows: the request's queries 0 .. Q-1, gallery row g at Q + g.  The
// resident graph is the gallery's own (G alone, gallery indices).  Sources:
// the queries and the touched gallery rows (their lists may differ from the
// resident ones).  A row of A* = (A + A^T) / 2 can change only when its
// out-list changed (a source) or its in-list did: a target of a source's old
// or new list.  Every other row is the resident row, indices shifted by Q.

// Sources and their old and new targets are marked; new edges counted per target.
__global__ void k3i_mark(const int32_t* __restrict__ knn, int k1, int64_t Q, const int32_t* __restrict__ touched,
                         const int32_t* __restrict__ n_touched, const int32_t* __restrict__ res_knn,
                         uint8_t* __restrict__ aff, uint8_t* __restrict__ src, int32_t* __restrict__ add_cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nsrc = Q + *n_touched;
  const int64_t wstride = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t f = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; f < nsrc; f += wstride) {
    const int64_t i = f < Q ? f : int64_t(touched[f - Q]);
    for (int r = lane; r < k1; r += kWarp) {
      const int32_t j = knn[i * k1 + r];
      aff[j] = 1;
      atomicAdd(&add_cnt[j], 1);
      if (i >= Q) aff[res_knn[(i - Q) * k1 + r] + Q] = 1;
    }
    if (lane == 0) {
      aff[i] = 1;
      src[i] = 1;
    }
  }
}

__global__ void k3i_scatter(const int32_t* __restrict__ knn, int k1, int64_t Q, const int32_t* __restrict__ touched,
                            const int32_t* __restrict__ n_touched, const int32_t* __restrict__ add_ptr,
                            int32_t* __restrict__ add_fill, int32_t* __restrict__ add_src) {
  const int lane = threadIdx.x & 31;
  const int64_t nsrc = Q + *n_touched;
  const int64_t wstride = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t f = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; f < nsrc; f += wstride) {
    const int64_t i = f < Q ? f : int64_t(touched[f - Q]);
    for (int r = lane; r < k1; r += kWarp) {
      const int32_t j = knn[i * k1 + r];
      add_src[add_ptr[j] + atomicAdd(&add_fill[j], 1)] = int32_t(i);
    }
  }
}

// Resident in-list of gallery row g, as read from its resident A* row: the
// columns with value 1 (reciprocal) and those with value 1/2 that are not in
// g's own resident out-list.  Kept for the request only when the source is
// not itself a source of the request (its new edges are in the added list).
__device__ __forceinline__ bool res_in_kept(int32_t c, float v, const int32_t* __restrict__ res_out, int k1,
                                            const uint8_t* __restrict__ src, int64_t Q) {
  if (src[Q + c]) return false;
  if (v == 1.0f) return true;
  for (int q = 0; q < k1; ++q)
    if (res_out[q] == c) return false;
  return true;
}

// Affected rows: the out-list and the added sources sorted by index (rank by
// counting), and the size of the new row of A*; other rows keep their length.
__global__ void k3i_count(int64_t n, int64_t Q, int k1, const int32_t* __restrict__ knn,
                          const uint8_t* __restrict__ aff, const uint8_t* __restrict__ src,
                          const int32_t* __restrict__ add_ptr, const int32_t* __restrict__ add_src,
                          const int64_t* __restrict__ rst, const int32_t* __restrict__ rln,
                          const int32_t* __restrict__ rcol, const float* __restrict__ rval,
                          const int32_t* __restrict__ res_knn, int32_t* __restrict__ out_sorted,
                          int32_t* __restrict__ add_sorted, int32_t* __restrict__ rowcnt) {
  const int64_t u = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n) return;
  if (!aff[u]) {
    if (lane == 0) rowcnt[u] = rln[u - Q];  // queries are always affected
    return;
  }
  const int32_t* o = knn + u * k1;
  for (int r = lane; r < k1; r += kWarp) {
    const int32_t v = o[r];
    int rank = 0;
    for (int q = 0; q < k1; ++q) rank += o[q] < v;
    out_sorted[u * k1 + rank] = v;
  }
  const int32_t a = add_ptr[u], m = add_ptr[u + 1] - a;
  for (int r = lane; r < m; r += kWarp) {
    const int32_t v = add_src[a + r];
    int rank = 0;
    for (int q = 0; q < m; ++q) rank += add_src[a + q] < v;
    add_sorted[a + rank] = v;
  }
  __syncwarp();
  // |in| = kept resident in-sources + added sources (disjoint); |row| = k1 + |in| - |out n in|.
  int kept = 0, both = 0;
  if (u >= Q) {
    const int64_t g = u - Q, ra = rst[g];
    const int32_t* rout = res_knn + g * k1;
    for (int p = lane; p < rln[g]; p += kWarp) {
      const int32_t c = rcol[ra + p];
      if (res_in_kept(c, rval[ra + p], rout, k1, src, Q)) {
        ++kept;
        for (int q = 0; q < k1; ++q) both += out_sorted[u * k1 + q] == c + int32_t(Q);
      }
    }
  }
  for (int r = lane; r < k1; r += kWarp) {
    const int32_t v = out_sorted[u * k1 + r];
    const int p = lower_bound(add_sorted + a, m, v);
    both += (p < m && add_sorted[a + p] == v);
  }
  kept = warp_sum(kept);
  both = warp_sum(both);
  if (lane == 0) rowcnt[u] = k1 + kept + m - both;
}

// Rows of A* into the layer-0 CSR: resident rows copied (indices shifted by
// Q), affected rows as the sorted union of out and in (1 where in both, else
// 1/2) by one lane.
__global__ void k3i_fill(int64_t n, int64_t Q, int k1, const uint8_t* __restrict__ aff,
                         const uint8_t* __restrict__ src, const int32_t* __restrict__ h0ptr,
                         const int32_t* __restrict__ out_sorted, const int32_t* __restrict__ add_ptr,
                         const int32_t* __restrict__ add_sorted, const int64_t* __restrict__ rst,
                         const int32_t* __restrict__ rln, const int32_t* __restrict__ rcol,
                         const float* __restrict__ rval, const int32_t* __restrict__ res_knn,
                         int32_t* __restrict__ col, float* __restrict__ val, int64_t* __restrict__ start,
                         int32_t* __restrict__ len, long long* __restrict__ nnz0) {
  const int64_t u = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n) return;
  const int32_t dst = h0ptr[u];
  if (lane == 0) {
    start[u] = dst;
    len[u] = h0ptr[u + 1] - dst;
    if (u == n - 1) {
      start[n] = h0ptr[n];
      if (nnz0) *nnz0 = h0ptr[n];
    }
  }
  if (!aff[u]) {
    const int64_t g = u - Q, ra = rst[g];
    for (int p = lane; p < rln[g]; p += kWarp) {
      col[dst + p] = rcol[ra + p] + int32_t(Q);
      val[dst + p] = rval[ra + p];
    }
    return;
  }
  if (lane != 0) return;
  const int32_t* o = out_sorted + u * k1;
  const int32_t a = add_ptr[u], m = add_ptr[u + 1] - a;
  const int32_t* ad = add_sorted + a;
  // The in-list in ascending order: kept resident in-sources and added sources.
  int64_t ra = 0, rn = 0;
  const int32_t* rout = nullptr;
  if (u >= Q) {
    const int64_t g = u - Q;
    ra = rst[g];
    rn = rln[g];
    rout = res_knn + g * k1;
  }
  int64_t rp = 0;
  int ap = 0, op = 0;
  int32_t pos = dst;
  auto next_res = [&]() -> int32_t {  // next kept resident in-source (union index), or INT_MAX
    while (rp < rn) {
      const int32_t c = rcol[ra + rp];
      const float v = rval[ra + rp];
      ++rp;
      if (res_in_kept(c, v, rout, k1, src, Q)) return c + int32_t(Q);
    }
    return kInvalidIdx;
  };
  int32_t rv = next_res();
  for (;;) {
    const int32_t av = ap < m ? ad[ap] : kInvalidIdx;
    const int32_t iv = rv < av ? rv : av;  // next in-source
    const int32_t ov = op < k1 ? o[op] : kInvalidIdx;
    if (iv == kInvalidIdx && ov == kInvalidIdx) break;
    if (ov == iv) {
      col[pos] = ov;
      val[pos] = 1.0f;
      ++op;
    } else if (ov < iv) {
      col[pos] = ov;
      val[pos] = 0.5f;
      ++op;
      ++pos;
      continue;
    } else {
      col[pos] = iv;
      val[pos] = 0.5f;
    }
    if (iv == rv) rv = next_res();
    else ++ap;
    ++pos;
  }
}

}  // namespace

int launch_graph_incremental(const Shape& sh, const Buffers& b, int64_t Q, const int32_t* touched,
                             const int32_t* n_touched, const int32_t* res_knn, const int64_t* rst,
                             const int32_t* rln, const int32_t* rcol, const float* rval, uint8_t* aff,
                             uint8_t* src, float alpha, int aggregator, long long* status, cudaStream_t s) {
  const int64_t n = sh.n;
  const int T = 256;
  const unsigned rows_grid = unsigned((n * kWarp + T - 1) / T);
  const unsigned src_grid = unsigned(std::min<int64_t>((n * kWarp + T - 1) / T, 1024));
  cudaMemsetAsync(aff, 0, size_t(n), s);
  cudaMemsetAsync(src, 0, size_t(n), s);
  cudaMemsetAsync(b.indeg, 0, sizeof(int32_t) * n, s);
  cudaMemsetAsync(b.fill, 0, sizeof(int32_t) * n, s);
  k3i_mark<<<src_grid, T, 0, s>>>(b.knn_idx, sh.k1, Q, touched, n_touched, res_knn, aff, src, b.indeg);
  launch_scan32(b.indeg, n, b.inptr, s);
  k3i_scatter<<<src_grid, T, 0, s>>>(b.knn_idx, sh.k1, Q, touched, n_touched, b.inptr, b.fill, b.insrc);
  k3i_count<<<rows_grid, T, 0, s>>>(n, Q, sh.k1, b.knn_idx, aff, src, b.inptr, b.insrc, rst, rln, rcol, rval,
                                    res_knn, b.out_sorted, b.in_sorted, b.rowcnt);
  launch_scan32(b.rowcnt, n, b.h0ptr, s);
  k3i_fill<<<rows_grid, T, 0, s>>>(n, Q, sh.k1, aff, src, b.h0ptr, b.out_sorted, b.inptr, b.in_sorted, rst, rln, rcol,
                                   rval, res_knn, b.col[2], b.val[2], b.start[2], b.len[2],
                                   status ? status + kStNnz0 : nullptr);
  k3_edges<<<unsigned((n + T - 1) / T), T, 0, s>>>(b.knn_idx, b.knn_score, n, sh.k1, sh.k2, alpha, aggregator, b.nbr,
                                                   b.nbr_w, b.nbr_n);
  return 8;
}

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

// K2: exact top-k1 neighbour lists (Eq. 8) from approximate candidates.
//
// The similarity stage returns, per row, K = k1 + m candidates ranked by an
// approximate score g with a known error bound eps_g (FP32 GEMM: an FMA chain
// of dp terms; BF16/FP8 GEMM: the quantisation bound).  For each row one warp
//   1. merges the per-chunk candidate lists (P-way merge, ties to the lower
//      index) and bounds every excluded column's approximate score by B;
//   2. rescores each candidate in FP32 from the unit rows: each lane runs an
//      FMA chain over dp/32 terms and the warp adds the 32 partials in a
//      5-level tree, so |s - S| <= eps_r = (dp/32 + 10) u (u = 2^-24; the
//      10 covers the tree and the rounding of the unit rows);
//   3. sorts the candidates by (s desc, index asc);
//   4. certifies the list: if s_(k1) - eps_r > B + eps_g, no excluded column
//      can belong to the true top-k1 (otherwise the row is redone exactly by
//      the fallback kernel below, which scores all n columns);
//   5. finds runs of consecutive candidates whose s values are within 2 eps_r
//      of each other and that reach into the top-k1; their members are
//      recomputed in FP64 from the caller's raw features, cos = x_i.x_j /
//      (||x_i|| ||x_j||), and each run is re-sorted by (FP64 value, index).
//      Outside such runs the FP32 order is already the exact order.
// Output: knn_idx[i][0..k1) and knn_score (the FP64 value where one was
// computed, else s).  Self gets S_ii = 1 exactly.
#include <algorithm>
#include <cfloat>
#include <cstdlib>

#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int KMAX = 64;
constexpr int WPB = 8;

struct WarpSmem {
  int idx[KMAX];
  float g[KMAX];
  float s[KMAX];
  double t[KMAX];
  int ord[KMAX];
  unsigned char need[KMAX];
};

struct RowIo {
  const void* xq;
  const void* xg;
  int64_t nq;
  int d;
  int dtype;
  const float* xhat;
  int dp;
  const double* norm;
  int32_t* knn_idx;
  float* knn_score;
  long long* status;
};

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ const void* raw_row(const RowIo& io, int64_t r, size_t& base) {
  if (r < io.nq) {
    base = size_t(r) * io.d;
    return io.xq;
  }
  base = size_t(r - io.nq) * io.d;
  return io.xg;
}

// Lane l's FMA chain over elements l, l + 32, ... in that order; the loads of
// eight steps are issued before their FMAs.
template <class T>
__device__ __forceinline__ double dot_fp64_chain(const T* fa, const T* fb, int d, int lane) {
  double acc = 0.0;
  int k = lane;
  for (; k + 7 * kWarp < d; k += 8 * kWarp) {
    float x[8], y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      x[u] = to_float(fa[k + u * kWarp]);
      y[u] = to_float(fb[k + u * kWarp]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = fma(double(x[u]), double(y[u]), acc);
  }
  for (; k < d; k += kWarp) acc = fma(double(to_float(fa[k])), double(to_float(fb[k])), acc);
  return acc;
}

__device__ double dot_fp64_raw(const RowIo& io, int64_t a, int64_t b, int lane) {
  size_t ba, bb;
  const void* pa = raw_row(io, a, ba);
  const void* pb = raw_row(io, b, bb);
  const double acc =
      io.dtype == 0
          ? dot_fp64_chain(static_cast<const float*>(pa) + ba, static_cast<const float*>(pb) + bb, io.d, lane)
          : dot_fp64_chain(static_cast<const __nv_bfloat16*>(pa) + ba, static_cast<const __nv_bfloat16*>(pb) + bb,
                           io.d, lane);
  return warp_sum(acc);
}

// Bulk prefetch of one candidate row (bytes: a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_row_l2(const float* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Two FP32 dot products of unit rows at once (independent chains for memory parallelism).
__device__ __forceinline__ void dot2_fp32(const float* xi, const float* y0, const float* y1, int dp, int lane,
                                          float& r0, float& r1) {
  const float4* a = reinterpret_cast<const float4*>(xi);
  const float4* b0 = reinterpret_cast<const float4*>(y0);
  const float4* b1 = reinterpret_cast<const float4*>(y1);
  float acc0 = 0.f, acc1 = 0.f;
  for (int q = lane; q < dp / 4; q += kWarp) {
    const float4 x = __ldg(a + q), u = __ldg(b0 + q), v = __ldg(b1 + q);
    acc0 = fmaf(x.x, u.x, acc0); acc0 = fmaf(x.y, u.y, acc0);
    acc0 = fmaf(x.z, u.z, acc0); acc0 = fmaf(x.w, u.w, acc0);
    acc1 = fmaf(x.x, v.x, acc1); acc1 = fmaf(x.y, v.y, acc1);
    acc1 = fmaf(x.z, v.z, acc1); acc1 = fmaf(x.w, v.w, acc1);
  }
  r0 = warp_sum(acc0);
  r1 = warp_sum(acc1);
}


// P-way merge of sorted candidate lists src[p*K .. p*K+K) for p < P (P <= 32),
// one list per lane.  Fills w.idx/w.g with the best K; returns the count and
// the bound B on every candidate that was not taken.  An index outside
// [0, n) ends its list (lists left unwritten by an aborted similarity stage
// must not send the refinement outside the feature rows).
__device__ int merge_lists(WarpSmem& w, const float* ls, const int32_t* li, int P, int K, int64_t n, int lane,
                           float& B) {
  int head = 0;
  float hs = -FLT_MAX;
  int hi = kInvalidIdx;
  if (lane < P) {
    hs = ls[lane * K];
    hi = li[lane * K];
    if (hi < 0 || hi >= n) hi = kInvalidIdx;
  }
  int cnt = 0;
  for (; cnt < K; ++cnt) {
    float bs = hs;
    int bi = hi, bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(kFull, bs, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      const int ol = __shfl_xor_sync(kFull, bl, o);
      if (ranks_before(os, oi, bs, bi)) {
        bs = os;
        bi = oi;
        bl = ol;
      }
    }
    if (bi == kInvalidIdx) break;
    if (lane == 0) {
      w.idx[cnt] = bi;
      w.g[cnt] = bs;
    }
    if (lane == bl) {
      ++head;
      if (head < K) {
        hs = ls[lane * K + head];
        hi = li[lane * K + head];
        if (hi < 0 || hi >= n) hi = kInvalidIdx;
      } else {
        hs = -FLT_MAX;
        hi = kInvalidIdx;
      }
    }
  }
  // Every column that is not a candidate scores at most the K-th candidate's
  // score: it was either dropped from a full chunk list (below that list's
  // K-th, which the merged K-th cannot undercut), skipped by a floor (another
  // chunk's K-th, same argument) or not taken by the merge.  With fewer than K
  // candidates nothing was dropped or skipped.
  __syncwarp();
  B = cnt == K ? w.g[K - 1] : -FLT_MAX;
  return cnt;
}

// Row i's unit row held in registers (dp <= 128 * RV), so that rescoring
// reads only the candidates' rows.  Lane l holds float4s l, l + 32, ...
// Four FP32 dot products with the register-resident row: the same per-lane
// FMA chains and warp tree as dot2_fp32, so the values are identical.
template <int RV>
__device__ __forceinline__ void dot4_reg(const float4 (&xr)[RV], int nv, const float* y0, const float* y1,
                                         const float* y2, const float* y3, int lane, float (&r)[4]) {
  const float4* b[4] = {reinterpret_cast<const float4*>(y0), reinterpret_cast<const float4*>(y1),
                        reinterpret_cast<const float4*>(y2), reinterpret_cast<const float4*>(y3)};
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int t = 0; t < RV; ++t) {
    if (t < nv) {
      const float4 x = xr[t];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float4 u = __ldg(b[c] + lane + 32 * t);
        acc[c] = fmaf(x.x, u.x, acc[c]);
        acc[c] = fmaf(x.y, u.y, acc[c]);
        acc[c] = fmaf(x.z, u.z, acc[c]);
        acc[c] = fmaf(x.w, u.w, acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) r[c] = warp_sum(acc[c]);
}

// Steps 2-5 for row i on candidates w.idx[0..K).  Returns false when the
// candidate list cannot be certified (then nothing is written unless `last`).
// RV > 0: keep row i in registers when dp <= 128 RV (the warp-per-row
// kernel; the fallback's 1024-thread CTAs have no registers to spare).
template <int RV>
__device__ bool refine_warp(WarpSmem& w, int Kc, int64_t i, int k1, float B, double eps_g, double eps_r,
                            const RowIo& io, bool last, int lane) {
  const float* xi = io.xhat + size_t(i) * io.dp;
  const int nq4 = io.dp / 4;  // float4s per row
  const bool reg = RV > 0 && nq4 <= 32 * RV;
  // Lane l's float4s are l, l + 32, ...: nv of them (the rest of the last step is zero padding).
  const int nv = (nq4 - lane + 31) / 32;
  constexpr int R = RV > 0 ? RV : 1;
  float4 xr[R];
  if (reg) {
#pragma unroll
    for (int t = 0; t < R; ++t)
      xr[t] = t < nv ? __ldg(reinterpret_cast<const float4*>(xi) + lane + 32 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // FP32 scores of candidates [c0, c1) into w.s.
  auto rescore = [&](int c0, int c1) {
    if (reg) {
      // The next group's rows are prefetched into L2 while this group is scored.
      const uint32_t row_bytes = uint32_t(io.dp) * 4u;
      if (lane < 4 && c0 + lane < c1) prefetch_row_l2(io.xhat + size_t(w.idx[c0 + lane]) * io.dp, row_bytes);
      for (int c = c0; c < c1; c += 4) {
        if (lane < 4 && c + 4 + lane < c1)
          prefetch_row_l2(io.xhat + size_t(w.idx[c + 4 + lane]) * io.dp, row_bytes);
        int j[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = w.idx[c + u < c1 ? c + u : c];
        float v[4];
        dot4_reg<R>(xr, nv, io.xhat + size_t(j[0]) * io.dp, io.xhat + size_t(j[1]) * io.dp,
                    io.xhat + size_t(j[2]) * io.dp, io.xhat + size_t(j[3]) * io.dp, lane, v);
        if (lane == 0) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (c + u < c1) w.s[c + u] = j[u] == i ? 1.0f : v[u];
        }
      }
    } else {
      for (int c = c0; c < c1; c += 2) {
        const int j0 = w.idx[c];
        const int j1 = c + 1 < c1 ? w.idx[c + 1] : j0;
        float v0, v1;
        dot2_fp32(xi, io.xhat + size_t(j0) * io.dp, io.xhat + size_t(j1) * io.dp, io.dp, lane, v0, v1);
        if (lane == 0) {
          w.s[c] = j0 == i ? 1.0f : v0;
          if (c + 1 < c1) w.s[c + 1] = j1 == i ? 1.0f : v1;
        }
      }
    }
    __syncwarp();
  };
  // Rank of each rescored candidate among [0, n): w.ord[rank] = candidate.
  // Candidates are distinct columns, so the ranks form a permutation; the
  // slots are filled with valid positions first, so that even a malformed
  // list (a repeated column) can never send a later read out of range.
  auto rank_all = [&](int n) {
    for (int c = lane; c < n; c += kWarp) w.ord[c] = c;
    __syncwarp();
    for (int c = lane; c < n; c += kWarp) {
      const float sc = w.s[c];
      const int ic = w.idx[c];
      int r = 0;
      for (int e = 0; e < n; ++e) r += ranks_before(w.s[e], w.idx[e], sc, ic) ? 1 : 0;
      w.ord[r] = c;
    }
    __syncwarp();
  };
  // Lazy rescoring: the candidates come sorted by approximate score; rescore
  // the first k1 + 4, then 8 more at a time, until the best approximate score
  // left (plus its bound) stays 3 eps_r below the k1-th rescored score.  The
  // rest cannot then reach the top-k1, nor a near-tie run inside it, so the
  // result is that of rescoring all Kc candidates.
  int K = tmin(Kc, (k1 + 7) & ~3);
  rescore(0, K);
  rank_all(K);
  while (K < Kc && !(double(w.s[w.ord[k1 - 1]]) - 3.0 * eps_r > double(w.g[K]) + eps_g)) {
    const int K2 = tmin(Kc, K + 8);
    rescore(K, K2);
    K = K2;
    rank_all(K);
  }
  for (int c = lane; c < K; c += kWarp) w.need[c] = 0;
  __syncwarp();

  // Certificate: every column outside the candidates scores at most B (approximately).
  bool ok = true;
  if (K == Kc && B > -FLT_MAX) ok = double(w.s[w.ord[k1 - 1]]) - eps_r > double(B) + eps_g;
  if (!ok && !last) return false;

  // Runs of near-equal FP32 scores that reach into the top-k1.
  if (lane == 0) {
    int r = 0;
    while (r < K) {
      int r1 = r;
      while (r1 + 1 < K && double(w.s[w.ord[r1]]) - double(w.s[w.ord[r1 + 1]]) <= 2.0 * eps_r) ++r1;
      if (r1 > r && r < k1)
        for (int q = r; q <= r1; ++q) w.need[w.ord[q]] = 1;
      r = r1 + 1;
    }
  }
  __syncwarp();
  int nneed = 0;
  for (int c = 0; c < K; ++c) {
    if (!w.need[c]) continue;
    const int j = w.idx[c];
    double t = 1.0;
    if (j != i) t = dot_fp64_raw(io, i, j, lane) / (io.norm[i] * io.norm[j]);
    if (lane == 0) w.t[c] = t;
    ++nneed;
  }
  __syncwarp();
  if (lane == 0) {
    if (nneed) atomicAdd(reinterpret_cast<unsigned long long*>(io.status + kStFp64), (unsigned long long)nneed);
    // Re-sort each run by (FP64 value desc, index asc); runs are maximal
    // blocks of consecutive needed positions whose gaps are <= 2 eps_r.
    int r = 0;
    while (r < K) {
      if (!w.need[w.ord[r]]) {
        ++r;
        continue;
      }
      int r1 = r;
      while (r1 + 1 < K && w.need[w.ord[r1 + 1]] &&
             double(w.s[w.ord[r1]]) - double(w.s[w.ord[r1 + 1]]) <= 2.0 * eps_r)
        ++r1;
      for (int a = r + 1; a <= r1; ++a) {
        const int c = w.ord[a];
        int b = a;
        while (b > r && ranks_before(w.t[c], w.idx[c], w.t[w.ord[b - 1]], w.idx[w.ord[b - 1]])) {
          w.ord[b] = w.ord[b - 1];
          --b;
        }
        w.ord[b] = c;
      }
      r = r1 + 1;
    }
  }
  __syncwarp();
  for (int r = lane; r < k1; r += kWarp) {
    const int c = w.ord[r];
    io.knn_idx[size_t(i) * k1 + r] = w.idx[c];
    io.knn_score[size_t(i) * k1 + r] = w.need[c] ? float(w.t[c]) : w.s[c];
  }
  if (!ok && lane == 0) set_error(io.status, kErrCertify);
  return ok;
}

// Bound on |approximate score - S_ij| for row i and any column j (unit rows).
__device__ __forceinline__ double row_eps_g(const ErrModel& em, int64_t i) {
  double eps_g = em.eps;
  if (em.kind == 1) {
    // one quantised copy q = x - e:  |<q_i,q_j> - <x_i,x_j>| <= e_i + e_max + e_i e_max
    const double ei = em.err[i], emx = em.emax[0];
    eps_g += ei + emx + ei * emx;
  } else if (em.kind == 3) {
    // the BF16 hi copy: ||x - hi|| = ||lo + r|| <= ||lo|| + ||r||, as for one quantised copy
    const double ei = double(em.err[em.np + i]) + double(em.err[2 * em.np + i]);
    const double emx = double(em.emax[1]) + double(em.emax[2]);
    eps_g += ei + emx + ei * emx;
  } else if (em.kind == 2) {
    // x = hi + lo + r exactly, S' = hi.hi + lo.hi + hi.lo, so S - S' = lo_i.lo_j + r_i.x_j +
    // (hi_i + lo_i).r_j and |S' - S| <= ||lo_i|| lo_max + ||r_i|| + r_max (with slack for ||x|| ~ 1):
    const double li = em.err[em.np + i], lmx = em.emax[1];
    const double ri = em.err[2 * em.np + i], rmx = em.emax[2];
    eps_g += li * lmx + 1.0001 * (ri + rmx);
  }
  return eps_g;
}

template <int RV>
__global__ void __launch_bounds__(WPB * kWarp)
k2_refine(RowIo io, int64_t n, const float* __restrict__ part_s, const int32_t* __restrict__ part_i, int P,
          int K, int k1, ErrModel em, double eps_r, const int32_t* __restrict__ rows,
          const int32_t* __restrict__ count, bool part_by_row, int32_t* fb_rows, int32_t* fb_count,
          int fb_stat) {
  __shared__ WarpSmem sm[WPB];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t limit = (rows && count) ? int64_t(*count) : n;
  // f: position of the row in this launch's row set (grid-stride: a gathered
  // row set's size is known on the device only)
  for (int64_t f = int64_t(blockIdx.x) * WPB + wib; f < limit; f += int64_t(gridDim.x) * WPB) {
    const int64_t i = rows ? int64_t(rows[f]) : f;
    const double eps_g = row_eps_g(em, i);
    WarpSmem& w = sm[wib];
    float B = -FLT_MAX;
    const size_t base = size_t(part_by_row ? i : f) * P * K;
    // After a similarity stage that timed out, its lists may be unwritten (any
    // bits, repeated columns): they are not read, and every row goes on to the
    // exact stage as one with no candidates.
    const bool aborted = (io.status[kStErr] & kErrTimeout) != 0;
    const int cnt = aborted ? 0 : merge_lists(w, part_s + base, part_i + base, P, K, n, lane, B);
    if (cnt == n) B = -FLT_MAX;  // every column is a candidate
    // Fewer than k1 candidates (only after an aborted similarity stage): the
    // row goes to the next, exact stage like an uncertified one.
    const bool ok = cnt >= k1 && refine_warp<RV>(w, cnt, i, k1, B, eps_g, eps_r, io, false, lane);
    if (!ok && lane == 0) {
      const int slot = atomicAdd(fb_count, 1);
      fb_rows[slot] = int32_t(i);
      atomicAdd(reinterpret_cast<unsigned long long*>(io.status + fb_stat), 1ull);
    }
    __syncwarp();
  }
}

// Merge of the P sorted candidate lists of a row by all threads of a CTA
// (the lists staged in shared memory, P * K <= MERGE_CAP): an entry's place in
// the merged order is its position in its own list plus, for every other
// list, the number of entries there that rank before it (a binary search;
// the lists are disjoint and sorted by (score desc, index asc)).  Entries
// ranked below K are dropped.  Same result as merge_lists.
constexpr int MERGE_CAP = 512;
struct MergeSmem {
  float s[MERGE_CAP];
  int32_t i[MERGE_CAP];
  int len[32];
};

__device__ int merge_lists_cta(WarpSmem& w, MergeSmem& m, const float* ls, const int32_t* li, int P, int K,
                               int64_t n, int t, int nthreads, float& B) {
  for (int e = t; e < P * K; e += nthreads) {
    m.s[e] = ls[e];
    m.i[e] = li[e];
  }
  __syncthreads();
  if (t < P) {
    // An index outside [0, n) ends its list (see merge_lists).
    int L = 0;
    while (L < K && m.i[t * K + L] >= 0 && m.i[t * K + L] < n) ++L;
    m.len[t] = L;
  }
  __syncthreads();
  for (int e = t; e < P * K; e += nthreads) {
    const int p = e / K, i = e - p * K;
    if (i >= m.len[p]) continue;
    const float sc = m.s[e];
    const int32_t ic = m.i[e];
    int rank = i;
    for (int q = 0; q < P && rank < K; ++q) {
      if (q == p) continue;
      int lo = 0, hi = m.len[q];
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ranks_before(m.s[q * K + mid], m.i[q * K + mid], sc, ic)) lo = mid + 1;
        else hi = mid;
      }
      rank += lo;
    }
    if (rank < K) {
      w.idx[rank] = ic;
      w.g[rank] = sc;
    }
  }
  int total = 0;
  for (int q = 0; q < P; ++q) total += m.len[q];
  __syncthreads();
  const int cnt = total < K ? total : K;
  B = cnt == K ? w.g[K - 1] : -FLT_MAX;
  return cnt;
}

// Two FP32 dot products of row i (in shared memory) with candidate rows: lane
// l's FMA chain over float4s l, l + 32, ... and the warp tree, as dot2_fp32
// and dot4_reg, so the values are identical to theirs.  The loads of two
// steps are issued before their FMAs (four in flight per lane: 0.62 against
// 0.69 ms for the first pass at d = 2048; four steps, or 32 warps per SM
// with more registers, measured slower).
__device__ __forceinline__ void dot2_shared(const float4* xi, const float* y0, const float* y1, int dp, int lane,
                                            float& r0, float& r1) {
  const float4* b0 = reinterpret_cast<const float4*>(y0);
  const float4* b1 = reinterpret_cast<const float4*>(y1);
  float acc0 = 0.f, acc1 = 0.f;
  const int nq4 = dp / 4;
  int q = lane;
  for (; q + 1 * kWarp < nq4; q += 2 * kWarp) {
    float4 u[2], v[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      u[s] = __ldg(b0 + q + s * kWarp);
      v[s] = __ldg(b1 + q + s * kWarp);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float4 x = xi[q + s * kWarp];
      acc0 = fmaf(x.x, u[s].x, acc0); acc0 = fmaf(x.y, u[s].y, acc0);
      acc0 = fmaf(x.z, u[s].z, acc0); acc0 = fmaf(x.w, u[s].w, acc0);
      acc1 = fmaf(x.x, v[s].x, acc1); acc1 = fmaf(x.y, v[s].y, acc1);
      acc1 = fmaf(x.z, v[s].z, acc1); acc1 = fmaf(x.w, v[s].w, acc1);
    }
  }
  for (; q < nq4; q += kWarp) {
    const float4 x = xi[q], u = __ldg(b0 + q), v = __ldg(b1 + q);
    acc0 = fmaf(x.x, u.x, acc0); acc0 = fmaf(x.y, u.y, acc0);
    acc0 = fmaf(x.z, u.z, acc0); acc0 = fmaf(x.w, u.w, acc0);
    acc1 = fmaf(x.x, v.x, acc1); acc1 = fmaf(x.y, v.y, acc1);
    acc1 = fmaf(x.z, v.z, acc1); acc1 = fmaf(x.w, v.w, acc1);
  }
  r0 = warp_sum(acc0);
  r1 = warp_sum(acc1);
}

// Steps 1-5 for one row with NW warps (the first pass): the row's unit row is
// staged in shared memory and the warps split every rescoring batch (two
// candidates per warp at a time), so a row has NW times the loads in flight
// of the warp-per-row kernel and a thread needs no registers for the row.
// Warp 0 merges, ranks, certifies and orders; the FP64 near-tie values are
// split over the warps.  Same arithmetic, same result as k2_refine.
template <int NW>
__global__ void __launch_bounds__(NW * kWarp, 48 / NW)
k2_refine_cta(RowIo io, int64_t n, const float* __restrict__ part_s, const int32_t* __restrict__ part_i, int P,
              int Kmax, int k1, ErrModel em, double eps_r, const int32_t* __restrict__ rows,
              const int32_t* __restrict__ count, bool part_by_row, int32_t* fb_rows, int32_t* fb_count,
              int fb_stat) {
  extern __shared__ float4 own[];  // dp / 4 float4: row i
  __shared__ WarpSmem w;
  __shared__ MergeSmem msm;
  __shared__ float sB;
  __shared__ int sh[4];            // [0] candidates, [1] next batch end (-1: done), [2] certified, [3] FP64 count
  const int t = threadIdx.x, wid = t >> 5, lane = t & 31;
  const int64_t limit = (rows && count) ? int64_t(*count) : n;
  for (int64_t f = blockIdx.x; f < limit; f += gridDim.x) {  // grid-stride, as in k2_refine
    const int64_t i = rows ? int64_t(rows[f]) : f;
    const double eps_g = row_eps_g(em, i);
    const float4* xi4 = reinterpret_cast<const float4*>(io.xhat + size_t(i) * io.dp);
    for (int q = t; q < io.dp / 4; q += NW * kWarp) own[q] = __ldg(xi4 + q);
    {
      float B = -FLT_MAX;
      const size_t base = size_t(part_by_row ? i : f) * P * Kmax;
      const bool aborted = (io.status[kStErr] & kErrTimeout) != 0;
      int cnt = 0;
      if (!aborted && P * Kmax <= MERGE_CAP) {
        cnt = merge_lists_cta(w, msm, part_s + base, part_i + base, P, Kmax, n, t, NW * kWarp, B);
      } else if (!aborted && wid == 0) {
        cnt = merge_lists(w, part_s + base, part_i + base, P, Kmax, n, lane, B);
      }
      if (cnt == n) B = -FLT_MAX;  // every column is a candidate
      if (t == 0) {
        sh[0] = cnt;
        sB = B;
      }
    }
    __syncthreads();
    const int Kc = sh[0];
    bool ok = Kc >= k1;
    if (ok) {
      // FP32 scores of candidates [c0, c1) into w.s, two per warp at a time.
      auto rescore = [&](int c0, int c1) {
        for (int c = c0 + 2 * wid; c < c1; c += 2 * NW) {
          const int j0 = w.idx[c];
          const int j1 = c + 1 < c1 ? w.idx[c + 1] : j0;
          float v0, v1;
          dot2_shared(own, io.xhat + size_t(j0) * io.dp, io.xhat + size_t(j1) * io.dp, io.dp, lane, v0, v1);
          if (lane == 0) {
            w.s[c] = j0 == i ? 1.0f : v0;
            if (c + 1 < c1) w.s[c + 1] = j1 == i ? 1.0f : v1;
          }
        }
        __syncthreads();
      };
      // Lazy rescoring as in refine_warp: the first k1 + 4, then 8 more at a
      // time, until the best approximate score left (plus its bound) stays
      // 3 eps_r below the k1-th rescored score.
      int K = tmin(Kc, (k1 + 7) & ~3);
      rescore(0, K);
      for (;;) {
        // rank of every rescored candidate (all threads), then the stop test
        for (int c = t; c < K; c += NW * kWarp) {
          const float sc = w.s[c];
          const int ic = w.idx[c];
          int r = 0;
          for (int e = 0; e < K; ++e) r += ranks_before(w.s[e], w.idx[e], sc, ic) ? 1 : 0;
          w.ord[r] = c;
        }
        __syncthreads();
        if (t == 0) {
          const bool more = K < Kc && !(double(w.s[w.ord[k1 - 1]]) - 3.0 * eps_r > double(w.g[K]) + eps_g);
          sh[1] = more ? tmin(Kc, K + 8) : -1;
        }
        __syncthreads();
        const int K2 = sh[1];
        if (K2 < 0) break;
        rescore(K, K2);
        K = K2;
      }
      // Certificate (every column outside the candidates scores at most B) and
      // the runs of near-equal FP32 scores that reach into the top-k1.
      if (wid == 0) {
        bool cert = true;
        if (K == Kc && sB > -FLT_MAX) cert = double(w.s[w.ord[k1 - 1]]) - eps_r > double(sB) + eps_g;
        // Runs of near-equal FP32 scores that reach into the top-k1, in
        // parallel: bit q of `gap` says sorted positions q and q + 1 are within
        // 2 eps_r; q is in a run when bit q - 1 or bit q is set, and the run
        // reaches into the top-k1 when q < k1 or bits k1 - 1 .. q - 1 are all
        // set (K <= 64: each lane takes positions lane and lane + 32).
        const int q0 = lane, q1 = lane + kWarp;
        const bool f0 = q0 + 1 < K && double(w.s[w.ord[q0]]) - double(w.s[w.ord[q0 + 1]]) <= 2.0 * eps_r;
        const bool f1 = q1 + 1 < K && double(w.s[w.ord[q1]]) - double(w.s[w.ord[q1 + 1]]) <= 2.0 * eps_r;
        const uint64_t gap = uint64_t(__ballot_sync(kFull, f0)) | (uint64_t(__ballot_sync(kFull, f1)) << 32);
        int nneed = 0;
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = h ? q1 : q0;
          if (q < K) {
            const bool inrun = ((gap >> q) & 1ull) || (q > 0 && ((gap >> (q - 1)) & 1ull));
            bool nd = inrun;
            if (q >= k1 && inrun) {
              const int span = q - (k1 - 1);  // bits k1 - 1 .. q - 1
              const uint64_t want = span >= 64 ? ~0ull : ((1ull << span) - 1ull);
              nd = ((gap >> (k1 - 1)) & want) == want;
            }
            nd = nd && cert;
            w.need[w.ord[q]] = nd ? 1 : 0;
            nneed += nd ? 1 : 0;
          }
        }
        nneed = warp_sum(nneed);
        if (lane == 0) {
          sh[2] = cert ? 1 : 0;
          sh[3] = nneed;
        }
      }
      __syncthreads();
      ok = sh[2] != 0;
      if (ok) {
        // FP64 values of the candidates in near-tie runs, one warp each.
        if (sh[3] > 0) {
          int seen = 0;
          for (int c = 0; c < K; ++c) {
            if (!w.need[c]) continue;
            if (seen++ % NW != wid) continue;
            const int j = w.idx[c];
            double tv = 1.0;
            if (j != i) tv = dot_fp64_raw(io, i, j, lane) / (io.norm[i] * io.norm[j]);
            if (lane == 0) w.t[c] = tv;
          }
        }
        __syncthreads();
        if (wid == 0) {
          if (lane == 0) {
            if (sh[3]) atomicAdd(reinterpret_cast<unsigned long long*>(io.status + kStFp64), (unsigned long long)sh[3]);
            // Re-sort each run by (FP64 value desc, index asc).
            int r = 0;
            while (r < K) {
              if (!w.need[w.ord[r]]) {
                ++r;
                continue;
              }
              int r1 = r;
              while (r1 + 1 < K && w.need[w.ord[r1 + 1]] &&
                     double(w.s[w.ord[r1]]) - double(w.s[w.ord[r1 + 1]]) <= 2.0 * eps_r)
                ++r1;
              for (int a = r + 1; a <= r1; ++a) {
                const int c = w.ord[a];
                int b = a;
                while (b > r && ranks_before(w.t[c], w.idx[c], w.t[w.ord[b - 1]], w.idx[w.ord[b - 1]])) {
                  w.ord[b] = w.ord[b - 1];
                  --b;
                }
                w.ord[b] = c;
              }
              r = r1 + 1;
            }
          }
          __syncwarp();
          for (int r = lane; r < k1; r += kWarp) {
            const int c = w.ord[r];
            io.knn_idx[size_t(i) * k1 + r] = w.idx[c];
            io.knn_score[size_t(i) * k1 + r] = w.need[c] ? float(w.t[c]) : w.s[c];
          }
        }
      }
    }
    if (!ok && t == 0) {
      const int slot = atomicAdd(fb_count, 1);
      fb_rows[slot] = int32_t(i);
      atomicAdd(reinterpret_cast<unsigned long long*>(io.status + fb_stat), 1ull);
    }
    __syncthreads();  // the shared row and lists are reused by the next row
  }
}

// Exact fallback: score all n columns of a flagged row with the accurate FP32
// dot, keep per-warp top-K lists, merge them, then refine with eps_g = eps_r.
constexpr int FB_WARPS = 32;
__global__ void __launch_bounds__(FB_WARPS * kWarp)
k2_fallback(RowIo io, int64_t n, int K, int k1, double eps_r, const int32_t* fb_rows, const int32_t* fb_count,
            float* scratch_s, int32_t* scratch_i) {
  __shared__ WarpSmem w;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int count = *fb_count;
  for (int f = blockIdx.x; f < count; f += gridDim.x) {
    const int64_t i = fb_rows[f];
    float* ls = scratch_s + (size_t(blockIdx.x) * FB_WARPS + warp) * K;
    int32_t* li = scratch_i + (size_t(blockIdx.x) * FB_WARPS + warp) * K;
    for (int e = lane; e < K; e += kWarp) {
      ls[e] = -FLT_MAX;
      li[e] = kInvalidIdx;
    }
    __syncwarp();
    float thr_s = -FLT_MAX;
    int thr_i = kInvalidIdx;
    const float* xi = io.xhat + size_t(i) * io.dp;
    for (int64_t c0 = warp; c0 < n; c0 += 2 * FB_WARPS) {
      const int64_t c1 = c0 + FB_WARPS < n ? c0 + FB_WARPS : c0;
      float v[2];
      dot2_fp32(xi, io.xhat + size_t(c0) * io.dp, io.xhat + size_t(c1) * io.dp, io.dp, lane, v[0], v[1]);
      const int64_t cs[2] = {c0, c1};
      const int m = c1 != c0 ? 2 : 1;
      if (lane == 0) {
        for (int q = 0; q < m; ++q) {
          const int col = int(cs[q]);
          const float s = col == i ? 1.0f : v[q];
          if (!ranks_before(s, col, thr_s, thr_i)) continue;
          int p = K - 1;
          while (p > 0 && ranks_before(s, col, ls[p - 1], li[p - 1])) {
            ls[p] = ls[p - 1];
            li[p] = li[p - 1];
            --p;
          }
          ls[p] = s;
          li[p] = col;
          thr_s = ls[K - 1];
          thr_i = li[K - 1];
        }
      }
      __syncwarp();
    }
    __threadfence_block();
    __syncthreads();
    if (warp == 0) {
      float B;
      const int cnt = merge_lists(w, scratch_s + size_t(blockIdx.x) * FB_WARPS * K,
                                  scratch_i + size_t(blockIdx.x) * FB_WARPS * K, FB_WARPS, K, n, lane, B);
      if (cnt == n) B = -FLT_MAX;
      if (cnt >= k1) refine_warp<0>(w, cnt, i, k1, B, eps_r, eps_r, io, true, lane);
      else if (lane == 0) set_error(io.status, kErrInternal);
    }
    __syncthreads();
  }
}

}  // namespace

static RowIo make_io(const Shape& sh, const void* xq, const void* xg, const float* xhat, const double* norm,
                     int32_t* knn_idx, float* knn_score, long long* status) {
  RowIo io;
  io.xq = xq;
  io.xg = xg;
  io.nq = sh.nq;
  io.d = sh.d;
  io.dtype = sh.dtype;
  io.xhat = xhat;
  io.dp = sh.dp;
  io.norm = norm;
  io.knn_idx = knn_idx;
  io.knn_score = knn_score;
  io.status = status;
  return io;
}

double rescore_eps(int dp) { return (dp / 32 + 10) * kU32 * 1.01; }

// Rows a launch over a gathered row set covers at once (both kernels loop):
// about one resident wave on 152 SMs.
constexpr int64_t kGatheredRows = 2048;

// Warps per row of the CTA-per-row refinement (0: warp-per-row kernel).  By
// default 4 for rows of 512 floats or more, where the warp-per-row kernel's
// register-resident row (16 to 64 registers) leaves too few warps per SM to
// cover the candidate gathers (measured: 0.69 against 1.07 ms at d = 2048,
// 0.74 against 0.80 ms at d = 512); RERANK_REFINE_CTA = 0, 2, 4 or 8 forces a choice
// (identical results); 2 is also accepted.
static int refine_cta_warps(int dp) {
  static const int forced = [] {
    const char* e = std::getenv("RERANK_REFINE_CTA");
    if (!e) return -1;
    const int x = std::atoi(e);
    return (x == 2 || x == 4 || x == 8) ? x : 0;
  }();
  if (forced >= 0) return forced;
  return dp >= 512 ? 4 : 0;
}

int launch_refine(const Shape& sh, const void* xq, const void* xg, const float* xhat, const double* norm,
                   const float* part_s, const int32_t* part_i, int P, const ErrModel& em, const int32_t* rows,
                   const int32_t* count, bool part_by_row, int32_t* knn_idx, float* knn_score,
                   int32_t* fb_rows, int32_t* fb_count,
                   long long* status, cudaStream_t s, int64_t grid_rows, int fb_stat) {
  RowIo io = make_io(sh, xq, xg, xhat, norm, knn_idx, knn_score, status);
  int64_t g = grid_rows > 0 && grid_rows < sh.n ? grid_rows : sh.n;
  // A gathered row set (size on the device): the kernels loop over it, so one
  // resident wave of rows is enough.
  if (rows && count) g = std::min<int64_t>(g, kGatheredRows);
  const unsigned blocks = unsigned((g + WPB - 1) / WPB);
  // First pass: uncertified rows go to the recheck; a recheck's failures go to the exact scan.
  const int stat = fb_stat >= 0 ? fb_stat : ((rows && !part_by_row) ? kStFallback2 : kStFallback);
  if (refine_cta_warps(sh.dp) > 0) {
    const size_t smem = size_t(sh.dp) * 4;
    if (refine_cta_warps(sh.dp) == 2)
      k2_refine_cta<2><<<unsigned(g), 2 * kWarp, smem, s>>>(io, sh.n, part_s, part_i, P, sh.K, sh.k1, em,
                                                             rescore_eps(sh.dp), rows, count, part_by_row, fb_rows,
                                                             fb_count, stat);
    else if (refine_cta_warps(sh.dp) == 8)
      k2_refine_cta<8><<<unsigned(g), 8 * kWarp, smem, s>>>(io, sh.n, part_s, part_i, P, sh.K, sh.k1, em,
                                                             rescore_eps(sh.dp), rows, count, part_by_row, fb_rows,
                                                             fb_count, stat);
    else
      k2_refine_cta<4><<<unsigned(g), 4 * kWarp, smem, s>>>(io, sh.n, part_s, part_i, P, sh.K, sh.k1, em,
                                                             rescore_eps(sh.dp), rows, count, part_by_row, fb_rows,
                                                             fb_count, stat);
    return 1;
  }
  // Row i in registers: 4 float4s per lane up to dp = 512, 16 up to 2048.
  if (sh.dp <= 512)
    k2_refine<4><<<blocks, WPB * kWarp, 0, s>>>(io, sh.n, part_s, part_i, P, sh.K, sh.k1, em, rescore_eps(sh.dp),
                                                rows, count, part_by_row, fb_rows, fb_count, stat);
  else
    k2_refine<16><<<blocks, WPB * kWarp, 0, s>>>(io, sh.n, part_s, part_i, P, sh.K, sh.k1, em, rescore_eps(sh.dp),
                                                 rows, count, part_by_row, fb_rows, fb_count, stat);
  return 1;
}

int launch_refine_fallback(const Shape& sh, const void* xq, const void* xg, const float* xhat,
                            const double* norm, int32_t* knn_idx, float* knn_score, const int32_t* fb_rows,
                            const int32_t* fb_count, float* scratch_s, int32_t* scratch_i, long long* status,
                            int sm_count, cudaStream_t s) {
  RowIo io = make_io(sh, xq, xg, xhat, norm, knn_idx, knn_score, status);
  k2_fallback<<<sm_count, FB_WARPS * kWarp, 0, s>>>(io, sh.n, fallback_k(sh), sh.k1, rescore_eps(sh.dp), fb_rows,
                                                    fb_count, scratch_s, scratch_i);
  return 1;
}

int refine_kmax() { return KMAX; }
int fallback_k(const Shape& sh) {
  const int64_t k = std::min<int64_t>(std::min<int64_t>(int64_t(sh.k1) + 16, sh.n), KMAX);
  return int(k);
}
int fallback_warps() { return FB_WARPS; }

}  // namespace rr

// Per-thread top-K selection used by the similarity kernels' epilogues.
//
// Each thread owns one row and keeps the best K (score, column) pairs seen so
// far in a binary min-heap in shared memory ("worst" element at the root,
// order: score ascending, then column descending), laid out [slot][row] so
// that the threads of a warp touch consecutive words.  Admission costs one
// comparison with the root; an insertion is an O(log K) sift.  At the end of
// a chunk the heap is sorted in place (heapsort) into the usual order:
// score descending, ties to the lower column.
//
// A row's selection may also be pruned by a floor: the K-th best score that
// another chunk of the same row already found.  Any column scoring below it
// cannot be in the row's overall top-K (K better columns exist), so skipping
// it loses nothing; ties with the floor are kept.
#pragma once

#include <cfloat>

#include "common.cuh"

namespace rr {

// Order-preserving map of a float to a signed int (for atomicMax on scores).
__device__ __forceinline__ int score_key(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : (b ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float key_score(int k) {
  return __int_as_float(k >= 0 ? k : (k ^ 0x7FFFFFFF));
}
// Byte pattern used to reset the floors (0x80808080, below every real score key).
constexpr int kFloorResetByte = 0x80;

__device__ __forceinline__ bool worse(float sa, int ia, float sb, int ib) {
  return sa < sb || (sa == sb && ia > ib);
}

template <int ROWS>
struct RowHeap {
  float* hs;  // [kmax][ROWS]
  int* hi;
  int r;      // this thread's row slot
  int K;
  int count;

  __device__ __forceinline__ float& s(int j) { return hs[j * ROWS + r]; }
  __device__ __forceinline__ int& i(int j) { return hi[j * ROWS + r]; }

  __device__ __forceinline__ void reset(int k) {
    K = k;
    count = 0;
  }
  // Would (sv, iv) enter the heap?
  __device__ __forceinline__ bool admits(float sv, int iv) {
    return count < K || ranks_before(sv, iv, s(0), i(0));
  }
  __device__ __forceinline__ void sift_down(int p, float sv, int iv, int n) {
    while (true) {
      int c = 2 * p + 1;
      if (c >= n) break;
      float cs = s(c);
      int ci = i(c);
      if (c + 1 < n) {
        const float c2s = s(c + 1);
        const int c2i = i(c + 1);
        if (worse(c2s, c2i, cs, ci)) {
          ++c;
          cs = c2s;
          ci = c2i;
        }
      }
      if (!worse(cs, ci, sv, iv)) break;
      s(p) = cs;
      i(p) = ci;
      p = c;
    }
    s(p) = sv;
    i(p) = iv;
  }
  __device__ __forceinline__ void push(float sv, int iv) {
    if (count < K) {
      int p = count++;
      while (p > 0) {
        const int q = (p - 1) >> 1;
        const float qs = s(q);
        const int qi = i(q);
        if (!worse(sv, iv, qs, qi)) break;
        s(p) = qs;
        i(p) = qi;
        p = q;
      }
      s(p) = sv;
      i(p) = iv;
    } else if (ranks_before(sv, iv, s(0), i(0))) {
      sift_down(0, sv, iv, K);
    }
  }
  __device__ __forceinline__ bool full() const { return count >= K; }
  __device__ __forceinline__ float root_score() { return s(0); }
  // Heapsort in place: afterwards slots 0..count-1 hold score descending,
  // ties by lower column; unused slots become (-FLT_MAX, invalid).
  __device__ __forceinline__ void sort_desc() {
    for (int n = count; n > 1; --n) {
      const float ts = s(0);
      const int ti = i(0);
      const float ls = s(n - 1);
      const int li = i(n - 1);
      s(n - 1) = ts;
      i(n - 1) = ti;
      sift_down(0, ls, li, n - 1);
    }
    for (int j = count; j < K; ++j) {
      s(j) = -FLT_MAX;
      i(j) = kInvalidIdx;
    }
  }
};

}  // namespace rr

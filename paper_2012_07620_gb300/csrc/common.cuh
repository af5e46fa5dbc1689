// Device helpers shared by the re-ranking kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace rr {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kInvalidIdx = 0x7fffffff;

// Bits of the device error word (ctx->d_err[0]).
enum : int {
  kErrNonFinite = 1,   // an input row holds NaN or Inf
  kErrZeroNorm = 2,    // an input row is all zero
  kErrOverflow = 4,    // a workspace region was too small; the host grows it and retries
  kErrCertify = 8,     // a row's neighbour list could not be certified even after the exact fallback
  kErrTimeout = 16,    // a bounded device wait ran out
  kErrInternal = 32,   // an index left its range (checked builds of the sparse stages)
};

// Slots of the device status block (int64 each).
enum : int {
  kStErr = 0,          // error bits (int)
  kStBadRow = 1,       // first offending input row
  kStFp64 = 2,         // candidates rescored in FP64
  kStFallback = 3,     // rows whose first candidate list was not certified
  kStFallback2 = 5,    // rows that needed the exact full-row scan
  kStNeed = 4,         // capacity needed by the stage that overflowed (elements)
  kStTouched = 6,      // serving: gallery rows whose neighbour list a request re-derived
  kStFallbackMid = 7,  // FP8 path: rows the single-product BF16 recheck stage could not certify
  kStNnz0 = 8,         // nnz of h^(l) at kStNnz0 + l, l <= 8
  kStRecomputed = 17,  // serving: layer rows recomputed (not taken from the gallery's own graph)
  kStCount = 32
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Ordering used everywhere: a before b when its score is larger, or equal with a lower index.
__device__ __forceinline__ bool ranks_before(float sa, int ia, float sb, int ib) {
  return sa > sb || (sa == sb && ia < ib);
}
__device__ __forceinline__ bool ranks_before(double sa, int ia, double sb, int ib) {
  return sa > sb || (sa == sb && ia < ib);
}

__device__ __forceinline__ void set_error(long long* st, int bits) {
  atomicOr(reinterpret_cast<unsigned long long*>(st + kStErr), (unsigned long long)bits);
}

// Loads of the caller's features: element k of row r, as float.
__device__ __forceinline__ float load_feat(const void* p, int dtype, size_t off) {
  if (dtype == 0) return __ldg(reinterpret_cast<const float*>(p) + off);
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[off]);
}

template <class T>
__host__ __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <class T>
__host__ __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Unit roundoff of binary32.
constexpr double kU32 = 5.9604644775390625e-08;

}  // namespace rr

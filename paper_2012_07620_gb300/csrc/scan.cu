// Exclusive prefix sums of int32 counts (one CTA; the arrays here hold one
// entry per vertex, so a single block of 1024 threads is enough).
// out[0..n) = exclusive scan, out[n] = total (n = 0: out[0] = 0).
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int ST = 1024;
constexpr int64_t TILE = int64_t(ST) * 8;  // elements per pass

// Four consecutive elements from idx (zeros past n); a 16-byte load when the
// array is 16-byte aligned and all four are in range.
template <bool VEC>
__device__ __forceinline__ int4 load4(const int32_t* __restrict__ in, int64_t idx, int64_t n) {
  if (VEC && idx + 3 < n) return __ldg(reinterpret_cast<const int4*>(in + idx));
  int4 v;
  v.x = idx < n ? in[idx] : 0;
  v.y = idx + 1 < n ? in[idx + 1] : 0;
  v.z = idx + 2 < n ? in[idx + 2] : 0;
  v.w = idx + 3 < n ? in[idx + 3] : 0;
  return v;
}

template <bool VEC, class T>
__device__ __forceinline__ void store4(T* __restrict__ out, int64_t idx, int64_t n, long long o0, long long o1,
                                       long long o2, long long o3) {
  if (VEC && idx + 3 < n) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<int4*>(out + idx) = make_int4(int(o0), int(o1), int(o2), int(o3));
    } else {
      reinterpret_cast<longlong2*>(out + idx)[0] = make_longlong2(o0, o1);
      reinterpret_cast<longlong2*>(out + idx)[1] = make_longlong2(o2, o3);
    }
    return;
  }
  if (idx < n) out[idx] = T(o0);
  if (idx + 1 < n) out[idx + 1] = T(o1);
  if (idx + 2 < n) out[idx + 2] = T(o2);
  if (idx + 3 < n) out[idx + 3] = T(o3);
}

// Passes of TILE elements; warp w owns the 256 consecutive elements from
// base + 256 w, lane l the groups of four at 4 l and 128 + 4 l, so every load
// and store instruction of a warp covers 512 contiguous input bytes.  Each
// group's sums are scanned across the warp with shuffles, the warp totals by
// warp 0, and a running carry links the passes; the next pass's values are
// loaded before this one is scanned.
template <bool VEC, class T>
__global__ void __launch_bounds__(ST) scan_single(const int32_t* __restrict__ in, int64_t n, T* __restrict__ out) {
  __shared__ long long warp_tot[ST / kWarp];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t my0 = int64_t(w) * 256 + 4 * lane, my1 = my0 + 128;
  long long carry = 0;
  int4 a = load4<VEC>(in, my0, n), b = load4<VEC>(in, my1, n);
  for (int64_t base = 0; base < n; base += TILE) {
    const int4 na = load4<VEC>(in, base + TILE + my0, n), nb = load4<VEC>(in, base + TILE + my1, n);
    const long long s0 = (long long)a.x + a.y + a.z + a.w, s1 = (long long)b.x + b.y + b.z + b.w;
    long long x0 = s0, x1 = s1;  // inclusive scans over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y0 = __shfl_up_sync(kFull, x0, o), y1 = __shfl_up_sync(kFull, x1, o);
      if (lane >= o) {
        x0 += y0;
        x1 += y1;
      }
    }
    const long long tot0 = __shfl_sync(kFull, x0, 31);
    if (lane == 31) warp_tot[w] = tot0 + x1;
    __syncthreads();
    if (w == 0) {
      long long u = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, u, o);
        if (lane >= o) u += y;
      }
      warp_tot[lane] = u;  // inclusive over warps
    }
    __syncthreads();
    const long long wb = carry + (w ? warp_tot[w - 1] : 0);
    long long o = wb + x0 - s0;
    store4<VEC>(out, base + my0, n, o, o + a.x, o + a.x + a.y, o + a.x + a.y + a.z);
    o = wb + tot0 + x1 - s1;
    store4<VEC>(out, base + my1, n, o, o + b.x, o + b.x + b.y, o + b.x + b.y + b.z);
    carry += warp_tot[ST / kWarp - 1];
    __syncthreads();  // warp_tot is rewritten by the next pass
    a = na;
    b = nb;
  }
  if (t == 0) out[n] = T(carry);
}

template <class T>
void scan_launch(const int32_t* in, int64_t n, T* out, cudaStream_t s) {
  const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  if (vec)
    scan_single<true, T><<<1, ST, 0, s>>>(in, n, out);
  else
    scan_single<false, T><<<1, ST, 0, s>>>(in, n, out);
}

}  // namespace

int launch_scan(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
  scan_launch<int64_t>(in, n, out, s);
  return 1;
}
int launch_scan32(const int32_t* in, int64_t n, int32_t* out, cudaStream_t s) {
  scan_launch<int32_t>(in, n, out, s);
  return 1;
}

}  // namespace rr

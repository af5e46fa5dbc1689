// Exclusive prefix sums of int32 counts (one CTA; the arrays here hold one
// entry per vertex, so a single block of 1024 threads is enough).
// out[0..n) = exclusive scan, out[n] = total.
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int ST = 1024;

template <class T>
__global__ void __launch_bounds__(ST) scan_single(const int32_t* __restrict__ in, int64_t n, T* __restrict__ out) {
  __shared__ long long warp_tot[ST / kWarp];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t chunk = (n + ST - 1) / ST;
  const int64_t a = tmin<int64_t>(n, int64_t(t) * chunk), b = tmin<int64_t>(n, a + chunk);
  long long s = 0;
  for (int64_t i = a; i < b; ++i) s += in[i];
  // inclusive warp scan
  long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    long long v = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += y;
    }
    warp_tot[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  long long off = x - s + (w ? warp_tot[w - 1] : 0);
  for (int64_t i = a; i < b; ++i) {
    out[i] = T(off);
    off += in[i];
  }
  if (t == ST - 1) out[n] = T(warp_tot[ST / kWarp - 1]);
}

}  // namespace

int launch_scan(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
  scan_single<int64_t><<<1, ST, 0, s>>>(in, n, out);
  return 1;
}
int launch_scan32(const int32_t* in, int64_t n, int32_t* out, cudaStream_t s) {
  scan_single<int32_t><<<1, ST, 0, s>>>(in, n, out);
  return 1;
}

}  // namespace rr

// K0: unit-normalise every vertex feature (the normalisation inside cos, Eq. 7)
// and, for the tensor-core path, write the low-precision copy with a bound on
// its error.
//
// One warp per row.  The squared norm is summed with the compensated "Dot2"
// scheme of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26(6), 2005): each square is split exactly with an FMA and the
// running sum is kept as an unevaluated float pair via TwoSum (Knuth), so the
// norm is as accurate as a double-precision sum at FP32 cost.  The warp then
// combines its 32 partials in double.  Outputs:
//   xhat[i][k] = x_ik * fl32(1 / ||x_i||)   (FP32, zero padded to dp columns)
//   norm[i]    = ||x_i||                    (double)
//   BF16 path: xlow = bf16(xhat)
//   FP8 path:  xlow = e4m3(xhat * s_i) with s_i = 448 / max_k |xhat_ik|,
//              inv_scale[i] = 1 / s_i
//   qerr[i]    >= || xhat_i - dequantised xlow_i ||_2, and qerr_max >= max_i qerr[i]
// A row with a NaN/Inf element or zero norm sets an error bit and its index.
#include <cuda_fp8.h>

#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// MODE: 0 = FP32 only, 1 = also BF16, 2 = also FP8-E4M3 with a per-row scale.
template <int MODE>
__global__ void __launch_bounds__(256) k0_normalize(const void* __restrict__ xq, const void* __restrict__ xg,
                                                    int64_t nq, int64_t n, int64_t np, int d, int dp, int dtype,
                                                    float* __restrict__ xhat, double* __restrict__ norm,
                                                    void* __restrict__ xlow, float* __restrict__ inv_scale,
                                                    float* __restrict__ qerr, float* __restrict__ qerr_max,
                                                    long long* __restrict__ status) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= np) return;
  float* out = xhat + row * dp;
  __nv_bfloat16* outb = MODE == 1 ? reinterpret_cast<__nv_bfloat16*>(xlow) + row * dp : nullptr;
  __nv_fp8_e4m3* out8 = MODE == 2 ? reinterpret_cast<__nv_fp8_e4m3*>(xlow) + row * dp : nullptr;
  auto zero_row = [&]() {
    for (int k = lane; k < dp; k += kWarp) {
      out[k] = 0.f;
      if (MODE == 1) outb[k] = __float2bfloat16_rn(0.f);
      if (MODE == 2) out8[k] = __nv_fp8_e4m3(0.f);
    }
    if (MODE != 0 && lane == 0) {
      qerr[row] = 0.f;
      if (MODE == 2) inv_scale[row] = 0.f;
    }
  };
  if (row >= n) {
    zero_row();
    return;
  }
  const void* src = row < nq ? xq : xg;
  const size_t base = size_t(row < nq ? row : row - nq) * size_t(d);

  float s = 0.f, c = 0.f;
  bool bad = false;
  for (int k = lane; k < d; k += kWarp) {
    float x = load_feat(src, dtype, base + k);
    bad |= !isfinite(x);
    float p = x * x;
    float ep = fmaf(x, x, -p);
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c += e + ep;
  }
  double tot = warp_sum(double(s) + double(c));
  bad = __any_sync(kFull, bad);
  if (bad || !(tot > 0.0)) {
    if (lane == 0) {
      set_error(status, bad ? kErrNonFinite : kErrZeroNorm);
      atomicMin(reinterpret_cast<unsigned long long*>(status + kStBadRow), (unsigned long long)row);
      norm[row] = 1.0;
    }
    zero_row();
    return;
  }
  const double nrm = sqrt(tot);
  const float r32 = float(1.0 / nrm);
  if (lane == 0) norm[row] = nrm;
  float err = 0.f, amax = 0.f;
  for (int k = lane; k < dp; k += kWarp) {
    const float v = k < d ? load_feat(src, dtype, base + k) * r32 : 0.f;
    out[k] = v;
    if (MODE == 1) {
      const __nv_bfloat16 b = __float2bfloat16_rn(v);
      outb[k] = b;
      const float dv = v - __bfloat162float(b);
      err = fmaf(dv, dv, err);
    }
    if (MODE == 2) amax = fmaxf(amax, fabsf(v));
  }
  if (MODE == 2) {
    amax = warp_max_f(amax);
    const float sc = 448.0f / amax;
    const float inv = amax / 448.0f;
    __syncwarp();
    for (int k = lane; k < dp; k += kWarp) {
      const float v = out[k];
      const __nv_fp8_e4m3 q(v * sc);
      out8[k] = q;
      const float dv = v - float(q) * inv;
      err = fmaf(dv, dv, err);
    }
    if (lane == 0) inv_scale[row] = inv;
  }
  if (MODE != 0) {
    err = warp_sum(err);
    // The FP32 sum of d squares is within (d/32 + 5) u of exact; round the bound up.
    const float e = sqrtf(err) * 1.0001f + 1e-30f;
    if (lane == 0) {
      qerr[row] = e;
      atomicMax(reinterpret_cast<int*>(qerr_max), __float_as_int(e));
    }
  }
}

}  // namespace

int launch_normalize(const Shape& sh, const void* xq, const void* xg, float* xhat, double* norm, void* xlow,
                     float* inv_scale, float* qerr, float* qerr_max, int precision, long long* status,
                     cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = unsigned((sh.np * kWarp + threads - 1) / threads);
  if (precision == RERANK_PREC_BF16) {
    cudaMemsetAsync(qerr_max, 0, sizeof(float), s);
    k0_normalize<1><<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm, xlow,
                                               inv_scale, qerr, qerr_max, status);
  } else if (precision == RERANK_PREC_FP8) {
    cudaMemsetAsync(qerr_max, 0, sizeof(float), s);
    k0_normalize<2><<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm, xlow,
                                               inv_scale, qerr, qerr_max, status);
  } else {
    k0_normalize<0><<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm,
                                               nullptr, nullptr, nullptr, nullptr, status);
  }
  return 1;
}

}  // namespace rr

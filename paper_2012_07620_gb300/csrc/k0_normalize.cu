// K0: unit-normalise every vertex feature (the normalisation inside cos, Eq. 7)
// and, for the tensor-core path, write the low-precision copies with bounds on
// their errors.
//
// One warp per row.  The squared norm is summed with the compensated "Dot2"
// scheme of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26(6), 2005): each square is split exactly with an FMA and the
// running sum is kept as an unevaluated float pair via TwoSum (Knuth), so the
// norm is as accurate as a double-precision sum at FP32 cost.  The warp then
// combines its 32 partials in double.  Outputs:
//   xhat[i][k] = x_ik * fl32(1 / ||x_i||)   (FP32, zero padded to dp columns)
//   norm[i]    = ||x_i||                    (double)
//   BF16 path: xlow = hi = bf16(xhat)
//   FP8 path:  xlow = e4m3(xhat * s_i) with s_i = 448 / max_k |xhat_ik|,
//              inv_scale[i] = 1 / s_i
//   both:      hi = bf16(xhat), lo = bf16(xhat - hi); xhat = hi + lo + r
//              exactly (each subtraction is exact in FP32)
//   err[0][i] >= || xhat_i - dequantised xlow_i ||,  err[1][i] >= ||lo_i||,
//   err[2][i] >= ||r_i||, and emax[0..2] >= their maxima over rows.
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

// The FP32 sum of squares is within (d/32 + 5) u of exact; round each bound up.
__device__ __forceinline__ float bound_of(float sumsq) { return sqrtf(sumsq) * 1.0001f + 1e-30f; }

// MODE: 0 = FP32 only, 1 = BF16 (xlow is hi), 2 = FP8-E4M3 with a per-row scale.
template <int MODE>
__global__ void __launch_bounds__(256) k0_normalize(const void* __restrict__ xq, const void* __restrict__ xg,
                                                    int64_t nq, int64_t n, int64_t np, int d, int dp, int dtype,
                                                    float* __restrict__ xhat, double* __restrict__ norm,
                                                    void* __restrict__ xlow, __nv_bfloat16* __restrict__ xhi,
                                                    __nv_bfloat16* __restrict__ xlo, float* __restrict__ inv_scale,
                                                    float* __restrict__ err, float* __restrict__ emax,
                                                    long long* __restrict__ status) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= np) return;
  float* out = xhat + row * dp;
  __nv_bfloat16* outh = MODE != 0 ? xhi + row * dp : nullptr;
  __nv_bfloat16* outl = MODE != 0 ? xlo + row * dp : nullptr;
  __nv_fp8_e4m3* out8 = MODE == 2 ? reinterpret_cast<__nv_fp8_e4m3*>(xlow) + row * dp : nullptr;
  auto zero_row = [&]() {
    for (int k = lane; k < dp; k += kWarp) {
      out[k] = 0.f;
      if (MODE != 0) {
        outh[k] = __float2bfloat16_rn(0.f);
        outl[k] = __float2bfloat16_rn(0.f);
      }
      if (MODE == 2) out8[k] = __nv_fp8_e4m3(0.f);
    }
    if (MODE != 0 && lane == 0) {
      err[row] = 0.f;
      err[np + row] = 0.f;
      err[2 * np + row] = 0.f;
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
  float e_lo = 0.f, e_r = 0.f, amax = 0.f;
  for (int k = lane; k < dp; k += kWarp) {
    const float v = k < d ? load_feat(src, dtype, base + k) * r32 : 0.f;
    out[k] = v;
    if (MODE != 0) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const float dh = v - __bfloat162float(h);          // exact
      const __nv_bfloat16 l = __float2bfloat16_rn(dh);
      const float rr = dh - __bfloat162float(l);          // exact
      outh[k] = h;
      outl[k] = l;
      e_lo = fmaf(__bfloat162float(l), __bfloat162float(l), e_lo);
      e_r = fmaf(rr, rr, e_r);
    }
    if (MODE == 2) amax = fmaxf(amax, fabsf(v));
  }
  float e_main = 0.f;
  if (MODE == 1) {
    // xlow = hi: its error is lo + r.
    for (int k = lane; k < dp; k += kWarp) {
      const float dv = out[k] - __bfloat162float(outh[k]);
      e_main = fmaf(dv, dv, e_main);
    }
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
      e_main = fmaf(dv, dv, e_main);
    }
    if (lane == 0) inv_scale[row] = inv;
  }
  if (MODE != 0) {
    const float b0 = bound_of(warp_sum(e_main));
    const float b1 = bound_of(warp_sum(e_lo));
    const float b2 = bound_of(warp_sum(e_r));
    if (lane == 0) {
      err[row] = b0;
      err[np + row] = b1;
      err[2 * np + row] = b2;
      atomicMax(reinterpret_cast<int*>(emax), __float_as_int(b0));
      atomicMax(reinterpret_cast<int*>(emax) + 1, __float_as_int(b1));
      atomicMax(reinterpret_cast<int*>(emax) + 2, __float_as_int(b2));
    }
  }
}

// The same for FP32 rows with d % 4 == 0 and dp <= 2048, with the row held in
// registers (16 float4 per lane at most): one read of the input, one write of
// each output.  Lane l owns float4s l, l + 32, ...; the compensated sum runs
// over them in that order.
constexpr int NV4 = 16;

template <int MODE>
__global__ void __launch_bounds__(256) k0_normalize_vec(const float* __restrict__ xq, const float* __restrict__ xg,
                                                        int64_t nq, int64_t n, int64_t np, int d, int dp,
                                                        float* __restrict__ xhat, double* __restrict__ norm,
                                                        void* __restrict__ xlow, __nv_bfloat16* __restrict__ xhi,
                                                        __nv_bfloat16* __restrict__ xlo, float* __restrict__ inv_scale,
                                                        float* __restrict__ err, float* __restrict__ emax,
                                                        long long* __restrict__ status) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= np) return;
  const int nv = d / 4, nvp = dp / 4;  // float4s of data and of the padded row
  float4* out = reinterpret_cast<float4*>(xhat + row * dp);
  auto store_low = [&](int q, float4 v) {
    if (MODE == 0) return;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y), h2 = __float2bfloat16_rn(v.z),
                        h3 = __float2bfloat16_rn(v.w);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v.x - __bfloat162float(h0)),
                        l1 = __float2bfloat16_rn(v.y - __bfloat162float(h1)),
                        l2 = __float2bfloat16_rn(v.z - __bfloat162float(h2)),
                        l3 = __float2bfloat16_rn(v.w - __bfloat162float(h3));
    __nv_bfloat162 hh[2] = {__halves2bfloat162(h0, h1), __halves2bfloat162(h2, h3)};
    __nv_bfloat162 ll[2] = {__halves2bfloat162(l0, l1), __halves2bfloat162(l2, l3)};
    reinterpret_cast<uint2*>(xhi + row * dp)[q] = *reinterpret_cast<uint2*>(hh);
    reinterpret_cast<uint2*>(xlo + row * dp)[q] = *reinterpret_cast<uint2*>(ll);
  };
  if (row >= n) {
    for (int q = lane; q < nvp; q += kWarp) {
      out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      store_low(q, make_float4(0.f, 0.f, 0.f, 0.f));
      if (MODE == 2) reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(xlow) + row * dp)[q] = 0u;
    }
    if (MODE != 0 && lane == 0) {
      err[row] = 0.f;
      err[np + row] = 0.f;
      err[2 * np + row] = 0.f;
      if (MODE == 2) inv_scale[row] = 0.f;
    }
    return;
  }
  const float4* src = reinterpret_cast<const float4*>(row < nq ? xq + row * int64_t(d) : xg + (row - nq) * int64_t(d));
  float4 xr[NV4];
  float s = 0.f, c = 0.f;
  bool bad = false;
#pragma unroll
  for (int t = 0; t < NV4; ++t) {
    const int q = lane + kWarp * t;
    xr[t] = q < nv ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int t = 0; t < NV4; ++t) {
    const float e4[4] = {xr[t].x, xr[t].y, xr[t].z, xr[t].w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float x = e4[u];
      bad |= !isfinite(x);
      const float p = x * x;
      const float ep = fmaf(x, x, -p);
      float tt, ee;
      two_sum(s, p, tt, ee);
      s = tt;
      c += ee + ep;
    }
  }
  const double tot = warp_sum(double(s) + double(c));
  bad = __any_sync(kFull, bad);
  if (bad || !(tot > 0.0)) {
    if (lane == 0) {
      set_error(status, bad ? kErrNonFinite : kErrZeroNorm);
      atomicMin(reinterpret_cast<unsigned long long*>(status + kStBadRow), (unsigned long long)row);
      norm[row] = 1.0;
    }
    for (int q = lane; q < nvp; q += kWarp) {
      out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      store_low(q, make_float4(0.f, 0.f, 0.f, 0.f));
      if (MODE == 2) reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(xlow) + row * dp)[q] = 0u;
    }
    if (MODE != 0 && lane == 0) {
      err[row] = 0.f;
      err[np + row] = 0.f;
      err[2 * np + row] = 0.f;
      if (MODE == 2) inv_scale[row] = 0.f;
    }
    return;
  }
  const double nrm = sqrt(tot);
  const float r32 = float(1.0 / nrm);
  if (lane == 0) norm[row] = nrm;
  float e_lo = 0.f, e_r = 0.f, e_main = 0.f, amax = 0.f;
#pragma unroll
  for (int t = 0; t < NV4; ++t) {
    const int q = lane + kWarp * t;
    if (q >= nvp) continue;
    float4 v = xr[t];
    v.x *= r32;
    v.y *= r32;
    v.z *= r32;
    v.w *= r32;
    xr[t] = v;
    out[q] = v;
    if (MODE != 0) {
      store_low(q, v);
      const float e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float h = __bfloat162float(__float2bfloat16_rn(e4[u]));
        const float dh = e4[u] - h;  // exact
        const float l = __bfloat162float(__float2bfloat16_rn(dh));
        const float rr = dh - l;      // exact
        e_lo = fmaf(l, l, e_lo);
        e_r = fmaf(rr, rr, e_r);
        if (MODE == 1) e_main = fmaf(dh, dh, e_main);
        if (MODE == 2) amax = fmaxf(amax, fabsf(e4[u]));
      }
    }
  }
  if (MODE == 2) {
    amax = warp_max_f(amax);
    const float sc = 448.0f / amax;
    const float inv = amax / 448.0f;
    uint32_t* o8 = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(xlow) + row * dp);
#pragma unroll
    for (int t = 0; t < NV4; ++t) {
      const int q = lane + kWarp * t;
      if (q >= nvp) continue;
      const float e4[4] = {xr[t].x, xr[t].y, xr[t].z, xr[t].w};
      uint32_t packed = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const __nv_fp8_e4m3 qv(e4[u] * sc);
        const float dv = e4[u] - float(qv) * inv;
        e_main = fmaf(dv, dv, e_main);
        packed |= uint32_t(qv.__x) << (8 * u);
      }
      o8[q] = packed;
    }
    if (lane == 0) inv_scale[row] = inv;
  }
  if (MODE != 0) {
    const float b0 = bound_of(warp_sum(e_main));
    const float b1 = bound_of(warp_sum(e_lo));
    const float b2 = bound_of(warp_sum(e_r));
    if (lane == 0) {
      err[row] = b0;
      err[np + row] = b1;
      err[2 * np + row] = b2;
      atomicMax(reinterpret_cast<int*>(emax), __float_as_int(b0));
      atomicMax(reinterpret_cast<int*>(emax) + 1, __float_as_int(b1));
      atomicMax(reinterpret_cast<int*>(emax) + 2, __float_as_int(b2));
    }
  }
}

}  // namespace

int launch_normalize(const Shape& sh, const void* xq, const void* xg, float* xhat, double* norm, void* xlow,
                     __nv_bfloat16* xhi, __nv_bfloat16* xlo, float* inv_scale, float* err, float* emax,
                     int precision, long long* status, cudaStream_t s) {
  // The register-resident row (about 96 registers a thread) allows 5 CTAs of
  // 128 threads per SM (20 warps) against 2 of 256 (16 warps).
  const bool vec_shape = sh.dtype == RERANK_DTYPE_F32 && sh.d % 4 == 0 && sh.dp <= 4 * kWarp * NV4;
  const int threads = vec_shape ? 128 : 256;
  const unsigned blocks = unsigned((sh.np * kWarp + threads - 1) / threads);
  const bool vec = sh.dtype == RERANK_DTYPE_F32 && sh.d % 4 == 0 && sh.dp <= 4 * kWarp * NV4 &&
                   (reinterpret_cast<uintptr_t>(xq) & 15) == 0 && (reinterpret_cast<uintptr_t>(xg) & 15) == 0;
  if (vec) {
    const float* fq = static_cast<const float*>(xq);
    const float* fg = static_cast<const float*>(xg);
    if (precision != RERANK_PREC_FP32) cudaMemsetAsync(emax, 0, 4 * sizeof(float), s);
    if (precision == RERANK_PREC_BF16)
      k0_normalize_vec<1><<<blocks, threads, 0, s>>>(fq, fg, sh.nq, sh.n, sh.np, sh.d, sh.dp, xhat, norm, xlow, xhi,
                                                     xlo, inv_scale, err, emax, status);
    else if (precision == RERANK_PREC_FP8)
      k0_normalize_vec<2><<<blocks, threads, 0, s>>>(fq, fg, sh.nq, sh.n, sh.np, sh.d, sh.dp, xhat, norm, xlow, xhi,
                                                     xlo, inv_scale, err, emax, status);
    else
      k0_normalize_vec<0><<<blocks, threads, 0, s>>>(fq, fg, sh.nq, sh.n, sh.np, sh.d, sh.dp, xhat, norm, nullptr,
                                                     nullptr, nullptr, nullptr, nullptr, nullptr, status);
    return 1;
  }
  if (precision == RERANK_PREC_BF16) {
    cudaMemsetAsync(emax, 0, 4 * sizeof(float), s);
    k0_normalize<1><<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm, xlow,
                                               xhi, xlo, inv_scale, err, emax, status);
  } else if (precision == RERANK_PREC_FP8) {
    cudaMemsetAsync(emax, 0, 4 * sizeof(float), s);
    k0_normalize<2><<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm, xlow,
                                               xhi, xlo, inv_scale, err, emax, status);
  } else {
    k0_normalize<0><<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm,
                                               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, status);
  }
  return 1;
}

}  // namespace rr

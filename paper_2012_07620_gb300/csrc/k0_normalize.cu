// K0: unit-normalise every vertex feature (the normalisation inside cos, Eq. 7).
//
// One warp per row.  The squared norm is summed with the compensated "Dot2"
// scheme of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26(6), 2005): each square is split exactly with an FMA and the
// running sum is kept as an unevaluated float pair via TwoSum (Knuth), so the
// norm is as accurate as a double-precision sum at FP32 cost.  The warp then
// combines its 32 partials in double.  Outputs:
//   xhat[i][k] = x_ik * fl32(1 / ||x_i||)   (FP32, zero padded to dp columns)
//   norm[i]    = ||x_i||                    (double)
//   xlow       BF16 copy of xhat            (tensor-core path, when requested)
// A row with a NaN/Inf element or zero norm sets an error bit and its index.
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(256) k0_normalize(const void* __restrict__ xq, const void* __restrict__ xg,
                                                    int64_t nq, int64_t n, int64_t np, int d, int dp,
                                                    int dtype, float* __restrict__ xhat,
                                                    double* __restrict__ norm,
                                                    __nv_bfloat16* __restrict__ xbf,
                                                    long long* __restrict__ status) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= np) return;
  float* out = xhat + row * dp;
  __nv_bfloat16* outb = xbf ? xbf + row * dp : nullptr;
  if (row >= n) {
    for (int k = lane; k < dp; k += kWarp) {
      out[k] = 0.f;
      if (outb) outb[k] = __float2bfloat16_rn(0.f);
    }
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
    for (int k = lane; k < dp; k += kWarp) {
      out[k] = 0.f;
      if (outb) outb[k] = __float2bfloat16_rn(0.f);
    }
    return;
  }
  const double nrm = sqrt(tot);
  const float r32 = float(1.0 / nrm);
  if (lane == 0) norm[row] = nrm;
  for (int k = lane; k < dp; k += kWarp) {
    float v = k < d ? load_feat(src, dtype, base + k) * r32 : 0.f;
    out[k] = v;
    if (outb) outb[k] = __float2bfloat16_rn(v);
  }
}

}  // namespace

int launch_normalize(const Shape& sh, const void* xq, const void* xg, float* xhat, double* norm,
                      void* xlow, float* xscale, int precision, long long* status, cudaStream_t s) {
  (void)xscale;
  const int threads = 256;
  const int64_t warps = sh.np;
  const unsigned blocks = unsigned((warps * kWarp + threads - 1) / threads);
  __nv_bfloat16* xbf = precision == RERANK_PREC_BF16 ? reinterpret_cast<__nv_bfloat16*>(xlow) : nullptr;
  k0_normalize<<<blocks, threads, 0, s>>>(xq, xg, sh.nq, sh.n, sh.np, sh.d, sh.dp, sh.dtype, xhat, norm,
                                          xbf, status);
  return 1;
}

}  // namespace rr

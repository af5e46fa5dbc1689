// Dense initial features h_i^(0) = x_i (Table 1, first column; Eq. 11 with
// the feature vector in place of the adjacency row): the propagation layers
// of Eq. 13-14 on dense N x d_p rows, and the final query-gallery cosines
// (Alg. 1 step 7).  With alpha = 0, the mean aggregator and one layer this is
// local query expansion (Sec. 3.4, Eq. 4) plus the residual of Eq. 13.
//
// Layer: one warp per row i walks the message list of i built by the graph
// stage (entries (j, c_j) in order, the residual folded into the self
// coefficient; max aggregator: the k2 weighted rows combined element-wise by
// max, then the residual entry marked by c = -1 added), lane l owning the
// float4 columns l, l + 32, ...; the row is divided by its L2 norm (a per-lane
// sum of squares, the 32 partials added in FP64).
//
// Scores: s(q, g) = <h_q, h_g> / (||h_q|| ||h_g||) for every query row q and
// gallery row g, 128 x 128 output tiles per CTA, 8 x 8 per thread.  Each
// 32-deep k-chunk is an FP32 FMA chain; the chunks are added in float-float
// (a TwoSum per chunk), so a score is as accurate as a chain of 32 products
// (about 1e-7 for unit rows) whatever d is; the norms are applied in FP64.
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int DK = 32;   // k-chunk of the scores

// out_i = normalise(sum_m c_m h_{j_m})  (sum / mean), or
// normalise(max_m (c_m h_{j_m}) + h_i)   (max; the residual entry has c < 0).
__global__ void k7_dense_layer(const float* __restrict__ hin, float* __restrict__ hout, int64_t n, int dp,
                               const int32_t* __restrict__ nbr, const float* __restrict__ nbr_w,
                               const int32_t* __restrict__ nbr_n, int k2, int agg_max) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int m = nbr_n[i];
  const int32_t* nb = nbr + i * (k2 + 1);
  const float* nw = nbr_w + i * (k2 + 1);
  const int nv = dp / 4;
  const float4* in4 = reinterpret_cast<const float4*>(hin);
  float4* out4 = reinterpret_cast<float4*>(hout) + i * nv;
  float ss = 0.f;
  // Two passes over the columns: the first builds the row and its sum of
  // squares, the second scales it (the row is re-read from this row's output).
  for (int q = lane; q < nv; q += kWarp) {
    float4 acc;
    if (agg_max) {
      acc = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
      float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = 0; e < m; ++e) {
        const float c = nw[e];
        const float4 v = __ldg(in4 + int64_t(nb[e]) * nv + q);
        if (c < 0.f) {
          res = v;
        } else {
          acc.x = fmaxf(acc.x, c * v.x);
          acc.y = fmaxf(acc.y, c * v.y);
          acc.z = fmaxf(acc.z, c * v.z);
          acc.w = fmaxf(acc.w, c * v.w);
        }
      }
      acc.x += res.x;
      acc.y += res.y;
      acc.z += res.z;
      acc.w += res.w;
    } else {
      acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = 0; e < m; ++e) {
        const float c = nw[e];
        const float4 v = __ldg(in4 + int64_t(nb[e]) * nv + q);
        acc.x = fmaf(c, v.x, acc.x);
        acc.y = fmaf(c, v.y, acc.y);
        acc.z = fmaf(c, v.z, acc.z);
        acc.w = fmaf(c, v.w, acc.w);
      }
    }
    ss = fmaf(acc.x, acc.x, ss);
    ss = fmaf(acc.y, acc.y, ss);
    ss = fmaf(acc.z, acc.z, ss);
    ss = fmaf(acc.w, acc.w, ss);
    out4[q] = acc;
  }
  const double tot = warp_sum(double(ss));
  const float inv = tot > 0.0 ? float(1.0 / sqrt(tot)) : 0.f;
  __syncwarp();
  for (int q = lane; q < nv; q += kWarp) {
    float4 v = out4[q];
    v.x *= inv;
    v.y *= inv;
    v.z *= inv;
    v.w *= inv;
    out4[q] = v;
  }
}

// 1 / ||h_i|| in FP64 (per-lane FP32 partials over float4 columns, FP64 warp sum).
__global__ void k7_dense_inv_norms(const float* __restrict__ h, int64_t n, int dp, double* __restrict__ inv) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int nv = dp / 4;
  const float4* r = reinterpret_cast<const float4*>(h) + i * nv;
  float ss = 0.f;
  for (int q = lane; q < nv; q += kWarp) {
    const float4 v = __ldg(r + q);
    ss = fmaf(v.x, v.x, ss);
    ss = fmaf(v.y, v.y, ss);
    ss = fmaf(v.z, v.z, ss);
    ss = fmaf(v.w, v.w, ss);
  }
  const double tot = warp_sum(double(ss));
  if (lane == 0) inv[i] = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
}

// Float-float accumulation: (hi, lo) += p, with Knuth's TwoSum for the rounding error.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float p) {
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err;
}

// Scores by 128 x 128 output tiles, 256 threads of 8 x 8 outputs each (rows
// 4 ty + a and 64 + 4 ty + a, columns 4 tx + b and 64 + 4 tx + b).  Each
// 32-deep k-chunk is an FP32 FMA chain per output in k order and is added to
// the output's (hi, lo) pair by TwoSum, so a score does not depend on the
// tile shape or on which thread computes it; 8 x 8 outputs per thread keep
// the shared-memory reads at a quarter of the FMAs' operands.  The chunk sums p and
// hi live in registers, lo in shared memory (read and written once per
// chunk).  The operand chunks are stored k-major (lane = row when loading, so
// the transposing stores are free of bank conflicts); the next chunk's global
// loads are issued before the current chunk is used.
constexpr int ST = 128;                 // output tile
constexpr int STHREADS = 256;
constexpr size_t SSMEM = size_t(2) * DK * ST * 4 + size_t(64) * STHREADS * 4;  // As, Bs, lo

__global__ void __launch_bounds__(STHREADS, 1)
k7_dense_scores(const float* __restrict__ h, int64_t nq, int64_t ng, int dp, const double* __restrict__ inv,
                float* __restrict__ S) {
  extern __shared__ float4 dyn4[];
  float* As = reinterpret_cast<float*>(dyn4);  // [DK][ST]
  float* Bs = As + DK * ST;                    // [DK][ST]
  float* lo = Bs + DK * ST;                    // [64][STHREADS]
  const int t = threadIdx.x, lane = t & 31, wq = t >> 5;
  const int tx = t & 15, ty = t >> 4;
  const int64_t q0 = int64_t(blockIdx.y) * ST, g0 = int64_t(blockIdx.x) * ST;
  float hi[64], p[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    hi[j] = 0.f;
    lo[j * STHREADS + t] = 0.f;
  }
  // Loader: warp wq moves k-group wq (4 consecutive k of the chunk) of rows
  // lane + 32 s, s = 0..3, for both operands.
  const float4* arow[4];
  const float4* brow[4];
  bool aok[4], bok[4];
#pragma unroll
  for (int sl = 0; sl < 4; ++sl) {
    const int64_t qa = q0 + lane + 32 * sl, ga = g0 + lane + 32 * sl;
    aok[sl] = qa < nq;
    bok[sl] = ga < ng;
    arow[sl] = reinterpret_cast<const float4*>(h + size_t(aok[sl] ? qa : 0) * dp) + wq;
    brow[sl] = reinterpret_cast<const float4*>(h + size_t(bok[sl] ? nq + ga : 0) * dp) + wq;
  }
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 va[4], vb[4];
#pragma unroll
  for (int sl = 0; sl < 4; ++sl) {
    va[sl] = aok[sl] ? __ldg(arow[sl]) : zero;
    vb[sl] = bok[sl] ? __ldg(brow[sl]) : zero;
  }
  for (int k0 = 0; k0 < dp; k0 += DK) {
    __syncthreads();  // the previous chunk is consumed
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      const int r = lane + 32 * sl, kk = 4 * wq;
      As[(kk + 0) * ST + r] = va[sl].x;
      As[(kk + 1) * ST + r] = va[sl].y;
      As[(kk + 2) * ST + r] = va[sl].z;
      As[(kk + 3) * ST + r] = va[sl].w;
      Bs[(kk + 0) * ST + r] = vb[sl].x;
      Bs[(kk + 1) * ST + r] = vb[sl].y;
      Bs[(kk + 2) * ST + r] = vb[sl].z;
      Bs[(kk + 3) * ST + r] = vb[sl].w;
    }
    __syncthreads();
    if (k0 + DK < dp) {
      const int step = (k0 + DK) / 4;
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        va[sl] = aok[sl] ? __ldg(arow[sl] + step) : zero;
        vb[sl] = bok[sl] ? __ldg(brow[sl] + step) : zero;
      }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) p[j] = 0.f;
#pragma unroll 4
    for (int k = 0; k < DK; ++k) {
      const float4 x0 = reinterpret_cast<const float4*>(As + k * ST)[ty];
      const float4 x1 = reinterpret_cast<const float4*>(As + k * ST)[16 + ty];
      const float4 y0 = reinterpret_cast<const float4*>(Bs + k * ST)[tx];
      const float4 y1 = reinterpret_cast<const float4*>(Bs + k * ST)[16 + tx];
      const float xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float yb[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) p[a * 8 + b] = fmaf(xa[a], yb[b], p[a * 8 + b]);
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      float l = lo[j * STHREADS + t];
      ff_add(hi[j], l, p[j]);
      lo[j * STHREADS + t] = l;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t q = q0 + (a < 4 ? 4 * ty + a : 64 + 4 * ty + (a - 4));
    if (q >= nq) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int64_t g = g0 + (b < 4 ? 4 * tx + b : 64 + 4 * tx + (b - 4));
      if (g >= ng) continue;
      const double dot = double(hi[a * 8 + b]) + double(lo[(a * 8 + b) * STHREADS + t]);
      S[q * ng + g] = float(dot * inv[q] * inv[nq + g]);
    }
  }
}

}  // namespace

int launch_dense_layer(const Shape& sh, const float* hin, float* hout, const int32_t* nbr, const float* nbr_w,
                       const int32_t* nbr_n, int aggregator, cudaStream_t s) {
  const int T = 256;
  k7_dense_layer<<<unsigned((sh.n * kWarp + T - 1) / T), T, 0, s>>>(hin, hout, sh.n, sh.dp, nbr, nbr_w, nbr_n,
                                                                   sh.k2, aggregator == RERANK_AGG_MAX ? 1 : 0);
  return 1;
}

int launch_dense_scores(const Shape& sh, const float* h, double* inv, float* S, cudaStream_t s) {
  const int T = 256;
  k7_dense_inv_norms<<<unsigned((sh.n * kWarp + T - 1) / T), T, 0, s>>>(h, sh.n, sh.dp, inv);
  dim3 grid(unsigned((sh.ng + ST - 1) / ST), unsigned((sh.nq + ST - 1) / ST));
  cudaFuncSetAttribute(k7_dense_scores, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SSMEM));
  k7_dense_scores<<<grid, STHREADS, SSMEM, s>>>(h, sh.nq, sh.ng, sh.dp, inv, S);
  return 2;
}

}  // namespace rr

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
// gallery row g, 64 x 64 output tiles per CTA, 4 x 4 per thread.  Each
// 32-deep k-chunk is an FP32 FMA chain; the chunks are added in float-float
// (a TwoSum per chunk), so a score is as accurate as a chain of 32 products
// (about 1e-7 for unit rows) whatever d is; the norms are applied in FP64.
#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int DT = 64;   // output tile (queries x gallery rows)
constexpr int DK = 32;   // k-chunk
constexpr int DTHREADS = 256;

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

__global__ void __launch_bounds__(DTHREADS)
k7_dense_scores(const float* __restrict__ h, int64_t nq, int64_t ng, int dp, const double* __restrict__ inv,
                float* __restrict__ S) {
  __shared__ float4 As[DK][DT / 4];  // k-major: As[k][r / 4] holds rows r .. r + 3
  __shared__ float4 Bs[DK][DT / 4];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  const int64_t q0 = int64_t(blockIdx.y) * DT, g0 = int64_t(blockIdx.x) * DT;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
  // Loader: thread t moves rows r = t / 4 (0..63) and columns (t % 4) * 8 .. + 7 of the chunk.
  const int lr = t >> 2, lc = (t & 3) * 8;
  const bool qa = q0 + lr < nq, ga = g0 + lr < ng;
  const float* qa_row = h + size_t(qa ? q0 + lr : 0) * dp;
  const float* ga_row = h + size_t(ga ? nq + g0 + lr : 0) * dp;
  for (int k0 = 0; k0 < dp; k0 += DK) {
    float va[8], vb[8];
    const float4 a0 = qa ? __ldg(reinterpret_cast<const float4*>(qa_row + k0 + lc)) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 a1 =
        qa ? __ldg(reinterpret_cast<const float4*>(qa_row + k0 + lc + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 b0 = ga ? __ldg(reinterpret_cast<const float4*>(ga_row + k0 + lc)) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 b1 =
        ga ? __ldg(reinterpret_cast<const float4*>(ga_row + k0 + lc + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
    va[0] = a0.x; va[1] = a0.y; va[2] = a0.z; va[3] = a0.w; va[4] = a1.x; va[5] = a1.y; va[6] = a1.z; va[7] = a1.w;
    vb[0] = b0.x; vb[1] = b0.y; vb[2] = b0.z; vb[3] = b0.w; vb[4] = b1.x; vb[5] = b1.y; vb[6] = b1.z; vb[7] = b1.w;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      reinterpret_cast<float*>(&As[lc + u][0])[lr] = va[u];
      reinterpret_cast<float*>(&Bs[lc + u][0])[lr] = vb[u];
    }
    __syncthreads();
    float p[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) p[a][b] = 0.f;
#pragma unroll 8
    for (int k = 0; k < DK; ++k) {
      const float4 x = As[k][ty], y = Bs[k][tx];
      const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[a][b] = fmaf(xa[a], yb[b], p[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) ff_add(hi[a][b], lo[a][b], p[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t q = q0 + ty * 4 + a;
    if (q >= nq) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t g = g0 + tx * 4 + b;
      if (g >= ng) continue;
      const double dot = double(hi[a][b]) + double(lo[a][b]);
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
  dim3 grid(unsigned((sh.ng + DT - 1) / DT), unsigned((sh.nq + DT - 1) / DT));
  k7_dense_scores<<<grid, DTHREADS, 0, s>>>(h, sh.nq, sh.ng, sh.dp, inv, S);
  return 2;
}

}  // namespace rr

// K1a: FP32 similarity S = Xhat Xhat^T (Eq. 7) with a fused per-row top-K (Eq. 8).
//
// S is never written to memory.  A CTA owns a block of 128 rows and a chunk of
// the column tiles; for every 128 x 128 tile it runs an FP32 SIMT GEMM over
// the full feature dimension (register-blocked 8 x 8 per thread, double
// buffered shared memory), stages the tile in shared memory, and the 128 row
// owners fold their row into a sorted top-K list kept in shared memory across
// the chunk.  Each row's list holds the K best columns of its chunk by
// (S desc, index asc), with S_ii set to exactly 1.  The per-chunk lists are
// merged and certified by the refinement stage (K2).
//
// Error bound of each S value (used by K2): one FMA chain over dp terms of
// unit-normalised rows, |S_fp32 - S| <= (dp + 10) u.
#include <cfloat>

#include "common.cuh"
#include "internal.hpp"
#include "topk_heap.cuh"

namespace rr {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;
constexpr int KMAX = 64;
constexpr int CSTRIDE = BN + 1;

struct SmemMain {
  float a[2][BK][BM + 4];
  float b[2][BK][BN + 4];
};
union SmemTile {
  SmemMain m;
  float c[BM][CSTRIDE];
};
struct Smem {
  SmemTile u;
  float ls[KMAX][BM];
  int li[KMAX][BM];
};

__global__ void __launch_bounds__(NT, 1)
k1_sgemm_topk(const float* __restrict__ x, int64_t n, int dp, int K, int P, int col_tiles,
              int* __restrict__ row_floor, float* __restrict__ part_s, int32_t* __restrict__ part_i) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // Row blocks vary fastest over the grid, so a row's later chunks start after
  // its earlier ones have published their floors.
  const int chunk = blockIdx.y;
  const int64_t row0 = int64_t(blockIdx.x) * BM;
  const int t_begin = int(int64_t(chunk) * col_tiles / P);
  const int t_end = int(int64_t(chunk + 1) * col_tiles / P);

  // Threads 0..127 own one row each: a top-K heap over this chunk's columns.
  const int64_t my_row = row0 + (tid & (BM - 1));
  const bool live = tid < BM && my_row < n;
  RowHeap<BM> heap{&sm.ls[0][0], &sm.li[0][0], tid & (BM - 1), K, 0};
  heap.reset(K);
  const float floor_s = live ? key_score(row_floor[my_row]) : FLT_MAX;
  float root_s = -FLT_MAX;
  int root_i = kInvalidIdx;
  bool heap_full = false;
  __syncthreads();

  const int lr = tid >> 2;        // loader row (and lr + 64)
  const int lk = (tid & 3) * 4;   // loader k offset
  const int nk = dp / BK;

  for (int ct = t_begin; ct < t_end; ++ct) {
    const int64_t col0 = int64_t(ct) * BN;
    const float* ag = x + (row0 + lr) * dp + lk;
    const float* bg = x + (col0 + lr) * dp + lk;
    const size_t half = size_t(64) * dp;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra0 = __ldg(reinterpret_cast<const float4*>(ag));
    float4 ra1 = __ldg(reinterpret_cast<const float4*>(ag + half));
    float4 rb0 = __ldg(reinterpret_cast<const float4*>(bg));
    float4 rb1 = __ldg(reinterpret_cast<const float4*>(bg + half));
    auto stash = [&](int st) {
      sm.u.m.a[st][lk + 0][lr] = ra0.x; sm.u.m.a[st][lk + 1][lr] = ra0.y;
      sm.u.m.a[st][lk + 2][lr] = ra0.z; sm.u.m.a[st][lk + 3][lr] = ra0.w;
      sm.u.m.a[st][lk + 0][lr + 64] = ra1.x; sm.u.m.a[st][lk + 1][lr + 64] = ra1.y;
      sm.u.m.a[st][lk + 2][lr + 64] = ra1.z; sm.u.m.a[st][lk + 3][lr + 64] = ra1.w;
      sm.u.m.b[st][lk + 0][lr] = rb0.x; sm.u.m.b[st][lk + 1][lr] = rb0.y;
      sm.u.m.b[st][lk + 2][lr] = rb0.z; sm.u.m.b[st][lk + 3][lr] = rb0.w;
      sm.u.m.b[st][lk + 0][lr + 64] = rb1.x; sm.u.m.b[st][lk + 1][lr + 64] = rb1.y;
      sm.u.m.b[st][lk + 2][lr + 64] = rb1.z; sm.u.m.b[st][lk + 3][lr + 64] = rb1.w;
    };
    stash(0);
    __syncthreads();

    for (int kt = 0; kt < nk; ++kt) {
      const int cur = kt & 1;
      if (kt + 1 < nk) {
        const int off = (kt + 1) * BK;
        ra0 = __ldg(reinterpret_cast<const float4*>(ag + off));
        ra1 = __ldg(reinterpret_cast<const float4*>(ag + half + off));
        rb0 = __ldg(reinterpret_cast<const float4*>(bg + off));
        rb1 = __ldg(reinterpret_cast<const float4*>(bg + half + off));
      }
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&sm.u.m.a[cur][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&sm.u.m.a[cur][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&sm.u.m.b[cur][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&sm.u.m.b[cur][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (kt + 1 < nk) stash(cur ^ 1);
      __syncthreads();
    }

    // Stage the tile (the union re-uses the operand buffers; all reads are done).
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4);
        sm.u.c[r][c] = acc[i][j];
      }
    }
    __syncthreads();

    if (tid < BM) {
      // Batches of 32 columns: admission test against the current root, then a
      // warp-convergent drain that folds in one admitted column per lane per round.
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t mask = 0;
        for (int j = 0; j < 32; ++j) {
          const int64_t col = col0 + c0 + j;
          const float v = (col == my_row) ? 1.0f : sm.u.c[tid][c0 + j];
          const bool adm = live && col < n && v >= floor_s &&
                           (!heap_full || ranks_before(v, int(col), root_s, root_i));
          mask |= adm ? (1u << j) : 0u;
        }
        while (__any_sync(kFull, mask != 0u)) {
          if (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1u;
            const int64_t col = col0 + c0 + j;
            heap.push((col == my_row) ? 1.0f : sm.u.c[tid][c0 + j], int(col));
          }
          heap_full = heap.full();
          if (heap_full) {
            root_s = heap.s(0);
            root_i = heap.i(0);
          }
        }
      }
    }
    __syncthreads();
  }

  // Write this chunk's list, sorted: part[(row * P + chunk) * K + r].
  if (live) {
    heap.sort_desc();
    if (heap_full) atomicMax(row_floor + my_row, score_key(sm.ls[K - 1][tid]));
  }
  __syncthreads();
  for (int e = tid; e < BM * K; e += NT) {
    const int r = e / K, j = e % K;
    const int64_t row = row0 + r;
    if (row < n) {
      const size_t o = (size_t(row) * P + chunk) * K + j;
      part_s[o] = sm.ls[j][r];
      part_i[o] = sm.li[j][r];
    }
  }
}

}  // namespace

int launch_sim_fp32_topk(const Shape& sh, const float* xhat, int* row_floor, float* part_s, int32_t* part_i,
                         int sm_count, cudaStream_t s) {
  (void)sm_count;
  const int col_tiles = int(sh.np / BN);
  const int row_blocks = int(sh.np / BM);
  const size_t smem = sizeof(Smem);
  cudaMemsetAsync(row_floor, kFloorResetByte, sizeof(int) * size_t(sh.n), s);
  cudaFuncSetAttribute(k1_sgemm_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  dim3 grid(row_blocks, sh.P);
  k1_sgemm_topk<<<grid, NT, smem, s>>>(xhat, sh.n, sh.dp, sh.K, sh.P, col_tiles, row_floor, part_s, part_i);
  return 1;
}

int sim_fp32_kmax() { return KMAX; }

}  // namespace rr

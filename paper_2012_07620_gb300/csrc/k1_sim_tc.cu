// K1b: similarity S = Xhat Xhat^T (Eq. 7) on the 5th-generation tensor cores
// (BF16 or FP8-E4M3 operands, FP32 accumulation in TMEM) with a fused per-row
// top-K (Eq. 8).  S never leaves the SM.
//
// One persistent CTA per SM walks work items (row block of 128 rows, chunk of
// 256-column tiles); items are ordered so that CTAs running together share
// the chunk, so the column tiles they stream are L2 hits.  Roles:
//   warp 0 (one thread)  TMA producer: per k-block, the 128-row A slab and
//                        the 256-row B slab (128-byte swizzle) into a
//                        3-stage shared-memory ring;
//   warp 1 (one thread)  MMA issuer: 4 tcgen05.mma (K = 16 BF16 / 32 FP8) per
//                        k-block into one of two 128 x 256 FP32 accumulators
//                        in TMEM (512 columns), commit frees the ring slot;
//                        the tile's last commit hands the accumulator over;
//   warps 2-5            epilogue: each thread owns one TMEM lane = one row,
//                        reads its 256 scores with tcgen05.ld (32 at a time),
//                        applies the FP8 row/column scales, sets S_ii = 1 and
//                        keeps a sorted top-K list (S desc, index asc) in
//                        shared memory; then releases the accumulator.
// The two accumulators let the MMA of tile t+1 run under the epilogue of
// tile t.  At the end of a work item the lists are written as one partial
// candidate list per (row, chunk), merged and certified by K2.
#include <cuda.h>
#include <cfloat>

#include "common.cuh"
#include "internal.hpp"
#include "tc_ptx.cuh"

namespace rr {
namespace {

constexpr int TBM = 128;
constexpr int TBN = 256;
constexpr int STAGES = 3;
constexpr int A_BYTES = TBM * 128;    // one 128-byte swizzle row per operand row
constexpr int B_BYTES = TBN * 128;
constexpr int KLIST = 64;
constexpr int THREADS = 192;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct alignas(1024) TcSmem {
  uint8_t a[STAGES][A_BYTES];
  uint8_t b[STAGES][B_BYTES];
  float ls[KLIST][TBM];
  int li[KLIST][TBM];
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

struct TcArgs {
  int64_t n;
  int row_blocks, col_tiles, chunks, kblocks, K;
  const float* inv_scale;  // FP8 only: 1 / s_i per row
  float* part_s;
  int32_t* part_i;
  long long* status;
};

__device__ __forceinline__ void item_range(const TcArgs& A, int item, int& rb, int& chunk, int& t0, int& t1) {
  rb = item % A.row_blocks;
  chunk = item / A.row_blocks;
  t0 = int(int64_t(chunk) * A.col_tiles / A.chunks);
  t1 = int(int64_t(chunk + 1) * A.col_tiles / A.chunks);
}

template <bool FP8>
__global__ void __launch_bounds__(THREADS, 1) k1_tc_topk(const __grid_constant__ CUtensorMap tmap, TcArgs A) {
  extern __shared__ uint8_t smem_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &sm.abort;
  const int items = A.row_blocks * A.chunks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&sm.full[s], 1);
      tc::mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&sm.tfull[b], 1);
      tc::mbar_init(&sm.tempty[b], 4);
    }
    tc::mbar_init(&sm.done, 1);
    sm.abort = 0;
    tc::fence_barrier_init();
    tc::tma_prefetch_desc(&tmap);
  }
  if (warp == 1) {
    tc::tmem_alloc(&sm.tmem_base, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0;  // bit s: slot s holds a load that may still be in flight
      uint32_t armed_phase = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        int rb, chunk, t0, t1;
        item_range(A, item, rb, chunk, t0, t1);
        for (int ct = t0; ct < t1 && ok; ++ct) {
          for (int kb = 0; kb < A.kblocks; ++kb) {
            if (!tc::mbar_wait(&sm.empty[stage], phase ^ 1u, abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&sm.full[stage], A_BYTES + B_BYTES);
            const int kx = kb * (FP8 ? 128 : 64);
            tc::tma_load_2d(sm.a[stage], &tmap, &sm.full[stage], kx, rb * TBM);
            tc::tma_load_2d(sm.b[stage], &tmap, &sm.full[stage], kx, ct * TBN);
            tc::tma_load_2d(sm.b[stage] + B_BYTES / 2, &tmap, &sm.full[stage], kx, ct * TBN + TBN / 2);
            armed |= 1u << stage;
            armed_phase = (armed_phase & ~(1u << stage)) | (phase << stage);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        *abort = 1;
        set_error(A.status, kErrTimeout);
        // Let loads already issued land before the CTA exits.
        for (int s = 0; s < STAGES; ++s)
          if (armed & (1u << s)) tc::mbar_wait(&sm.full[s], (armed_phase >> s) & 1u, abort, WAIT_LIMIT);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = tc::instr_desc(FP8 ? 0u : 1u, TBM, TBN);
      uint32_t stage = 0, phase = 0, tcount = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        int rb, chunk, t0, t1;
        item_range(A, item, rb, chunk, t0, t1);
        for (int ct = t0; ct < t1 && ok; ++ct) {
          const uint32_t ab = tcount & 1u, tph = (tcount >> 1) & 1u;
          if (!tc::mbar_wait(&sm.tempty[ab], tph ^ 1u, abort, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t d = tmem + ab * TBN;
          for (int kb = 0; kb < A.kblocks; ++kb) {
            if (!tc::mbar_wait(&sm.full[stage], phase, abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const uint64_t da = tc::desc_sw128(sm.a[stage]);
            const uint64_t db = tc::desc_sw128(sm.b[stage]);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // 32 bytes of K per instruction: advance the start address by 2 (16-byte units).
              if (FP8)
                tc::mma_fp8(d, da + 2u * kk, db + 2u * kk, idesc, (kb | kk) != 0);
              else
                tc::mma_bf16(d, da + 2u * kk, db + 2u * kk, idesc, (kb | kk) != 0);
            }
            tc::mma_commit(&sm.empty[stage]);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          tc::mma_commit(&sm.tfull[ab]);
          ++tcount;
        }
      }
      if (!ok) {
        *abort = 1;
        set_error(A.status, kErrTimeout);
      }
      // Every MMA issued by this thread has completed once `done` fires.
      tc::mma_commit(&sm.done);
      tc::mbar_wait(&sm.done, 0, abort, WAIT_LIMIT);
    }
  } else {
    // ---------------- epilogue: warps 2..5 ----------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    const uint32_t tlane = tmem + (uint32_t(q * 32) << 16);
    uint32_t tcount = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int rb, chunk, t0, t1;
      item_range(A, item, rb, chunk, t0, t1);
      const int64_t grow = int64_t(rb) * TBM + r;
      const bool live = grow < A.n;
      for (int j = 0; j < A.K; ++j) {
        sm.ls[j][r] = -FLT_MAX;
        sm.li[j][r] = kInvalidIdx;
      }
      float thr_s = -FLT_MAX;
      int thr_i = kInvalidIdx;
      const float rinv = (FP8 && live) ? A.inv_scale[grow] : 1.0f;
      for (int ct = t0; ct < t1; ++ct) {
        const uint32_t ab = tcount & 1u, tph = (tcount >> 1) & 1u;
        if (!tc::mbar_wait(&sm.tfull[ab], tph, abort, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        for (int cb = 0; cb < TBN / 32; ++cb) {
          uint32_t v[32];
          tc::tmem_ld32(tlane + ab * TBN + cb * 32, v);
          tc::tmem_wait_ld();
          if (live) {
            const int64_t cbase = int64_t(ct) * TBN + cb * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int64_t col = cbase + j;
              if (col >= A.n) break;
              float s = __uint_as_float(v[j]);
              if (FP8) s = s * rinv * __ldg(A.inv_scale + col);
              if (col == grow) s = 1.0f;
              if (ranks_before(s, int(col), thr_s, thr_i)) {
                int p = A.K - 1;
                while (p > 0) {
                  const float ps = sm.ls[p - 1][r];
                  const int pi = sm.li[p - 1][r];
                  if (!ranks_before(s, int(col), ps, pi)) break;
                  sm.ls[p][r] = ps;
                  sm.li[p][r] = pi;
                  --p;
                }
                sm.ls[p][r] = s;
                sm.li[p][r] = int(col);
                thr_s = sm.ls[A.K - 1][r];
                thr_i = sm.li[A.K - 1][r];
              }
            }
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&sm.tempty[ab]);
        ++tcount;
      }
      if (!ok) break;
      if (live) {
        const size_t o = (size_t(grow) * A.chunks + chunk) * A.K;
        for (int j = 0; j < A.K; ++j) {
          A.part_s[o + j] = sm.ls[j][r];
          A.part_i[o + j] = sm.li[j][r];
        }
      }
    }
    if (!ok) {
      *abort = 1;
      set_error(A.status, kErrTimeout);
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

}  // namespace

size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }
int tc_kmax() { return KLIST; }
int tc_tile_rows() { return TBM; }
int tc_tile_cols() { return TBN; }

// Returns the number of kernels launched (1), or a negative value when the
// tensor map cannot be encoded.
int launch_sim_tc_topk(const Shape& sh, const void* xlow, bool fp8, const float* inv_scale, float* part_s,
                       int32_t* part_i, long long* status, int sm_count, cudaStream_t s) {
  EncodeFn enc = get_encode();
  if (!enc) return -1;
  CUtensorMap map;
  const cuuint64_t dims[2] = {cuuint64_t(sh.dp), cuuint64_t(sh.np)};
  const cuuint64_t strides[1] = {cuuint64_t(sh.dp) * (fp8 ? 1 : 2)};
  const cuuint32_t box[2] = {fp8 ? 128u : 64u, 128u};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(xlow), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return -1;
  TcArgs A;
  A.n = sh.n;
  A.row_blocks = int(sh.np / TBM);
  A.col_tiles = int(sh.np / TBN);
  A.chunks = sh.P;
  A.kblocks = fp8 ? sh.dp / 128 : sh.dp / 64;
  A.K = sh.K;
  A.inv_scale = inv_scale;
  A.part_s = part_s;
  A.part_i = part_i;
  A.status = status;
  const int items = A.row_blocks * A.chunks;
  const int grid = items < sm_count ? items : sm_count;
  const size_t smem = tc_smem_bytes();
  if (fp8) {
    cudaFuncSetAttribute(k1_tc_topk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k1_tc_topk<true><<<grid, THREADS, smem, s>>>(map, A);
  } else {
    cudaFuncSetAttribute(k1_tc_topk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k1_tc_topk<false><<<grid, THREADS, smem, s>>>(map, A);
  }
  return 1;
}

}  // namespace rr

// K1b: similarity S = Xhat Xhat^T (Eq. 7) on the 5th-generation tensor cores
// (BF16 or FP8-E4M3 operands, FP32 accumulation in TMEM) with a fused per-row
// top-K (Eq. 8).  S never leaves the SM.
//
// One persistent CTA per SM walks work items (row block of 128 rows, chunk of
// 256-column tiles); items are ordered so that CTAs running together share
// the chunk, so the column tiles they stream are L2 hits, and so that a row's
// later chunks run after its earlier ones (see the floors below).  Roles:
//   warp 0 (one thread)  TMA producer: per k-block, the 128-row A slab and
//                        the 256-row B slab (128-byte swizzle) into a
//                        4-stage shared-memory ring;
//   warp 1 (one thread)  MMA issuer: 4 tcgen05.mma (K = 16 BF16 / 32 FP8) per
//                        k-block into one of two 128 x 256 FP32 accumulators
//                        in TMEM (512 columns), commit frees the ring slot;
//                        the tile's last commit hands the accumulator over;
//   warps 2-5            epilogue: each thread owns one TMEM lane = one row,
//                        reads its 256 scores with tcgen05.ld (32 at a time),
//                        applies the FP8 row/column scales, sets S_ii = 1 and
//                        folds admitted columns into a sorted top-K list held
//                        in registers; then releases the accumulator.
// The two accumulators let the MMA of tile t+1 run under the epilogue of
// tile t.  At the end of a work item the list is written as one
// partial candidate list per (row, chunk), merged and certified by K2.
//
// Split mode (the recheck of rows whose list could not be certified): the
// operands are the hi/lo BF16 halves of the unit rows, x = hi + lo + r, and
// the k-loop runs three times over the feature dimension so that the one
// accumulator collects hi_i.hi_j + lo_i.hi_j + hi_i.lo_j.  The A rows are the
// gathered rows being rechecked; their count is read on the device.
#include <cuda.h>
#include <cfloat>
#include <climits>

#include <cstdlib>
#include <type_traits>

#include "common.cuh"
#include "internal.hpp"
#include "tc_ptx.cuh"
#include "topk_heap.cuh"  // score_key / key_score

namespace rr {
namespace {

constexpr int TBM = 128;
constexpr int TBN = 256;
constexpr int STAGES = 4;
constexpr int A_BYTES = TBM * 128;    // one 128-byte swizzle row per operand row
constexpr int B_BYTES = TBN * 128;
constexpr int KLIST = 64;  // largest candidate list the kernel supports
// Epilogue warp groups: group g owns columns [g, g+1) * TBN / EG of every tile
// and keeps its own list per row (EG lists per row and chunk).  Two groups
// when the MMA work per tile is short (K depth <= 1024), so that the
// epilogue keeps pace; one otherwise (fewer, longer lists).
constexpr int EG_MAX = 2;
constexpr int threads_of(int eg) { return 64 + 128 * eg; }  // TMA warp, MMA warp, 4 epilogue warps per group
constexpr uint32_t WAIT_LIMIT = 1u << 22;

// BF16 / FP8: one matrix against itself (or a rectangular block);
// SPLIT: gathered rows, hi/lo products; GATHER: gathered rows, one BF16 product.
enum { MODE_BF16 = 0, MODE_FP8 = 1, MODE_SPLIT = 2, MODE_GATHER = 3 };
__host__ __device__ constexpr bool gathered(int mode) { return mode == MODE_SPLIT || mode == MODE_GATHER; }

// Shared memory of one CTA.  A CTA of a pair holds only its half of the B
// rows (128 of the tile's 256), so the same space holds more stages.  EGN
// epilogue groups; QC > 0: each row's queue of QC admitted (score, column)
// pairs not yet in its list (paired kernels).
template <int STG, int BBYTES, int EGN, int QC>
struct alignas(1024) TcSmemT {
  static constexpr int kStages = STG;
  uint8_t a[STG][A_BYTES];
  uint8_t b[STG][BBYTES];
  float batch[EGN][32][TBM];  // per group: scores of the 32 columns being folded in
  float qsc[QC > 0 ? EGN : 1][QC > 0 ? QC : 1][TBM];
  int32_t qcol[QC > 0 ? EGN : 1][QC > 0 ? QC : 1][TBM];
  uint64_t full[STG];
  uint64_t empty[STG];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t done;
  // Dynamic item order: the publisher's ring of item numbers.
  int item_q[4];
  uint64_t ifull[4];
  uint64_t iempty[4];
  uint32_t tmem_base;
  int abort;
};
constexpr int IQ = 4;  // item ring depth
constexpr int QCAP = 8;  // entries of a row's insertion queue (paired kernels)
using TcSmem = TcSmemT<STAGES, B_BYTES, EG_MAX, 0>;
// Pairs: 32 KB stages; six of them with one epilogue group, five with two.
template <int EG>
using TcSmemPair = TcSmemT<EG == 1 ? 6 : 5, B_BYTES / 2, EG, QCAP>;
template <bool PAIR, int EG>
using SmemOf = typename std::conditional<PAIR, TcSmemPair<EG>, TcSmem>::type;

// Batched launches: up to kMaxBatchInst instances, each a matrix against
// itself; their tensor maps travel as one kernel parameter.
constexpr int kMaxBatchInst = 64;
struct TcMaps {
  CUtensorMap m[kMaxBatchInst];
};
struct TcInst {
  int64_t n;                // rows = columns of the instance
  int row_blocks, col_tiles, chunks, kblocks, K;
  int item_begin;           // first item of the instance in the launch's item space
  const float* inv_scale;
  int* row_floor;
  float* part_s;
  int32_t* part_i;
  long long* status;
};

struct TcArgs {
  int64_t n;                // columns of B (valid column indices 0 .. n-1)
  int64_t a_rows;           // outside split mode: valid rows of A
  int64_t row0;             // outside split mode: vertex index of A row 0
  int64_t col0;             // vertex index of B column 0
  int row_blocks;           // outside split mode
  int col_tiles, chunks, kblocks, K;
  const float* inv_scale;   // FP8 only: 1 / s_i per row
  const int32_t* rows;      // split mode: global row of each A row
  const int32_t* count;     // split mode: number of A rows
  int* row_floor;           // per A row: score_key of the best K-th score any finished chunk found
  int stall;                // test hook: the TMA warp issues nothing, so every wait runs out
  float* part_s;
  int32_t* part_i;
  long long* status;
  const TcInst* insts;      // batched launch: the instances (device memory), else null
  int ninst, items_total;
  int* work;                // non-null: items are taken in order from this counter (zero at launch)
};

// One work item (a row block against a chunk of column tiles) with the
// parameters of its instance.
struct TcItem {
  const CUtensorMap* ma0;
  const CUtensorMap* ma1;
  const CUtensorMap* mb0;
  const CUtensorMap* mb1;
  int rb, chunk, t0, t1, kblocks, K, chunks;
  int64_t n, nrows, row0, col0;
  const float* inv_scale;
  int* row_floor;
  float* part_s;
  int32_t* part_i;
};

// Gathered launches (recheck): the row count is known on the device only, so
// the number of column chunks is chosen there, by the host's rule (whole waves
// of items over the grid, each chunk charged three tiles for its cold start),
// up to the A.chunks lists per row the caller reads.
__device__ __forceinline__ int pick_chunks(int row_blocks, int maxc, int col_tiles, int grid) {
  int best = maxc;
  long long best_cost = LLONG_MAX;
  for (int c = 1; c <= maxc; ++c) {
    const long long waves = (static_cast<long long>(row_blocks) * c + grid - 1) / grid;
    const long long cost = waves * ((col_tiles + c - 1) / c + 3);
    if (cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

// chunks: column chunks of this launch (<= A.chunks, the lists per row in the output).
template <bool BATCH>
__device__ __forceinline__ void get_item(const TcArgs& A, const CUtensorMap* ma0, const CUtensorMap* ma1,
                                         const CUtensorMap* mb0, const CUtensorMap* mb1, const CUtensorMap* bmaps,
                                         int row_blocks, int64_t nrows, int item, TcItem& it, int chunks) {
  if (!BATCH) {
    it.ma0 = ma0;
    it.ma1 = ma1;
    it.mb0 = mb0;
    it.mb1 = mb1;
    it.rb = item % row_blocks;
    it.chunk = item / row_blocks;
    it.t0 = int(int64_t(it.chunk) * A.col_tiles / chunks);
    it.t1 = int(int64_t(it.chunk + 1) * A.col_tiles / chunks);
    it.kblocks = A.kblocks;
    it.K = A.K;
    it.chunks = A.chunks;
    it.n = A.n;
    it.nrows = nrows;
    it.row0 = A.row0;
    it.col0 = A.col0;
    it.inv_scale = A.inv_scale;
    it.row_floor = A.row_floor;
    it.part_s = A.part_s;
    it.part_i = A.part_i;
  } else {
    int lo = 0, hi = A.ninst - 1;  // last instance whose items begin at or before `item`
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (A.insts[mid].item_begin <= item) lo = mid;
      else hi = mid - 1;
    }
    const TcInst& I = A.insts[lo];
    const int local = item - I.item_begin;
    it.ma0 = it.ma1 = it.mb0 = it.mb1 = bmaps + lo;
    it.rb = local % I.row_blocks;
    it.chunk = local / I.row_blocks;
    it.t0 = int(int64_t(it.chunk) * I.col_tiles / I.chunks);
    it.t1 = int(int64_t(it.chunk + 1) * I.col_tiles / I.chunks);
    it.kblocks = I.kblocks;
    it.K = I.K;
    it.chunks = I.chunks;
    it.n = I.n;
    it.nrows = I.n;
    it.row0 = 0;
    it.col0 = 0;
    it.inv_scale = I.inv_scale;
    it.row_floor = I.row_floor;
    it.part_s = I.part_s;
    it.part_i = I.part_i;
  }
}

// Timeout: every instance of the launch reports it.
template <bool BATCH>
__device__ void report_timeout(const TcArgs& A) {
  if (!BATCH) {
    set_error(A.status, kErrTimeout);
  } else {
    for (int k = 0; k < A.ninst; ++k) set_error(A.insts[k].status, kErrTimeout);
  }
}



// Give loads this CTA issued time to land before it leaves (pair mode, after a
// timeout: their bytes complete on the even CTA's barrier, which this CTA
// cannot poll).  A tile load takes microseconds; wait about 200 us.
__device__ __forceinline__ void drain_delay() {
  for (int k = 0; k < 200; ++k) __nanosleep(1000);
}

// Insert (cs, ci) into a row's sorted list: slot j takes cs where cs first
// beats ls[j], and slot j-1's old entry for every later slot.  For the sorted
// scores that is max(min(ls[j-1], cs), ls[j]); the columns follow the same
// choice.  All tests use the old list: no serial dependency.  Columns arrive
// in increasing order, so an equal score keeps the earlier, lower column in
// front (score desc, column asc); cs = -inf changes nothing.
template <int KL>
__device__ __forceinline__ void list_insert(float (&ls)[KL], int (&li)[KL], float cs, int ci) {
#pragma unroll
  for (int j = KL - 1; j > 0; --j) {
    const bool bj = cs > ls[j], bp = cs > ls[j - 1];
    li[j] = bp ? li[j - 1] : (bj ? ci : li[j]);
    ls[j] = fmaxf(fminf(ls[j - 1], cs), ls[j]);
  }
  li[0] = cs > ls[0] ? ci : li[0];
  ls[0] = fmaxf(cs, ls[0]);
}

// Item order.  Static: unit, unit + units, ...  Dynamic (A.work set): the
// publisher (the TMA thread of a CTA, or of the even CTA of a pair) takes the
// next item number from the global counter and hands it to every consumer of
// the work through a ring in shared memory (both CTAs' rings for a pair):
// the MMA thread, the epilogue warps and, in the odd CTA of a pair, its TMA
// thread.  A slot is reused once all consumers released it on the even CTA's
// `iempty`.  Items still come in increasing order overall, but a unit that
// finishes early takes more of them, which evens out the per-item cost of the
// top-K epilogue.  Every consumer reads the same sequence; the first number
// >= items ends it.
struct ItemRing {
  uint32_t qs = 0, qph = 0;
};

template <bool PAIR, class Smem>
__device__ __forceinline__ int next_item(Smem& sm, const TcArgs& A, bool publisher, bool leader, int prev, int unit,
                                         int units, ItemRing& rg, volatile int* abort, bool& ok) {
  if (!A.work) return prev < 0 ? unit : prev + units;
  int it = INT_MAX;
  if (publisher) {
    it = atomicAdd(A.work, 1);
    if (!tc::mbar_wait(&sm.iempty[rg.qs], rg.qph ^ 1u, abort, WAIT_LIMIT)) {
      ok = false;
      return INT_MAX;
    }
    reinterpret_cast<volatile int*>(sm.item_q)[rg.qs] = it;
    if (PAIR) {
      tc::st_cluster(tc::map_to_rank(&sm.item_q[rg.qs], 1), it);
      tc::mbar_arrive_cluster(tc::map_to_rank(&sm.ifull[rg.qs], 1));
    }
    tc::mbar_arrive(&sm.ifull[rg.qs]);
  } else {
    const bool got = PAIR ? tc::mbar_wait_cluster(&sm.ifull[rg.qs], rg.qph, abort, WAIT_LIMIT)
                          : tc::mbar_wait(&sm.ifull[rg.qs], rg.qph, abort, WAIT_LIMIT);
    if (!got) {
      ok = false;
      return INT_MAX;
    }
    it = reinterpret_cast<volatile int*>(sm.item_q)[rg.qs];
    if (PAIR && !leader) tc::mbar_arrive_cluster(tc::map_to_rank(&sm.iempty[rg.qs], 0));
    else tc::mbar_arrive(&sm.iempty[rg.qs]);
  }
  if (++rg.qs == IQ) {
    rg.qs = 0;
    rg.qph ^= 1u;
  }
  return it;
}

// PAIR: the CTAs of a cluster of two compute 256-row tiles together with
// tcgen05 cta_group::2.  The even CTA ("leader") issues the MMAs; each CTA
// loads its own 128 rows of A and its 128 of the tile's 256 B rows, counted
// on the leader's `full` barrier; the MMA's commits reach both CTAs'
// `empty` / `tfull` barriers; both CTAs' epilogue warps release an
// accumulator on the leader's `tempty`.
template <int MODE, int KL, int EGROUPS, bool BATCH, bool PAIR>
__device__ __forceinline__ void tc_body(const CUtensorMap* pA0, const CUtensorMap* pA1, const CUtensorMap* pB0,
                                        const CUtensorMap* pB1, const CUtensorMap* bmaps, const TcArgs& A) {
  using Smem = SmemOf<PAIR, EGROUPS>;
  constexpr int STG = Smem::kStages;
  constexpr bool QUEUE = PAIR;  // insertion queues (see the epilogue)
  constexpr int ROWS = PAIR ? 2 * TBM : TBM;  // A rows of one work item
  extern __shared__ uint8_t smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &sm.abort;
  constexpr int SEGS = MODE == MODE_SPLIT ? 3 : 1;
  const uint32_t rank = PAIR ? tc::cluster_rank() : 0u;
  const bool leader = rank == 0;
  const int unit = PAIR ? int(blockIdx.x >> 1) : int(blockIdx.x);   // cluster (pair) or CTA
  const int units = PAIR ? int(gridDim.x >> 1) : int(gridDim.x);
  const int64_t nrows = gathered(MODE) ? int64_t(*A.count) : A.a_rows;
  const int row_blocks = gathered(MODE) ? int((nrows + ROWS - 1) / ROWS) : A.row_blocks;
  const int chunks = gathered(MODE) ? pick_chunks(row_blocks, A.chunks, A.col_tiles, units) : A.chunks;
  const int items = BATCH ? A.items_total : row_blocks * chunks;

  if (threadIdx.x == 0) {
    for (int st = 0; st < STG; ++st) {
      tc::mbar_init(&sm.full[st], 1);
      tc::mbar_init(&sm.empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&sm.tfull[b], 1);
      tc::mbar_init(&sm.tempty[b], 4 * EGROUPS * (PAIR ? 2 : 1));
    }
    tc::mbar_init(&sm.done, 1);
    for (int q = 0; q < IQ; ++q) {
      tc::mbar_init(&sm.ifull[q], 1);
      // consumers: the MMA thread and the epilogue warps; for a pair also the
      // odd CTA's TMA thread and epilogue warps (they release on the even CTA's)
      tc::mbar_init(&sm.iempty[q], PAIR ? 2 + 8 * EGROUPS : 1 + 4 * EGROUPS);
    }
    sm.abort = 0;
    tc::fence_barrier_init();
    if (!BATCH) {
      tc::tma_prefetch_desc(pA0);
      tc::tma_prefetch_desc(pB0);
      if (MODE == MODE_SPLIT) {
        tc::tma_prefetch_desc(pA1);
        tc::tma_prefetch_desc(pB1);
      }
    }
  }
  if (warp == 1) {
    if (PAIR) {
      tc::tmem_alloc_pair(&sm.tmem_base, 512);
      tc::tmem_relinquish_pair();
    } else {
      tc::tmem_alloc(&sm.tmem_base, 512);
      tc::tmem_relinquish();
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (PAIR) tc::cluster_sync();  // the peer's barriers are initialised before any cross-CTA signal
  tc::tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0;  // bit s: slot s holds a load that may still be in flight
      uint32_t armed_phase = 0;
      bool ok = true;
      ItemRing rg;
      const bool publisher = !PAIR || leader;
      for (int item = A.stall ? INT_MAX : next_item<PAIR>(sm, A, publisher, leader, -1, unit, units, rg, abort, ok);
           item < items && ok;
           item = next_item<PAIR>(sm, A, publisher, leader, item, unit, units, rg, abort, ok)) {
        TcItem it;
        get_item<BATCH>(A, pA0, pA1, pB0, pB1, bmaps, row_blocks, nrows, item, it, chunks);
        const int rb = it.rb;
        const int kb_total = it.kblocks * SEGS;
        for (int ct = it.t0; ct < it.t1 && ok; ++ct) {
          for (int kt = 0; kt < kb_total; ++kt) {
            if (!tc::mbar_wait(&sm.empty[stage], phase ^ 1u, abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            const int seg = kt / it.kblocks, kb = kt - seg * it.kblocks;
            const CUtensorMap* ma = seg == 1 ? it.ma1 : it.ma0;
            const CUtensorMap* mb = seg == 2 ? it.mb1 : it.mb0;
            const int kx = kb * (MODE == MODE_FP8 ? 128 : 64);
            if (PAIR) {
              // this CTA's A rows and its half of the tile's B rows; bytes counted on the leader
              const uint32_t bar = tc::map_to_rank(&sm.full[stage], 0);
              if (leader) tc::mbar_arrive_expect_tx(&sm.full[stage], 2 * (A_BYTES + B_BYTES / 2));
              tc::tma_load_2d_pair(sm.a[stage], ma, bar, kx, rb * ROWS + int(rank) * TBM);
              tc::tma_load_2d_pair(sm.b[stage], mb, bar, kx, ct * TBN + int(rank) * (TBN / 2));
            } else {
              tc::mbar_arrive_expect_tx(&sm.full[stage], A_BYTES + B_BYTES);
              tc::tma_load_2d(sm.a[stage], ma, &sm.full[stage], kx, rb * TBM);
              tc::tma_load_2d(sm.b[stage], mb, &sm.full[stage], kx, ct * TBN);
              tc::tma_load_2d(sm.b[stage] + B_BYTES / 2, mb, &sm.full[stage], kx, ct * TBN + TBN / 2);
            }
            armed |= 1u << stage;
            armed_phase = (armed_phase & ~(1u << stage)) | (phase << stage);
            if (++stage == STG) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        *abort = 1;
        report_timeout<BATCH>(A);
        // Let loads already issued land before the CTA exits.
        if (PAIR && !leader) {
          if (armed) drain_delay();
        } else {
          for (int st = 0; st < STG; ++st)
            if (armed & (1u << st)) tc::mbar_wait(&sm.full[st], (armed_phase >> st) & 1u, abort, WAIT_LIMIT);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (the leader of a pair) ----------------
      constexpr uint32_t idesc = tc::instr_desc(MODE == MODE_FP8 ? 0u : 1u, ROWS, TBN);
      constexpr uint16_t both = 3;
      uint32_t stage = 0, phase = 0, tcount = 0;
      bool ok = true;
      ItemRing rg;
      for (int item = next_item<PAIR>(sm, A, false, leader, -1, unit, units, rg, abort, ok); item < items && ok;
           item = next_item<PAIR>(sm, A, false, leader, item, unit, units, rg, abort, ok)) {
        TcItem it;
        get_item<BATCH>(A, pA0, pA1, pB0, pB1, bmaps, row_blocks, nrows, item, it, chunks);
        const int kb_total = it.kblocks * SEGS;
        for (int ct = it.t0; ct < it.t1 && ok; ++ct) {
          const uint32_t ab = tcount & 1u, tph = (tcount >> 1) & 1u;
          if (!tc::mbar_wait(&sm.tempty[ab], tph ^ 1u, abort, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t d = tmem + ab * TBN;
          for (int kt = 0; kt < kb_total; ++kt) {
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
              const uint32_t acc = (kt | kk) != 0;
              if (PAIR) {
                if (MODE == MODE_FP8) tc::mma_fp8_pair(d, da + 2u * kk, db + 2u * kk, idesc, acc);
                else tc::mma_bf16_pair(d, da + 2u * kk, db + 2u * kk, idesc, acc);
              } else {
                if (MODE == MODE_FP8) tc::mma_fp8(d, da + 2u * kk, db + 2u * kk, idesc, acc);
                else tc::mma_bf16(d, da + 2u * kk, db + 2u * kk, idesc, acc);
              }
            }
            if (PAIR) tc::mma_commit_pair(&sm.empty[stage], both);
            else tc::mma_commit(&sm.empty[stage]);
            if (++stage == STG) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          if (PAIR) tc::mma_commit_pair(&sm.tfull[ab], both);
          else tc::mma_commit(&sm.tfull[ab]);
          ++tcount;
        }
      }
      if (!ok) {
        *abort = 1;
        report_timeout<BATCH>(A);
      }
      // Every MMA issued by this thread has completed once `done` fires.
      if (PAIR) tc::mma_commit_pair(&sm.done, 1);
      else tc::mma_commit(&sm.done);
      tc::mbar_wait(&sm.done, 0, abort, WAIT_LIMIT);
    }
  } else {
    // ---------------- epilogue: warps 2 .. 2 + 4 EGROUPS ----------------
    // Warp w may read TMEM lanes 32 (w % 4) .. + 31 (its rows); the groups split
    // the tile's columns, and each keeps its own list per row (EGROUPS lists per chunk).
    const int q = warp & 3;
    const int eg = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const uint32_t tlane = tmem + (uint32_t(q * 32) << 16);
    const uint32_t tempty_leader0 = PAIR ? tc::map_to_rank(&sm.tempty[0], 0) : 0u;
    const uint32_t tempty_leader1 = PAIR ? tc::map_to_rank(&sm.tempty[1], 0) : 0u;
    uint32_t tcount = 0;
    bool ok = true;
    // This row's best KL columns of the current chunk: scores ls (descending)
    // and columns li, in registers.  Columns arrive in increasing order, so a
    // new column beats a slot only with a strictly larger score: an equal
    // score keeps the earlier, lower column in front (score desc, column asc).
    float ls[KL];
    int li[KL];
    // Paired kernels queue a row's admitted columns in shared memory and fold
    // them into the list only when some row's queue would overflow or the
    // item ends: a warp pays, per drain, the largest count among its 32 rows,
    // and that maximum is far smaller over many batches than summed batch by
    // batch (a warm row admits ~0.3 columns per batch).  Columns still enter
    // a list in increasing order.
    int qn = 0;
    auto drain_queue = [&]() {
      int rq = qn;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rq = max(rq, __shfl_xor_sync(kFull, rq, o));
#pragma unroll 1
      for (int rd = 0; rd < rq; ++rd) {
        float cs = -INFINITY;
        int ci = kInvalidIdx;
        if (rd < qn) {
          cs = sm.qsc[QUEUE ? eg : 0][rd][r];
          ci = sm.qcol[QUEUE ? eg : 0][rd][r];
        }
        list_insert<KL>(ls, li, cs, ci);
      }
      qn = 0;
    };
    ItemRing rg;
    // one lane of the warp takes the item from the ring, the warp shares it
    auto take = [&](int prev) {
      int v = 0;
      bool good = true;
      if (lane == 0) v = next_item<PAIR>(sm, A, false, leader, prev, unit, units, rg, abort, good);
      v = __shfl_sync(kFull, v, 0);
      good = __shfl_sync(kFull, good ? 1 : 0, 0) != 0;
      if (!good) ok = false;
      return v;
    };
    for (int item = take(-1); item < items && ok; item = take(item)) {
      TcItem it;
      get_item<BATCH>(A, pA0, pA1, pB0, pB1, bmaps, row_blocks, nrows, item, it, chunks);
      const int chunk = it.chunk;
      const int64_t arow = int64_t(it.rb) * ROWS + int(rank) * TBM + r;   // row of the A operand
      const bool live = arow < it.nrows;
      const int64_t grow = gathered(MODE) ? (live ? int64_t(A.rows[arow]) : -1) : it.row0 + arow;  // vertex
#pragma unroll
      for (int j = 0; j < KL; ++j) {
        ls[j] = -FLT_MAX;
        li[j] = kInvalidIdx;
      }
      qn = 0;
      // Admission: beat the last slot and reach the row's floor (s >= floor,
      // i.e. s > the float below it).  The floor is the best K-th score any
      // chunk of this row has published: chunks publish their running K-th
      // after every tile, and an item re-reads the floor before every tile,
      // so chunks of a row that run at the same time raise each other's bar.
      // A partial list's K-th best is at most the row's final K-th best, so a
      // column below the floor can never be among the row's K best.
      int seen = live ? __ldcg(it.row_floor + arow) : INT_MAX;  // floor key in use (also: last published)
      float floor_below = live ? nextafterf(key_score(seen), -INFINITY) : INFINITY;
      const float rinv = (MODE == MODE_FP8 && live) ? it.inv_scale[grow] : 1.0f;
      for (int ct = it.t0; ct < it.t1; ++ct) {
        const int fk = (live && ct > it.t0) ? __ldcg(it.row_floor + arow) : seen;
        const uint32_t ab = tcount & 1u, tph = (tcount >> 1) & 1u;
        if (!tc::mbar_wait(&sm.tfull[ab], tph, abort, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        if (fk > seen) {
          seen = fk;
          floor_below = nextafterf(key_score(fk), -INFINITY);
        }
#pragma unroll 1
        for (int cb = eg * (TBN / 32 / EGROUPS); cb < (eg + 1) * (TBN / 32 / EGROUPS); ++cb) {
          uint32_t v[32];
          tc::tmem_ld32(tlane + ab * TBN + cb * 32, v);
          tc::tmem_wait_ld();
          // Admission test of the 32 columns, then a warp-convergent drain:
          // every round each lane inserts at most one admitted column with a
          // branch-free pass over its list, so the warp pays per round.
          const int64_t lbase = int64_t(ct) * TBN + cb * 32;  // B column
          const int64_t cbase = it.col0 + lbase;               // its vertex
          const int nvalid = int(tmin<int64_t>(it.n - lbase, 32));
          const int64_t dself = grow - cbase;
          const int jself = (dself >= 0 && dself < 32) ? int(dself) : -1;
          const float thr = fmaxf(ls[KL - 1], floor_below);
          uint32_t mask = 0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float sc = __uint_as_float(v[j]);
            if (MODE == MODE_FP8) sc = sc * rinv * __ldg(it.inv_scale + (j < nvalid ? cbase + j : 0));
            if (j == jself) sc = 1.0f;
            if (j >= nvalid) sc = -INFINITY;
            sm.batch[eg][j][r] = sc;
            mask |= (sc > thr) ? (1u << j) : 0u;
          }
          int rounds = __popc(mask);
          if constexpr (QUEUE) {
            if (__any_sync(kFull, qn + rounds > QCAP)) {
              // No room: empty the queues, then fold this batch in directly,
              // tested again against the raised lists.
              drain_queue();
              const float thr2 = fmaxf(ls[KL - 1], floor_below);
              uint32_t keep = 0;
              for (uint32_t mm = mask; mm; mm &= mm - 1u) {
                const int j = __ffs(mm) - 1;
                if (sm.batch[eg][j][r] > thr2) keep |= 1u << j;
              }
              mask = keep;
              rounds = __popc(mask);
            } else {
              while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1u;
                sm.qsc[QUEUE ? eg : 0][qn][r] = sm.batch[eg][j][r];
                sm.qcol[QUEUE ? eg : 0][qn][r] = int(cbase + j);
                ++qn;
              }
              rounds = 0;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(kFull, rounds, o));
#pragma unroll 1
          for (int rd = 0; rd < rounds; ++rd) {
            float cs = -INFINITY;
            int ci = kInvalidIdx;
            if (mask) {
              const int j = __ffs(mask) - 1;
              mask &= mask - 1u;
              cs = sm.batch[eg][j][r];
              ci = int(cbase + j);
            }
            list_insert<KL>(ls, li, cs, ci);
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (PAIR && !leader) tc::mbar_arrive_cluster(ab ? tempty_leader1 : tempty_leader0);
          else tc::mbar_arrive(&sm.tempty[ab]);
        }
        ++tcount;
        // Publish this chunk's running K-th best when it raises the row's floor.
        if (live && ct + 1 < it.t1) {
          float kth = FLT_MAX;
#pragma unroll
          for (int j = 0; j < KL; ++j)
            if (j < it.K) kth = fminf(kth, ls[j]);
          if (kth != -FLT_MAX) {
            const int key = score_key(kth);
            if (key > seen) {
              atomicMax(it.row_floor + arow, key);
              seen = key;
              floor_below = nextafterf(kth, -INFINITY);
            }
          }
        }
      }
      if (!ok) break;
      if (QUEUE) drain_queue();
      if (live) {
        const size_t o = ((size_t(arow) * it.chunks + chunk) * EGROUPS + eg) * it.K;
        // The K-th best as a running minimum over the first K slots (the list
        // is never indexed dynamically, so it stays in registers).
        float kth = FLT_MAX;
#pragma unroll
        for (int j = 0; j < KL; ++j) {
          if (j < it.K) {
            it.part_s[o + j] = ls[j];
            it.part_i[o + j] = li[j];
            kth = fminf(kth, ls[j]);
          }
        }
        // This chunk's K-th best becomes a floor for the row's later chunks.
        if (kth != -FLT_MAX) atomicMax(it.row_floor + arow, score_key(kth));
        // Lists of chunks this launch does not use are empty (first entry invalid).
        if (gathered(MODE) && chunk == 0)
          for (int c = chunks; c < it.chunks; ++c) {
            const size_t oe = ((size_t(arow) * it.chunks + c) * EGROUPS + eg) * it.K;
            it.part_s[oe] = -FLT_MAX;
            it.part_i[oe] = kInvalidIdx;
          }
      }
    }
    if (!ok) {
      *abort = 1;
      report_timeout<BATCH>(A);
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  if (PAIR) tc::cluster_sync();  // neither CTA leaves while the pair's MMAs or signals may touch it
  tc::tc_fence_after();
  if (warp == 1) {
    if (PAIR) tc::tmem_dealloc_pair(tmem, 512);
    else tc::tmem_dealloc(tmem, 512);
  }
}

template <int MODE, int KL, int EGROUPS>
__global__ void __launch_bounds__(threads_of(EGROUPS), 1)
k1_tc_topk(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
           const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, TcArgs A) {
  tc_body<MODE, KL, EGROUPS, false, false>(&mA0, &mA1, &mB0, &mB1, nullptr, A);
}

// CTA pairs (launched in clusters of two): 256-row items, one cta_group::2
// MMA per k-step for both SMs.
template <int MODE, int KL, int EGROUPS>
__global__ void __launch_bounds__(threads_of(EGROUPS), 1)
k1_tc2_topk(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
            const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, TcArgs A) {
  tc_body<MODE, KL, EGROUPS, false, true>(&mA0, &mA1, &mB0, &mB1, nullptr, A);
}

// Many instances in one persistent launch: the items of all instances form one
// list that the CTAs walk; each item carries its instance's parameters.
template <int MODE, int KL, int EGROUPS>
__global__ void __launch_bounds__(threads_of(EGROUPS), 1)
k1_tc_topk_batch(const __grid_constant__ TcMaps maps, TcArgs A) {
  tc_body<MODE, KL, EGROUPS, true, false>(nullptr, nullptr, nullptr, nullptr, maps.m, A);
}

// Test hook: RERANK_TEST_TC_STALL set in the environment makes the kernels'
// TMA warp issue nothing, so the MMA and epilogue waits run out and the call
// returns ETIMEOUT (no copy or MMA is ever in flight on that path).
int stall_hook() { return std::getenv("RERANK_TEST_TC_STALL") ? 1 : 0; }

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

// Row-major rows x dp matrix, boxes of 128 rows x 128 bytes, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int dp, bool fp8) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  const cuuint64_t dims[2] = {cuuint64_t(dp), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(dp) * (fp8 ? 1 : 2)};
  const cuuint32_t box[2] = {fp8 ? 128u : 64u, 128u};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int KL, int EG>
void launch_kl(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0, const CUtensorMap& b1,
               const TcArgs& A, int grid, cudaStream_t s) {
  const size_t smem = sizeof(TcSmem) + 1024;
  cudaFuncSetAttribute(k1_tc_topk<MODE, KL, EG>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  k1_tc_topk<MODE, KL, EG><<<grid, threads_of(EG), smem, s>>>(a0, a1, b0, b1, A);
}

// Pairs that can be resident at once (clusters of two, one CTA per SM); 0 if
// the query fails.
template <int MODE, int KL, int EG>
int pair_units(int sm_count) {
  static int cached = -1;
  if (cached < 0) {
    const size_t smem = sizeof(TcSmemPair<EG>) + 1024;
    cudaFuncSetAttribute(k1_tc2_topk<MODE, KL, EG>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(unsigned(sm_count & ~1));
    cfg.blockDim = dim3(threads_of(EG));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k1_tc2_topk<MODE, KL, EG>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    cached = n;
  }
  return cached;
}

template <int MODE, int KL, int EG>
bool launch_kl_pair(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0, const CUtensorMap& b1,
                    const TcArgs& A, int items, int sm_count, cudaStream_t s) {
  const int units = pair_units<MODE, KL, EG>(sm_count);
  if (units < 1) return false;
  const size_t smem = sizeof(TcSmemPair<EG>) + 1024;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(2 * (items < units ? items : units)));
  cfg.blockDim = dim3(threads_of(EG));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k1_tc2_topk<MODE, KL, EG>, a0, a1, b0, b1, A) == cudaSuccess;
}

// items: work items of the launch, or INT_MAX when only the device knows
// them (gathered rows): then every resident pair is launched.
template <int MODE>
bool launch_mode_pair(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0, const CUtensorMap& b1,
                      const TcArgs& A, int eg, int items, int sm_count, cudaStream_t s) {
  if (A.K <= 48)
    return eg == 2 ? launch_kl_pair<MODE, 48, 2>(a0, a1, b0, b1, A, items, sm_count, s)
                   : launch_kl_pair<MODE, 48, 1>(a0, a1, b0, b1, A, items, sm_count, s);
  return eg == 2 ? launch_kl_pair<MODE, KLIST, 2>(a0, a1, b0, b1, A, items, sm_count, s)
                 : launch_kl_pair<MODE, KLIST, 1>(a0, a1, b0, b1, A, items, sm_count, s);
}

// The per-row list lives in registers, so its length is a compile-time choice.
template <int MODE>
void launch_mode(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0, const CUtensorMap& b1,
                 const TcArgs& A, int eg, int grid, cudaStream_t s) {
  if (A.K <= 48) {
    if (eg == 2)
      launch_kl<MODE, 48, 2>(a0, a1, b0, b1, A, grid, s);
    else
      launch_kl<MODE, 48, 1>(a0, a1, b0, b1, A, grid, s);
  } else {
    if (eg == 2)
      launch_kl<MODE, KLIST, 2>(a0, a1, b0, b1, A, grid, s);
    else
      launch_kl<MODE, KLIST, 1>(a0, a1, b0, b1, A, grid, s);
  }
}

__global__ void k_gather_rows(const int32_t* __restrict__ rows, const int32_t* __restrict__ count,
                              const uint4* __restrict__ hi, const uint4* __restrict__ lo, uint4* __restrict__ dhi,
                              uint4* __restrict__ dlo, int64_t n, int vecs) {
  const int64_t f = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= n || f >= *count) return;
  const int64_t src = rows[f];
  for (int k = lane; k < vecs; k += kWarp) {
    dhi[f * vecs + k] = hi[src * vecs + k];
    dlo[f * vecs + k] = lo[src * vecs + k];
  }
}

}  // namespace

size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }
static_assert(sizeof(TcSmemPair<1>) + 1024 <= 227 * 1024, "shared memory of the paired tensor-core kernel");
static_assert(sizeof(TcSmemPair<2>) + 1024 <= 227 * 1024, "shared memory of the paired tensor-core kernel");
// Whether the main similarity pass runs on CTA pairs (cta_group::2).  Both
// kernels give identical lists; RERANK_TC_PAIRS=0 selects the single-CTA one.
bool tc_pairs() {
  static const int on = [] {
    const char* e = std::getenv("RERANK_TC_PAIRS");
    return (e && e[0] == '0') ? 0 : 1;
  }();
  return on != 0;
}
int tc_item_rows() { return tc_pairs() ? 2 * TBM : TBM; }
// Whether the main pass takes its items dynamically (see next_item);
// RERANK_TC_DYNAMIC=0 selects the static order (identical lists).
bool tc_dynamic() {
  static const int on = [] {
    const char* e = std::getenv("RERANK_TC_DYNAMIC");
    return (e && e[0] == '0') ? 0 : 1;
  }();
  return on != 0;
}
int tc_lists_per_chunk(int dp, int segs) { return dp * segs <= 1024 ? 2 : 1; }
static_assert(sizeof(TcSmem) + 1024 <= 227 * 1024, "shared memory of the tensor-core kernel");
int tc_kmax() { return KLIST; }
int tc_tile_rows() { return TBM; }
int tc_tile_cols() { return TBN; }

// Returns the number of kernels launched (1), or a negative value when the
// tensor map cannot be encoded.
int launch_sim_tc_topk(const Shape& sh, const void* xlow, bool fp8, const float* inv_scale, int* row_floor,
                       float* part_s, int32_t* part_i, long long* status, int sm_count, cudaStream_t s,
                       int32_t* work) {
  CUtensorMap map;
  if (!make_map(&map, xlow, sh.np, sh.dp, fp8)) return -1;
  cudaMemsetAsync(row_floor, kFloorResetByte, sizeof(int) * size_t(sh.n), s);
  const bool pairs = tc_pairs() && sm_count >= 2 && sh.np % (2 * TBM) == 0;
  TcArgs A{};
  A.n = sh.n;
  A.a_rows = sh.n;
  A.row_blocks = int(sh.np / (pairs ? 2 * TBM : TBM));
  A.col_tiles = int(sh.np / TBN);
  const int eg = tc_lists_per_chunk(sh.dp, 1);
  A.chunks = sh.P / eg;  // sh.P counts lists per row
  if (A.chunks < 1 || A.chunks * eg != sh.P || A.chunks > A.col_tiles) return -1;
  A.kblocks = fp8 ? sh.dp / 128 : sh.dp / 64;
  A.K = sh.K;
  A.inv_scale = inv_scale;
  A.row_floor = row_floor;
  A.part_s = part_s;
  A.part_i = part_i;
  A.status = status;
  A.stall = stall_hook();
  if (work && tc_dynamic()) {
    cudaMemsetAsync(work, 0, sizeof(int32_t), s);
    A.work = work;
  }
  const int items = A.row_blocks * A.chunks;
  if (pairs) {
    const bool ok = fp8 ? launch_mode_pair<MODE_FP8>(map, map, map, map, A, eg, items, sm_count, s)
                        : launch_mode_pair<MODE_BF16>(map, map, map, map, A, eg, items, sm_count, s);
    return ok ? 1 : -1;
  }
  const int grid = items < sm_count ? items : sm_count;
  if (fp8)
    launch_mode<MODE_FP8>(map, map, map, map, A, eg, grid, s);
  else
    launch_mode<MODE_BF16>(map, map, map, map, A, eg, grid, s);
  return 1;
}

int launch_sim_tc_rect_topk(const Shape& sh, const void* a, int64_t a_rows, int64_t row0, const void* b,
                            int64_t b_cols, int64_t col0, int chunks, bool fp8, const float* inv_scale,
                            int* row_floor, float* part_s, int32_t* part_i, long long* status, int sm_count,
                            cudaStream_t s) {
  // The maps span at least one full tile (the caller's buffers hold that many rows).
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, a_rows > TBN ? a_rows : TBN, sh.dp, fp8) ||
      !make_map(&mb, b, b_cols > TBN ? b_cols : TBN, sh.dp, fp8))
    return -1;
  cudaMemsetAsync(row_floor, kFloorResetByte, sizeof(int) * size_t(a_rows), s);
  TcArgs A{};
  A.n = b_cols;
  A.a_rows = a_rows;
  A.row0 = row0;
  A.col0 = col0;
  A.row_blocks = int((a_rows + TBM - 1) / TBM);
  A.col_tiles = int((b_cols + TBN - 1) / TBN);
  if (chunks < 1 || chunks > A.col_tiles) return -1;  // the caller reads chunks * tc_lists_per_chunk lists per row
  A.chunks = chunks;
  const int eg = tc_lists_per_chunk(sh.dp, 1);
  A.kblocks = fp8 ? sh.dp / 128 : sh.dp / 64;
  A.K = sh.K;
  A.inv_scale = inv_scale;
  A.row_floor = row_floor;
  A.part_s = part_s;
  A.part_i = part_i;
  A.status = status;
  A.stall = stall_hook();
  const int items = A.row_blocks * A.chunks;
  const int grid = items < sm_count ? items : sm_count;
  if (fp8)
    launch_mode<MODE_FP8>(ma, ma, mb, mb, A, eg, grid, s);
  else
    launch_mode<MODE_BF16>(ma, ma, mb, mb, A, eg, grid, s);
  return 1;
}

int launch_sim_tc_split_topk(const Shape& sh, int P3, const __nv_bfloat16* ahi, const __nv_bfloat16* alo,
                             const __nv_bfloat16* bhi, const __nv_bfloat16* blo, const int32_t* rows,
                             const int32_t* count, int* row_floor, float* part_s, int32_t* part_i,
                             long long* status, int sm_count, cudaStream_t s) {
  CUtensorMap a0, a1, b0, b1;
  if (!make_map(&a0, ahi, sh.np, sh.dp, false) || !make_map(&a1, alo, sh.np, sh.dp, false) ||
      !make_map(&b0, bhi, sh.np, sh.dp, false) || !make_map(&b1, blo, sh.np, sh.dp, false))
    return -1;
  cudaMemsetAsync(row_floor, kFloorResetByte, sizeof(int) * size_t(sh.n), s);
  TcArgs A{};
  A.n = sh.n;
  A.row_blocks = 0;
  A.col_tiles = int(sh.np / TBN);
  const int eg = tc_lists_per_chunk(sh.dp, 3);
  A.chunks = P3 / eg;  // P3 counts lists per row
  if (A.chunks < 1 || A.chunks * eg != P3 || A.chunks > A.col_tiles) return -1;
  A.kblocks = sh.dp / 64;
  A.K = sh.K;
  A.rows = rows;
  A.count = count;
  A.row_floor = row_floor;
  A.part_s = part_s;
  A.part_i = part_i;
  A.status = status;
  A.stall = stall_hook();
  // CTA pairs when the rows come in whole 256-row blocks of the padded buffers.
  if (tc_pairs() && sm_count >= 2 && sh.np % (2 * TBM) == 0)
    return launch_mode_pair<MODE_SPLIT>(a0, a1, b0, b1, A, eg, INT_MAX, sm_count, s) ? 1 : -1;
  launch_mode<MODE_SPLIT>(a0, a1, b0, b1, A, eg, sm_count, s);
  return 1;
}

size_t tc_batch_inst_bytes() { return sizeof(TcInst); }
int tc_batch_max_inst() { return kMaxBatchInst; }
int tc_stall_hook() { return stall_hook(); }

int launch_sim_tc_batch(const TcBatchInst* in, int ninst, bool fp8, void* insts_dev, void* staging, int sm_count,
                        cudaStream_t s) {
  if (ninst < 1 || ninst > kMaxBatchInst) return -1;
  const int eg = tc_lists_per_chunk(in[0].dp, 1);
  TcMaps maps;
  TcInst* hi = static_cast<TcInst*>(staging);
  int items = 0, kmax = 0;
  for (int k = 0; k < ninst; ++k) {
    const TcBatchInst& b = in[k];
    if (tc_lists_per_chunk(b.dp, 1) != eg) return -1;
    if (!make_map(&maps.m[k], b.xlow, b.np, b.dp, fp8)) return -1;
    TcInst& t = hi[k];
    t.n = b.n;
    t.row_blocks = int(b.np / TBM);
    t.col_tiles = int(b.np / TBN);
    t.chunks = b.P / eg;
    if (t.chunks < 1 || t.chunks * eg != b.P || t.chunks > t.col_tiles) return -1;
    t.kblocks = fp8 ? b.dp / 128 : b.dp / 64;
    t.K = b.K;
    t.item_begin = items;
    t.inv_scale = b.inv_scale;
    t.row_floor = b.row_floor;
    t.part_s = b.part_s;
    t.part_i = b.part_i;
    t.status = b.status;
    items += t.row_blocks * t.chunks;
    kmax = b.K > kmax ? b.K : kmax;
    cudaMemsetAsync(b.row_floor, kFloorResetByte, sizeof(int) * size_t(b.n), s);
  }
  cudaMemcpyAsync(insts_dev, staging, sizeof(TcInst) * size_t(ninst), cudaMemcpyHostToDevice, s);
  TcArgs A{};
  A.insts = static_cast<const TcInst*>(insts_dev);
  A.ninst = ninst;
  A.items_total = items;
  A.status = in[0].status;
  A.stall = stall_hook();
  const int grid = items < sm_count ? items : sm_count;
  const size_t smem = sizeof(TcSmem) + 1024;
  auto go = [&](auto kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    kernel<<<grid, threads_of(eg), smem, s>>>(maps, A);
  };
  const bool k48 = kmax <= 48;
  if (fp8) {
    if (eg == 2) k48 ? go(k1_tc_topk_batch<MODE_FP8, 48, 2>) : go(k1_tc_topk_batch<MODE_FP8, KLIST, 2>);
    else k48 ? go(k1_tc_topk_batch<MODE_FP8, 48, 1>) : go(k1_tc_topk_batch<MODE_FP8, KLIST, 1>);
  } else {
    if (eg == 2) k48 ? go(k1_tc_topk_batch<MODE_BF16, 48, 2>) : go(k1_tc_topk_batch<MODE_BF16, KLIST, 2>);
    else k48 ? go(k1_tc_topk_batch<MODE_BF16, 48, 1>) : go(k1_tc_topk_batch<MODE_BF16, KLIST, 1>);
  }
  return 1;
}

int launch_sim_tc_gather_topk(const Shape& sh, int P, const __nv_bfloat16* ahi, const __nv_bfloat16* bhi,
                              const int32_t* rows, const int32_t* count, int* row_floor, float* part_s,
                              int32_t* part_i, long long* status, int sm_count, cudaStream_t s) {
  CUtensorMap a0, b0;
  if (!make_map(&a0, ahi, sh.np, sh.dp, false) || !make_map(&b0, bhi, sh.np, sh.dp, false)) return -1;
  cudaMemsetAsync(row_floor, kFloorResetByte, sizeof(int) * size_t(sh.n), s);
  TcArgs A{};
  A.n = sh.n;
  A.row_blocks = 0;
  A.col_tiles = int(sh.np / TBN);
  const int eg = tc_lists_per_chunk(sh.dp, 1);
  A.chunks = P / eg;  // P counts lists per row
  if (A.chunks < 1 || A.chunks * eg != P || A.chunks > A.col_tiles) return -1;
  A.kblocks = sh.dp / 64;
  A.K = sh.K;
  A.rows = rows;
  A.count = count;
  A.row_floor = row_floor;
  A.part_s = part_s;
  A.part_i = part_i;
  A.status = status;
  A.stall = stall_hook();
  if (tc_pairs() && sm_count >= 2 && sh.np % (2 * TBM) == 0)
    return launch_mode_pair<MODE_GATHER>(a0, a0, b0, b0, A, eg, INT_MAX, sm_count, s) ? 1 : -1;
  launch_mode<MODE_GATHER>(a0, a0, b0, b0, A, eg, sm_count, s);
  return 1;
}

int launch_gather_rows(const int32_t* rows, const int32_t* count, const __nv_bfloat16* hi, const __nv_bfloat16* lo,
                       __nv_bfloat16* dst_hi, __nv_bfloat16* dst_lo, int64_t n, int dp, cudaStream_t s) {
  const int T = 256;
  k_gather_rows<<<unsigned((n * kWarp + T - 1) / T), T, 0, s>>>(
      rows, count, reinterpret_cast<const uint4*>(hi), reinterpret_cast<const uint4*>(lo),
      reinterpret_cast<uint4*>(dst_hi), reinterpret_cast<uint4*>(dst_lo), n, dp / 8);
  return 1;
}

}  // namespace rr

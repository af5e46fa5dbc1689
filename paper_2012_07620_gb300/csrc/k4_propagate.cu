// K4: one message-passing layer (Eq. 13-14, sum, mean or max aggregator)
// followed by L2 normalisation (Sec. 3.3), on sparse vertex features.
//
//   h_i <- normalise( sum_{(j, c_j) in M(i)} c_j h_j )
//
// where M(i) is the message list built by K3 (N(i, k2) with c_j = e_ij^alpha,
// the residual h_i folded into c_i).  Max aggregator: entries with c_j >= 0
// are combined by element-wise max (every value is >= 0, so a missing column
// counts as 0), and the last entry, c_i = -1, adds the residual h_i on top;
// max is exact, so the result does not depend on the order either.  Features
// are stored as padded CSR: row
// i occupies [start_i, start_i + len_i) of (col, val), each column at most
// once, in no particular order (h^(0) from K3 is ascending).  start_i is an
// exclusive scan of ub_i = sum_j len_j, an upper bound on the output row, so
// every row can be written without a second pass.
//
// Rows whose distinct columns fit three quarters of a 512-slot table (almost
// all): one warp per row with a private open-addressing hash table in shared
// memory (columns as keys), 4 KB per warp so up to 48 warps share an SM.  The warp
// walks the message list in order and adds c_j * val into the table, one
// list at a time, so every output value is summed in message-list order and
// the result does not depend on scheduling.  The occupied slots are
// compacted in table order, scaled by 1/||row|| and written: a column's
// position in the row never matters (a later layer folds each column's terms
// in message order wherever they sit, and the norm is summed exactly as
// 128-bit fixed point, so it does not depend on the order either).
// Rows that overflow that table (or whose bound exceeds 2,048) are listed and
// taken by one more launch (k4_spmm_rest, one CTA of 12 warps per SM): when
// there are many, each warp retries them with a 2,048-slot table (16 KB), the
// same code; the rows that overflow that too, or all of them when there are
// few, go to one CTA per row with a dense accumulator and a bitmap of touched
// columns in global memory, whose scan emits the columns in order.
#include <cstdlib>

#include "common.cuh"
#include "internal.hpp"

namespace rr {
namespace {

constexpr int WSLOTS = 512;   // hash slots per warp (4 KB: up to 48 warps per SM)
constexpr int WDIRECT = 4 * WSLOTS;  // ub above this skips the first pass
constexpr int MSLOTS = 2048;  // hash slots per warp of the second pass (16 KB)
constexpr int RWARPS = 12;    // warps of k4_spmm_rest (192 KB of tables, one CTA per SM)
constexpr int RTHREADS = RWARPS * 32;
constexpr int KEY_EMPTY = -1;

__global__ void k4_ub(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nbr_n, int k2p1,
                      const int32_t* __restrict__ len, int64_t n, int32_t* __restrict__ ub,
                      int32_t* __restrict__ big_rows, int32_t* __restrict__ big_count,
                      const long long* __restrict__ status, LayerReuse reuse) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (status[kStErr] & kErrOverflow) {
    ub[i] = 0;
    return;
  }
  int64_t u = 0;
  const int m = nbr_n[i];
  for (int q = 0; q < m; ++q) u += len[nbr[i * k2p1 + q]];
  if (u > n) u = n;
  const bool copied = reuse.changed && !reuse.changed[i];
  if (copied) u = max(u, int64_t(reuse.rlen[i - reuse.shift]));  // room for the copied row
  ub[i] = int32_t(u);
  if (u > WDIRECT && !copied) big_rows[atomicAdd(big_count, 1)] = int32_t(i);
}

__device__ __forceinline__ bool capacity_ok(const int64_t* dstart, int64_t n, int64_t cap, long long* status) {
  if (status[kStErr] & kErrOverflow) return false;
  const int64_t need = dstart[n];
  if (need > cap) {
    if (threadIdx.x == 0) {
      set_error(status, kErrOverflow);
      atomicMax(reinterpret_cast<unsigned long long*>(status + kStNeed), (unsigned long long)need);
    }
    return false;
  }
  return true;
}

// Adds v to the entry of `col` (or, with take_max, raises it to v; entries
// start at 0 and every value is >= 0); returns true when this call created it.
__device__ __forceinline__ bool hash_add(volatile int* keys, float* vals, int mask, int shift, int col, float v,
                                         long long* status, bool take_max = false) {
  const unsigned h = (unsigned(col) * 2654435761u) >> shift;
  for (int probe = 0; probe <= mask; ++probe) {
    const int slot = int((h + unsigned(probe)) & unsigned(mask));
    const int k = keys[slot];
    if (k == col) {
      vals[slot] = take_max ? fmaxf(vals[slot], v) : vals[slot] + v;
      return false;
    }
    if (k == KEY_EMPTY) {
      const int old = atomicCAS(const_cast<int*>(keys) + slot, KEY_EMPTY, col);
      if (old == KEY_EMPTY || old == col) {
        vals[slot] = take_max ? fmaxf(vals[slot], v) : vals[slot] + v;
        return old == KEY_EMPTY;
      }
    }
  }
  set_error(status, kErrInternal);
  return false;
}

// v^2 as a 128-bit fixed-point number, truncated to a multiple of 2^-64:
// (hi, lo) = (floor(v^2), floor(frac(v^2) 2^64)).  For |v| < 1 (every value of
// a normalised layer) it is m^2 2^(2e + 18) for v = m 2^(e - 23), in 64-bit
// integer arithmetic; otherwise from the exact square in double.  Both give the
// same bits.
__device__ __forceinline__ void sq_fixed(float v, unsigned long long& hi, unsigned long long& lo) {
  const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
  const int ef = int(b >> 23);
  if (ef >= 127) {
    const double d = double(v) * double(v);
    const double ip = floor(d);
    hi = static_cast<unsigned long long>(ip);
    lo = static_cast<unsigned long long>((d - ip) * 18446744073709551616.0);  // x 2^64
    return;
  }
  const unsigned long long m = ef ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu);
  const int s = 2 * (ef ? ef - 127 : -126) + 18;
  const unsigned long long m2 = m * m;
  hi = 0;
  lo = s >= 0 ? (m2 << s) : (s > -64 ? (m2 >> -s) : 0ull);
}

// Sum of squares of v[0 .. cnt) by one warp, independent of the order of the
// values: each square is exact, is truncated to a multiple of 2^-64, and the
// truncated squares are added as 128-bit integers.
__device__ float warp_sumsq_exact(const float* v, int cnt, int lane) {
  unsigned long long hi = 0, lo = 0;
  for (int p = lane; p < cnt; p += kWarp) {
    unsigned long long h, l;
    sq_fixed(v[p], h, l);
    lo += l;
    hi += h + (lo < l ? 1ull : 0ull);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oh = __shfl_xor_sync(kFull, hi, o), ol = __shfl_xor_sync(kFull, lo, o);
    const unsigned long long nl = lo + ol;
    hi = hi + oh + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  return float(double(hi) + double(lo) * 5.421010862427522e-20);  // 2^-64
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

constexpr int kMaxPropWarps = 24;  // 24 warps x 4 KB of tables: 96 KB per CTA

// Row i through one warp's SLOTS-entry table (keys / vals: empty on entry and
// on return).  Returns false when the row was written (lane 0 adds its length
// to nnz), true when its distinct columns filled three quarters of the table:
// then nothing is written and the caller hands the row on.
template <int SLOTS>
__device__ bool warp_row(int64_t i, int u, volatile int* keys, float* vals, const int64_t* __restrict__ sstart,
                         const int32_t* __restrict__ slen, const int32_t* __restrict__ scol,
                         const float* __restrict__ sval, const int32_t* __restrict__ nbr,
                         const float* __restrict__ nbr_w, const int32_t* __restrict__ nbr_n, int k2p1,
                         const int64_t* __restrict__ dstart, int32_t* __restrict__ dlen, int32_t* __restrict__ dcol,
                         float* __restrict__ dval, long long* __restrict__ status, bool agg_max, int lane,
                         unsigned long long& nnz) {
  const unsigned lt = (1u << lane) - 1u;
  // Table of at least twice the bound on distinct columns, at most SLOTS; when
  // the bound is larger the row is tried here and handed on if its distinct
  // columns fill three quarters of the table.
  const int T = min(SLOTS, next_pow2(max(64, 2 * min(u, SLOTS))));
  const int mask = T - 1, shift = 32 - (31 - __clz(T));
  const int limit = (3 * T) / 4;
  const int m = nbr_n[i];
  int distinct = 0;
  bool spilled = false;
  // Lane q < m holds message q's source row (start, length) and weight; the
  // messages are folded in order, 32 entries per step, and the entries of
  // the next step are loaded while this step is added to the table.
  int64_t qa = 0;
  int ql = 0;
  float qc = 0.f;
  if (m > kWarp) {
    // more messages than lanes (k2 >= 32): one message at a time
    for (int q = 0; q < m && !spilled; ++q) {
      const int32_t j = nbr[i * k2p1 + q];
      const float cj = nbr_w[i * k2p1 + q];
      const int64_t a = sstart[j];
      const int lj = slen[j];
      for (int e0 = 0; e0 < lj; e0 += kWarp) {
        const int e = e0 + lane;
        bool fresh = false;
        if (e < lj)
          fresh = hash_add(keys, vals, mask, shift, scol[a + e], fabsf(cj) * sval[a + e], status,
                           agg_max && cj >= 0.f);
        distinct += __popc(__ballot_sync(kFull, fresh));
        __syncwarp();
        if (distinct > limit) {
          spilled = true;
          break;
        }
      }
    }
  }
  const int mq = m > kWarp ? 0 : m;  // messages handled by the pipelined loop
  if (lane < mq) {
    const int32_t j = nbr[i * k2p1 + lane];
    qc = nbr_w[i * k2p1 + lane];
    qa = sstart[j];
    ql = slen[j];
  }
  int q = 0, e0 = 0;
  while (q < mq && __shfl_sync(kFull, ql, q) == 0) ++q;
  int col = -1;
  float val = 0.f;
  if (q < mq) {
    const int64_t a = __shfl_sync(kFull, qa, q);
    const int lj = __shfl_sync(kFull, ql, q);
    if (lane < lj) {
      col = scol[a + lane];
      val = sval[a + lane];
    }
  }
  while (q < mq) {
    // next step: (q, e0 + 32) or the next non-empty message
    int nq = q, ne0 = e0 + kWarp;
    if (ne0 >= __shfl_sync(kFull, ql, q)) {
      ne0 = 0;
      ++nq;
      while (nq < mq && __shfl_sync(kFull, ql, nq) == 0) ++nq;
    }
    int ncol = -1;
    float nval = 0.f;
    if (nq < mq) {
      const int64_t a = __shfl_sync(kFull, qa, nq);
      const int lj = __shfl_sync(kFull, ql, nq);
      if (ne0 + lane < lj) {
        ncol = scol[a + ne0 + lane];
        nval = sval[a + ne0 + lane];
      }
    }
    const float cj = __shfl_sync(kFull, qc, q);
    bool fresh = false;
    if (col >= 0) fresh = hash_add(keys, vals, mask, shift, col, fabsf(cj) * val, status, agg_max && cj >= 0.f);
    distinct += __popc(__ballot_sync(kFull, fresh));
    __syncwarp();  // this step's table writes are visible to the next step
    if (distinct > limit) {
      spilled = true;
      break;
    }
    q = nq;
    e0 = ne0;
    col = ncol;
    val = nval;
  }
  if (spilled) {
    for (int s = lane; s < T; s += kWarp) {
      keys[s] = KEY_EMPTY;
      vals[s] = 0.f;
    }
    __syncwarp();
    return true;
  }
  // Compact occupied slots to the front (order-preserving, in place).
  int cnt = 0;
  for (int s0 = 0; s0 < T; s0 += kWarp) {
    const int k = keys[s0 + lane];
    const float v = vals[s0 + lane];
    const bool occ = k != KEY_EMPTY;
    const unsigned bal = __ballot_sync(kFull, occ);
    const int pos = cnt + __popc(bal & lt);
    __syncwarp();
    if (occ) {
      keys[pos] = k;
      vals[pos] = v;
    }
    cnt += __popc(bal);
    __syncwarp();
  }
  // The row is written in table order: its columns' order never matters
  // downstream (each column occurs once per row, so a later layer folds a
  // column's terms in message order whatever the positions), and the norm
  // below is independent of the order.
  const float ss = warp_sumsq_exact(vals, cnt, lane);
  const float inv = 1.0f / sqrtf(ss);
  const int64_t o = dstart[i];
  for (int p = lane; p < cnt; p += kWarp) {
    dcol[o + p] = keys[p];
    dval[o + p] = vals[p] * inv;
  }
  if (lane == 0) {
    dlen[i] = cnt;
    nnz += unsigned(cnt);
  }
  __syncwarp();
  for (int s = lane; s < T; s += kWarp) {
    keys[s] = KEY_EMPTY;
    vals[s] = 0.f;
  }
  __syncwarp();
  return false;
}

// First pass: warp per row, 512-slot tables; rows that overflow them, or
// whose bound is above WDIRECT, are listed in big_rows for k4_spmm_rest.
__global__ void __launch_bounds__(kMaxPropWarps * kWarp)
k4_spmm_warp(const int64_t* __restrict__ sstart, const int32_t* __restrict__ slen, const int32_t* __restrict__ scol,
             const float* __restrict__ sval, const int32_t* __restrict__ nbr, const float* __restrict__ nbr_w,
             const int32_t* __restrict__ nbr_n, int k2p1, const int32_t* __restrict__ ub,
             const int64_t* __restrict__ dstart, int32_t* __restrict__ dlen, int32_t* __restrict__ dcol,
             float* __restrict__ dval, int64_t n, int64_t cap, int32_t* __restrict__ big_rows,
             int32_t* __restrict__ big_count, int32_t* __restrict__ next_row, long long* __restrict__ status,
             bool agg_max, LayerReuse reuse, unsigned long long* __restrict__ nnz_out) {
  extern __shared__ int smem_i[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* keys = smem_i + wib * WSLOTS * 2;
  float* vals = reinterpret_cast<float*>(smem_i + wib * WSLOTS * 2 + WSLOTS);
  if (!capacity_ok(dstart, n, cap, status)) return;
  for (int s = lane; s < WSLOTS; s += kWarp) {
    keys[s] = KEY_EMPTY;
    vals[s] = 0.f;
  }
  __syncwarp();
  unsigned long long nnz = 0;  // entries this warp wrote (lane 0)
  // Rows are taken one at a time from a counter: their cost varies with the
  // length of their message rows, and a static split left the busiest SM
  // with twice the average work (market, second layer).
  for (;;) {
    int64_t i = 0;
    if (lane == 0) i = atomicAdd(next_row, 1);
    i = __shfl_sync(kFull, i, 0);
    if (i >= n) break;
    if (reuse.changed && !reuse.changed[i]) {
      // inputs unchanged: the known row, in its own column order
      const int64_t g = i - reuse.shift, a = reuse.rstart[g], o = dstart[i];
      const int m = reuse.rlen[g];
      for (int p = lane; p < m; p += kWarp) {
        dcol[o + p] = int32_t(reuse.rcol[a + p] + reuse.shift);
        dval[o + p] = reuse.rval[a + p];
      }
      if (lane == 0) {
        dlen[i] = m;
        nnz += unsigned(m);
      }
      continue;
    }
    const int u = ub[i];
    if (u > WDIRECT) continue;
    if (warp_row<WSLOTS>(i, u, keys, vals, sstart, slen, scol, sval, nbr, nbr_w, nbr_n, k2p1, dstart, dlen, dcol,
                         dval, status, agg_max, lane, nnz) &&
        lane == 0)
      big_rows[atomicAdd(big_count, 1)] = int32_t(i);
  }
  if (nnz_out && lane == 0 && nnz) atomicAdd(nnz_out, nnz);
}

// Row i by the whole CTA (RTHREADS threads): a dense accumulator and a bitmap
// of touched columns in this CTA's part of the global scratch; messages in
// order (one barrier each), the bitmap scan emits the columns in ascending
// order, and the norm is the exact fixed-point sum of warp_row.
__device__ void cta_row(int64_t i, const int64_t* __restrict__ sstart, const int32_t* __restrict__ slen,
                        const int32_t* __restrict__ scol, const float* __restrict__ sval,
                        const int32_t* __restrict__ nbr, const float* __restrict__ nbr_w,
                        const int32_t* __restrict__ nbr_n, int k2p1, const int64_t* __restrict__ dstart,
                        int32_t* __restrict__ dlen, int32_t* __restrict__ dcol, float* __restrict__ dval, int64_t n,
                        float* __restrict__ acc, uint32_t* __restrict__ bm, bool agg_max, int* scan_s,
                        unsigned long long* red_hi, unsigned long long* red_lo, unsigned long long& nnz) {
  const int tid = threadIdx.x;
  const int64_t nwords = (n + 31) / 32;
  const int64_t wpt = (nwords + RTHREADS - 1) / RTHREADS;
  const int64_t w0 = tmin<int64_t>(nwords, tid * wpt), w1 = tmin<int64_t>(nwords, w0 + wpt);
  const int m = nbr_n[i];
  for (int q = 0; q < m; ++q) {
    const int32_t j = nbr[i * k2p1 + q];
    const float cj = nbr_w[i * k2p1 + q];
    const int64_t a = sstart[j];
    const int lj = slen[j];
    for (int e = tid; e < lj; e += RTHREADS) {
      const int c = scol[a + e];
      const float v = fabsf(cj) * sval[a + e];
      acc[c] = (agg_max && cj >= 0.f) ? fmaxf(acc[c], v) : acc[c] + v;
      atomicOr(&bm[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
  }
  int mine = 0;
  for (int64_t w = w0; w < w1; ++w) mine += __popc(bm[w]);
  scan_s[tid] = mine;
  __syncthreads();
  for (int o = 1; o < RTHREADS; o <<= 1) {
    const int v = tid >= o ? scan_s[tid - o] : 0;
    __syncthreads();
    scan_s[tid] += v;
    __syncthreads();
  }
  const int total = scan_s[RTHREADS - 1];
  int pos = scan_s[tid] - mine;
  const int64_t o = dstart[i];
  for (int64_t w = w0; w < w1; ++w) {
    uint32_t b = bm[w];
    while (b) {
      const int bit = __ffs(b) - 1;
      b &= b - 1;
      const int c = int(w * 32 + bit);
      dcol[o + pos] = c;
      dval[o + pos] = acc[c];
      acc[c] = 0.f;
      ++pos;
    }
    bm[w] = 0u;
  }
  __syncthreads();  // the row's values are written
  // The sum of squares as in warp_sumsq_exact (exact squares truncated to
  // 2^-64, added as 128-bit integers), so a row gets the same norm, bit for
  // bit, on every path; the entries are split evenly over the threads.
  unsigned long long shi = 0, slo = 0;
  for (int p = tid; p < total; p += RTHREADS) {
    unsigned long long h, l;
    sq_fixed(dval[o + p], h, l);
    slo += l;
    shi += h + (slo < l ? 1ull : 0ull);
  }
  red_hi[tid] = shi;
  red_lo[tid] = slo;
  __syncthreads();
  for (int st = 256; st > 0; st >>= 1) {  // RTHREADS <= 512
    if (tid < st && tid + st < RTHREADS) {
      const unsigned long long nl = red_lo[tid] + red_lo[tid + st];
      red_hi[tid] = red_hi[tid] + red_hi[tid + st] + (nl < red_lo[tid] ? 1ull : 0ull);
      red_lo[tid] = nl;
    }
    __syncthreads();
  }
  const float ss = float(double(red_hi[0]) + double(red_lo[0]) * 5.421010862427522e-20);  // 2^-64
  const float inv = 1.0f / sqrtf(ss);
  for (int p = tid; p < total; p += RTHREADS) dval[o + p] *= inv;
  if (tid == 0) {
    dlen[i] = total;
    nnz += unsigned(total);
  }
  __syncthreads();
}

// The rows the first pass listed, one CTA per SM.  With at least min_rows of
// them (dense layers: many) each of the RWARPS warps takes rows through a
// 2,048-slot table (16 KB), and the CTA then takes the rows its own warps
// could not hold (flagged in spill[], indexed like big_rows) with cta_row;
// with fewer, every listed row goes to cta_row, which is faster for a few rows.
// Every path gives the same values, bit for bit.
__global__ void __launch_bounds__(RTHREADS)
k4_spmm_rest(const int64_t* __restrict__ sstart, const int32_t* __restrict__ slen, const int32_t* __restrict__ scol,
             const float* __restrict__ sval, const int32_t* __restrict__ nbr, const float* __restrict__ nbr_w,
             const int32_t* __restrict__ nbr_n, int k2p1, const int32_t* __restrict__ ub,
             const int32_t* __restrict__ big_rows, const int32_t* __restrict__ big_count, int min_rows,
             int32_t* __restrict__ spill, const int64_t* __restrict__ dstart, int32_t* __restrict__ dlen,
             int32_t* __restrict__ dcol, float* __restrict__ dval, int64_t n, int64_t cap, float* __restrict__ dense,
             uint32_t* __restrict__ bits, long long* __restrict__ status, bool agg_max,
             unsigned long long* __restrict__ nnz_out) {
  extern __shared__ int smem_i[];
  __shared__ int scan_s[RTHREADS];
  __shared__ unsigned long long red_hi[RTHREADS], red_lo[RTHREADS];
  if (!capacity_ok(dstart, n, cap, status)) return;
  const int count = *big_count;
  if (count == 0) return;
  const int tid = threadIdx.x, wib = tid >> 5, lane = tid & 31;
  float* acc = dense + size_t(blockIdx.x) * n;
  uint32_t* bm = bits + size_t(blockIdx.x) * ((n + 31) / 32);
  unsigned long long nnz = 0;      // entries written by this thread's warp (lane 0) or CTA (thread 0)
  if (count >= min_rows) {
    volatile int* keys = smem_i + wib * MSLOTS * 2;
    float* vals = reinterpret_cast<float*>(smem_i + wib * MSLOTS * 2 + MSLOTS);
    for (int sl = lane; sl < MSLOTS; sl += kWarp) {
      keys[sl] = KEY_EMPTY;
      vals[sl] = 0.f;
    }
    __syncwarp();
    for (int64_t f = int64_t(blockIdx.x) * RWARPS + wib; f < count; f += int64_t(gridDim.x) * RWARPS) {
      const int64_t i = big_rows[f];
      const bool sp = warp_row<MSLOTS>(i, ub[i], keys, vals, sstart, slen, scol, sval, nbr, nbr_w, nbr_n, k2p1,
                                       dstart, dlen, dcol, dval, status, agg_max, lane, nnz);
      if (lane == 0) spill[f] = sp ? 1 : 0;
    }
    __syncthreads();  // this CTA's flags are written
    for (int64_t f0 = int64_t(blockIdx.x) * RWARPS; f0 < count; f0 += int64_t(gridDim.x) * RWARPS)
      for (int w = 0; w < RWARPS && f0 + w < count; ++w)
        if (spill[f0 + w])
          cta_row(big_rows[f0 + w], sstart, slen, scol, sval, nbr, nbr_w, nbr_n, k2p1, dstart, dlen, dcol, dval, n,
                  acc, bm, agg_max, scan_s, red_hi, red_lo, nnz);
  } else {
    // The tables are not needed: when the dense accumulator and its bitmap fit
    // the shared memory (n up to ~47,000), they live there (zeroed once; every
    // row leaves them zero) instead of in the global scratch.
    const int64_t nwords = (n + 31) / 32;
    const bool local = (n + nwords) * 4 <= int64_t(RWARPS) * MSLOTS * 2 * int64_t(sizeof(int));
    float* a2 = local ? reinterpret_cast<float*>(smem_i) : acc;
    uint32_t* b2 = local ? reinterpret_cast<uint32_t*>(smem_i) + n : bm;
    if (local) {
      for (int64_t e = tid; e < n + nwords; e += RTHREADS) smem_i[e] = 0;
      __syncthreads();
    }
    for (int64_t f = blockIdx.x; f < count; f += gridDim.x)
      cta_row(big_rows[f], sstart, slen, scol, sval, nbr, nbr_w, nbr_n, k2p1, dstart, dlen, dcol, dval, n, a2, b2,
              agg_max, scan_s, red_hi, red_lo, nnz);
  }
  if (nnz_out && lane == 0 && nnz) atomicAdd(nnz_out, nnz);
}

__global__ void k4_row_norms(const int64_t* __restrict__ start, const int32_t* __restrict__ len,
                             const float* __restrict__ val, int64_t n, float* __restrict__ rn,
                             const long long* __restrict__ status, const uint8_t* __restrict__ sel) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  // After an overflowing layer the row lengths of its output were never written.
  if (i >= n || (status[kStErr] & kErrOverflow) || (sel && !sel[i])) return;
  const int64_t a = start[i];
  const int m = len[i];
  const float ss = warp_sumsq_exact(val + a, m, lane);
  if (lane == 0) rn[i] = 1.0f / sqrtf(ss);
}

__global__ void k4_compact(int64_t n, const int64_t* __restrict__ start, const int32_t* __restrict__ len,
                           const int32_t* __restrict__ col, const float* __restrict__ val,
                           const int64_t* __restrict__ cstart, int32_t* __restrict__ ccol, float* __restrict__ cval) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t a = start[i], o = cstart[i];
  const int m = len[i];
  for (int p = lane; p < m; p += kWarp) {
    ccol[o + p] = col[a + p];
    cval[o + p] = val[a + p];
  }
}

}  // namespace

int launch_layer_compact(int64_t n, const int64_t* start, const int32_t* len, const int32_t* col, const float* val,
                         const int64_t* cstart, int32_t* ccol, float* cval, cudaStream_t s) {
  const int T = 256;
  k4_compact<<<unsigned((n * kWarp + T - 1) / T), T, 0, s>>>(n, start, len, col, val, cstart, ccol, cval);
  return 1;
}

int propagate_warp_slots() { return WSLOTS; }

int launch_propagate(const Shape& sh, const Buffers& b, int src, int dst, int aggregator, long long* status,
                      int sm_count, const Tuning& t, cudaStream_t s, const LayerReuse* reuse, long long* nnz_slot) {
  unsigned long long* nnz_out = reinterpret_cast<unsigned long long*>(nnz_slot);
  const int64_t n = sh.n;
  const int k2p1 = sh.k2 + 1;
  const int T = 256;
  cudaMemsetAsync(b.big_count, 0, 2 * sizeof(int32_t), s);  // [0]: rows handed on, [1]: next row of the first pass
  const LayerReuse ru = reuse ? *reuse : LayerReuse{};
  k4_ub<<<unsigned((n + T - 1) / T), T, 0, s>>>(b.nbr, b.nbr_n, k2p1, b.len[src], n, b.ub, b.big_rows, b.big_count,
                                                 status, ru);
  launch_scan(b.ub, n, b.start[dst], s);
  const int warps = t.prop_warps < 1 ? 1 : (t.prop_warps > kMaxPropWarps ? kMaxPropWarps : t.prop_warps);
  const size_t smem = size_t(warps) * WSLOTS * 2 * sizeof(int);
  cudaFuncSetAttribute(k4_spmm_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int64_t blocks_needed = (n + warps - 1) / warps;
  const int per_sm = smem ? int((227 * 1024) / smem) : 1;
  const unsigned blocks = unsigned(tmin<int64_t>(blocks_needed, int64_t(sm_count) * (per_sm > 0 ? per_sm : 1)));
  k4_spmm_warp<<<blocks, warps * kWarp, smem, s>>>(b.start[src], b.len[src], b.col[src], b.val[src], b.nbr, b.nbr_w,
                                                   b.nbr_n, k2p1, b.ub, b.start[dst], b.len[dst], b.col[dst],
                                                   b.val[dst], n, sh.cap_h, b.big_rows, b.big_count,
                                                   b.big_count + 1, status, aggregator == RERANK_AGG_MAX, ru,
                                                   nnz_out);
  // The rows the first pass listed: 2,048-slot tables when there are at least
  // 4 per SM (market_hard: 21,906 rows, propagation 2.20 -> 1.13 ms), else the
  // CTA path (market: 549 rows, faster there).
  static const int min_override = [] {
    const char* e = std::getenv("RERANK_TEST_PROP_SECOND_MIN");  // test hook: the row count that takes the tables
    return e ? std::atoi(e) : -1;
  }();
  const int min_rows = min_override >= 0 ? min_override : 4 * sm_count;
  const size_t rsmem = size_t(RWARPS) * MSLOTS * 2 * sizeof(int);
  cudaFuncSetAttribute(k4_spmm_rest, cudaFuncAttributeMaxDynamicSharedMemorySize, int(rsmem));
  k4_spmm_rest<<<sm_count, RTHREADS, rsmem, s>>>(
      b.start[src], b.len[src], b.col[src], b.val[src], b.nbr, b.nbr_w, b.nbr_n, k2p1, b.ub, b.big_rows, b.big_count,
      min_rows, b.prop_spill, b.start[dst], b.len[dst], b.col[dst], b.val[dst], n, sh.cap_h, b.hash_keys_vals,
      reinterpret_cast<uint32_t*>(b.hash_keys_vals + size_t(sm_count) * n), status, aggregator == RERANK_AGG_MAX,
      nnz_out);
  return 4;
}

int launch_row_norms(const Shape& sh, const Buffers& b, int src, const long long* status, cudaStream_t s,
                     const uint8_t* rows_sel) {
  const int T = 256;
  k4_row_norms<<<unsigned((sh.n * kWarp + T - 1) / T), T, 0, s>>>(b.start[src], b.len[src], b.val[src], sh.n,
                                                                   b.rnorm, status, rows_sel);
  return 1;
}

}  // namespace rr

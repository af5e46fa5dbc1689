// K5 + K6: the final ranking (Alg. 1 step 7): for every query q the gallery
// sorted by cos(h_q, h_g), descending, ties to the lower gallery index;
// returned as (gallery index, 1 - cos).
//
// K5 transposes the gallery rows of H (scaled to unit norm) into CSC, so the
// column c lists every gallery vertex g with h_g[c] != 0.
// K6 takes one query per CTA and computes all of its scores at once,
// Gustavson style: s_g = sum_{c in supp(h_q)} h_q[c] * h_g[c].  Products are
// accumulated as unsigned fixed point (2^-31 units) with shared-memory atomics;
// integer addition is associative, so the score does not depend on the order
// in which warps add their terms.  Zero scores (disjoint supports, the bulk of
// the gallery) are exact.  The non-zero scores become 64-bit sort keys
// (bit-inverted score, gallery index): all distinct, and their ascending order
// is the ranking (equal scores in ascending gallery index).  They are put in
// order by one bucket pass: the bucket of a score is its binary exponent and
// the next 7 bits (4,096 log-spaced buckets, monotone in the score), keys are
// scattered to their bucket's range, and each key's place inside its bucket is
// the number of smaller keys there.  The keys live in shared memory up to
// 8,192 of them, beyond that in the CTA's global scratch, where full lists cut
// each bucket into ceil(count / 4) equal value ranges first.  Queries with a
// bucket too crowded for the counting step (massive ties) use a stable LSD
// radix sort in global memory (four 8-bit passes, per-warp digit histograms,
// __match_any_sync ranks).  The zero tail follows in ascending gallery index.
#include "common.cuh"
#include "internal.hpp"

#include <cstdio>
#include <cstdlib>

namespace rr {
namespace {

constexpr int RT = 1024;                // threads per ranking CTA
constexpr int RW = RT / kWarp;
constexpr int SORT_CAP = 8192;          // non-zeros sorted in shared memory
constexpr float kFix = 2147483648.0f;   // 2^31
constexpr float kUnfix = 4.656612873077393e-10f;  // 2^-31

__global__ void k5_count(const int64_t* __restrict__ start, const int32_t* __restrict__ len,
                         const int32_t* __restrict__ col, int64_t nq, int64_t n, int32_t* __restrict__ colcnt,
                         const long long* __restrict__ status, const uint8_t* __restrict__ sel) {
  const int64_t r = nq + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n || (status[kStErr] & kErrOverflow) || (sel && !sel[r])) return;
  const int64_t a = start[r];
  const int m = len[r];
  for (int p = lane; p < m; p += kWarp) atomicAdd(&colcnt[col[a + p]], 1);
}

__global__ void k5_fill(const int64_t* __restrict__ start, const int32_t* __restrict__ len,
                        const int32_t* __restrict__ col, const float* __restrict__ val, const float* __restrict__ rn,
                        int64_t nq, int64_t n, const int64_t* __restrict__ colptr, int32_t* __restrict__ fill,
                        int32_t* __restrict__ csc_row, float* __restrict__ csc_val,
                        const long long* __restrict__ status, const uint8_t* __restrict__ sel) {
  const int64_t r = nq + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n || (status[kStErr] & kErrOverflow) || (sel && !sel[r])) return;
  const int64_t a = start[r];
  const int m = len[r];
  const float s = rn[r];
  for (int p = lane; p < m; p += kWarp) {
    const int c = col[a + p];
    const int64_t pos = colptr[c] + atomicAdd(&fill[c], 1);
    csc_row[pos] = int32_t(r - nq);
    csc_val[pos] = val[a + p] * s;
  }
}

// Exclusive block scan of one int per thread; returns the total.
__device__ int block_exscan(int v, int* tmp, int& excl) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < RW ? tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += y;
    }
    tmp[lane] = s;
  }
  __syncthreads();
  excl = x - v + (w ? tmp[w - 1] : 0);
  const int total = tmp[RW - 1];
  __syncthreads();
  return total;
}

// Stable LSD radix sort of (key, val) ascending by key, four 8-bit passes.
// Each warp owns a contiguous segment and counts its digits; the scatter
// offsets are one exclusive scan over the (digit, warp) counts in digit-major
// order, so equal digits keep their order across warps, and __match_any_sync
// ranks them within a warp.  All threads of the block must call it; the
// result ends in (keys, vals), whose pointers are swapped as passes run.
__device__ void block_radix_sort(uint32_t*& keys, uint32_t*& vals, uint32_t*& tkeys, uint32_t*& tvals, int cnt,
                                 uint32_t* hist, int* tmp, int* skip) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int seg = (cnt + RW - 1) / RW;
  const int a = min(cnt, w * seg), b = min(cnt, a + seg);
  // Scan ownership: thread t holds digit d = t / 4 and warps 8 (t % 4) .. + 7.
  const int sd = t >> 2, sw = (t & 3) * 8;
  for (int shift = 0; shift < 32; shift += 8) {
    for (int e = t; e < RW * 256; e += RT) hist[e] = 0;
    if (t == 0) *skip = 0;
    __syncthreads();
    for (int p = a + lane; p < b; p += kWarp) atomicAdd(&hist[w * 256 + ((keys[p] >> shift) & 255)], 1u);
    __syncthreads();
    uint32_t c[8];
    int part = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c[k] = hist[(sw + k) * 256 + sd];
      part += int(c[k]);
    }
    int dig = part;  // total of digit sd over all warps (4 consecutive lanes)
    dig += __shfl_xor_sync(kFull, dig, 1);
    dig += __shfl_xor_sync(kFull, dig, 2);
    if ((t & 3) == 0 && dig == cnt) *skip = 1;  // one digit holds every key: nothing would move
    int base;
    block_exscan(part, tmp, base);
    if (*skip) continue;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      hist[(sw + k) * 256 + sd] = uint32_t(base);
      base += int(c[k]);
    }
    __syncthreads();
    for (int p0 = a; p0 < b; p0 += kWarp) {
      const int p = p0 + lane;
      const bool valid = p < b;
      const uint32_t k = valid ? keys[p] : 0u;
      const uint32_t v = valid ? vals[p] : 0u;
      const int d = valid ? int((k >> shift) & 255) : 256 + lane;
      const unsigned peers = __match_any_sync(kFull, d);
      const int rank = __popc(peers & lt);
      const uint32_t pos = valid ? hist[w * 256 + d] + uint32_t(rank) : 0u;
      __syncwarp();
      if (valid) {
        tkeys[pos] = k;
        tvals[pos] = v;
        if ((peers & lt) == 0) hist[w * 256 + d] += uint32_t(__popc(peers));
      }
      __syncwarp();
    }
    __syncthreads();
    uint32_t* x = keys; keys = tkeys; tkeys = x;
    x = vals; vals = tvals; tvals = x;
  }
}

struct RankArgs {
  const int64_t* start;
  const int32_t* len;
  const int32_t* col;
  const float* val;
  const float* rn;
  const int64_t* colptr;
  const int32_t* csc_row;
  const float* csc_val;
  int64_t nq, ng, topk;
  int64_t q_begin, q_end;  // queries ranked by this launch
  int32_t* out_idx;
  float* out_dist;
  uint32_t* gscratch;   // per CTA (rank_scratch_words): acc (ng) [if !acc_smem] + 4 * ng sort buffers
  int acc_smem;
  RankReuse reuse;  // resident gallery lists (colptr null: none)
  int sort_cap;    // most non-zeros the shared-memory sort takes (SORT_CAP unless a test lowers it)
  int bucket_cap;  // largest bucket it takes (BUCKET_CAP unless a test lowers it)
  long long* status;
};

constexpr int NB = 4096;         // score buckets of the shared-memory sort
constexpr int BUCKET_CAP = 256;  // largest bucket the counting step takes
static_assert(NB % RT == 0 && NB <= RW * 256, "bucket counters share the radix histogram space");

// Bucket of a non-zero fixed-point score x: the position of its leading bit
// and the 7 bits after it, so f(x) never decreases as x grows; reversed, so
// that higher scores come first.
__device__ __forceinline__ int score_bucket(uint32_t x) {
  const int lz = __clz(x);
  const uint32_t below = (x << lz) << 1;  // the bits after the leading one, left-aligned
  const int f = ((31 - lz) << 7) | int(below >> 25);
  return (NB - 1) - f;
}

__device__ __forceinline__ uint64_t rank_key(uint32_t x, uint32_t g) { return (uint64_t(~x) << 32) | g; }

// Global scratch per ranking CTA, in 32-bit words (even, so every CTA's part
// is 8-byte aligned): the accumulator when shared memory cannot hold it, then
// either two 64-bit key arrays (bucket sort beyond SORT_CAP keys) or four
// 32-bit arrays (radix sort).
__host__ __device__ inline int64_t scratch_words(int64_t ng) { return (5 * ng + 9) & ~int64_t(1); }

__global__ void __launch_bounds__(RT, 1) k6_rank(RankArgs A) {
  extern __shared__ uint32_t sm[];
  if (A.status[kStErr] & kErrOverflow) return;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ng = A.ng;
  const int nwords = int((ng + 31) / 32);
  uint32_t* hist = sm;                                   // RW * 256 (radix) or NB (buckets)
  int* tmp = reinterpret_cast<int*>(hist + RW * 256);    // 32
  int* misc = tmp + 32;                                  // 32: [0] skip flag, [1] largest bucket, [2] bstar
  uint32_t* bits = reinterpret_cast<uint32_t*>(misc + 32);  // nwords
  uint64_t* kb = reinterpret_cast<uint64_t*>(bits + ((nwords + 3) & ~3));  // SORT_CAP keys, bucket order
  uint32_t* region = reinterpret_cast<uint32_t*>(kb + SORT_CAP);  // acc (when acc_smem), later sorted keys
  uint64_t* ks = reinterpret_cast<uint64_t*>(region);   // SORT_CAP sorted keys (the accumulator is dead by then)
  uint32_t* gbase = A.gscratch + size_t(blockIdx.x) * size_t(scratch_words(ng));
  uint32_t* acc = A.acc_smem ? region : gbase;
  uint32_t* gk0 = gbase + ng;
  uint32_t* gv0 = gk0 + ng;
  uint32_t* gk1 = gv0 + ng;
  uint32_t* gv1 = gk1 + ng;
  uint64_t* kbg = reinterpret_cast<uint64_t*>(gbase + ((ng + 1) & ~int64_t(1)));  // ng keys, bucket order
  uint64_t* ksg = kbg + ng;                                                       // ng sorted keys
  const int64_t T = A.topk;

  for (int64_t q = A.q_begin + blockIdx.x; q < A.q_end; q += gridDim.x) {
    for (int64_t g = t; g < ng; g += RT) acc[g] = 0u;
    for (int e = t; e < NB; e += RT) hist[e] = 0u;
    if (t == 0) misc[1] = 0;
    __syncthreads();
    const int64_t a = A.start[q];
    const int m = A.len[q];
    const float rq = A.rn[q];
    // Warp w takes entries w, w + RW, ...; the next entry's column bounds are
    // loaded while the current column is added, four column steps per round.
    {
      int e = w;
      float v = 0.f;
      int64_t p0 = 0, p1 = 0;
      if (e < m) {
        const int c = A.col[a + e];
        v = A.val[a + e] * rq;
        p0 = A.colptr[c];
        p1 = A.colptr[c + 1];
      }
      while (e < m) {
        const int en = e + RW;
        float vn = 0.f;
        int64_t n0 = 0, n1 = 0;
        if (en < m) {
          const int cn = A.col[a + en];
          vn = A.val[a + en] * rq;
          n0 = A.colptr[cn];
          n1 = A.colptr[cn + 1];
        }
        for (int64_t p = p0 + lane; p < p1; p += 4 * kWarp) {
          int r[4];
          float x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t pp = p + u * kWarp;
            r[u] = pp < p1 ? A.csc_row[pp] : -1;
            x[u] = pp < p1 ? A.csc_val[pp] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float prod = v * x[u];
            if (r[u] >= 0) atomicAdd(&acc[r[u]], __float2uint_rn(prod * kFix));
          }
        }
        e = en;
        v = vn;
        p0 = n0;
        p1 = n1;
      }
    }
    if (A.reuse.colptr) {
      // The same over the resident lists of the columns of gallery vertices,
      // for the gallery rows the request left unchanged.
      const RankReuse& R = A.reuse;
      for (int e = w; e < m; e += RW) {
        const int64_t c = A.col[a + e] - R.shift;
        if (c < 0) continue;
        const float v = A.val[a + e] * rq;
        const int64_t p1 = R.colptr[c + 1];
        for (int64_t p = R.colptr[c] + lane; p < p1; p += 4 * kWarp) {
          int r[4];
          float x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t pp = p + u * kWarp;
            r[u] = pp < p1 ? R.row[pp] : -1;
            x[u] = pp < p1 ? R.val[pp] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (r[u] >= 0 && !R.changed[r[u]]) atomicAdd(&acc[r[u]], __float2uint_rn(v * x[u] * kFix));
        }
      }
    }
    __syncthreads();
    // Non-zero bitmap, bucket histogram and count, warp-cooperative: warp w
    // owns words [w0, w1) (32 gallery entries each, lane = entry); the ballot
    // of a word is its bitmap word.
    const int wpw = (nwords + RW - 1) / RW;
    const int w0 = min(nwords, w * wpw), w1 = min(nwords, w0 + wpw);
    int mine = 0;
    // Four words per step: independent loads in flight (the accumulator may live in global memory).
    for (int wd = w0; wd < w1; wd += 4) {
      uint32_t x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t g = int64_t(wd + u) * 32 + lane;
        x[u] = (wd + u < w1 && g < ng) ? acc[g] : 0u;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned bal = __ballot_sync(kFull, x[u] != 0u);
        if (lane == 0 && wd + u < w1) bits[wd + u] = bal;
        if (x[u] != 0u) atomicAdd(&hist[score_bucket(x[u])], 1u);
        mine += __popc(bal);
      }
    }
    int off;
    const int cnt = block_exscan(lane == 0 ? mine : 0, tmp, off);  // one count per warp (lane 0)
    off = __shfl_sync(kFull, off, 0);
    // Zeros before this warp's words: all earlier words are whole, so 32 w0 - (non-zeros before).
    const int64_t zeros_before = int64_t(w0) * 32 - off;
    // Only the first `cut` places are returned: the buckets up to the one
    // holding place cut - 1 (bstar) are sorted, later ones are left out.
    const int cut = int(tmin<int64_t>(T, cnt));
    int bstar = -1;
    // Keys of the bucket sort in shared memory up to sort_cap of them, else in
    // this CTA's global scratch (L1/L2-resident); the radix sort only when a
    // bucket is too crowded for the counting step.
    // Full lists whose keys go to global scratch (dense final features: every
    // gallery score non-zero, about 20 keys per log bucket on average): each
    // log bucket of c keys is cut into ceil(c / 4) equal value ranges, the
    // sub-buckets, in the same order, so that the in-bucket counting reads a
    // few keys per key.  Sub-bucket bases and counters live in the bucket-key
    // space of shared memory (unused when the keys are in global scratch).
    // When the sub-buckets do not fit, or one is still crowded, the query
    // takes the log buckets below; the lists are the same either way.
    bool done = false;
    if (cnt > A.sort_cap && T >= cnt) {
      uint32_t* sbase = reinterpret_cast<uint32_t*>(kb);  // NB: first sub-bucket of each log bucket
      uint32_t* h2 = sbase + NB;                           // sub-bucket counters, then their ends
      const int H2CAP = 2 * SORT_CAP - NB;
      uint32_t c[NB / RT];
      int part = 0;
#pragma unroll
      for (int k = 0; k < NB / RT; ++k) {
        c[k] = (hist[t * (NB / RT) + k] + 3u) >> 2;
        part += int(c[k]);
      }
      int base;
      const int nb2 = block_exscan(part, tmp, base);
      if (nb2 <= H2CAP) {
#pragma unroll
        for (int k = 0; k < NB / RT; ++k) {
          sbase[t * (NB / RT) + k] = uint32_t(base);
          base += int(c[k]);
        }
        for (int e = t; e < nb2; e += RT) h2[e] = 0u;
        if (t == 0) misc[3] = 0;
        __syncthreads();
        // Sub-bucket of a non-zero x: its place inside its log bucket (the
        // bits below the leading 8), scaled onto the bucket's ceil(c / 4)
        // ranges, higher x first.
        auto sub_bucket = [&](uint32_t x) {
          const int bk = score_bucket(x);
          const int sh = max(0, 24 - __clz(x));  // bits below the leading one and the 7 after it
          const uint32_t r = x & ((1u << sh) - 1u);
          const uint32_t ns = (hist[bk] + 3u) >> 2;
          const uint32_t sub = uint32_t((uint64_t(r) * ns) >> sh);
          return int(sbase[bk] + (ns - 1u - sub));
        };
        for (int wd = w0; wd < w1; wd += 4) {
          uint32_t bal[4], x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            bal[u] = wd + u < w1 ? bits[wd + u] : 0u;
            x[u] = ((bal[u] >> lane) & 1u) ? acc[int64_t(wd + u) * 32 + lane] : 0u;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if ((bal[u] >> lane) & 1u) atomicAdd(&h2[sub_bucket(x[u])], 1u);
        }
        __syncthreads();
        // Sub-bucket starts (a contiguous range per thread) and the largest one.
        const int per = (nb2 + RT - 1) / RT;
        const int e0 = min(nb2, t * per), e1 = min(nb2, e0 + per);
        int loc = 0, big = 0;
        for (int e = e0; e < e1; ++e) {
          loc += int(h2[e]);
          big = max(big, int(h2[e]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) big = max(big, __shfl_xor_sync(kFull, big, o));
        if (lane == 0 && big > 0) atomicMax(&misc[3], big);
        int run;
        block_exscan(loc, tmp, run);  // its barriers also publish misc[3]
        if (misc[3] <= A.bucket_cap) {
          for (int e = e0; e < e1; ++e) {
            const uint32_t v = h2[e];
            h2[e] = uint32_t(run);
            run += int(v);
          }
          __syncthreads();
          for (int wd = w0; wd < w1; wd += 4) {
            uint32_t bal[4], x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              bal[u] = wd + u < w1 ? bits[wd + u] : 0u;
              x[u] = ((bal[u] >> lane) & 1u) ? acc[int64_t(wd + u) * 32 + lane] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if ((bal[u] >> lane) & 1u) {
                const uint32_t pos = atomicAdd(&h2[sub_bucket(x[u])], 1u);
                kbg[pos] = rank_key(x[u], uint32_t(int64_t(wd + u) * 32 + lane));
              }
            }
          }
          __syncthreads();  // h2[i] is now the end of sub-bucket i
          for (int64_t p = t; p < cnt; p += RT) {
            const uint64_t key = kbg[p];
            const uint32_t x = ~uint32_t(key >> 32);
            const int i2 = sub_bucket(x);
            const int b0 = i2 ? int(h2[i2 - 1]) : 0, b1 = int(h2[i2]);
            int r = 0;
            for (int j = b0; j < b1; ++j) r += kbg[j] < key;
            const int64_t pos = b0 + r;
            A.out_idx[q * T + pos] = int32_t(uint32_t(key));
            A.out_dist[q * T + pos] = 1.0f - __uint2float_rn(x) * kUnfix;
          }
          done = true;
        }
      }
      __syncthreads();  // the bucket-key space and misc are free again
    }
    if (!done) {
      const bool keys_smem = cnt <= A.sort_cap;
      uint64_t* const kbx = keys_smem ? kb : kbg;
      uint64_t* const ksx = keys_smem ? ks : ksg;
      bool small = true;
      {
        // Bucket starts: exclusive scan of the histogram, four buckets per thread;
        // the largest bucket up to bstar decides whether the counting step may run.
        const bool whole = cut == cnt;  // every non-zero is returned: bstar is the last bucket
        uint32_t c[NB / RT];
        int part = 0, big = 0;
  #pragma unroll
        for (int k = 0; k < NB / RT; ++k) {
          c[k] = hist[t * (NB / RT) + k];
          part += int(c[k]);
          big = max(big, int(c[k]));
        }
        if (whole) {
  #pragma unroll
          for (int o = 16; o > 0; o >>= 1) big = max(big, __shfl_xor_sync(kFull, big, o));
          if (lane == 0 && big > 0) atomicMax(&misc[1], big);
        }
        int base;
        block_exscan(part, tmp, base);  // its barriers also publish misc[1]
  #pragma unroll
        for (int k = 0; k < NB / RT; ++k) {
          hist[t * (NB / RT) + k] = uint32_t(base);
          if (!whole && base <= cut - 1 && cut - 1 < base + int(c[k])) misc[2] = t * (NB / RT) + k;
          base += int(c[k]);
        }
        __syncthreads();
        if (whole) {
          bstar = cnt > 0 ? NB - 1 : -1;
        } else {
          bstar = misc[2];
          big = 0;
  #pragma unroll
          for (int k = 0; k < NB / RT; ++k)
            if (t * (NB / RT) + k <= bstar) big = max(big, int(c[k]));
  #pragma unroll
          for (int o = 16; o > 0; o >>= 1) big = max(big, __shfl_xor_sync(kFull, big, o));
          if (lane == 0 && big > 0) atomicMax(&misc[1], big);
          __syncthreads();
        }
        small = misc[1] <= A.bucket_cap;
      }
      if (small) {
        // Scatter the non-zeros of buckets 0 .. bstar to their bucket's range
        // (any order inside it); afterwards hist[b] is the end of bucket b.
        for (int wd = w0; wd < w1; wd += 4) {
          uint32_t bal[4], x[4];
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            bal[u] = wd + u < w1 ? bits[wd + u] : 0u;
            x[u] = ((bal[u] >> lane) & 1u) ? acc[int64_t(wd + u) * 32 + lane] : 0u;
          }
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            if ((bal[u] >> lane) & 1u) {
              const int bk = score_bucket(x[u]);
              if (bk <= bstar) {
                const uint32_t pos = atomicAdd(&hist[bk], 1u);
                kbx[pos] = rank_key(x[u], uint32_t(int64_t(wd + u) * 32 + lane));
              }
            }
          }
        }
        __syncthreads();
        // Place of a key = its bucket's start + the number of smaller keys in
        // the bucket (keys are distinct); the accumulator is no longer needed.
        const int nsel = bstar >= 0 ? int(hist[bstar]) : 0;
        for (int p = t; p < nsel; p += RT) {
          const uint64_t key = kbx[p];
          const int bk = score_bucket(~uint32_t(key >> 32));
          const int b0 = bk ? int(hist[bk - 1]) : 0, b1 = int(hist[bk]);
          int r = 0;
          for (int j = b0; j < b1; ++j) r += kbx[j] < key;
          ksx[b0 + r] = key;
        }
        __syncthreads();
        const int64_t nout = tmin<int64_t>(T, cnt);
        for (int64_t p = t; p < nout; p += RT) {
          const uint64_t key = ksx[p];
          A.out_idx[q * T + p] = int32_t(uint32_t(key));
          A.out_dist[q * T + p] = 1.0f - __uint2float_rn(~uint32_t(key >> 32)) * kUnfix;
        }
      } else {
        // Global-memory path: non-zeros compacted in gallery order, then the
        // stable radix sort.
        for (int wd = w0; wd < w1; wd += 4) {
          uint32_t bal[4], x[4];
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            bal[u] = wd + u < w1 ? bits[wd + u] : 0u;
            x[u] = ((bal[u] >> lane) & 1u) ? acc[int64_t(wd + u) * 32 + lane] : 0u;
          }
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            if ((bal[u] >> lane) & 1u) {
              const int pos = off + __popc(bal[u] & lt);
              gk0[pos] = ~x[u];
              gv0[pos] = uint32_t(int64_t(wd + u) * 32 + lane);
            }
            off += __popc(bal[u]);
          }
        }
        __syncthreads();
        uint32_t* k0 = gk0;
        uint32_t* v0 = gv0;
        uint32_t* k1 = gk1;
        uint32_t* v1 = gv1;
        block_radix_sort(k0, v0, k1, v1, cnt, hist, tmp, misc);
        const int64_t nout = tmin<int64_t>(T, cnt);
        for (int64_t p = t; p < nout; p += RT) {
          const float s = __uint2float_rn(~k0[p]) * kUnfix;
          A.out_idx[q * T + p] = int32_t(v0[p]);
          A.out_dist[q * T + p] = 1.0f - s;
        }
      }
    }
    // The zero tail in gallery order.  Its distances are all 1: plain
    // block-wide stores, 16 bytes each once aligned.  Its indices: warp w
    // writes the zeros of its words (a warp scan of 32 words' zero counts,
    // then one coalesced store per word).
    if (T > cnt) {
      float* dq = A.out_dist + q * T;
      const int64_t head = tmin<int64_t>((4 - int((reinterpret_cast<uintptr_t>(dq + cnt) >> 2) & 3)) & 3, T - cnt);
      if (t < head) dq[cnt + t] = 1.0f;
      const int64_t p0 = cnt + head, nv = (T - p0) >> 2;
      float4* dv = reinterpret_cast<float4*>(dq + p0);
      for (int64_t v = t; v < nv; v += RT) dv[v] = make_float4(1.f, 1.f, 1.f, 1.f);
      for (int64_t p = p0 + 4 * nv + t; p < T; p += RT) dq[p] = 1.0f;
      int32_t* iq = A.out_idx + q * T;
      // The warp's words 32 at a time: lane l takes word c0 + l, its zeros and
      // their count; a warp scan of the counts gives every word's first place,
      // then the warp writes the words' indices one word at a time.
      int64_t run = int64_t(cnt) + zeros_before;
      for (int c0 = w0; c0 < w1 && run < T; c0 += kWarp) {
        const int nw = min(kWarp, w1 - c0);
        uint32_t zl = 0u;
        if (lane < nw) {
          const int wd = c0 + lane;
          const int valid = int(tmin<int64_t>(32, ng - int64_t(wd) * 32));
          const uint32_t vm = valid == 32 ? kFull : ((1u << valid) - 1u);
          zl = ~bits[wd] & vm;
        }
        const int cz = __popc(zl);
        int incl = cz;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int64_t wbase = run + (incl - cz);
        for (int j = 0; j < nw; ++j) {
          const uint32_t zj = __shfl_sync(kFull, zl, j);
          const int64_t bj = __shfl_sync(kFull, wbase, j);
          if ((zj >> lane) & 1u) {
            const int64_t p = bj + __popc(zj & lt);
            if (p < T) iq[p] = int32_t(int64_t(c0 + j) * 32 + lane);
          }
        }
        run += __shfl_sync(kFull, incl, 31);
      }
    }
    __syncthreads();
  }
}

// Shared memory without the accumulator: radix histograms (RW x 256 words,
// also the NB bucket counters), scan scratch, the bitmap and the bucket-order
// keys; the region after them holds the accumulator (when it fits) and then
// the sorted keys, so it is never smaller than SORT_CAP keys.
size_t rank_smem_fixed(int64_t ng) {
  const int64_t nwords = (ng + 31) / 32;
  return sizeof(uint32_t) * (RW * 256 + 64 + ((nwords + 3) & ~int64_t(3))) + sizeof(uint64_t) * SORT_CAP;
}

// Dense final features (h^(0) = x_i): one query per CTA ranks all its gallery
// scores S[q][0 .. ng), which may be negative.  A score's 32-bit sort key is
// its IEEE bits mapped to an unsigned order (negatives reversed, -0 taken as
// +0), inverted so that ascending keys are descending scores; with the
// gallery index below it (64-bit key) the keys are distinct and their
// ascending order is the ranking (equal scores in ascending gallery index).
// Buckets in two levels, so that they hold a few keys each whatever the
// distribution: level one splits the key space into 8,192 bins of 2^19 keys
// (a sixteenth of an octave of the score), and a bin of c keys is cut into
// ceil(c / 4) equal key ranges, the buckets (in key order).  Keys are
// scattered to their bucket's range in the CTA's global scratch (L2-resident)
// and a key's place in its bucket is the number of smaller keys there.  A
// query with more than NBD2 buckets or a bucket of more than bucket_cap keys
// (e.g. many equal scores) takes the stable LSD radix sort in the same
// scratch instead (4 ng words).
constexpr int NBD1 = 8192;        // level-one bins (2^19 keys each)
constexpr int NBD2 = 16384;       // buckets
constexpr int DBUCKET_CAP = 256;  // largest bucket the counting step takes
constexpr size_t DENSE_SMEM = sizeof(uint32_t) * (2 * NBD1 + NBD2);  // bin counts, bin bases, bucket counters

__device__ __forceinline__ uint32_t dense_key(float sc) {
  const uint32_t u = sc == 0.0f ? 0u : __float_as_uint(sc);
  const uint32_t up = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // ascending with the score
  return ~up;
}

__global__ void __launch_bounds__(RT, 1)
k6_rank_dense(const float* __restrict__ S, int64_t nq, int64_t ng, int64_t topk, int32_t* __restrict__ out_idx,
              float* __restrict__ out_dist, uint32_t* __restrict__ gscratch, int bucket_cap,
              const long long* __restrict__ status) {
  extern __shared__ uint32_t dsm[];
  uint32_t* bcnt = dsm;              // NBD1: keys per bin
  uint32_t* bbase = dsm + NBD1;      // NBD1: first bucket of each bin
  uint32_t* hist = dsm + 2 * NBD1;   // NBD2 bucket counters (also the radix histograms)
  __shared__ int tmp[32];
  __shared__ uint32_t wmax[RW];
  __shared__ int skip;
  if (status[kStErr] & kErrOverflow) return;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t* base = gscratch + size_t(blockIdx.x) * size_t(scratch_words(ng));
  uint64_t* kb = reinterpret_cast<uint64_t*>(base);  // ng keys in bucket order (2 ng words)
  auto bucket = [&](uint32_t k) {
    const int bin = int(k >> 19);
    return int(bbase[bin] + ((uint64_t(k & 0x7ffffu) * ((bcnt[bin] + 3u) >> 2)) >> 19));
  };
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const float* sq = S + q * ng;
    for (int e = t; e < NBD1; e += RT) bcnt[e] = 0u;
    for (int e = t; e < NBD2; e += RT) hist[e] = 0u;
    __syncthreads();
    for (int64_t g = t; g < ng; g += RT) atomicAdd(&bcnt[dense_key(sq[g]) >> 19], 1u);
    __syncthreads();
    {
      // bbase = exclusive scan of ceil(bcnt / 4), eight bins per thread.
      uint32_t c[NBD1 / RT];
      int part = 0;
#pragma unroll
      for (int k = 0; k < NBD1 / RT; ++k) {
        c[k] = (bcnt[t * (NBD1 / RT) + k] + 3u) >> 2;
        part += int(c[k]);
      }
      int start;
      const int nbk = block_exscan(part, tmp, start);
#pragma unroll
      for (int k = 0; k < NBD1 / RT; ++k) {
        bbase[t * (NBD1 / RT) + k] = uint32_t(start);
        start += int(c[k]);
      }
      if (t == 0) skip = nbk > NBD2 ? 1 : 0;
      __syncthreads();
    }
    bool small = skip == 0;
    if (small) {
      for (int64_t g = t; g < ng; g += RT) atomicAdd(&hist[bucket(dense_key(sq[g]))], 1u);
      __syncthreads();
      uint32_t c[NBD2 / RT];
      int part = 0, big = 0;
#pragma unroll
      for (int k = 0; k < NBD2 / RT; ++k) {
        c[k] = hist[t * (NBD2 / RT) + k];
        part += int(c[k]);
        big = max(big, int(c[k]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) big = max(big, __shfl_xor_sync(kFull, big, o));
      if (lane == 0) wmax[w] = uint32_t(big);
      int start;
      block_exscan(part, tmp, start);  // its barriers also publish wmax
      for (int k = 0; k < RW; ++k) small = small && int(wmax[k]) <= bucket_cap;
      if (small) {
#pragma unroll
        for (int k = 0; k < NBD2 / RT; ++k) {
          hist[t * (NBD2 / RT) + k] = uint32_t(start);
          start += int(c[k]);
        }
        __syncthreads();
        for (int64_t g = t; g < ng; g += RT) {
          const uint32_t k = dense_key(sq[g]);
          const uint32_t pos = atomicAdd(&hist[bucket(k)], 1u);
          kb[pos] = (uint64_t(k) << 32) | uint64_t(g);
        }
        __syncthreads();  // hist[b] is now the end of bucket b
        for (int64_t p = t; p < ng; p += RT) {
          const uint64_t key = kb[p];
          const int bk = bucket(uint32_t(key >> 32));
          const int b0 = bk ? int(hist[bk - 1]) : 0, b1 = int(hist[bk]);
          int r = 0;
          for (int j = b0; j < b1; ++j) r += kb[j] < key;
          const int64_t pos = b0 + r;
          if (pos < topk) {
            const uint32_t g = uint32_t(key);
            out_idx[q * topk + pos] = int32_t(g);
            out_dist[q * topk + pos] = 1.0f - sq[g];
          }
        }
      }
    }
    if (!small) {
      uint32_t* keys = base;
      uint32_t* vals = base + ng;
      uint32_t* tkeys = base + 2 * ng;
      uint32_t* tvals = base + 3 * ng;
      for (int64_t g = t; g < ng; g += RT) {
        keys[g] = dense_key(sq[g]);
        vals[g] = uint32_t(g);
      }
      __syncthreads();
      block_radix_sort(keys, vals, tkeys, tvals, int(ng), hist, tmp, &skip);
      for (int64_t p = t; p < topk; p += RT) {
        const uint32_t g = vals[p];
        out_idx[q * topk + p] = int32_t(g);
        out_dist[q * topk + p] = 1.0f - sq[g];
      }
    }
    __syncthreads();
  }
}

// Test hook: RERANK_TEST_RANK_CAPS = "sort_cap,bucket_cap" lowers the limits,
// so that small inputs take the global-key and radix paths; all paths give
// identical lists.
void rank_caps(int* sort_cap, int* bucket_cap) {
  *sort_cap = SORT_CAP;
  *bucket_cap = BUCKET_CAP;
  if (const char* e = std::getenv("RERANK_TEST_RANK_CAPS")) {
    int s = SORT_CAP, b = BUCKET_CAP;
    if (std::sscanf(e, "%d,%d", &s, &b) == 2) {
      *sort_cap = s < SORT_CAP ? s : SORT_CAP;
      *bucket_cap = b < BUCKET_CAP ? b : BUCKET_CAP;
    }
  }
}

}  // namespace

int64_t rank_scratch_words(int64_t ng) { return scratch_words(ng); }

size_t rank_smem_bytes(int64_t ng, int threads) {
  (void)threads;
  const size_t fixed = rank_smem_fixed(ng);
  const size_t sorted = sizeof(uint64_t) * SORT_CAP;
  const size_t with_acc = fixed + (sizeof(uint32_t) * size_t(ng) > sorted ? sizeof(uint32_t) * size_t(ng) : sorted);
  return with_acc <= 227 * 1024 ? with_acc : fixed + sorted;
}

int launch_rank(const Shape& sh, const Buffers& b, int src, int32_t* out_idx, float* out_dist, long long* status,
                 int sm_count, const Tuning& tune, cudaStream_t s) {
  int nl = launch_rank_prep(sh, b, src, status, s);
  nl += launch_rank_queries(sh, b, src, out_idx, out_dist, 0, sh.nq, status, sm_count, tune, s);
  return nl;
}

int launch_rank_prep(const Shape& sh, const Buffers& b, int src, long long* status, cudaStream_t s,
                     const uint8_t* rows_sel) {
  const int64_t n = sh.n, nq = sh.nq, ng = sh.ng;
  const int T = 256;
  cudaMemsetAsync(b.colcnt, 0, sizeof(int32_t) * (n + 1), s);
  k5_count<<<unsigned((ng * kWarp + T - 1) / T), T, 0, s>>>(b.start[src], b.len[src], b.col[src], nq, n, b.colcnt,
                                                            status, rows_sel);
  launch_scan(b.colcnt, n, b.colptr, s);
  cudaMemsetAsync(b.colcnt, 0, sizeof(int32_t) * (n + 1), s);
  k5_fill<<<unsigned((ng * kWarp + T - 1) / T), T, 0, s>>>(b.start[src], b.len[src], b.col[src], b.val[src], b.rnorm,
                                                           nq, n, b.colptr, b.colcnt, b.csc_row, b.csc_val, status,
                                                           rows_sel);
  return 3;
}

int launch_rank_queries(const Shape& sh, const Buffers& b, int src, int32_t* out_idx, float* out_dist, int64_t q0,
                        int64_t q1, long long* status, int sm_count, const Tuning& tune, cudaStream_t s,
                        const RankReuse* reuse) {
  (void)tune;
  (void)sm_count;
  const int64_t nq = sh.nq, ng = sh.ng;
  RankArgs A;
  A.start = b.start[src];
  A.len = b.len[src];
  A.col = b.col[src];
  A.val = b.val[src];
  A.rn = b.rnorm;
  A.colptr = b.colptr;
  A.csc_row = b.csc_row;
  A.csc_val = b.csc_val;
  A.nq = nq;
  A.ng = ng;
  A.topk = sh.topk;
  A.q_begin = q0;
  A.q_end = q1;
  A.out_idx = out_idx;
  A.out_dist = out_dist;
  A.gscratch = b.rank_scratch;
  A.reuse = reuse ? *reuse : RankReuse{};
  const size_t smem = rank_smem_bytes(ng, RT);
  A.acc_smem = smem - rank_smem_fixed(ng) >= sizeof(uint32_t) * size_t(ng);
  rank_caps(&A.sort_cap, &A.bucket_cap);
  A.status = status;
  cudaFuncSetAttribute(k6_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int64_t nqry = q1 - q0;
  const unsigned grid = unsigned(nqry < sh.rank_ctas ? (nqry > 0 ? nqry : 1) : sh.rank_ctas);
  k6_rank<<<grid, RT, smem, s>>>(A);
  return 1;
}

int rank_threads() { return RT; }

int launch_rank_dense(const Shape& sh, const float* S, int32_t* out_idx, float* out_dist, uint32_t* scratch,
                      long long* status, cudaStream_t s) {
  const unsigned grid = unsigned(sh.nq < sh.rank_ctas ? sh.nq : sh.rank_ctas);
  int sort_cap = 0, bucket_cap = 0;
  rank_caps(&sort_cap, &bucket_cap);  // a test lowering the bucket cap sends queries to the radix sort
  cudaFuncSetAttribute(k6_rank_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, int(DENSE_SMEM));
  k6_rank_dense<<<grid, RT, DENSE_SMEM, s>>>(S, sh.nq, sh.ng, sh.topk, out_idx, out_dist, scratch,
                                             bucket_cap < DBUCKET_CAP ? bucket_cap : DBUCKET_CAP, status);
  return 1;
}

}  // namespace rr

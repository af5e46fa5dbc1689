// Serving: a resident gallery and a request loop with continuous batching.
//
// A request with Q queries is Algorithm 1 on X_u = (its queries) u G, queries
// first (Sec. 3.3).  What depends on G alone is computed once, at load: the
// unit rows, their BF16/FP8 copies and error bounds, every gallery row's K
// best columns of G by the tensor-core score (its candidate list), and its
// exact top-k1 list over G.  Per request, on a slot of its own:
//   1. the queries are normalised into the rows just before the slot's copy
//      of the gallery, so that X_u is one contiguous block;
//   2. tensor-core scores of the query rows against X_u (their candidate
//      lists) and of the gallery rows against the queries;
//   3. a gallery row keeps its resident exact list (indices shifted by Q)
//      when no query can enter it: its best approximate query score plus that
//      score's error bound stays below s_(k1) - eps_r, so every query's S is
//      below the row's k1-th score and the k1 best columns of X_u are the k1
//      best of G.  Otherwise ("touched") its candidate list over X_u is the
//      merge of its resident list and its query lists (the K best of a union
//      are the K best of the parts' K best) and it is refined like any row;
//   4. the refinement, recheck, exact scan, graph, propagation and ranking
//      stages, as in rerank_run, on X_u; a propagation layer recomputes only
//      the rows whose inputs differ from the gallery's own graph (G alone,
//      computed at load): a row whose message list and whose sources' rows of
//      the previous layer are unchanged gets the resident row, columns shifted
//      by Q.  Its values are those of a recomputation (each column is summed
//      in message order, norms are exact), only their order in the row differs.
// Every slot owns a stream and all the buffers of one request, so requests
// on different slots overlap on the GPU and never see each other's data.
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.hpp"

namespace rr {

double rescore_eps(int dp);
int fallback_warps();

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

constexpr int kMaxSlots = 8;
constexpr int64_t kMaxQuery = 1024;  // query columns of a request: at most 4 tiles of 256
constexpr int kMaxQueryLists = 8;    // lists per gallery row against the queries: 4 chunks x 2
constexpr int64_t kPad = 256;  // zero rows after the gallery: one full tensor-core tile

struct Server;

struct Slot {
  Server* srv = nullptr;
  int index = 0;
  cudaStream_t stream = nullptr;
  char* mem = nullptr;
  // X_u feature arrays over internal rows [0, S + G + kPad); union row u is
  // internal row S - Q + u, the gallery starts at internal row S.
  float* xhat = nullptr;
  void* xlow = nullptr;
  __nv_bfloat16* xhi = nullptr;
  __nv_bfloat16* xlo = nullptr;
  float* xscale = nullptr;
  double* norm = nullptr;
  float* err = nullptr;   // 3 x rowstride
  float* emax = nullptr;  // 4: maxima over X_u
  // per request
  float* err_q = nullptr;   // 3 x S: the queries' bounds, before they move into `err`
  float* emax_q = nullptr;  // 4: maxima over the queries
  int32_t* iota = nullptr;  // 0 .. S-1
  int32_t* scal = nullptr;  // [0] = Q, [1] = touched rows
  float* pa_s = nullptr;    // S x Pa x K: query rows against X_u
  int32_t* pa_i = nullptr;
  float* pb_s = nullptr;    // G x Pb x K: gallery rows against the queries
  int32_t* pb_i = nullptr;
  float* pm_s = nullptr;    // G x K: merged lists of the touched rows (by position)
  int32_t* pm_i = nullptr;
  int32_t* touched = nullptr;
  uint8_t* chg[2] = {nullptr, nullptr};  // per union row: layer input changed (two layers in turn)
  uint8_t* msgchg = nullptr;             // per union row: message list differs from the resident one
  int* floor_a = nullptr;
  int* floor_b = nullptr;
  void* xq_stage = nullptr;  // S x d: host queries staged here
  Buffers b;                 // the pipeline's own buffers, sized for Q = S
  long long* d_status = nullptr;
  long long* h_status = nullptr;
  // the request in flight
  uint64_t ticket = 0;
  bool busy = false;
  Clock::time_point t_done;
};

struct Pending {
  rerank_request req{};
  cudaEvent_t ready = nullptr;  // recorded on the caller's stream at submit
  Clock::time_point t_submit, t_start, t_done;
  rerank_status status = RERANK_OK;
  bool done = false;
  int slot = -1;
};

struct Server {
  rerank_ctx* ctx = nullptr;
  int64_t G = 0, S = 0, rowstride = 0;
  int d = 0, dp = 0, dtype = 0, k1 = 0, k2 = 0, layers = 0, prec = 0, K = 0;
  int64_t cap_h = 0;
  char* res_mem = nullptr;
  void* xg_raw = nullptr;         // the caller's gallery, copied
  float* res_s = nullptr;         // G x K candidate lists (approximate scores, gallery indices)
  int32_t* res_i = nullptr;
  int32_t* res_knn_idx = nullptr; // G x k1 exact lists over G
  float* res_knn_score = nullptr;
  float* res_emax = nullptr;      // 4: maxima of the gallery's bounds
  // The gallery's own graph (G alone): message lists and layers 0 .. L as
  // compact CSR, gallery indices.  Empty when they did not fit the budget.
  struct ResLayer {
    int64_t* start = nullptr;
    int32_t* len = nullptr;
    int32_t* col = nullptr;
    float* val = nullptr;
  };
  std::vector<ResLayer> res_layers;
  int64_t* res_colptr = nullptr;  // the last layer as CSC (row norms applied): gallery columns
  int32_t* res_csc_row = nullptr;
  float* res_csc_val = nullptr;
  int32_t* res_nbr = nullptr;
  float* res_nbr_w = nullptr;
  int32_t* res_nbr_n = nullptr;
  std::vector<void*> res_extra;   // allocations of the above
  bool reuse = false;
  std::vector<Slot> slots;
  size_t resident_bytes = 0, slot_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;     // worker wake-ups and waiters
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Pending> reqs;
  std::vector<int> finished;      // slots whose work has completed
  uint64_t next = 1;
  bool stop = false;
  int in_flight = 0, max_in_flight = 0;
  int64_t completed = 0, touched_rows = 0, recomputed_rows = 0;
  std::thread worker;
};

size_t esize(int prec) { return prec == RERANK_PREC_FP8 ? 1 : 2; }

// Bytes of one slot: the X_u arrays, the per-request lists and the pipeline workspace.
size_t slot_layout(const Server& v, Slot* sl, char* base, const Shape& shmax, int sm_count) {
  Carver c;
  c.base = base;
  const size_t rows = size_t(v.rowstride), dp = size_t(v.dp);
  const int pa_max = 32, pb_max = int((v.S + 255) / 256) * tc_lists_per_chunk(v.dp, 1);
  Slot t;
  t.xhat = c.take<float>(rows * dp);
  t.xlow = c.take<char>(rows * dp * esize(v.prec));
  t.xhi = v.prec == RERANK_PREC_BF16 ? static_cast<__nv_bfloat16*>(t.xlow) : c.take<__nv_bfloat16>(rows * dp);
  t.xlo = c.take<__nv_bfloat16>(rows * dp);
  t.xscale = c.take<float>(rows);
  t.norm = c.take<double>(rows);
  t.err = c.take<float>(3 * rows);
  t.emax = c.take<float>(4);
  t.err_q = c.take<float>(3 * size_t(v.S));
  t.emax_q = c.take<float>(4);
  t.iota = c.take<int32_t>(size_t(v.S));
  t.scal = c.take<int32_t>(4);
  t.pa_s = c.take<float>(size_t(v.S) * pa_max * v.K);
  t.pa_i = c.take<int32_t>(size_t(v.S) * pa_max * v.K);
  t.pb_s = c.take<float>(size_t(v.G) * pb_max * v.K);
  t.pb_i = c.take<int32_t>(size_t(v.G) * pb_max * v.K);
  t.pm_s = c.take<float>(size_t(v.G) * v.K);
  t.pm_i = c.take<int32_t>(size_t(v.G) * v.K);
  t.touched = c.take<int32_t>(size_t(v.G));
  t.chg[0] = c.take<uint8_t>(size_t(v.S + v.G));
  t.chg[1] = c.take<uint8_t>(size_t(v.S + v.G));
  t.msgchg = c.take<uint8_t>(size_t(v.S + v.G));
  t.floor_a = c.take<int>(size_t(v.S));
  t.floor_b = c.take<int>(size_t(v.G));
  t.xq_stage = c.take<char>(size_t(v.S) * v.d * type_size(v.dtype));
  t.d_status = c.take<long long>(kStCount);
  Carver w;
  w.base = base ? base + ((c.used + 255) & ~size_t(255)) : nullptr;
  Buffers b;
  const size_t ws = carve(w, shmax, b, sm_count, v.prec);
  if (sl) {
    const Slot keep = *sl;
    *sl = t;
    sl->srv = keep.srv;
    sl->index = keep.index;
    sl->stream = keep.stream;
    sl->mem = keep.mem;
    sl->h_status = keep.h_status;
    sl->b = b;
  }
  return ((c.used + 255) & ~size_t(255)) + ws;
}

// Layer-0 marks of a request's union rows (queries first, gallery row g at
// union row Q + g): h0 changed when the row of A* differs from the gallery
// graph's, msgchg when the message list (sources or weights) differs.
__global__ void k_mark_h0(int64_t n, int64_t Q, const int64_t* __restrict__ st, const int32_t* __restrict__ ln,
                          const int32_t* __restrict__ cl, const float* __restrict__ vl,
                          const int64_t* __restrict__ rst, const int32_t* __restrict__ rln,
                          const int32_t* __restrict__ rcl, const float* __restrict__ rvl,
                          const int32_t* __restrict__ nbr, const float* __restrict__ nbr_w,
                          const int32_t* __restrict__ nbr_n, const int32_t* __restrict__ rnbr,
                          const float* __restrict__ rnbr_w, const int32_t* __restrict__ rnbr_n, int k2p1,
                          const uint8_t* __restrict__ aff, uint8_t* __restrict__ h0chg,
                          uint8_t* __restrict__ msgchg) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < Q) {
    h0chg[i] = 1;
    msgchg[i] = 1;
    return;
  }
  const int64_t g = i - Q;
  const int m = nbr_n[i];
  bool mc = m != rnbr_n[g];
  for (int q = 0; q < m && !mc; ++q)
    mc = nbr[i * k2p1 + q] != rnbr[g * k2p1 + q] + Q || nbr_w[i * k2p1 + q] != rnbr_w[g * k2p1 + q];
  // Rows the incremental graph did not rebuild (aff clear) are resident copies.
  const int len = ln[i];
  bool hc = len != rln[g];
  const int64_t a = st[i], ra = rst[g];
  if (!aff || aff[i])
    for (int p = 0; p < len && !hc; ++p) hc = cl[a + p] != rcl[ra + p] + Q || vl[a + p] != rvl[ra + p];
  h0chg[i] = hc ? 1 : 0;
  msgchg[i] = mc ? 1 : 0;
}

// Marks of the next layer: a row's output changes when its message list or a
// source's row of the previous layer did.
__global__ void k_mark_next(int64_t n, const uint8_t* __restrict__ prev, const uint8_t* __restrict__ msgchg,
                            const int32_t* __restrict__ nbr, const int32_t* __restrict__ nbr_n, int k2p1,
                            uint8_t* __restrict__ next, long long* __restrict__ status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  bool c = false;
  if (i < n) {
    c = msgchg[i] != 0;
    const int m = nbr_n[i];
    for (int q = 0; q < m && !c; ++q) c = prev[nbr[i * k2p1 + q]] != 0;
    next[i] = c ? 1 : 0;
  }
  const unsigned bal = __ballot_sync(kFull, c);
  if ((threadIdx.x & 31) == 0 && bal)
    atomicAdd(reinterpret_cast<unsigned long long*>(status + kStRecomputed), (unsigned long long)__popc(bal));
}

__global__ void k_iota(int32_t* p, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = int32_t(i);
}

// Device-to-device copy of a block of rows (source and destination rows are contiguous).
void copy_rows(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

// The queries' bounds move to their rows of X_u; maxima over X_u; Q for the refinement.
__global__ void k_serve_prep(const float* __restrict__ err_q, int64_t Q, float* __restrict__ err_u,
                             int64_t stride, const float* __restrict__ emax_q, const float* __restrict__ emax_g,
                             float* __restrict__ emax_u, int32_t* __restrict__ scal) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < Q)
    for (int k = 0; k < 3; ++k) err_u[k * stride + r] = err_q[k * Q + r];
  if (r < 4) emax_u[r] = fmaxf(emax_q[r], emax_g[r]);
  if (r == 0) scal[0] = int32_t(Q);
}

// One warp per gallery row: keep the resident exact list, or merge the
// candidate lists of a row that a query may enter (see step 3 above).
constexpr int AWPB = 8;
__global__ void __launch_bounds__(AWPB * kWarp)
k_serve_assemble(int64_t G, int64_t Q, int K, int k1, int Pb, const float* __restrict__ res_s,
                 const int32_t* __restrict__ res_i, const int32_t* __restrict__ res_knn_idx,
                 const float* __restrict__ res_knn_score, const float* __restrict__ pb_s,
                 const int32_t* __restrict__ pb_i, const float* __restrict__ err_u, const float* __restrict__ emax_q,
                 double eps_acc, double eps_r, int32_t* __restrict__ knn_idx, float* __restrict__ knn_score,
                 float* __restrict__ pm_s, int32_t* __restrict__ pm_i, int32_t* __restrict__ touched,
                 int32_t* __restrict__ n_touched, long long* status) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = int64_t(blockIdx.x) * AWPB + wib;
  if (g >= G) return;
  const int64_t u = Q + g;  // the row's index in X_u
  // Best approximate score of any query column (each list is sorted, best first).
  float bq = -FLT_MAX;
  for (int p = 0; p < Pb; ++p) {
    const size_t o = (size_t(g) * Pb + p) * K;
    if (pb_i[o] != kInvalidIdx) bq = fmaxf(bq, pb_s[o]);
  }
  // |approximate - S| for this row against any query: one quantised copy on each side.
  const double ei = err_u[u], eq = emax_q[0];
  const double eps_q = eps_acc + ei + eq + ei * eq;
  const double sk = res_knn_score[size_t(g) * k1 + k1 - 1];
  const bool hit = bq != -FLT_MAX && double(bq) + eps_q >= sk - eps_r;
  if (!hit) {
    for (int r = lane; r < k1; r += kWarp) {
      knn_idx[size_t(u) * k1 + r] = res_knn_idx[size_t(g) * k1 + r] + int32_t(Q);
      knn_score[size_t(u) * k1 + r] = res_knn_score[size_t(g) * k1 + r];
    }
    return;
  }
  int pos = 0;
  if (lane == 0) {
    pos = atomicAdd(n_touched, 1);
    touched[pos] = int32_t(u);
    atomicAdd(reinterpret_cast<unsigned long long*>(status + kStTouched), 1ull);
  }
  pos = __shfl_sync(kFull, pos, 0);
  if (lane != 0) return;
  // Merge (1 + Pb) sorted lists into the K best by (score desc, index asc).
  int head[1 + kMaxQueryLists] = {};
  const int L = 1 + Pb;
  for (int e = 0; e < K; ++e) {
    int best = -1;
    float bs = -FLT_MAX;
    int bi = kInvalidIdx;
    for (int l = 0; l < L; ++l) {
      if (head[l] >= K) continue;
      float s;
      int c;
      if (l == 0) {
        s = res_s[size_t(g) * K + head[0]];
        c = res_i[size_t(g) * K + head[0]];
        if (c != kInvalidIdx) c += int(Q);
      } else {
        const size_t o = (size_t(g) * Pb + (l - 1)) * K + head[l];
        s = pb_s[o];
        c = pb_i[o];
      }
      if (c == kInvalidIdx) continue;
      if (best < 0 || ranks_before(s, c, bs, bi)) {
        best = l;
        bs = s;
        bi = c;
      }
    }
    if (best >= 0) ++head[best];
    pm_s[size_t(pos) * K + e] = best >= 0 ? bs : -FLT_MAX;
    pm_i[size_t(pos) * K + e] = best >= 0 ? bi : kInvalidIdx;
  }
}

// K best of P sorted lists per row (the gallery's candidate lists after load).
__global__ void __launch_bounds__(AWPB * kWarp)
k_merge_parts(int64_t n, int P, int K, const float* __restrict__ ps, const int32_t* __restrict__ pi,
              float* __restrict__ out_s, int32_t* __restrict__ out_i) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = int64_t(blockIdx.x) * AWPB + wib;
  if (r >= n) return;
  const size_t base = size_t(r) * P * K;
  int head = 0;  // lane p walks list p
  for (int e = 0; e < K; ++e) {
    float s = -FLT_MAX;
    int c = kInvalidIdx;
    if (lane < P && head < K) {
      s = ps[base + size_t(lane) * K + head];
      c = pi[base + size_t(lane) * K + head];
    }
    float bs = s;
    int bc = c, bl = c == kInvalidIdx ? 64 : lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(kFull, bs, o);
      const int oc = __shfl_xor_sync(kFull, bc, o);
      const int ol = __shfl_xor_sync(kFull, bl, o);
      const bool take = (ol != 64) && (bl == 64 || ranks_before(os, oc, bs, bc));
      if (take) {
        bs = os;
        bc = oc;
        bl = ol;
      }
    }
    if (lane == bl) ++head;
    if (lane == 0) {
      out_s[size_t(r) * K + e] = bl == 64 ? -FLT_MAX : bs;
      out_i[size_t(r) * K + e] = bl == 64 ? kInvalidIdx : bc;
    }
  }
}

void CUDART_CB on_done(void* p) {
  Slot* sl = static_cast<Slot*>(p);
  Server* v = sl->srv;
  std::lock_guard<std::mutex> lk(v->mu);
  sl->t_done = Clock::now();
  v->finished.push_back(sl->index);
  v->cv.notify_all();
}

// Enqueue one request on its slot.  No host synchronisation.
rerank_status enqueue_request(Server& v, Slot& sl, const rerank_request& rq, cudaEvent_t ready) {
  nvtxRangePushA("rerank request");
  struct PopRange {
    ~PopRange() { nvtxRangePop(); }
  } pop_range;
  rerank_ctx* ctx = v.ctx;
  const int64_t Q = rq.nq, G = v.G, n = G + Q, base = v.S - Q;
  const int64_t topk = rq.topk_out ? rq.topk_out : G;
  const bool host_out = is_host_ptr(rq.out_idx) || is_host_ptr(rq.out_dist);
  Shape sh;
  // The resident lists were made with the context's rescore_m: requests use it too.
  Tuning tq = lookup_tuning(ctx, v.prec, G + Q, v.d);
  tq.rescore_m = -1;
  rerank_status st =
      plan_shape(ctx, Q, G, v.d, v.dtype, v.k1, v.k2, v.layers, topk, false, false, host_out, 0, &sh, &tq);
  if (st != RERANK_OK) return st;
  sh.ext_feat = true;
  sh.cap_h = v.cap_h;
  const bool fp8 = v.prec == RERANK_PREC_FP8;
  const size_t es = esize(v.prec), dp = size_t(v.dp);
  Buffers b = sl.b;
  b.xhat = sl.xhat + size_t(base) * dp;
  b.xlow = static_cast<char*>(sl.xlow) + size_t(base) * dp * es;
  b.xhi = sl.xhi + size_t(base) * dp;
  b.xlo = sl.xlo + size_t(base) * dp;
  b.xscale = sl.xscale + base;
  b.norm = sl.norm + base;
  b.err = sl.err + base;
  b.emax = sl.emax;
  cudaStream_t s = sl.stream;
  long long* status = sl.d_status;
  const int sm = ctx->sm_count;
  if (ready) RR_CUDA(cudaStreamWaitEvent(s, ready, 0));

  launch_status_reset(status, s);
  RR_CUDA(cudaMemsetAsync(b.fb_count, 0, sizeof(int32_t), s));
  RR_CUDA(cudaMemsetAsync(b.fb2_count, 0, sizeof(int32_t), s));
  RR_CUDA(cudaMemsetAsync(sl.scal, 0, 4 * sizeof(int32_t), s));
  const void* dq = rq.xq;
  if (is_host_ptr(rq.xq)) {
    RR_CUDA(cudaMemcpyAsync(sl.xq_stage, rq.xq, size_t(Q) * v.d * type_size(v.dtype), cudaMemcpyHostToDevice, s));
    dq = sl.xq_stage;
  }
  // 1. the queries' unit rows and copies, straight into their rows of X_u
  Shape shq = sh;
  shq.nq = Q;
  shq.ng = 0;
  shq.n = Q;
  shq.np = Q;
  launch_normalize(shq, dq, dq, b.xhat, b.norm, b.xlow, b.xhi, b.xlo, b.xscale, sl.err_q, sl.emax_q, v.prec, status,
                   s);
  k_serve_prep<<<unsigned((Q + 255) / 256), 256, 0, s>>>(sl.err_q, Q, b.err, v.rowstride, sl.emax_q, v.res_emax,
                                                         sl.emax, sl.scal);
  ErrModel em;
  em.kind = 1;
  em.err = b.err;
  em.emax = b.emax;
  em.np = v.rowstride;
  em.eps = (v.dp / 16 + 32) * 2.0 * kU32 + 8.0 * kU32;
  // 2. query rows against X_u; gallery rows against the queries
  const int lpc = tc_lists_per_chunk(v.dp, 1);
  const int pa = std::min(choose_chunks((Q + 127) / 128, sh.np / 256, sm, sh.tune.sim_chunks), 32 / lpc);
  const int pb = int((Q + 255) / 256);  // chunks; the lists per row are lpc times as many
  char* xl = static_cast<char*>(b.xlow);
  if (launch_sim_tc_rect_topk(sh, xl, Q, 0, xl, n, 0, pa, fp8, b.xscale, sl.floor_a, sl.pa_s, sl.pa_i, status, sm,
                              s) < 0)
    return RERANK_ECUDA;
  if (launch_sim_tc_rect_topk(sh, xl + size_t(Q) * dp * es, G, Q, xl, Q, 0, pb, fp8, b.xscale, sl.floor_b, sl.pb_s,
                              sl.pb_i, status, sm, s) < 0)
    return RERANK_ECUDA;
  // 3. resident or re-derived gallery lists
  const double eps_r = rescore_eps(v.dp);
  k_serve_assemble<<<unsigned((G + AWPB - 1) / AWPB), AWPB * kWarp, 0, s>>>(
      G, Q, v.K, v.k1, pb * lpc, v.res_s, v.res_i, v.res_knn_idx, v.res_knn_score, sl.pb_s, sl.pb_i, b.err, sl.emax_q,
      em.eps, eps_r, b.knn_idx, b.knn_score, sl.pm_s, sl.pm_i, sl.touched, sl.scal + 1, status);
  // 4. refinement of the query rows and of the touched gallery rows
  const void* dg = v.xg_raw;
  launch_refine(sh, dq, dg, b.xhat, b.norm, sl.pa_s, sl.pa_i, pa * lpc, em, sl.iota, sl.scal, true, b.knn_idx,
                b.knn_score, b.fb_rows, b.fb_count, status, s, Q);
  launch_refine(sh, dq, dg, b.xhat, b.norm, sl.pm_s, sl.pm_i, 1, em, sl.touched, sl.scal + 1, false, b.knn_idx,
                b.knn_score, b.fb_rows, b.fb_count, status, s, G);
  // recheck of uncertified rows with the hi/lo split, then the exact scan
  launch_gather_rows(b.fb_rows, b.fb_count, b.xhi, b.xlo, b.ahi, b.alo, n, v.dp, s);
  if (launch_sim_tc_split_topk(sh, sh.P3, b.ahi, b.alo, b.xhi, b.xlo, b.fb_rows, b.fb_count, b.row_floor3,
                               b.part3_s, b.part3_i, status, sm, s) < 0)
    return RERANK_ECUDA;
  ErrModel e3 = em;
  e3.kind = 2;
  e3.eps = (3 * (v.dp / 16) + 32) * 2.0 * kU32 + 8.0 * kU32;
  launch_refine(sh, dq, dg, b.xhat, b.norm, b.part3_s, b.part3_i, sh.P3, e3, b.fb_rows, b.fb_count, false, b.knn_idx,
                b.knn_score, b.fb2_rows, b.fb2_count, status, s);
  float* fb_s = reinterpret_cast<float*>(b.scan_tmp);
  int32_t* fb_i = reinterpret_cast<int32_t*>(fb_s + size_t(sm) * fallback_warps() * fallback_k(sh));
  launch_refine_fallback(sh, dq, dg, b.xhat, b.norm, b.knn_idx, b.knn_score, b.fb2_rows, b.fb2_count, fb_s, fb_i,
                         status, sm, s);
  // 5. graph, propagation, ranking on X_u.  With the gallery's own graph kept,
  // only the rows of A* the request can change are built (aff marks them).
  uint8_t* aff = nullptr;
  if (v.reuse && ctx->cfg.feature_mode == RERANK_FEAT_ASTAR) {
    aff = reinterpret_cast<uint8_t*>(b.label);  // 4n bytes, free once the refinement is done
    const Server::ResLayer& r0 = v.res_layers[0];
    launch_graph_incremental(sh, b, Q, sl.touched, sl.scal + 1, v.res_knn_idx, r0.start, r0.len, r0.col, r0.val, aff,
                             aff + n, ctx->cfg.alpha, ctx->cfg.aggregator, status, s);
  } else {
    launch_graph(sh, b, ctx->cfg.alpha, ctx->cfg.aggregator, ctx->cfg.feature_mode, status, s);
  }
  RR_CUDA(cudaMemsetAsync(b.hash_keys_vals, 0, sizeof(float) * size_t(sm) * (size_t(n) + size_t((n + 31) / 32)), s));
  const int k2p1 = v.k2 + 1;
  const unsigned mg = unsigned((n + 255) / 256);
  if (v.reuse) {
    const Server::ResLayer& r0 = v.res_layers[0];
    k_mark_h0<<<mg, 256, 0, s>>>(n, Q, b.start[2], b.len[2], b.col[2], b.val[2], r0.start, r0.len, r0.col, r0.val,
                                 b.nbr, b.nbr_w, b.nbr_n, v.res_nbr, v.res_nbr_w, v.res_nbr_n, k2p1, aff, sl.chg[0],
                                 sl.msgchg);
  }
  int src = 2;
  for (int l = 0; l < v.layers; ++l) {
    const int dst = l & 1;
    LayerReuse ru;
    if (v.reuse) {
      k_mark_next<<<mg, 256, 0, s>>>(n, sl.chg[l & 1], sl.msgchg, b.nbr, b.nbr_n, k2p1, sl.chg[(l + 1) & 1],
                                     status);
      const Server::ResLayer& rl = v.res_layers[size_t(l) + 1];
      ru.changed = sl.chg[(l + 1) & 1];
      ru.rstart = rl.start;
      ru.rlen = rl.len;
      ru.rcol = rl.col;
      ru.rval = rl.val;
      ru.shift = Q;
    }
    launch_propagate(sh, b, src, dst, ctx->cfg.aggregator, status, sm, sh.tune, s, v.reuse ? &ru : nullptr);
    src = dst;
  }
  // With the gallery graph kept, only the rows whose last layer changed (the
  // queries among them) need their norm: the others' are in the resident lists.
  launch_row_norms(sh, b, src, status, s, v.reuse ? sl.chg[v.layers & 1] : nullptr);
  int32_t* oi = host_out ? b.out_idx : rq.out_idx;
  float* od = host_out ? b.out_dist : rq.out_dist;
  if (v.reuse) {
    // the gallery rows of the last layer that changed get new column lists;
    // the others' entries come from the gallery graph's own lists
    const uint8_t* last = sl.chg[v.layers & 1];
    RankReuse rr;
    rr.colptr = v.res_colptr;
    rr.row = v.res_csc_row;
    rr.val = v.res_csc_val;
    rr.changed = last + Q;
    rr.shift = Q;
    launch_rank_prep(sh, b, src, status, s, last);
    launch_rank_queries(sh, b, src, oi, od, 0, Q, status, sm, sh.tune, s, &rr);
  } else {
    launch_rank(sh, b, src, oi, od, status, sm, sh.tune, s);
  }
  if (host_out) {
    const size_t cnt = size_t(Q) * size_t(topk);
    RR_CUDA(cudaMemcpyAsync(rq.out_idx, b.out_idx, cnt * 4, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaMemcpyAsync(rq.out_dist, b.out_dist, cnt * 4, cudaMemcpyDeviceToHost, s));
  }
  RR_CUDA(cudaMemcpyAsync(sl.h_status, status, sizeof(long long) * kStCount, cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaGetLastError());
  RR_CUDA(cudaLaunchHostFunc(s, on_done, &sl));
  return RERANK_OK;
}

void worker_loop(Server* v) {
  cudaSetDevice(v->ctx->device);
  std::unique_lock<std::mutex> lk(v->mu);
  for (;;) {
    v->cv.wait(lk, [&] {
      if (!v->finished.empty()) return true;
      if (v->stop && v->queue.empty() && v->in_flight == 0) return true;
      if (v->queue.empty()) return false;
      for (const Slot& s : v->slots)
        if (!s.busy) return true;
      return false;
    });
    // Retire the slots whose work completed.
    for (int si : v->finished) {
      Slot& sl = v->slots[size_t(si)];
      auto it = v->reqs.find(sl.ticket);
      if (it != v->reqs.end()) {
        rerank_info inf{};
        int64_t need = 0;
        rerank_status st = map_status(sl.h_status, v->prec, &inf, &need);
        it->second.status = st;
        it->second.t_done = sl.t_done;
        it->second.done = true;
      }
      v->touched_rows += sl.h_status[kStTouched];
      v->recomputed_rows += sl.h_status[kStRecomputed];
      sl.busy = false;
      --v->in_flight;
      ++v->completed;
    }
    if (!v->finished.empty()) v->cv.notify_all();
    v->finished.clear();
    // Admit queued requests into free slots.
    for (Slot& sl : v->slots) {
      if (v->queue.empty()) break;
      if (sl.busy) continue;
      const uint64_t t = v->queue.front();
      v->queue.pop_front();
      Pending& p = v->reqs[t];
      sl.busy = true;
      sl.ticket = t;
      p.slot = sl.index;
      p.t_start = Clock::now();
      ++v->in_flight;
      v->max_in_flight = std::max(v->max_in_flight, v->in_flight);
      const rerank_request rq = p.req;
      const cudaEvent_t ready = p.ready;
      lk.unlock();
      rerank_status st = enqueue_request(*v, sl, rq, ready);
      if (st != RERANK_OK) cudaStreamSynchronize(sl.stream);
      lk.lock();
      if (st != RERANK_OK) {
        Pending& q = v->reqs[t];
        q.status = st;
        q.t_done = Clock::now();
        q.done = true;
        sl.busy = false;
        --v->in_flight;
        ++v->completed;
        v->cv.notify_all();
      }
    }
    if (v->stop && v->queue.empty() && v->in_flight == 0) break;
  }
}

void free_server(Server* v) {
  for (Slot& s : v->slots) {
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.mem) cudaFree(s.mem);
    if (s.h_status) cudaFreeHost(s.h_status);
  }
  if (v->res_mem) cudaFree(v->res_mem);
  for (void* p : v->res_extra) cudaFree(p);
  delete v;
}

}  // namespace

rerank_status serve_stop(rerank_ctx* ctx) {
  Server* v = reinterpret_cast<Server*>(ctx->serve);
  if (!v) return RERANK_OK;
  {
    std::lock_guard<std::mutex> lk(v->mu);
    v->stop = true;
    v->cv.notify_all();
  }
  if (v->worker.joinable()) v->worker.join();
  cudaSetDevice(ctx->device);
  for (Slot& s : v->slots)
    if (s.stream) cudaStreamSynchronize(s.stream);
  free_server(v);
  ctx->serve = nullptr;
  return RERANK_OK;
}

// The gallery's own graph (G alone), built on slot 0's buffers at load: the
// message lists and layers 0 .. L, kept as compact CSR.  When they do not fit
// what the HBM budget leaves (budget_left; 0 = no budget), they are dropped
// and requests recompute every row.  Returns a failure only for CUDA errors.
rerank_status build_resident_graph(Server& v, cudaStream_t s0, long long* gst, size_t budget_left) {
  rerank_ctx* ctx = v.ctx;
  const Buffers& b = v.slots[0].b;
  const int64_t G = v.G;
  Shape sg;
  sg.nq = 0;
  sg.ng = G;
  sg.n = G;
  sg.np = G;
  sg.k1 = v.k1;
  sg.k2 = v.k2;
  sg.layers = v.layers;
  sg.cap_h = v.cap_h;
  sg.tune = lookup_tuning(ctx, v.prec, G, v.d);
  const size_t e1 = size_t(G) * size_t(v.k1), k2p1 = size_t(v.k2) + 1;
  copy_rows(b.knn_idx, v.res_knn_idx, e1 * 4, s0);
  copy_rows(b.knn_score, v.res_knn_score, e1 * 4, s0);
  launch_status_reset(gst, s0);
  launch_graph(sg, b, ctx->cfg.alpha, ctx->cfg.aggregator, ctx->cfg.feature_mode, gst, s0);
  RR_CUDA(cudaMemsetAsync(b.hash_keys_vals, 0,
                          sizeof(float) * size_t(ctx->sm_count) * (size_t(G) + size_t((G + 31) / 32)), s0));
  size_t used = 0;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    used += (bytes + 255) & ~size_t(255);
    if (budget_left && used > budget_left) return nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    v.res_extra.push_back(p);
    return p;
  };
  auto drop = [&]() {
    for (void* p : v.res_extra) cudaFree(p);
    v.res_extra.clear();
    v.res_layers.clear();
    v.res_nbr = nullptr;
    v.res_nbr_w = nullptr;
    v.res_nbr_n = nullptr;
    v.res_colptr = nullptr;
    v.res_csc_row = nullptr;
    v.res_csc_val = nullptr;
    v.reuse = false;
  };
  bool ok = true;
  v.res_nbr = static_cast<int32_t*>(alloc(size_t(G) * k2p1 * 4));
  v.res_nbr_w = static_cast<float*>(alloc(size_t(G) * k2p1 * 4));
  v.res_nbr_n = static_cast<int32_t*>(alloc(size_t(G) * 4));
  ok = v.res_nbr && v.res_nbr_w && v.res_nbr_n;
  if (ok) {
    copy_rows(v.res_nbr, b.nbr, size_t(G) * k2p1 * 4, s0);
    copy_rows(v.res_nbr_w, b.nbr_w, size_t(G) * k2p1 * 4, s0);
    copy_rows(v.res_nbr_n, b.nbr_n, size_t(G) * 4, s0);
  }
  auto keep = [&](int layer) -> bool {
    Server::ResLayer r;
    r.start = static_cast<int64_t*>(alloc(size_t(G + 1) * 8));
    r.len = static_cast<int32_t*>(alloc(size_t(G) * 4));
    if (!r.start || !r.len) return false;
    launch_scan(b.len[layer], G, r.start, s0);
    copy_rows(r.len, b.len[layer], size_t(G) * 4, s0);
    int64_t nnz = 0;
    if (cudaMemcpyAsync(&nnz, r.start + G, sizeof(nnz), cudaMemcpyDeviceToHost, s0) != cudaSuccess ||
        cudaStreamSynchronize(s0) != cudaSuccess)
      return false;
    r.col = static_cast<int32_t*>(alloc(size_t(std::max<int64_t>(nnz, 1)) * 4));
    r.val = static_cast<float*>(alloc(size_t(std::max<int64_t>(nnz, 1)) * 4));
    if (!r.col || !r.val) return false;
    launch_layer_compact(G, b.start[layer], b.len[layer], b.col[layer], b.val[layer], r.start, r.col, r.val, s0);
    v.res_layers.push_back(r);
    return true;
  };
  ok = ok && keep(2);  // layer 0: the rows of A* (or A)
  int src = 2;
  for (int l = 0; ok && l < v.layers; ++l) {
    const int dst = l & 1;
    launch_propagate(sg, b, src, dst, ctx->cfg.aggregator, gst, ctx->sm_count, sg.tune, s0);
    ok = keep(dst);
    src = dst;
  }
  if (ok) {
    // the last layer's column lists, as the ranking uses them
    launch_row_norms(sg, b, src, gst, s0);
    launch_rank_prep(sg, b, src, gst, s0);
    int64_t nnz = 0;
    v.res_colptr = static_cast<int64_t*>(alloc(size_t(G + 1) * 8));
    ok = v.res_colptr != nullptr;
    if (ok) {
      copy_rows(v.res_colptr, b.colptr, size_t(G + 1) * 8, s0);
      ok = cudaMemcpyAsync(&nnz, b.colptr + G, sizeof(nnz), cudaMemcpyDeviceToHost, s0) == cudaSuccess &&
           cudaStreamSynchronize(s0) == cudaSuccess;
    }
    if (ok) {
      v.res_csc_row = static_cast<int32_t*>(alloc(size_t(std::max<int64_t>(nnz, 1)) * 4));
      v.res_csc_val = static_cast<float*>(alloc(size_t(std::max<int64_t>(nnz, 1)) * 4));
      ok = v.res_csc_row && v.res_csc_val;
    }
    if (ok) {
      copy_rows(v.res_csc_row, b.csc_row, size_t(nnz) * 4, s0);
      copy_rows(v.res_csc_val, b.csc_val, size_t(nnz) * 4, s0);
    }
  }
  long long hst[kStCount];
  RR_CUDA(cudaMemcpyAsync(hst, gst, sizeof(hst), cudaMemcpyDeviceToHost, s0));
  RR_CUDA(cudaStreamSynchronize(s0));
  RR_CUDA(cudaGetLastError());
  if (!ok || hst[kStErr] != 0) {
    drop();
    return RERANK_OK;
  }
  v.reuse = true;
  v.resident_bytes += used;
  return RERANK_OK;
}

rerank_status serve_load(rerank_ctx* ctx, const void* xg, int64_t ng, int d, int dtype,
                         const rerank_serve_config* sc) {
  const int prec = ctx->cfg.precision;
  if (prec == RERANK_PREC_FP32) return RERANK_EUNSUPPORTED;
  if (ctx->serve) return RERANK_EUNSUPPORTED;
  if (ctx->cfg.feature_mode == RERANK_FEAT_X) return RERANK_EUNSUPPORTED;  // dense features: rerank_run only
  const int64_t S = sc->max_query;
  const int k1 = sc->k1, k2 = sc->k2, layers = sc->layers;
  rerank_status st = rerank_check_args(S, ng, d, dtype, k1, k2, layers, 0);
  if (st != RERANK_OK) return st;
  if (ng < int64_t(k1) + ctx->cfg.rescore_m || sc->slots < 0 || S > kMaxQuery) return RERANK_EINVAL;
  RR_CUDA(cudaSetDevice(ctx->device));

  Server* v = new Server();
  v->ctx = ctx;
  v->G = ng;
  v->S = S;
  v->rowstride = S + ng + kPad;
  v->d = d;
  v->dtype = dtype;
  v->k1 = k1;
  v->k2 = k2;
  v->layers = layers;
  v->prec = prec;
  // 1. the gallery's own exact neighbour lists: the rerank_knn pipeline on G
  Shape shg;
  Tuning tg = lookup_tuning(ctx, prec, ng, d);
  tg.rescore_m = -1;
  st = plan_shape(ctx, ng, 0, d, dtype, k1, 1, 0, 0, true, false, false, 0, &shg, &tg);
  if (st != RERANK_OK) {
    delete v;
    return st;
  }
  v->dp = shg.dp;
  v->K = shg.K;
  Shape shmax;
  Tuning tm = lookup_tuning(ctx, prec, S + ng, d);
  tm.rescore_m = -1;
  st = plan_shape(ctx, S, ng, d, dtype, k1, k2, layers, ng, false, false, true, 0, &shmax, &tm);
  if (st != RERANK_OK) {
    delete v;
    return st;
  }
  if (shmax.K != v->K) {  // both are k1 + rescore_m once ng >= k1 + rescore_m
    delete v;
    return RERANK_EINTERNAL;
  }
  shmax.ext_feat = true;
  v->cap_h = shmax.cap_h;
  Buffers bg;
  Carver dry;
  const size_t gws = carve(dry, shg, bg, ctx->sm_count, prec);
  const size_t raw = size_t(ng) * d * type_size(dtype);
  Carver rc;
  rc.take<char>(raw);
  rc.take<float>(size_t(ng) * v->K);
  rc.take<int32_t>(size_t(ng) * v->K);
  rc.take<int32_t>(size_t(ng) * k1);
  rc.take<float>(size_t(ng) * k1);
  rc.take<float>(4);
  v->resident_bytes = rc.used;
  v->slot_bytes = slot_layout(*v, nullptr, nullptr, shmax, ctx->sm_count);
  const size_t budget = ctx->cfg.hbm_budget;
  // The gallery's temporary workspace is freed before the slots are made.
  int nslots = sc->slots ? std::min(sc->slots, kMaxSlots) : kMaxSlots;
  if (budget) {
    // The gallery's temporary workspace lives until the slots hold their copies.
    if (v->resident_bytes + gws + v->slot_bytes > budget) {
      delete v;
      return RERANK_EBUDGET;
    }
    nslots = int(std::min<size_t>(size_t(nslots), (budget - v->resident_bytes - gws) / v->slot_bytes));
  }
  if (cudaMalloc(&v->res_mem, v->resident_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete v;
    return RERANK_ENOMEM;
  }
  rc.base = v->res_mem;
  rc.used = 0;
  v->xg_raw = rc.take<char>(raw);
  v->res_s = rc.take<float>(size_t(ng) * v->K);
  v->res_i = rc.take<int32_t>(size_t(ng) * v->K);
  v->res_knn_idx = rc.take<int32_t>(size_t(ng) * k1);
  v->res_knn_score = rc.take<float>(size_t(ng) * k1);
  v->res_emax = rc.take<float>(4);
  auto fail = [&](rerank_status e) {
    free_server(v);
    return e;
  };
  cudaStream_t s0 = nullptr;
  if (cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess) return fail(RERANK_ECUDA);
  char* gmem = nullptr;
  long long* gst = nullptr;
  long long hst[kStCount];
  rerank_status res = RERANK_OK;
  do {
    if (cudaMemcpyAsync(v->xg_raw, xg, raw, cudaMemcpyDefault, s0) != cudaSuccess) {
      res = RERANK_ECUDA;
      break;
    }
    if (cudaMalloc(&gmem, gws) != cudaSuccess || cudaMalloc(&gst, sizeof(long long) * kStCount) != cudaSuccess) {
      res = RERANK_ENOMEM;
      break;
    }
    JobRun j;
    j.sh = shg;
    Carver gc;
    gc.base = gmem;
    carve(gc, shg, j.b, ctx->sm_count, prec);
    j.st = gst;
    j.xq = v->xg_raw;
    j.xg = v->xg_raw;
    j.out_idx = v->res_knn_idx;
    j.out_dist = v->res_knn_score;
    int64_t nl = 0;
    res = enqueue_job(ctx, j, s0, nullptr, &nl);
    if (res != RERANK_OK) break;
    k_merge_parts<<<unsigned((ng + AWPB - 1) / AWPB), AWPB * kWarp, 0, s0>>>(ng, shg.P, v->K, j.b.part_s,
                                                                              j.b.part_i, v->res_s, v->res_i);
    cudaMemcpyAsync(v->res_emax, j.b.emax, 4 * sizeof(float), cudaMemcpyDeviceToDevice, s0);
    cudaMemcpyAsync(hst, gst, sizeof(hst), cudaMemcpyDeviceToHost, s0);
    if (cudaStreamSynchronize(s0) != cudaSuccess) {
      res = RERANK_ECUDA;
      break;
    }
    rerank_info inf{};
    int64_t need = 0;
    res = map_status(hst, prec, &inf, &need);
    if (res != RERANK_OK) break;
    // 2. the slots, each with its own copy of the gallery's rows of X_u
    v->slots.reserve(size_t(nslots));
    for (int k = 0; k < nslots && res == RERANK_OK; ++k) {
      v->slots.emplace_back();
      Slot& sl = v->slots.back();
      sl.srv = v;
      sl.index = k;
      if (cudaMalloc(&sl.mem, v->slot_bytes) != cudaSuccess ||
          cudaMallocHost(&sl.h_status, sizeof(long long) * kStCount) != cudaSuccess ||
          cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (sl.mem) cudaFree(sl.mem);
        if (sl.h_status) cudaFreeHost(sl.h_status);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        v->slots.pop_back();
        if (k == 0) res = RERANK_ENOMEM;
        break;
      }
      slot_layout(*v, &sl, sl.mem, shmax, ctx->sm_count);
      const size_t dp = size_t(v->dp), es = esize(prec), gS = size_t(S), gN = size_t(ng);
      // zero pad rows after the gallery
      cudaMemsetAsync(sl.xhat + (gS + gN) * dp, 0, size_t(kPad) * dp * 4, s0);
      cudaMemsetAsync(static_cast<char*>(sl.xlow) + (gS + gN) * dp * es, 0, size_t(kPad) * dp * es, s0);
      if (prec == RERANK_PREC_FP8) cudaMemsetAsync(sl.xhi + (gS + gN) * dp, 0, size_t(kPad) * dp * 2, s0);
      cudaMemsetAsync(sl.xlo + (gS + gN) * dp, 0, size_t(kPad) * dp * 2, s0);
      copy_rows(sl.xhat + gS * dp, j.b.xhat, gN * dp * 4, s0);
      copy_rows(static_cast<char*>(sl.xlow) + gS * dp * es, j.b.xlow, gN * dp * es, s0);
      if (prec == RERANK_PREC_FP8) copy_rows(sl.xhi + gS * dp, j.b.xhi, gN * dp * 2, s0);
      copy_rows(sl.xlo + gS * dp, j.b.xlo, gN * dp * 2, s0);
      copy_rows(sl.xscale + gS, j.b.xscale, gN * 4, s0);
      copy_rows(sl.norm + gS, j.b.norm, gN * 8, s0);
      for (int e = 0; e < 3; ++e)
        copy_rows(sl.err + size_t(e) * size_t(v->rowstride) + gS, j.b.err + size_t(e) * size_t(shg.np), gN * 4, s0);
      k_iota<<<unsigned((S + 255) / 256), 256, 0, s0>>>(sl.iota, S);
    }
    if (res != RERANK_OK) break;
    if (cudaStreamSynchronize(s0) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      res = RERANK_ECUDA;
      break;
    }
    // 3. the gallery's own graph and layers, for the rows a request leaves unchanged
    size_t left = 0;
    if (budget) {
      const size_t spent = v->resident_bytes + gws + v->slots.size() * v->slot_bytes;
      left = budget > spent ? budget - spent : 1;
    }
    res = build_resident_graph(*v, s0, gst, left);
  } while (false);
  if (gmem) cudaFree(gmem);
  if (gst) cudaFree(gst);
  cudaStreamDestroy(s0);
  if (res != RERANK_OK) return fail(res);
  ctx->serve = reinterpret_cast<ServeHandle*>(v);
  v->worker = std::thread(worker_loop, v);
  return RERANK_OK;
}

rerank_status serve_submit(rerank_ctx* ctx, const rerank_request* rq, uint64_t* ticket) {
  Server* v = reinterpret_cast<Server*>(ctx->serve);
  if (!v) return RERANK_EUNSUPPORTED;
  if (!rq || !ticket || !rq->xq || !rq->out_idx || !rq->out_dist) return RERANK_EINVAL;
  if (rq->nq < 1 || rq->nq > v->S || rq->topk_out < 0 || rq->topk_out > v->G) return RERANK_EINVAL;
  // Order the request after the caller's work on its stream.
  RR_CUDA(cudaSetDevice(ctx->device));
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ready, static_cast<cudaStream_t>(rq->stream)) != cudaSuccess) {
    cudaGetLastError();
    if (ready) cudaEventDestroy(ready);
    return RERANK_ECUDA;
  }
  std::lock_guard<std::mutex> lk(v->mu);
  if (v->stop) {
    cudaEventDestroy(ready);
    return RERANK_EUNSUPPORTED;
  }
  const uint64_t t = v->next++;
  Pending& p = v->reqs[t];
  p.req = *rq;
  p.ready = ready;
  p.t_submit = Clock::now();
  v->queue.push_back(t);
  *ticket = t;
  v->cv.notify_all();
  return RERANK_OK;
}

rerank_status serve_wait(rerank_ctx* ctx, uint64_t ticket, int timeout_ms, rerank_ticket_info* info) {
  Server* v = reinterpret_cast<Server*>(ctx->serve);
  if (!v) return RERANK_EUNSUPPORTED;
  std::unique_lock<std::mutex> lk(v->mu);
  auto it = v->reqs.find(ticket);
  if (it == v->reqs.end()) return RERANK_EINVAL;
  auto ready = [&] { return v->reqs[ticket].done; };
  if (timeout_ms < 0)
    v->cv.wait(lk, ready);
  else if (!v->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return RERANK_EAGAIN;
  Pending& p = v->reqs[ticket];
  const rerank_status st = p.status;
  if (p.ready) cudaEventDestroy(p.ready);
  if (info) {
    info->status = st;
    info->queue_ms = p.slot >= 0 ? ms_between(p.t_submit, p.t_start) : 0.0;
    info->total_ms = ms_between(p.t_submit, p.t_done);
    info->slot = p.slot;
  }
  v->reqs.erase(ticket);
  return st;
}

rerank_status serve_info(const rerank_ctx* ctx, rerank_serve_info* info) {
  Server* v = reinterpret_cast<Server*>(ctx->serve);
  if (!v) return RERANK_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(v->mu);
  info->slots = int(v->slots.size());
  info->max_in_flight = v->max_in_flight;
  info->completed = v->completed;
  info->touched_rows = v->touched_rows;
  info->resident_bytes = int64_t(v->resident_bytes);
  info->slot_bytes = int64_t(v->slot_bytes);
  info->reuse_layers = v->reuse ? 1 : 0;
  info->recomputed_rows = v->recomputed_rows;
  return RERANK_OK;
}

}  // namespace rr

using namespace rr;

extern "C" {

rerank_status rerank_gallery_load(rerank_ctx* ctx, const void* xg, int64_t ng, int d, int dtype,
                                  const rerank_serve_config* sc) {
  if (!ctx || !xg || !sc) return RERANK_EINVAL;
  return serve_load(ctx, xg, ng, d, dtype, sc);
}

rerank_status rerank_submit(rerank_ctx* ctx, const rerank_request* req, uint64_t* ticket) {
  if (!ctx) return RERANK_EINVAL;
  return serve_submit(ctx, req, ticket);
}

rerank_status rerank_wait(rerank_ctx* ctx, uint64_t ticket, int timeout_ms, rerank_ticket_info* info) {
  if (!ctx) return RERANK_EINVAL;
  return serve_wait(ctx, ticket, timeout_ms, info);
}

rerank_status rerank_serve_info_get(const rerank_ctx* ctx, rerank_serve_info* info) {
  if (!ctx || !info) return RERANK_EINVAL;
  return serve_info(ctx, info);
}

rerank_status rerank_gallery_unload(rerank_ctx* ctx) {
  if (!ctx) return RERANK_EINVAL;
  return serve_stop(ctx);
}

}  // extern "C"

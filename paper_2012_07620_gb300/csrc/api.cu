// The C ABI (include/rerank.h): argument checks, workspace planning, stage
// sequencing on the caller's stream, and the end-of-call error read-back.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.hpp"

namespace rr {

static thread_local std::string g_last_cuda;

rerank_status cuda_fail(cudaError_t e, const char* what) {
  g_last_cuda = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return RERANK_ENOMEM;
  return RERANK_ECUDA;
}
const char* last_cuda_error_text() { return g_last_cuda.c_str(); }

void StageTimer::mark(const char* name) {
  if (!on) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, stream);
  ev.push_back(e);
  names.push_back(name);
}

double rescore_eps(int dp);
int sim_fp32_kmax();
int refine_kmax();
int fallback_warps();

__global__ void k_status_reset(long long* st) {
  const int t = threadIdx.x;
  if (t < kStCount) st[t] = (t == kStBadRow) ? LLONG_MAX : 0;
}

int launch_status_reset(long long* st, cudaStream_t s) {
  k_status_reset<<<1, 64, 0, s>>>(st);
  return 1;
}

bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int choose_chunks(int64_t row_blocks, int64_t col_tiles, int sm_count, int forced) {
  if (forced > 0) return int(std::min<int64_t>(std::min<int64_t>(forced, 32), col_tiles));
  int best = 1;
  double best_cost = 1e300;
  for (int p = 1; p <= 32 && p <= col_tiles; ++p) {
    const int64_t ctas = row_blocks * p;
    const int64_t waves = (ctas + sm_count - 1) / sm_count;
    const int64_t tiles = (col_tiles + p - 1) / p;
    // Every chunk starts its lists cold (no floor yet): charge it about three tiles.
    const double cost = double(waves) * (double(tiles) + 3.0);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = p;
    }
  }
  return best;
}

size_t type_size(int dtype) { return dtype == RERANK_DTYPE_BF16 ? 2 : 4; }

// Carve every buffer of the run out of one block (dry pass when base == nullptr).
size_t carve(Carver& c, const Shape& sh, Buffers& b, int sm_count, int precision) {
  const int64_t n = sh.n, np = sh.np;
  const int k1 = sh.k1, k2 = sh.k2;
  if (sh.host_in) {
    b.xq = c.take<char>(size_t(sh.nq) * sh.d * type_size(sh.dtype));
    b.xg = c.take<char>(size_t(sh.ng ? sh.ng : 1) * sh.d * type_size(sh.dtype));
  }
  if (sh.host_out) {
    b.out_idx = c.take<int32_t>(size_t(sh.nq) * (sh.knn_only ? k1 : sh.topk));
    b.out_dist = c.take<float>(size_t(sh.nq) * (sh.knn_only ? k1 : sh.topk));
  }
  if (!sh.ext_feat) {
    b.xhat = c.take<float>(size_t(np) * sh.dp);
    b.xlow = precision == RERANK_PREC_FP32
                 ? nullptr
                 : c.take<char>(size_t(np) * sh.dp * (precision == RERANK_PREC_FP8 ? 1 : 2));
    b.xscale = c.take<float>(size_t(np));
    b.err = c.take<float>(3 * size_t(np));
    b.emax = c.take<float>(4);
    b.norm = c.take<double>(size_t(np));
  }
  if (precision != RERANK_PREC_FP32) {
    if (!sh.ext_feat) {
      b.xhi = precision == RERANK_PREC_BF16 ? static_cast<__nv_bfloat16*>(b.xlow)
                                            : c.take<__nv_bfloat16>(size_t(np) * sh.dp);
      b.xlo = c.take<__nv_bfloat16>(size_t(np) * sh.dp);
    }
    b.ahi = c.take<__nv_bfloat16>(size_t(np) * sh.dp);
    b.alo = c.take<__nv_bfloat16>(size_t(np) * sh.dp);
    const size_t p3k = std::max(size_t(sh.P3) * sh.K, size_t(sh.P3g) * sh.K3);
    b.part3_s = c.take<float>(size_t(n) * p3k);
    b.part3_i = c.take<int32_t>(size_t(n) * p3k);
    b.row_floor3 = c.take<int>(size_t(n));
    b.fb2_rows = c.take<int32_t>(size_t(n));
    b.fb2_count = c.take<int32_t>(4);
    b.fb3_rows = c.take<int32_t>(size_t(n));
    b.fb3_count = c.take<int32_t>(4);
  }
  b.row_floor = c.take<int>(size_t(n));
  b.work = c.take<int32_t>(16);
  b.nb4 = c.take<int32_t>(4 * size_t(n));
  b.label = c.take<int32_t>(size_t(n));
  b.order = c.take<int32_t>(size_t(n));
  b.ord_cnt = c.take<int32_t>(size_t(n) + 1);
  b.ord_start = c.take<int32_t>(size_t(n) + 1);
  b.ord_fill = c.take<int32_t>(size_t(n));
  b.part_s = c.take<float>(size_t(n) * sh.P * sh.K);
  b.part_i = c.take<int32_t>(size_t(n) * sh.P * sh.K);
  b.knn_idx = c.take<int32_t>(size_t(n) * k1);
  b.knn_score = c.take<float>(size_t(n) * k1);
  b.fb_rows = c.take<int32_t>(size_t(n));
  b.fb_count = c.take<int32_t>(4);
  // fallback per-warp lists (scores then indices)
  b.scan_tmp = c.take<int64_t>(size_t(sm_count) * fallback_warps() * std::max(sh.K, fallback_k(sh)));
  if (sh.knn_only) return c.used;
  b.indeg = c.take<int32_t>(size_t(n));
  b.fill = c.take<int32_t>(size_t(n));
  b.inptr = c.take<int32_t>(size_t(n) + 1);
  b.insrc = c.take<int32_t>(size_t(n) * k1);
  b.out_sorted = c.take<int32_t>(size_t(n) * k1);
  b.in_sorted = c.take<int32_t>(size_t(n) * k1);
  b.rowcnt = c.take<int32_t>(size_t(n));
  b.h0ptr = c.take<int32_t>(size_t(n) + 1);
  b.nbr = c.take<int32_t>(size_t(n) * (k2 + 1));
  b.nbr_w = c.take<float>(size_t(n) * (k2 + 1));
  b.nbr_n = c.take<int32_t>(size_t(n));
  for (int l = 0; l < 3; ++l) {
    const size_t cap = l < 2 ? size_t(sh.cap_h) : size_t(2) * n * k1;
    b.start[l] = c.take<int64_t>(size_t(n) + 1);
    b.len[l] = c.take<int32_t>(size_t(n));
    b.col[l] = c.take<int32_t>(cap);
    b.val[l] = c.take<float>(cap);
  }
  b.ub = c.take<int32_t>(size_t(n));
  b.big_rows = c.take<int32_t>(size_t(n));
  b.prop_spill = c.take<int32_t>(size_t(n));
  b.big_count = c.take<int32_t>(4);
  b.hash_keys_vals = c.take<float>(size_t(sm_count) * (size_t(n) + size_t((n + 31) / 32)));
  b.rnorm = c.take<float>(size_t(n));
  b.colcnt = c.take<int32_t>(size_t(n) + 1);
  b.colptr = c.take<int64_t>(size_t(n) + 1);
  b.csc_row = c.take<int32_t>(size_t(sh.cap_h));
  b.csc_val = c.take<float>(size_t(sh.cap_h));
  b.rank_scratch = c.take<uint32_t>(size_t(sh.rank_ctas) * size_t(rank_scratch_words(sh.ng)));
  if (sh.dense) {
    b.hd[0] = c.take<float>(size_t(np) * sh.dp);
    b.hd[1] = c.take<float>(size_t(np) * sh.dp);
    b.hinv = c.take<double>(size_t(np));
    b.xscore = c.take<float>(size_t(sh.nq) * size_t(sh.ng));
  }
  return c.used;
}

void free_graph(BatchGraph* g);

// Cached batch graphs hold copy and memset nodes on the workspace and on the
// pinned status block; a new allocation can come back at the same address
// (so a key of pointers would still match), so every graph goes with the old one.
void drop_graphs(rerank_ctx* ctx) {
  for (BatchGraph* g : ctx->graphs) free_graph(g);
  ctx->graphs.clear();
  ctx->graph_seen.clear();
}

rerank_status ensure_workspace(rerank_ctx* ctx, size_t bytes) {
  if (ctx->cfg.hbm_budget && bytes > ctx->cfg.hbm_budget) return RERANK_EBUDGET;
  if (bytes <= ctx->ws_bytes) return RERANK_OK;
  drop_graphs(ctx);
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  const size_t want = bytes + bytes / 8;
  const size_t alloc = (ctx->cfg.hbm_budget && want > ctx->cfg.hbm_budget) ? bytes : want;
  RR_CUDA(cudaMalloc(&ctx->ws, alloc));
  ctx->ws_bytes = alloc;
  return RERANK_OK;
}

rerank_status collect(rerank_ctx* ctx, cudaStream_t s) {
  RR_CUDA(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(long long) * kStCount, cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  RR_CUDA(cudaGetLastError());
  return RERANK_OK;
}

void finish_timing(rerank_ctx* ctx) {
  ctx->stage_ms.clear();
  ctx->stage_names.clear();
  auto& tm = ctx->timer;
  for (size_t i = 1; i < tm.ev.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tm.ev[i - 1], tm.ev[i]);
    ctx->stage_ms.push_back(ms);
    ctx->stage_names.push_back(tm.names[i]);
  }
  for (auto e : tm.ev) cudaEventDestroy(e);
  tm.ev.clear();
  tm.names.clear();
}

// Enqueue every stage of one instance on `s` (no host synchronisation).
cudaError_t ensure_copy_stream(rerank_ctx* ctx) {
  if (ctx->copy_stream) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
  for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) ctx->copy_events.push_back(ev);
  }
  return e;
}

rerank_status enqueue_job(rerank_ctx* ctx, const JobRun& j, cudaStream_t s, StageTimer* tm, int64_t* launches,
                          bool copy_overlap, int phases) {
  const Shape& sh = j.sh;
  const Buffers& b = j.b;
  long long* status = j.st;
  // NVTX: one range per instance on the host timeline, a marker per stage
  // (no-ops unless a profiler is attached).
  nvtxRangePushA("rerank instance");
  struct PopRange {
    ~PopRange() { nvtxRangePop(); }
  } pop_range;
  auto mark = [&](const char* name) {
    nvtxMarkA(name);
    if (tm) tm->mark(name);
  };
  int64_t nl = 0;
  const void* dq = sh.host_in ? b.xq : j.xq;
  const void* dg = sh.host_in ? b.xg : j.xg;
  const int prec = ctx->cfg.precision;
  if (phases & kPhasePre) {
    k_status_reset<<<1, 64, 0, s>>>(status);
    ++nl;
    RR_CUDA(cudaMemsetAsync(b.fb_count, 0, sizeof(int32_t), s));
    if (b.fb2_count) RR_CUDA(cudaMemsetAsync(b.fb2_count, 0, sizeof(int32_t), s));
    if (b.fb3_count) RR_CUDA(cudaMemsetAsync(b.fb3_count, 0, sizeof(int32_t), s));
    if (sh.host_in) {
      const size_t es = type_size(sh.dtype);
      RR_CUDA(cudaMemcpyAsync(b.xq, j.xq, size_t(sh.nq) * sh.d * es, cudaMemcpyHostToDevice, s));
      if (sh.ng) RR_CUDA(cudaMemcpyAsync(b.xg, j.xg, size_t(sh.ng) * sh.d * es, cudaMemcpyHostToDevice, s));
      mark("h2d");
    }
    nl += launch_normalize(sh, dq, dg, b.xhat, b.norm, b.xlow, b.xhi, b.xlo, b.xscale, b.err, b.emax, prec, status,
                           s);
    mark("normalize");
  }
  ErrModel em;
  em.err = b.err;
  em.emax = b.emax;
  em.np = sh.np;
  if (prec == RERANK_PREC_FP32) {
    // One FMA chain of dp terms over unit rows.
    em.kind = 0;
    em.eps = (sh.dp + 10) * kU32 * 1.01;
  } else {
    // Quantisation error enters per row; on top: the FP32 accumulation of dp/16
    // (BF16) or dp/32 (FP8) tensor-core partial sums, each charged 2u, the
    // rounding of the unit rows (4u) and of the FP8 scale products (2u).
    em.kind = 1;
    em.eps = (sh.dp / 16 + 32) * 2.0 * kU32 + 8.0 * kU32;
  }
  if (phases & kPhaseSim) {
    if (prec == RERANK_PREC_FP32) {
      nl += launch_sim_fp32_topk(sh, b.xhat, b.row_floor, b.part_s, b.part_i, ctx->sm_count, s);
    } else {
      const int r = launch_sim_tc_topk(sh, b.xlow, prec == RERANK_PREC_FP8, b.xscale, b.row_floor, b.part_s,
                                       b.part_i, status, ctx->sm_count, s, b.work);
      if (r < 0) return RERANK_ECUDA;
      nl += r;
    }
    RR_CUDA(cudaGetLastError());
    mark("similarity_topk");
  }
  if (!(phases & kPhasePost)) {
    *launches += nl;
    return RERANK_OK;
  }
  const int32_t* order = nullptr;
  if (sh.tune.refine_order) {
    nl += launch_cluster_order(sh, b.part_s, b.part_i, b.nb4, b.label, b.ord_cnt, b.ord_start, b.ord_fill, b.order,
                               s);
    order = b.order;
  }
  nl += launch_refine(sh, dq, dg, b.xhat, b.norm, b.part_s, b.part_i, sh.P, em, order, nullptr, true, b.knn_idx,
                      b.knn_score, b.fb_rows, b.fb_count, status, s);
  RR_CUDA(cudaGetLastError());
  mark("refine");
  const int32_t* exact_rows = b.fb_rows;
  const int32_t* exact_count = b.fb_count;
  if (prec != RERANK_PREC_FP32) {
    // Recheck the uncertified rows with the hi/lo split on the tensor cores:
    // |S' - S| is ~1e-5 instead of ~1e-3, enough for rows whose k1-th
    // neighbour sits among many near-equal scores.
    nl += launch_gather_rows(b.fb_rows, b.fb_count, b.xhi, b.xlo, b.ahi, b.alo, sh.n, sh.dp, s);
    const int32_t* split_rows = b.fb_rows;
    const int32_t* split_count = b.fb_count;
    if (prec == RERANK_PREC_FP8) {
      // FP8 leaves most rows uncertified (its bound is ~0.07): a single-product
      // BF16 stage (the hi copies, bound ~3e-3) with the longest candidate
      // lists (K3 = 64) first, the hi/lo split only for what that cannot
      // certify.  (For BF16 rows the same stage certifies nearly every row
      // but costs as much as the split: its loose bound makes the rescoring
      // go ~50 candidates deep instead of ~27.)
      Shape sh3 = sh;
      sh3.K = sh.K3;
      const int rg = launch_sim_tc_gather_topk(sh3, sh.P3g, b.ahi, b.xhi, b.fb_rows, b.fb_count, b.row_floor3,
                                               b.part3_s, b.part3_i, status, ctx->sm_count, s);
      if (rg < 0) return RERANK_ECUDA;
      nl += rg;
      // the hi copy is not the FP8 copy: its own bound ||x - hi|| = ||lo + r||
      ErrModel eh = em;
      eh.kind = 3;
      eh.eps = (sh.dp / 16 + 32) * 2.0 * kU32 + 8.0 * kU32;
      nl += launch_refine(sh3, dq, dg, b.xhat, b.norm, b.part3_s, b.part3_i, sh.P3g, eh, b.fb_rows, b.fb_count,
                          false, b.knn_idx, b.knn_score, b.fb3_rows, b.fb3_count, status, s, -1, kStFallbackMid);
      nl += launch_gather_rows(b.fb3_rows, b.fb3_count, b.xhi, b.xlo, b.ahi, b.alo, sh.n, sh.dp, s);
      split_rows = b.fb3_rows;
      split_count = b.fb3_count;
    }
    const int r = launch_sim_tc_split_topk(sh, sh.P3, b.ahi, b.alo, b.xhi, b.xlo, split_rows, split_count,
                                           b.row_floor3, b.part3_s, b.part3_i, status, ctx->sm_count, s);
    if (r < 0) return RERANK_ECUDA;
    nl += r;
    ErrModel e3 = em;
    e3.kind = 2;
    e3.eps = (3 * (sh.dp / 16) + 32) * 2.0 * kU32 + 8.0 * kU32;
    nl += launch_refine(sh, dq, dg, b.xhat, b.norm, b.part3_s, b.part3_i, sh.P3, e3, split_rows, split_count, false,
                        b.knn_idx, b.knn_score, b.fb2_rows, b.fb2_count, status, s, -1, kStFallback2);
    exact_rows = b.fb2_rows;
    exact_count = b.fb2_count;
    RR_CUDA(cudaGetLastError());
    mark("recheck");
  }
  float* fb_s = reinterpret_cast<float*>(b.scan_tmp);
  int32_t* fb_i = reinterpret_cast<int32_t*>(fb_s + size_t(ctx->sm_count) * fallback_warps() * fallback_k(sh));
  nl += launch_refine_fallback(sh, dq, dg, b.xhat, b.norm, b.knn_idx, b.knn_score, exact_rows, exact_count, fb_s, fb_i,
                               status, ctx->sm_count, s);
  mark("exact_scan");
  if (sh.knn_only) {
    const size_t bytes = size_t(sh.n) * sh.k1;
    int32_t* oi = sh.host_out ? b.out_idx : j.out_idx;
    float* os = sh.host_out ? b.out_dist : j.out_dist;
    RR_CUDA(cudaMemcpyAsync(oi, b.knn_idx, bytes * 4, cudaMemcpyDeviceToDevice, s));
    RR_CUDA(cudaMemcpyAsync(os, b.knn_score, bytes * 4, cudaMemcpyDeviceToDevice, s));
    if (sh.host_out) {
      RR_CUDA(cudaMemcpyAsync(j.out_idx, b.out_idx, bytes * 4, cudaMemcpyDeviceToHost, s));
      RR_CUDA(cudaMemcpyAsync(j.out_dist, b.out_dist, bytes * 4, cudaMemcpyDeviceToHost, s));
    }
  } else {
    nl += launch_graph(sh, b, ctx->cfg.alpha, ctx->cfg.aggregator, ctx->cfg.feature_mode, status, s);
    RR_CUDA(cudaGetLastError());
    mark("graph");
    if (sh.dense) {
      // h^(0) = the unit rows x_i / ||x_i||; L dense layers; cosines over d; ranking.
      const float* h = b.xhat;
      for (int l = 0; l < sh.layers; ++l) {
        nl += launch_dense_layer(sh, h, b.hd[l & 1], b.nbr, b.nbr_w, b.nbr_n, ctx->cfg.aggregator, s);
        h = b.hd[l & 1];
      }
      RR_CUDA(cudaGetLastError());
      mark("propagate");
      int32_t* oi = sh.host_out ? b.out_idx : j.out_idx;
      float* od = sh.host_out ? b.out_dist : j.out_dist;
      nl += launch_dense_scores(sh, h, b.hinv, b.xscore, s);
      nl += launch_rank_dense(sh, b.xscore, oi, od, b.rank_scratch, status, s);
      RR_CUDA(cudaGetLastError());
      mark("rank");
      if (sh.host_out) {
        const size_t cnt = size_t(sh.nq) * sh.topk;
        RR_CUDA(cudaMemcpyAsync(j.out_idx, b.out_idx, cnt * 4, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaMemcpyAsync(j.out_dist, b.out_dist, cnt * 4, cudaMemcpyDeviceToHost, s));
        mark("d2h");
      }
      *launches += nl;
      return RERANK_OK;
    }
    RR_CUDA(cudaMemsetAsync(b.hash_keys_vals, 0,
                            sizeof(float) * size_t(ctx->sm_count) * (size_t(sh.n) + size_t((sh.n + 31) / 32)), s));
    int src = 2;
    for (int l = 0; l < sh.layers; ++l) {
      const int dst = l & 1;
      nl += launch_propagate(sh, b, src, dst, ctx->cfg.aggregator, status, ctx->sm_count, sh.tune, s, nullptr,
                             l < 8 ? status + kStNnz0 + l + 1 : nullptr);
      src = dst;
    }
    RR_CUDA(cudaGetLastError());
    mark("propagate");
    nl += launch_row_norms(sh, b, src, status, s);
    int32_t* oi = sh.host_out ? b.out_idx : j.out_idx;
    float* od = sh.host_out ? b.out_dist : j.out_dist;
    if (sh.host_out && copy_overlap && sh.nq >= 4 * int64_t(ctx->sm_count)) {
      // Host outputs: rank the queries in four parts and copy each part back on
      // a second stream while the next part is ranked.
      RR_CUDA(ensure_copy_stream(ctx));
      nl += launch_rank_prep(sh, b, src, status, s);
      const int parts = 4;
      for (int p = 0; p < parts; ++p) {
        const int64_t q0 = sh.nq * p / parts, q1 = sh.nq * (p + 1) / parts;
        nl += launch_rank_queries(sh, b, src, oi, od, q0, q1, status, ctx->sm_count, sh.tune, s);
        RR_CUDA(cudaEventRecord(ctx->copy_events[size_t(p)], s));
        RR_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_events[size_t(p)], 0));
        const size_t off = size_t(q0) * size_t(sh.topk), cnt = size_t(q1 - q0) * size_t(sh.topk);
        RR_CUDA(cudaMemcpyAsync(j.out_idx + off, oi + off, cnt * 4, cudaMemcpyDeviceToHost, ctx->copy_stream));
        RR_CUDA(cudaMemcpyAsync(j.out_dist + off, od + off, cnt * 4, cudaMemcpyDeviceToHost, ctx->copy_stream));
      }
      RR_CUDA(cudaEventRecord(ctx->copy_events[size_t(parts)], ctx->copy_stream));
      RR_CUDA(cudaStreamWaitEvent(s, ctx->copy_events[size_t(parts)], 0));
      RR_CUDA(cudaGetLastError());
      mark("rank_d2h");
    } else {
      nl += launch_rank(sh, b, src, oi, od, status, ctx->sm_count, sh.tune, s);
      RR_CUDA(cudaGetLastError());
      mark("rank");
      if (sh.host_out) {
        const size_t cnt = size_t(sh.nq) * sh.topk;
        RR_CUDA(cudaMemcpyAsync(j.out_idx, b.out_idx, cnt * 4, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaMemcpyAsync(j.out_dist, b.out_dist, cnt * 4, cudaMemcpyDeviceToHost, s));
        mark("d2h");
      }
    }
  }
  *launches += nl;
  return RERANK_OK;
}

// Map one instance's device status block to a return code; fills the info counters.
// On a layer-buffer overflow, *need receives the capacity the layer asked for.
rerank_status map_status(const long long* h, int precision, rerank_info* info, int64_t* need) {
  info->fp64_rescored = h[kStFp64];
  info->fallback_rows = h[kStFallback];
  info->exact_scan_rows = precision == RERANK_PREC_FP32 ? h[kStFallback] : h[kStFallback2];
  info->error_bits = int32_t(h[kStErr]);
  info->bad_row = h[kStBadRow] == LLONG_MAX ? -1 : int32_t(h[kStBadRow]);
  for (int l = 0; l < 9; ++l) info->h_nnz[l] = h[kStNnz0 + l];
  const int e = int(h[kStErr]);
  *need = 0;
  if (e & (kErrNonFinite | kErrZeroNorm)) return RERANK_EINVAL;
  if (e & kErrOverflow) {
    *need = int64_t(h[kStNeed]);
    return RERANK_ENOMEM;
  }
  if (e & kErrTimeout) return RERANK_ETIMEOUT;
  if (e & (kErrCertify | kErrInternal)) return RERANK_EINTERNAL;
  return RERANK_OK;
}

// One attempt of the pipeline.  Returns OK, or the mapped device error.
rerank_status run_once(rerank_ctx* ctx, const void* xq, const void* xg, int32_t* out_idx, float* out_dist,
                       cudaStream_t s) {
  JobRun j;
  j.sh = ctx->shape;
  Carver dry;
  const size_t need = carve(dry, j.sh, j.b, ctx->sm_count, ctx->cfg.precision);
  rerank_status st = ensure_workspace(ctx, need);
  if (st != RERANK_OK) return st;
  Carver real;
  real.base = ctx->ws;
  carve(real, j.sh, j.b, ctx->sm_count, ctx->cfg.precision);
  ctx->buf = j.b;
  j.st = ctx->d_status;
  j.xq = xq;
  j.xg = xg;
  j.out_idx = out_idx;
  j.out_dist = out_dist;

  auto& tm = ctx->timer;
  tm.on = ctx->cfg.stage_timing != 0;
  tm.stream = s;
  tm.mark("begin");
  int64_t nl = 0;
  st = enqueue_job(ctx, j, s, &tm, &nl, true);
  if (st != RERANK_OK) return st;
  ctx->launches = nl;
  RR_CUDA(cudaGetLastError());
  st = collect(ctx, s);
  if (tm.on) finish_timing(ctx);
  if (st != RERANK_OK) return st;
  int64_t want = 0;
  st = map_status(ctx->h_status, ctx->cfg.precision, &ctx->info, &want);
  // The caller of run_once retries an overflow with the larger capacity.
  if (st == RERANK_ENOMEM) ctx->cap_h_hint = std::max<int64_t>(ctx->cap_h_hint, want + want / 4 + 1024);
  return st;
}

// Shape of one instance.  cap_hint: a layer capacity learned from an earlier overflow.
rerank_status plan_shape(const rerank_ctx* ctx, int64_t nq, int64_t ng, int d, int dtype, int k1, int k2, int layers,
                         int64_t topk, bool knn_only, bool host_in, bool host_out, int64_t cap_hint, Shape* out,
                         const Tuning* tune) {
  Shape sh;
  sh.nq = nq;
  sh.ng = ng;
  sh.n = nq + ng;
  const int prec = ctx->cfg.precision;
  const bool tc = prec != RERANK_PREC_FP32;
  // Tensor-core tiles are 128 rows x 256 columns; FP8 k-blocks are 128 bytes = 128 elements.
  sh.np = round_up(sh.n, tc ? 256 : 128);
  sh.d = d;
  sh.dp = int(round_up(d, prec == RERANK_PREC_FP8 ? 128 : 64));
  sh.dtype = dtype;
  sh.k1 = k1;
  sh.k2 = k2;
  sh.layers = layers;
  sh.topk = topk;
  sh.knn_only = knn_only;
  sh.host_in = host_in;
  sh.host_out = host_out;
  const int kmax = std::min(tc ? tc_kmax() : sim_fp32_kmax(), refine_kmax());
  if (k1 > RERANK_MAX_K1 || k1 > kmax) return RERANK_EUNSUPPORTED;
  sh.tune = tune ? *tune : (ctx->force_tune ? *ctx->force_tune : lookup_tuning(ctx, prec, sh.n, d));
  const int m = sh.tune.rescore_m >= 0 ? sh.tune.rescore_m : ctx->cfg.rescore_m;
  int64_t K = std::min<int64_t>(int64_t(k1) + std::max(m, 0), sh.n);
  K = std::min<int64_t>(K, kmax);
  sh.K = int(K);
  // P counts candidate lists per row: one per column chunk on the FP32 path; the
  // tensor-core kernel writes tc_lists_per_chunk() per chunk, and the refinement
  // merges at most 32 lists.
  const int lpc = tc ? tc_lists_per_chunk(sh.dp, 1) : 1;
  const int lpc3 = tc ? tc_lists_per_chunk(sh.dp, 3) : 1;
  // Work items of the main pass: row blocks of tc_item_rows() rows (CTA pairs
  // take 256) times column chunks, spread over the SMs (or SM pairs).
  const int irows = tc ? tc_item_rows() : 128;
  const int units = ctx->sm_count * 128 / irows;
  const int chunks = choose_chunks(sh.np / irows, sh.np / (tc ? 256 : 128), units, sh.tune.sim_chunks);
  sh.P = std::min(chunks, 32 / lpc) * lpc;
  // The recheck covers an unknown, usually small, set of rows: many short chunks keep every SM busy.
  sh.P3 = tc ? int(std::min<int64_t>(32 / lpc3, sh.np / 256)) * lpc3 : 0;
  sh.P3g = prec == RERANK_PREC_FP8 ? int(std::min<int64_t>(32 / lpc, sh.np / 256)) * lpc : 0;
  sh.K3 = prec == RERANK_PREC_FP8 ? int(std::max<int64_t>(sh.K, std::min<int64_t>(kmax, sh.n))) : 0;
  // Capacity of a propagation layer: sum over rows of ub_i <= min(n, sum_j len_j).
  // n^2 bounds it exactly for small graphs; otherwise a generous guess, grown on overflow.
  int64_t guess = std::max<int64_t>(2 * sh.n * k1, std::min<int64_t>(sh.n * sh.n, sh.n * int64_t(k2 + 1) * 160));
  if (ctx->test_cap_h > 0) guess = ctx->test_cap_h;
  sh.cap_h = std::max<int64_t>(guess, cap_hint);
  sh.dense = !knn_only && ctx->cfg.feature_mode == RERANK_FEAT_X;
  if (sh.dense) sh.cap_h = 1;  // the sparse layer buffers are not used
  sh.rank_ctas = ctx->sm_count;
  if (sh.n * int64_t(k1) >= (int64_t(1) << 31) || sh.n >= (int64_t(1) << 31) - 1) return RERANK_EUNSUPPORTED;
  *out = sh;
  return RERANK_OK;
}

rerank_status plan(rerank_ctx* ctx, int64_t nq, int64_t ng, int d, int dtype, int k1, int k2, int layers,
                   int64_t topk, bool knn_only, bool host_in, bool host_out) {
  return plan_shape(ctx, nq, ng, d, dtype, k1, k2, layers, topk, knn_only, host_in, host_out, ctx->cap_h_hint,
                    &ctx->shape);
}

rerank_status run_with_retry(rerank_ctx* ctx, const void* xq, const void* xg, int32_t* oi, float* od,
                             cudaStream_t s) {
  rerank_status st = RERANK_OK;
  for (int attempt = 0; attempt < 4; ++attempt) {
    st = run_once(ctx, xq, xg, oi, od, s);
    if (!(st == RERANK_ENOMEM && (ctx->info.error_bits & kErrOverflow))) break;
    ctx->shape.cap_h = std::max(ctx->shape.cap_h, ctx->cap_h_hint);
  }
  ctx->info.workspace_bytes = int64_t(ctx->ws_bytes);
  ctx->info.kernel_launches = ctx->launches;
  ctx->info.n_vertices = ctx->shape.n;
  ctx->info.candidates_per_row = ctx->shape.K;
  return st;
}

constexpr int kBatchStreams = 16;

rerank_status ensure_streams(rerank_ctx* ctx) {
  if (!ctx->streams.empty()) return RERANK_OK;
  for (int i = 0; i < kBatchStreams; ++i) {
    cudaStream_t st = nullptr;
    RR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ctx->streams.push_back(st);
  }
  for (int i = 0; i <= kBatchStreams; ++i) {
    cudaEvent_t e = nullptr;
    RR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->events.push_back(e);
  }
  return RERANK_OK;
}

rerank_status ensure_host_status(rerank_ctx* ctx, size_t count) {
  if (count <= ctx->h_batch_count) return RERANK_OK;
  drop_graphs(ctx);
  if (ctx->h_batch) cudaFreeHost(ctx->h_batch);
  ctx->h_batch = nullptr;
  ctx->h_batch_count = 0;
  RR_CUDA(cudaMallocHost(&ctx->h_batch, count * sizeof(long long)));
  ctx->h_batch_count = count;
  return RERANK_OK;
}

rerank_status ensure_host_stage(rerank_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->h_stage_bytes) return RERANK_OK;
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  ctx->h_stage = nullptr;
  ctx->h_stage_bytes = 0;
  RR_CUDA(cudaMallocHost(&ctx->h_stage, bytes));
  ctx->h_stage_bytes = bytes;
  return RERANK_OK;
}

// Memory the GPU cannot reach from a graph's copy nodes without staging.
bool is_pageable(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered;
}

using PtrAttrFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);

// Process-wide unique id of the allocation holding p, 0 when the driver does
// not know p.  Graph keys carry it beside each pointer, so a buffer freed and
// allocated again at the same address does not match a graph of the old one.
uint64_t buffer_id(const void* p) {
  static const PtrAttrFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PtrAttrFn>(f);
  }();
  unsigned long long id = 0;
  if (!fn || !p || fn(&id, CU_POINTER_ATTRIBUTE_BUFFER_ID, reinterpret_cast<CUdeviceptr>(p)) != CUDA_SUCCESS) return 0;
  return id;
}

// Every field of a planned instance: together with the job's pointers and
// workspace offset they fix everything a batched call enqueues for it.
void shape_key(const Shape& sh, std::vector<int64_t>& k) {
  const int64_t v[] = {sh.nq, sh.ng, sh.n, sh.np, sh.d, sh.dp, sh.dtype, sh.k1, sh.k2, sh.layers, sh.K, sh.P, sh.P3,
                       sh.P3g, sh.K3, sh.topk, sh.host_in, sh.host_out, sh.knn_only, sh.ext_feat, sh.cap_h, sh.cap_csc,
                       sh.hash_slots, sh.rank_ctas, sh.rank_scratch_per_cta, sh.tune.sim_chunks, sh.tune.prop_warps,
                       sh.tune.refine_order, sh.tune.rescore_m, sh.tune.rank_threads};
  k.insert(k.end(), std::begin(v), std::end(v));
}

uint64_t key_hash(const std::vector<int64_t>& k) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the 64-bit words
  for (int64_t v : k) h = (h ^ uint64_t(v)) * 1099511628211ull;
  return h;
}

void free_graph(BatchGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->stage) cudaFreeHost(g->stage);
  delete g;
}

// Capture what `enqueue` issues into a new graph of the context's cache
// (evicting the least recently used one beyond kMaxGraphs).  *out stays null
// when the capture itself was refused (the caller then enqueues directly).
constexpr size_t kMaxGraphs = 4;
template <class F>
rerank_status capture_batch_graph(rerank_ctx* ctx, std::vector<int64_t>&& key, size_t stage_bytes, int64_t* nl,
                                  F& enqueue, BatchGraph** out) {
  *out = nullptr;
  if (!ctx->cap_stream) RR_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  BatchGraph* g = new BatchGraph;
  g->key = std::move(key);
  if (cudaMallocHost(&g->stage, stage_bytes ? stage_bytes : 16) != cudaSuccess) {
    g->stage = nullptr;
    free_graph(g);
    return cuda_fail(cudaGetLastError(), "cudaMallocHost");
  }
  *nl = 0;
  if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    free_graph(g);
    return RERANK_OK;
  }
  const rerank_status st = enqueue(ctx->cap_stream, g->stage);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
  cudaError_t ei = cudaErrorUnknown;
  if (st == RERANK_OK && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&g->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st != RERANK_OK || ei != cudaSuccess) {
    cudaGetLastError();
    g->exec = nullptr;
    free_graph(g);
    return st;
  }
  g->launches = *nl;
  if (ctx->graphs.size() >= kMaxGraphs) {
    auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                [](const BatchGraph* a, const BatchGraph* b) { return a->stamp < b->stamp; });
    free_graph(*lru);
    ctx->graphs.erase(lru);
  }
  ctx->graphs.push_back(g);
  *out = g;
  return RERANK_OK;
}

// Rough device cost of an instance, used to spread instances over the streams.
double job_cost(const Shape& sh) {
  return double(sh.np) * double(sh.np) * double(sh.dp) + 4.0e4 * double(sh.n) * double(sh.k1);
}

rerank_status run_batch(rerank_ctx* ctx, rerank_job* jobs, int njobs, cudaStream_t s) {
  std::vector<JobRun> runs(static_cast<size_t>(njobs));
  size_t total = 0;
  const size_t st_bytes = sizeof(long long) * kStCount;
  std::vector<size_t> off(static_cast<size_t>(njobs));
  for (int i = 0; i < njobs; ++i) {
    const rerank_job& jb = jobs[i];
    const bool host_in = is_host_ptr(jb.xq) || is_host_ptr(jb.xg);
    const bool host_out = is_host_ptr(jb.out_idx) || is_host_ptr(jb.out_dist);
    const int64_t topk = jb.topk_out ? jb.topk_out : jb.ng;
    rerank_status st = plan_shape(ctx, jb.nq, jb.ng, jb.d, jb.dtype, jb.k1, jb.k2, jb.layers, topk, false, host_in,
                                  host_out, 0, &runs[size_t(i)].sh);
    if (st != RERANK_OK) return st;
    Carver dry;
    const size_t need = carve(dry, runs[size_t(i)].sh, runs[size_t(i)].b, ctx->sm_count, ctx->cfg.precision);
    total = (total + 255) & ~size_t(255);
    off[size_t(i)] = total;
    total += ((st_bytes + 255) & ~size_t(255)) + need;
  }
  // Tensor-core precisions: the similarity stage of all instances runs as
  // persistent launches over many instances (their tables live here).
  const bool tc_batch = ctx->cfg.precision != RERANK_PREC_FP32;
  const size_t inst_bytes = tc_batch_inst_bytes() * size_t(njobs);
  total = (total + 255) & ~size_t(255);
  const size_t inst_off = total;
  if (tc_batch) total += inst_bytes;
  rerank_status st = ensure_workspace(ctx, total);
  if (st != RERANK_OK) return st;
  st = ensure_streams(ctx);
  if (st != RERANK_OK) return st;
  st = ensure_host_status(ctx, size_t(njobs) * kStCount);
  if (st != RERANK_OK) return st;
  if (tc_batch) {
    st = ensure_host_stage(ctx, inst_bytes);
    if (st != RERANK_OK) return st;
  }
  for (int i = 0; i < njobs; ++i) {
    JobRun& j = runs[size_t(i)];
    j.st = reinterpret_cast<long long*>(ctx->ws + off[size_t(i)]);
    Carver real;
    real.base = ctx->ws + off[size_t(i)] + ((st_bytes + 255) & ~size_t(255));
    carve(real, j.sh, j.b, ctx->sm_count, ctx->cfg.precision);
    j.xq = jobs[i].xq;
    j.xg = jobs[i].xg;
    j.out_idx = jobs[i].out_idx;
    j.out_dist = jobs[i].out_dist;
  }
  // Largest instances first, each onto the least loaded stream.
  std::vector<int> idx(static_cast<size_t>(njobs));
  for (int i = 0; i < njobs; ++i) idx[size_t(i)] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    const double ca = job_cost(runs[size_t(a)].sh), cb = job_cost(runs[size_t(b)].sh);
    return ca != cb ? ca > cb : a < b;
  });
  const int ns = std::min<int>(kBatchStreams, njobs);
  std::vector<double> load(static_cast<size_t>(ns), 0.0);
  std::vector<int> lane(static_cast<size_t>(njobs), 0);
  for (int i : idx) {
    int k = 0;
    for (int t = 1; t < ns; ++t)
      if (load[size_t(t)] < load[size_t(k)]) k = t;
    load[size_t(k)] += job_cost(runs[size_t(i)].sh);
    lane[size_t(i)] = k;
  }
  int64_t nl = 0;
  // Everything the call enqueues, from stream `o`: fork onto the streams,
  // each phase of every instance on its stream, join back into `o`; the
  // status blocks are copied to the host last.  `stage`: pinned memory for the
  // instance tables of the batched similarity launches.
  auto enqueue_all = [&](cudaStream_t o, void* stage) -> rerank_status {
    auto fan_out = [&](int phases) -> rerank_status {
      RR_CUDA(cudaEventRecord(ctx->events[0], o));
      for (int k = 0; k < ns; ++k) RR_CUDA(cudaStreamWaitEvent(ctx->streams[size_t(k)], ctx->events[0], 0));
      rerank_status r = RERANK_OK;
      for (int i : idx) {
        r = enqueue_job(ctx, runs[size_t(i)], ctx->streams[size_t(lane[size_t(i)])], nullptr, &nl, false, phases);
        if (r != RERANK_OK) break;
      }
      for (int k = 0; k < ns; ++k) {
        RR_CUDA(cudaEventRecord(ctx->events[size_t(1 + k)], ctx->streams[size_t(k)]));
        RR_CUDA(cudaStreamWaitEvent(o, ctx->events[size_t(1 + k)], 0));
      }
      return r;
    };
    rerank_status r = RERANK_OK;
    if (!tc_batch) {
      r = fan_out(kPhaseAll);
    } else {
      r = fan_out(kPhasePre);
      if (r == RERANK_OK) {
        // Similarity + top-K: instances with the same epilogue layout share a
        // launch, largest first (up to the launch's instance limit).
        const bool fp8 = ctx->cfg.precision == RERANK_PREC_FP8;
        std::vector<TcBatchInst> group;
        size_t used = 0;
        for (int eg = 1; eg <= 2 && r == RERANK_OK; ++eg) {
          group.clear();
          for (size_t p = 0; p <= idx.size(); ++p) {
            const bool end = p == idx.size();
            if (!end) {
              const JobRun& j = runs[size_t(idx[p])];
              if (tc_lists_per_chunk(j.sh.dp, 1) != eg) continue;
              TcBatchInst t{};
              t.xlow = j.b.xlow;
              t.n = j.sh.n;
              t.np = j.sh.np;
              t.dp = j.sh.dp;
              t.P = j.sh.P;
              t.K = j.sh.K;
              t.inv_scale = j.b.xscale;
              t.row_floor = j.b.row_floor;
              t.part_s = j.b.part_s;
              t.part_i = j.b.part_i;
              t.status = j.st;
              group.push_back(t);
            }
            if (!group.empty() && (end || int(group.size()) == tc_batch_max_inst())) {
              const int k = launch_sim_tc_batch(group.data(), int(group.size()), fp8, ctx->ws + inst_off + used,
                                                static_cast<uint8_t*>(stage) + used, ctx->sm_count, o);
              if (k < 0) {
                r = RERANK_ECUDA;
                break;
              }
              nl += k;
              used += tc_batch_inst_bytes() * group.size();
              group.clear();
            }
          }
        }
        if (r == RERANK_OK) RR_CUDA(cudaGetLastError());
      }
      if (r == RERANK_OK) r = fan_out(kPhasePost);
    }
    if (r != RERANK_OK) return r;
    for (int i = 0; i < njobs; ++i)
      RR_CUDA(cudaMemcpyAsync(ctx->h_batch + size_t(i) * kStCount, runs[size_t(i)].st, st_bytes,
                              cudaMemcpyDeviceToHost, o));
    return RERANK_OK;
  };
  // A call whose buffers are all device or pinned memory is captured once as a
  // CUDA graph and replayed by later calls with the same key (thousands of
  // small launches become one graph launch).
  bool graphable = true;
  for (int i = 0; i < njobs && graphable; ++i) {
    const rerank_job& jb = jobs[i];
    graphable = !is_pageable(jb.xq) && !is_pageable(jb.xg) && !is_pageable(jb.out_idx) && !is_pageable(jb.out_dist);
  }
  if (graphable) {
    std::vector<int64_t> key;
    key.reserve(size_t(njobs) * 44 + 10);
    key.push_back(int64_t(reinterpret_cast<uintptr_t>(ctx->ws)));
    key.push_back(int64_t(buffer_id(ctx->ws)));
    key.push_back(int64_t(total));
    key.push_back(int64_t(reinterpret_cast<uintptr_t>(ctx->h_batch)));
    key.push_back(int64_t(buffer_id(ctx->h_batch)));
    key.push_back(tc_stall_hook());
    for (int i = 0; i < njobs; ++i) {
      const rerank_job& jb = jobs[i];
      key.push_back(int64_t(reinterpret_cast<uintptr_t>(jb.xq)));
      key.push_back(int64_t(reinterpret_cast<uintptr_t>(jb.xg)));
      key.push_back(int64_t(reinterpret_cast<uintptr_t>(jb.out_idx)));
      key.push_back(int64_t(reinterpret_cast<uintptr_t>(jb.out_dist)));
      for (const void* p : {jb.xq, jb.xg, static_cast<const void*>(jb.out_idx), static_cast<const void*>(jb.out_dist)})
        key.push_back(int64_t(buffer_id(p)));
      key.push_back(int64_t(off[size_t(i)]));
      shape_key(runs[size_t(i)].sh, key);
    }
    BatchGraph* g = nullptr;
    for (BatchGraph* c : ctx->graphs)
      if (c->key == key) g = c;
    if (!g) {
      // Capture only a key seen before: a one-off call is enqueued directly
      // and pays no instantiation.
      const uint64_t h = key_hash(key);
      const bool seen = std::find(ctx->graph_seen.begin(), ctx->graph_seen.end(), h) != ctx->graph_seen.end();
      if (seen) {
        st = capture_batch_graph(ctx, std::move(key), inst_bytes, &nl, enqueue_all, &g);
        if (st != RERANK_OK) return st;
      } else {
        if (ctx->graph_seen.size() >= 16) ctx->graph_seen.erase(ctx->graph_seen.begin());
        ctx->graph_seen.push_back(h);
      }
    }
    if (g) {
      g->stamp = ++ctx->graph_clock;
      RR_CUDA(cudaGraphLaunch(g->exec, s));
      nl = g->launches;
    } else {
      graphable = false;  // the capture was refused: enqueue directly
    }
  }
  if (!graphable) {
    nl = 0;
    st = enqueue_all(s, ctx->h_stage);
    if (st != RERANK_OK) return st;
  }
  RR_CUDA(cudaStreamSynchronize(s));
  RR_CUDA(cudaGetLastError());
  ctx->launches = nl;
  rerank_status first = RERANK_OK;
  rerank_info agg{};
  for (int i = 0; i < njobs; ++i) {
    rerank_info inf{};
    int64_t want = 0;
    rerank_status js = map_status(ctx->h_batch + size_t(i) * kStCount, ctx->cfg.precision, &inf, &want);
    if (js == RERANK_ENOMEM) {
      // Overflowed propagation buffers: rerun this instance alone with the capacity it asked for.
      ctx->cap_h_hint = std::max<int64_t>(ctx->cap_h_hint, want + want / 4 + 1024);
      const rerank_job& jb = jobs[i];
      js = plan(ctx, jb.nq, jb.ng, jb.d, jb.dtype, jb.k1, jb.k2, jb.layers, runs[size_t(i)].sh.topk, false,
                runs[size_t(i)].sh.host_in, runs[size_t(i)].sh.host_out);
      if (js == RERANK_OK) js = run_with_retry(ctx, jb.xq, jb.xg, jb.out_idx, jb.out_dist, s);
      nl += ctx->launches;
      inf = ctx->info;
    }
    jobs[i].status = js;
    if (js != RERANK_OK && first == RERANK_OK) first = js;
    agg.n_vertices += runs[size_t(i)].sh.n;
    agg.fp64_rescored += inf.fp64_rescored;
    agg.fallback_rows += inf.fallback_rows;
    agg.exact_scan_rows += inf.exact_scan_rows;
    agg.error_bits |= inf.error_bits;
  }
  agg.bad_row = -1;
  agg.workspace_bytes = int64_t(ctx->ws_bytes);
  agg.kernel_launches = nl;
  ctx->info = agg;
  ctx->launches = nl;
  return first;
}

bool valid_enum(const rerank_config* c) {
  return c->precision >= 0 && c->precision <= 2 && c->aggregator >= 0 && c->aggregator <= 2 &&
         c->feature_mode >= 0 && c->feature_mode <= 2 && c->rescore_m >= 0 && c->rescore_m <= 256;
}

}  // namespace rr

using namespace rr;

extern "C" {

void rerank_config_init(rerank_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->precision = RERANK_PREC_FP32;
  cfg->rescore_m = 16;
  cfg->alpha = 2.0f;
  cfg->aggregator = RERANK_AGG_SUM;
  cfg->feature_mode = RERANK_FEAT_ASTAR;
  cfg->hbm_budget = 0;
  cfg->autotune_path = nullptr;
  cfg->stage_timing = 0;
}

const char* rerank_last_cuda_error(void) { return rr::last_cuda_error_text(); }

const char* rerank_strerror(rerank_status s) {
  switch (s) {
    case RERANK_OK: return "ok";
    case RERANK_EINVAL: return "invalid argument or input row";
    case RERANK_ENOMEM: return "out of memory";
    case RERANK_EBUDGET: return "workspace exceeds the HBM budget";
    case RERANK_ECUDA: return "CUDA error";
    case RERANK_ETIMEOUT: return "device wait timed out";
    case RERANK_EINTERNAL: return "internal check failed";
    case RERANK_EUNSUPPORTED: return "unsupported combination";
    case RERANK_EAGAIN: return "not ready";
  }
  return "unknown status";
}

rerank_status rerank_check_args(int64_t nq, int64_t ng, int d, int dtype, int k1, int k2, int layers,
                                int64_t topk_out) {
  if (nq < 1 || ng < 1 || d < 1) return RERANK_EINVAL;
  if (dtype != RERANK_DTYPE_F32 && dtype != RERANK_DTYPE_BF16) return RERANK_EINVAL;
  if (k1 < 1 || k2 < 1 || k2 > k1 || int64_t(k1) > nq + ng) return RERANK_EINVAL;
  if (layers < 0 || topk_out < 0 || topk_out > ng) return RERANK_EINVAL;
  return RERANK_OK;
}

rerank_status rerank_create(rerank_ctx** out, const rerank_config* cfg) {
  if (!out || !cfg) return RERANK_EINVAL;
  *out = nullptr;
  if (!valid_enum(cfg)) return RERANK_EINVAL;
  int ndev = 0;
  const cudaError_t ec = cudaGetDeviceCount(&ndev);
  if (ec != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(ec, "cudaGetDeviceCount");
  }
  if (cfg->device < 0 || cfg->device >= ndev) return cuda_fail(cudaErrorInvalidDevice, "rerank_create: device index");
  cudaDeviceProp prop;
  RR_CUDA(cudaGetDeviceProperties(&prop, cfg->device));
  if (prop.major != 10 || prop.minor != 3)
    return cuda_fail(cudaErrorNoKernelImageForDevice, "rerank_create: not a compute capability 10.3 device");
  RR_CUDA(cudaSetDevice(cfg->device));
  rerank_ctx* ctx = new (std::nothrow) rerank_ctx();
  if (!ctx) return RERANK_ENOMEM;
  ctx->cfg = *cfg;
  if (cfg->autotune_path) {
    ctx->tune_path = cfg->autotune_path;
    read_tune_file(ctx->tune_path, &ctx->tune_table);  // a missing file is an empty table
  }
  ctx->cfg.autotune_path = nullptr;
  ctx->device = cfg->device;
  ctx->sm_count = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  // Test hook: start the propagation buffers this small to exercise the overflow-and-retry path.
  if (const char* e = std::getenv("RERANK_TEST_CAP_H")) ctx->test_cap_h = std::atoll(e);
  if (cudaMalloc(&ctx->d_status, sizeof(long long) * kStCount) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(long long) * kStCount) != cudaSuccess) {
    cudaGetLastError();
    rerank_destroy(ctx);
    return RERANK_ENOMEM;
  }
  *out = ctx;
  return RERANK_OK;
}

rerank_status rerank_destroy(rerank_ctx* ctx) {
  if (!ctx) return RERANK_OK;
  serve_stop(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  for (auto e : ctx->timer.ev) cudaEventDestroy(e);
  for (auto st : ctx->streams) cudaStreamDestroy(st);
  for (auto e : ctx->events) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  for (BatchGraph* g : ctx->graphs) free_graph(g);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto e : ctx->copy_events) cudaEventDestroy(e);
  if (ctx->h_batch) cudaFreeHost(ctx->h_batch);
  delete ctx;
  return RERANK_OK;
}

rerank_status rerank_run(rerank_ctx* ctx, const void* xq, int64_t nq, const void* xg, int64_t ng, int d, int dtype,
                         int k1, int k2, int layers, int64_t topk_out, int32_t* out_idx, float* out_dist,
                         void* stream) {
  if (!ctx || !xq || !xg || !out_idx || !out_dist) return RERANK_EINVAL;
  rerank_status st = rerank_check_args(nq, ng, d, dtype, k1, k2, layers, topk_out);
  if (st != RERANK_OK) return st;
  RR_CUDA(cudaSetDevice(ctx->device));
  const bool host_in = is_host_ptr(xq) || is_host_ptr(xg);
  const bool host_out = is_host_ptr(out_idx) || is_host_ptr(out_dist);
  const int64_t topk = topk_out ? topk_out : ng;
  st = plan(ctx, nq, ng, d, dtype, k1, k2, layers, topk, false, host_in, host_out);
  if (st != RERANK_OK) return st;
  return run_with_retry(ctx, xq, xg, out_idx, out_dist, static_cast<cudaStream_t>(stream));
}

rerank_status rerank_run_batch(rerank_ctx* ctx, rerank_job* jobs, int njobs, void* stream) {
  if (!ctx || !jobs || njobs < 1) return RERANK_EINVAL;
  if (ctx->cfg.feature_mode == RERANK_FEAT_X) return RERANK_EUNSUPPORTED;
  rerank_status bad = RERANK_OK;
  for (int i = 0; i < njobs; ++i) {
    rerank_job& j = jobs[i];
    j.status = (!j.xq || !j.xg || !j.out_idx || !j.out_dist)
                   ? RERANK_EINVAL
                   : rerank_check_args(j.nq, j.ng, j.d, j.dtype, j.k1, j.k2, j.layers, j.topk_out);
    if (j.status != RERANK_OK && bad == RERANK_OK) bad = j.status;
  }
  if (bad != RERANK_OK) return bad;
  RR_CUDA(cudaSetDevice(ctx->device));
  return run_batch(ctx, jobs, njobs, static_cast<cudaStream_t>(stream));
}

rerank_status rerank_knn(rerank_ctx* ctx, const void* x, int64_t n, int d, int dtype, int k, int32_t* out_idx,
                         float* out_score, void* stream) {
  if (!ctx || !x || !out_idx || !out_score) return RERANK_EINVAL;
  if (n < 1 || d < 1 || k < 1 || k > n || (dtype != RERANK_DTYPE_F32 && dtype != RERANK_DTYPE_BF16))
    return RERANK_EINVAL;
  RR_CUDA(cudaSetDevice(ctx->device));
  const bool host_in = is_host_ptr(x);
  const bool host_out = is_host_ptr(out_idx) || is_host_ptr(out_score);
  rerank_status st = plan(ctx, n, 0, d, dtype, k, 1, 0, 0, true, host_in, host_out);
  if (st != RERANK_OK) return st;
  return run_with_retry(ctx, x, x, out_idx, out_score, static_cast<cudaStream_t>(stream));
}

rerank_status rerank_last_info(const rerank_ctx* ctx, rerank_info* info) {
  if (!ctx || !info) return RERANK_EINVAL;
  *info = ctx->info;
  return RERANK_OK;
}

rerank_status rerank_stage_times(const rerank_ctx* ctx, float* ms, const char** names, int cap, int* count) {
  if (!ctx || !count) return RERANK_EINVAL;
  if (!ctx->cfg.stage_timing) return RERANK_EINVAL;
  const int nstage = int(ctx->stage_ms.size());
  *count = nstage;
  for (int i = 0; i < nstage && i < cap; ++i) {
    if (ms) ms[i] = ctx->stage_ms[i];
    if (names) names[i] = ctx->stage_names[i];
  }
  return RERANK_OK;
}

rerank_status rerank_debug_copy(const rerank_ctx* ctx, int what, void* dst, size_t cap, size_t* bytes) {
  if (!ctx || !bytes) return RERANK_EINVAL;
  const Shape& sh = ctx->shape;
  const Buffers& b = ctx->buf;
  const int last = sh.layers == 0 ? 2 : (sh.layers - 1) & 1;
  const void* src = nullptr;
  size_t nb = 0;
  switch (what) {
    case RERANK_DBG_KNN_IDX: src = b.knn_idx; nb = size_t(sh.n) * sh.k1 * 4; break;
    case RERANK_DBG_KNN_SCORE: src = b.knn_score; nb = size_t(sh.n) * sh.k1 * 4; break;
    case RERANK_DBG_H0_ROWPTR: src = b.h0ptr; nb = (size_t(sh.n) + 1) * 4; break;
    case RERANK_DBG_H0_COL: src = b.col[2]; nb = size_t(2) * sh.n * sh.k1 * 4; break;
    case RERANK_DBG_H0_VAL: src = b.val[2]; nb = size_t(2) * sh.n * sh.k1 * 4; break;
    case RERANK_DBG_HL_START: src = b.start[last]; nb = size_t(sh.n) * 8; break;
    case RERANK_DBG_HL_LEN: src = b.len[last]; nb = size_t(sh.n) * 4; break;
    case RERANK_DBG_HL_COL: src = b.col[last]; nb = size_t(last == 2 ? 2 * sh.n * sh.k1 : sh.cap_h) * 4; break;
    case RERANK_DBG_HL_VAL: src = b.val[last]; nb = size_t(last == 2 ? 2 * sh.n * sh.k1 : sh.cap_h) * 4; break;
    case RERANK_DBG_PART_S: src = b.part_s; nb = size_t(sh.n) * sh.P * sh.K * 4; break;
    case RERANK_DBG_PART_I: src = b.part_i; nb = size_t(sh.n) * sh.P * sh.K * 4; break;
    case RERANK_DBG_QERR: src = b.err; nb = size_t(sh.np) * 4; break;
    case RERANK_DBG_HL_DENSE:
      if (!sh.dense) return RERANK_EINVAL;
      src = sh.layers == 0 ? b.xhat : b.hd[(sh.layers - 1) & 1];
      nb = size_t(sh.n) * sh.dp * 4;
      break;
    default: return RERANK_EINVAL;
  }
  if (sh.knn_only && what > RERANK_DBG_KNN_SCORE && what < RERANK_DBG_PART_S) return RERANK_EINVAL;
  if (what == RERANK_DBG_QERR && ctx->cfg.precision == RERANK_PREC_FP32) return RERANK_EINVAL;
  *bytes = nb;
  if (!dst) return RERANK_OK;
  if (cap < nb || !src) return RERANK_EINVAL;
  RR_CUDA(cudaSetDevice(ctx->device));
  RR_CUDA(cudaMemcpy(dst, src, nb, cudaMemcpyDefault));
  return RERANK_OK;
}

}  // extern "C"

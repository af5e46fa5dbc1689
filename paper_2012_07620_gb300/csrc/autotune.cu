// Autotuner: launch shapes per (precision, d, vertex-count bucket), measured
// on the caller's own data and kept in a JSON table.
//
// Knobs (none changes a result, only the work decomposition):
//   sim_chunks    column chunks P of the similarity top-K kernel: more chunks
//                 fill more SMs for small N, fewer keep more columns per list
//                 and let the cross-chunk floors prune harder;
//   prop_warps    warps per CTA of the propagation kernel (one hash table of
//                 4 KB per warp in shared memory);
//   refine_order  refine rows cluster by cluster (candidate rows shared in L1)
//                 or in index order (no ordering pass);
//   rescore_m     candidates kept beyond k1 (K = k1 + m): a longer list costs
//                 the similarity epilogue and the refinement more, and leaves
//                 fewer rows uncertified for the hi/lo recheck.
// The GEMM tile (128 x 256 x 64 bytes of K, 4-stage TMA ring, one CTA per SM)
// is fixed: it is the largest tile whose accumulators (2 x 256 TMEM columns)
// and operand ring fit one SM, and the per-row top-K epilogue needs a whole
// 128-row block per CTA.
//
// Search: coordinate descent, one knob at a time from the defaults, each
// candidate timed by the stage it affects (median of three runs with CUDA
// events), the whole pipeline run each time so caches see a real mix.
//
// Table format (written by write_tune_file, read back by read_tune_file):
//   {"version": 1, "entries": [
//     {"precision": 1, "d": 2048, "n_bucket": 29, "sim_chunks": 4,
//      "prop_warps": 8, "refine_order": 1, "rescore_m": 22, "ms": 6.4}, ...]}
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.hpp"

namespace rr {

int tune_bucket(int64_t n) {
  int b = 0;
  // floor(2 log2 n), exactly: the largest b with 2^b <= n^2.
  const double n2 = double(n) * double(n);
  while (b < 126 && std::ldexp(1.0, b + 1) <= n2) ++b;
  return b;
}

Tuning lookup_tuning(const rerank_ctx* ctx, int precision, int64_t n, int d) {
  const int nb = tune_bucket(n);
  for (const TuneEntry& e : ctx->tune_table)
    if (e.precision == precision && e.d == d && e.n_bucket == nb) return e.t;
  return Tuning{};
}

namespace {

// Value of "key": <number> inside one JSON object's text; false if absent.
bool field(const std::string& obj, const char* key, double* out) {
  const std::string k = std::string("\"") + key + "\"";
  const size_t p = obj.find(k);
  if (p == std::string::npos) return false;
  size_t c = obj.find(':', p + k.size());
  if (c == std::string::npos) return false;
  const char* s = obj.c_str() + c + 1;
  char* end = nullptr;
  const double v = std::strtod(s, &end);
  if (end == s) return false;
  *out = v;
  return true;
}

}  // namespace

bool read_tune_file(const std::string& path, std::vector<TuneEntry>* out) {
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  const size_t list = text.find("\"entries\"");
  if (list == std::string::npos) return false;
  std::vector<TuneEntry> entries;
  size_t p = text.find('[', list);
  while (p != std::string::npos) {
    const size_t a = text.find('{', p);
    if (a == std::string::npos) break;
    const size_t b = text.find('}', a);
    if (b == std::string::npos) break;
    const std::string obj = text.substr(a, b - a + 1);
    double prec, d, nb, pc, pw, ro, ms = 0.0, rm = -1.0;
    if (field(obj, "precision", &prec) && field(obj, "d", &d) && field(obj, "n_bucket", &nb) &&
        field(obj, "sim_chunks", &pc) && field(obj, "prop_warps", &pw) && field(obj, "refine_order", &ro)) {
      field(obj, "ms", &ms);
      field(obj, "rescore_m", &rm);
      TuneEntry e;
      e.precision = int(prec);
      e.d = int(d);
      e.n_bucket = int(nb);
      e.t.sim_chunks = std::max(0, std::min(32, int(pc)));
      e.t.prop_warps = std::max(1, std::min(24, int(pw)));
      e.t.refine_order = ro != 0.0 ? 1 : 0;
      e.t.rescore_m = std::max(-1, std::min(256, int(rm)));
      e.ms = ms;
      entries.push_back(e);
    }
    p = b + 1;
  }
  *out = entries;
  return true;
}

bool write_tune_file(const std::string& path, const std::vector<TuneEntry>& entries) {
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "{\"version\": 1, \"entries\": [");
  for (size_t i = 0; i < entries.size(); ++i) {
    const TuneEntry& e = entries[i];
    std::fprintf(f,
                 "%s\n  {\"precision\": %d, \"d\": %d, \"n_bucket\": %d, \"sim_chunks\": %d, \"prop_warps\": %d, "
                 "\"refine_order\": %d, \"rescore_m\": %d, \"ms\": %.4f}",
                 i ? "," : "", e.precision, e.d, e.n_bucket, e.t.sim_chunks, e.t.prop_warps, e.t.refine_order,
                 e.t.rescore_m, e.ms);
  }
  std::fprintf(f, "\n]}\n");
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace rr

using namespace rr;

namespace {

// One timed pipeline run under `t`; returns the named stage's time (or the total).
rerank_status timed_run(rerank_ctx* ctx, const Tuning& t, const void* xq, int64_t nq, const void* xg, int64_t ng,
                        int d, int dtype, int k1, int k2, int layers, int32_t* oi, float* od, void* stream,
                        const char* stage, double* ms_out) {
  std::vector<double> v;
  for (int r = 0; r < 3; ++r) {
    ctx->force_tune = &t;
    const rerank_status st = rerank_run(ctx, xq, nq, xg, ng, d, dtype, k1, k2, layers, 0, oi, od, stream);
    ctx->force_tune = nullptr;
    if (st != RERANK_OK) return st;
    double ms = 0.0;
    for (size_t i = 0; i < ctx->stage_ms.size(); ++i)
      if (!stage || std::strcmp(ctx->stage_names[i], stage) == 0) ms += ctx->stage_ms[i];
    v.push_back(ms);
  }
  std::sort(v.begin(), v.end());
  *ms_out = v[1];
  return RERANK_OK;
}

}  // namespace

extern "C" {

rerank_status rerank_autotune(rerank_ctx* ctx, const void* xq, int64_t nq, const void* xg, int64_t ng, int d,
                              int dtype, int k1, int k2, int layers, rerank_tuning* out, void* stream) {
  if (!ctx || !xq || !xg) return RERANK_EINVAL;
  rerank_status st = rerank_check_args(nq, ng, d, dtype, k1, k2, layers, 0);
  if (st != RERANK_OK) return st;
  RR_CUDA(cudaSetDevice(ctx->device));
  int32_t* oi = nullptr;
  float* od = nullptr;
  RR_CUDA(cudaMalloc(&oi, sizeof(int32_t) * size_t(nq) * size_t(ng)));
  if (cudaMalloc(&od, sizeof(float) * size_t(nq) * size_t(ng)) != cudaSuccess) {
    cudaFree(oi);
    return RERANK_ENOMEM;
  }
  const int saved_timing = ctx->cfg.stage_timing;
  ctx->cfg.stage_timing = 1;
  const int prec = ctx->cfg.precision;
  const int64_t n = nq + ng;
  const int64_t col_tiles = (n + (prec == RERANK_PREC_FP32 ? 127 : 255)) / (prec == RERANK_PREC_FP32 ? 128 : 256);
  Tuning best = lookup_tuning(ctx, prec, n, d);
  best.sim_chunks = 0;
  double best_ms = 0.0;
  do {
    // 0. candidates kept beyond k1: more cost in the similarity epilogue and
    //    the refinement, fewer rows left for the recheck
    {
      double t0_best = 1e300;
      const int m_set[] = {-1, 8, 22, 30, 38};  // 38: the full 64-entry list for k1 = 26
      Tuning base0 = best;
      for (int m : m_set) {
        Tuning t = base0;
        t.rescore_m = m;
        double ms = 0.0;
        st = timed_run(ctx, t, xq, nq, xg, ng, d, dtype, k1, k2, layers, oi, od, stream, nullptr, &ms);
        if (st != RERANK_OK) break;
        if (ms < t0_best * 0.99) {
          t0_best = ms;
          best.rescore_m = m;
        }
      }
      if (st != RERANK_OK) break;
    }
    // 1. column chunks of the similarity stage (0 = the SM-count heuristic)
    const int chunk_set[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
    double t_best = 1e300;
    for (int c : chunk_set) {
      if (c > col_tiles) continue;
      Tuning t = best;
      t.sim_chunks = c;
      double ms = 0.0;
      st = timed_run(ctx, t, xq, nq, xg, ng, d, dtype, k1, k2, layers, oi, od, stream, "similarity_topk", &ms);
      if (st != RERANK_OK) break;
      if (ms < t_best * 0.99) {
        t_best = ms;
        best.sim_chunks = c;
      }
    }
    if (st != RERANK_OK) break;
    // 2. refinement order
    t_best = 1e300;
    Tuning base = best;
    for (int o : {1, 0}) {
      Tuning t = base;
      t.refine_order = o;
      double ms = 0.0;
      // the ordering pass is timed with the refinement it serves
      st = timed_run(ctx, t, xq, nq, xg, ng, d, dtype, k1, k2, layers, oi, od, stream, "refine", &ms);
      if (st != RERANK_OK) break;
      if (ms < t_best * 0.99) {
        t_best = ms;
        best.refine_order = o;
      }
    }
    if (st != RERANK_OK) break;
    // 3. propagation CTA width
    t_best = 1e300;
    base = best;
    for (int w : {8, 4, 16, 24}) {
      Tuning t = base;
      t.prop_warps = w;
      double ms = 0.0;
      st = timed_run(ctx, t, xq, nq, xg, ng, d, dtype, k1, k2, layers, oi, od, stream, "propagate", &ms);
      if (st != RERANK_OK) break;
      if (ms < t_best * 0.99) {
        t_best = ms;
        best.prop_warps = w;
      }
    }
    if (st != RERANK_OK) break;
    st = timed_run(ctx, best, xq, nq, xg, ng, d, dtype, k1, k2, layers, oi, od, stream, nullptr, &best_ms);
  } while (false);
  ctx->cfg.stage_timing = saved_timing;
  cudaFree(oi);
  cudaFree(od);
  if (st != RERANK_OK) return st;
  TuneEntry e;
  e.precision = prec;
  e.d = d;
  e.n_bucket = tune_bucket(n);
  e.t = best;
  e.ms = best_ms;
  bool replaced = false;
  for (TuneEntry& x : ctx->tune_table)
    if (x.precision == e.precision && x.d == e.d && x.n_bucket == e.n_bucket) {
      x = e;
      replaced = true;
    }
  if (!replaced) ctx->tune_table.push_back(e);
  if (!ctx->tune_path.empty() && !write_tune_file(ctx->tune_path, ctx->tune_table)) return RERANK_EINVAL;
  if (out) {
    out->sim_chunks = best.sim_chunks;
    out->prop_warps = best.prop_warps;
    out->refine_order = best.refine_order;
    out->rescore_m = best.rescore_m;
    out->n_bucket = e.n_bucket;
    out->ms = best_ms;
  }
  return RERANK_OK;
}

rerank_status rerank_tuning_lookup(const char* path, int precision, int64_t n, int d, rerank_tuning* out) {
  if (!path || !out || n < 1 || d < 1) return RERANK_EINVAL;
  std::vector<TuneEntry> entries;
  if (!read_tune_file(path, &entries)) return RERANK_EINVAL;
  const int nb = tune_bucket(n);
  for (const TuneEntry& e : entries)
    if (e.precision == precision && e.d == d && e.n_bucket == nb) {
      out->sim_chunks = e.t.sim_chunks;
      out->prop_warps = e.t.prop_warps;
      out->refine_order = e.t.refine_order;
      out->rescore_m = e.t.rescore_m;
      out->n_bucket = nb;
      out->ms = e.ms;
      return RERANK_OK;
    }
  return RERANK_EAGAIN;
}

}  // extern "C"

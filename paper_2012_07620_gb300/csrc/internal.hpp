// Host-side internals: the context, its device workspace, and the stage launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rerank.h"

namespace rr {

#define RR_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::rr::cuda_fail(e_, #call); \
  } while (0)

rerank_status cuda_fail(cudaError_t e, const char* what);
const char* last_cuda_error_text();

// Bump allocator over one device block.  A dry pass (base == nullptr) only
// measures; the real pass hands out 256-byte aligned sub-buffers.
struct Carver {
  char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

// Launch shapes chosen per (precision, d, n) by the autotuner or its defaults.
// None of them changes a result: only which thread computes what, and when.
struct Tuning {
  int sim_chunks = 0;      // column chunks P of the similarity top-K kernel (0 = from the SM count)
  int prop_warps = 8;      // warps per CTA of the propagation kernel
  int refine_order = 1;    // 1: refine rows cluster by cluster, 0: in index order
  int rescore_m = -1;      // candidates kept beyond k1 (-1: the context's cfg.rescore_m)
  int rank_threads = 1024; // threads per CTA of the final ranking kernel
};
struct TuneEntry {
  int precision = 0, d = 0, n_bucket = 0;
  Tuning t;
  double ms = 0.0;  // pipeline time measured with this entry
};
int tune_bucket(int64_t n);  // half-octave bucket of the vertex count

// Device pointers of one pipeline run (all inside the workspace block).
struct Buffers {
  // inputs staged from host memory, when the caller passed host buffers
  void* xq = nullptr;
  void* xg = nullptr;
  int32_t* out_idx = nullptr;
  float* out_dist = nullptr;
  // K0
  float* xhat = nullptr;         // np x dp, unit rows, zero padding
  void* xlow = nullptr;          // np x dp bf16 / fp8 copy for the tensor-core path
  float* xscale = nullptr;       // np fp8 row scales (1 / s_i)
  __nv_bfloat16* xhi = nullptr;  // np x dp: bf16(xhat) (the same array as xlow on the BF16 path)
  __nv_bfloat16* xlo = nullptr;  // np x dp: bf16(xhat - hi)
  float* err = nullptr;          // 3 x np: bounds on ||xhat - xlow||, ||lo||, ||xhat - hi - lo|| per row
  float* emax = nullptr;         // 4: their maxima
  // recheck of uncertified rows with the hi/lo split ("BF16x3")
  __nv_bfloat16* ahi = nullptr;  // np x dp: hi rows of the rows being rechecked, gathered
  __nv_bfloat16* alo = nullptr;  // np x dp: lo rows, gathered
  float* part3_s = nullptr;      // n x P3 x K
  int32_t* part3_i = nullptr;
  int* row_floor3 = nullptr;     // n
  int32_t* fb2_rows = nullptr;   // n: rows left for the exact scan
  int32_t* fb2_count = nullptr;
  int32_t* fb3_rows = nullptr;   // n: FP8 path, rows left after the single-product BF16 recheck stage
  int32_t* fb3_count = nullptr;
  int* row_floor = nullptr;      // n, shared K-th best per row (similarity kernels)
  int32_t* nb4 = nullptr;        // 4n: best candidates per row (processing order)
  int32_t* label = nullptr;      // n
  int32_t* order = nullptr;      // n: rows grouped by cluster
  int32_t* ord_cnt = nullptr;    // n + 1 scratch of the counting sort
  int32_t* ord_start = nullptr;  // n + 1
  int32_t* ord_fill = nullptr;   // n
  double* norm = nullptr;        // n, ||x_i|| in FP64 accuracy
  // K1 / K2
  float* part_s = nullptr;       // n x P x K
  int32_t* part_i = nullptr;
  int32_t* knn_idx = nullptr;    // n x k1
  float* knn_score = nullptr;
  int32_t* fb_rows = nullptr;    // rows to redo exactly (count in status)
  int32_t* fb_count = nullptr;
  // K3
  int32_t* indeg = nullptr;
  int32_t* fill = nullptr;
  int32_t* inptr = nullptr;      // n + 1
  int32_t* insrc = nullptr;      // n * k1
  int32_t* out_sorted = nullptr; // n * k1
  int32_t* in_sorted = nullptr;  // n * k1
  int32_t* rowcnt = nullptr;     // n
  int32_t* h0ptr = nullptr;      // n + 1
  int32_t* nbr = nullptr;        // n x (k2 + 1)
  float* nbr_w = nullptr;        // n x (k2 + 1)
  int32_t* nbr_n = nullptr;      // n
  // padded-CSR feature buffers: slots 0 and 1 alternate between layers,
  // slot 2 holds h^(0) (capacity 2 n k1)
  int64_t* start[3] = {nullptr, nullptr, nullptr};  // n + 1 (exclusive scan; [n] = total)
  int32_t* len[3] = {nullptr, nullptr, nullptr};
  int32_t* col[3] = {nullptr, nullptr, nullptr};
  float* val[3] = {nullptr, nullptr, nullptr};
  int32_t* ub = nullptr;         // n
  int32_t* big_rows = nullptr;    // n: rows the first propagation pass hands on
  int32_t* prop_spill = nullptr;  // n: per listed row, 1 when its 2,048-slot table overflowed
  int32_t* big_count = nullptr;
  float* hash_keys_vals = nullptr; // global hash tables of the big-row path
  float* rnorm = nullptr;        // n, 1/||h_i^(L)||
  // K5 / K6
  int32_t* colcnt = nullptr;     // n
  int64_t* colptr = nullptr;     // n + 1
  int32_t* csc_row = nullptr;
  float* csc_val = nullptr;
  uint32_t* rank_scratch = nullptr;
  int32_t* work = nullptr;       // 16: item counter of the similarity kernel
  // dense features (RERANK_FEAT_X)
  float* hd[2] = {nullptr, nullptr};  // np x dp each, alternating layers
  double* hinv = nullptr;             // np: 1 / ||h_i^(L)||
  float* xscore = nullptr;            // nq x ng final cosines
  // scan scratch
  int64_t* scan_tmp = nullptr;
};

struct Shape {
  int64_t nq = 0, ng = 0, n = 0, np = 0;
  int d = 0, dp = 0, dtype = 0;
  int k1 = 0, k2 = 0, layers = 0, K = 0, P = 0;
  int P3 = 0;              // candidate lists per row of the hi/lo recheck
  int P3g = 0;             // FP8 path: lists per row of the single-product BF16 recheck stage
  int K3 = 0;              // FP8 path: candidates per list of that stage (the longest list the kernels hold)
  int64_t topk = 0;
  bool host_in = false, host_out = false;
  bool knn_only = false;
  bool ext_feat = false;   // the unit rows and their copies live outside the workspace (serving)
  bool dense = false;      // h^(0) = x_i: dense layers and final cosines (RERANK_FEAT_X)
  int64_t cap_h = 0;       // elements per padded-CSR layer buffer
  int64_t cap_csc = 0;
  int hash_slots = 0;      // slots of each global hash table (big-row path)
  int rank_ctas = 0;
  int64_t rank_scratch_per_cta = 0;
  Tuning tune;             // launch shapes of this instance
};

struct ServeHandle;  // the request loop of a loaded gallery (serve.cu)

// A batched call captured as a CUDA graph.  key: everything the capture
// depended on (workspace, pointers, planned shapes); stage: the pinned
// instance tables its copy nodes upload.
struct BatchGraph {
  std::vector<int64_t> key;
  cudaGraphExec_t exec = nullptr;
  void* stage = nullptr;
  int64_t launches = 0;
  uint64_t stamp = 0;
};

struct StageTimer {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<const char*> names;
  cudaStream_t stream = nullptr;
  void mark(const char* name);
};

}  // namespace rr

struct rerank_ctx {
  rerank_config cfg{};
  int device = 0;
  int sm_count = 0;
  size_t smem_optin = 0;
  char* ws = nullptr;          // device workspace block
  size_t ws_bytes = 0;
  long long* d_status = nullptr;  // device status block (rr::kStCount int64)
  long long* h_status = nullptr;  // pinned host copy
  std::vector<rr::TuneEntry> tune_table;  // loaded from / written to tune_path
  const rr::Tuning* force_tune = nullptr;  // set while the autotuner measures a candidate
  std::string tune_path;
  int64_t cap_h_hint = 0;      // layer-buffer capacity learned from earlier overflows
  int64_t test_cap_h = 0;      // initial layer capacity forced by RERANK_TEST_CAP_H (tests only)
  int64_t cap_csc_hint = 0;
  rr::StageTimer timer;
  std::vector<float> stage_ms;
  std::vector<const char*> stage_names;
  rerank_info info{};
  int64_t launches = 0;
  rr::Buffers buf{};
  rr::Shape shape{};
  // batched calls: internal streams forked from the caller's, fork/join events,
  // and a pinned copy of every instance's status block
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;   // [0] fork, [1 + i] join of streams[i]
  // single calls with host outputs: results copied back while later queries are ranked
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> copy_events;
  long long* h_batch = nullptr;
  size_t h_batch_count = 0;
  void* h_stage = nullptr;  // pinned: instance tables of batched similarity launches
  size_t h_stage_bytes = 0;
  // batched calls replayed as CUDA graphs (least recently used evicted); all
  // dropped when the workspace or the pinned status block is reallocated,
  // since their copy and memset nodes name those allocations
  std::vector<rr::BatchGraph*> graphs;
  uint64_t graph_clock = 0;
  std::vector<uint64_t> graph_seen;  // hashes of recent keys not yet captured
  cudaStream_t cap_stream = nullptr;
  rr::ServeHandle* serve = nullptr;
};

namespace rr {

// ---- stage launchers (each enqueues on `s`; no host synchronisation) ----
int launch_normalize(const Shape& sh, const void* xq, const void* xg, float* xhat, double* norm, void* xlow,
                     __nv_bfloat16* xhi, __nv_bfloat16* xlo, float* inv_scale, float* err, float* emax,
                     int precision, long long* status, cudaStream_t s);
// Copy the hi/lo rows listed in rows[0 .. *count) to dst_hi/dst_lo[0 .. *count).
int launch_gather_rows(const int32_t* rows, const int32_t* count, const __nv_bfloat16* hi, const __nv_bfloat16* lo,
                       __nv_bfloat16* dst_hi, __nv_bfloat16* dst_lo, int64_t n, int dp, cudaStream_t s);
// row_floor: n ints of scratch (reset by the launcher) through which chunks of
// a row share their K-th best score.
int launch_sim_fp32_topk(const Shape& sh, const float* xhat, int* row_floor, float* part_s, int32_t* part_i,
                         int sm_count, cudaStream_t s);
// work (4 bytes, nullable): counter for the dynamic item order of the main pass.
int launch_sim_tc_topk(const Shape& sh, const void* xlow, bool fp8, const float* inv_scale, int* row_floor,
                       float* part_s, int32_t* part_i, long long* status, int sm_count, cudaStream_t s,
                       int32_t* work = nullptr);
// Rectangular block: rows of `a` (a_rows of them, vertices row0 ..) against the
// columns of `b` (b_cols, vertices col0 ..); per row P lists of its best K
// columns (vertex indices) in part_s/part_i [a_rows][P][K].  Rows and columns
// beyond the counts are never listed; `a` and `b` must hold at least
// max(count, 256) rows (the tensor maps span whole tiles).
int launch_sim_tc_rect_topk(const Shape& sh, const void* a, int64_t a_rows, int64_t row0, const void* b,
                            int64_t b_cols, int64_t col0, int chunks, bool fp8, const float* inv_scale,
                            int* row_floor, float* part_s, int32_t* part_i, long long* status, int sm_count,
                            cudaStream_t s);
// hi/lo split: S' = hi_i.hi_j + lo_i.hi_j + hi_i.lo_j for the rows rows[0 .. *count)
// (their hi/lo copies gathered in ahi/alo) against every column; lists indexed by
// position in `rows`, P3 chunks.
int launch_sim_tc_split_topk(const Shape& sh, int P3, const __nv_bfloat16* ahi, const __nv_bfloat16* alo,
                             const __nv_bfloat16* bhi, const __nv_bfloat16* blo, const int32_t* rows,
                             const int32_t* count, int* row_floor, float* part_s, int32_t* part_i,
                             long long* status, int sm_count, cudaStream_t s);

// One instance of a batched similarity launch: the instance's low-precision
// copy (np x dp) against itself, P lists of K per row.
struct TcBatchInst {
  const void* xlow;
  int64_t n, np;
  int dp, P, K;
  const float* inv_scale;
  int* row_floor;
  float* part_s;
  int32_t* part_i;
  long long* status;
};
// Up to 64 instances with the same tc_lists_per_chunk(dp, 1) in one persistent
// launch.  insts_dev: ninst * tc_batch_inst_bytes() of device memory; staging:
// as many bytes of pinned host memory, untouched until the launch has run.
int launch_sim_tc_batch(const TcBatchInst* in, int ninst, bool fp8, void* insts_dev, void* staging, int sm_count,
                        cudaStream_t s);
size_t tc_batch_inst_bytes();
int tc_batch_max_inst();
int tc_stall_hook();  // nonzero while the tensor-core kernels' test stall is set

// Gathered rows rows[0 .. *count) (their BF16 hi copies in ahi) against every
// column's hi copy, one product: the middle stage of the FP8 path's recheck.
int launch_sim_tc_gather_topk(const Shape& sh, int P, const __nv_bfloat16* ahi, const __nv_bfloat16* bhi,
                              const int32_t* rows, const int32_t* count, int* row_floor, float* part_s,
                              int32_t* part_i, long long* status, int sm_count, cudaStream_t s);

// Bound on |approximate score - S_ij| used to certify a row's candidate list.
struct ErrModel {
  int kind = 0;                  // 0: eps only; 1: one quantised copy; 2: hi/lo split; 3: the hi copy
  double eps = 0.0;              // accumulation and rounding part
  const float* err = nullptr;    // 3 x np per-row bounds (see Buffers::err)
  const float* emax = nullptr;
  int64_t np = 0;
};
// Rows: all n in index order; or rows[0 .. *count) (count == nullptr: n) in that order,
// with the candidate lists indexed by row (part_by_row) or by position in `rows`.
int launch_refine(const Shape& sh, const void* xq, const void* xg, const float* xhat,
                   const double* norm, const float* part_s, const int32_t* part_i, int P, const ErrModel& em,
                   const int32_t* rows, const int32_t* count, bool part_by_row,
                   int32_t* knn_idx, float* knn_score, int32_t* fb_rows, int32_t* fb_count,
                   long long* status, cudaStream_t s, int64_t grid_rows = -1,  // grid_rows: bound on the row count
                   int fb_stat = -1);  // status slot counting the rows passed on (-1: by the row set)
size_t tc_smem_bytes();
bool tc_pairs();      // main similarity pass on CTA pairs (cta_group::2)
int tc_item_rows();   // A rows per work item of the main pass: 256 on pairs, else 128
int tc_kmax();
// Candidate lists per row and column chunk written by the tensor-core kernels
// (their epilogue warp groups) for K depth dp and `segs` products per k-block.
int tc_lists_per_chunk(int dp, int segs);
// Candidates per row kept by the exact last-resort scan: k1 + 16 (at most
// the list capacity and n), whatever margin the first pass used.
int fallback_k(const Shape& sh);
int launch_refine_fallback(const Shape& sh, const void* xq, const void* xg, const float* xhat,
                            const double* norm, int32_t* knn_idx, float* knn_score,
                            const int32_t* fb_rows, const int32_t* fb_count, float* scratch_s,
                            int32_t* scratch_i, long long* status, int sm_count, cudaStream_t s);
// Rows grouped cluster by cluster (label propagation over the best 4 candidates).
int launch_cluster_order(const Shape& sh, const float* part_s, const int32_t* part_i, int32_t* nb, int32_t* label,
                         int32_t* cnt, int32_t* start, int32_t* fill, int32_t* order, cudaStream_t s);
int launch_scan(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s);
int launch_scan32(const int32_t* in, int64_t n, int32_t* out, cudaStream_t s);
int launch_graph(const Shape& sh, const Buffers& b, float alpha, int aggregator, int feature,
                  long long* status, cudaStream_t s);
// A serving request's graph (A* features) from the resident gallery graph:
// only rows whose A* row can change (the queries, the touched gallery rows
// touched[0 .. *n_touched) and the old and new targets of their lists) are
// built; the others are the resident rows (rst / rln / rcol / rval, gallery
// indices) shifted by Q.  aff / src: n bytes of scratch each.  Same CSR,
// message lists and nnz counter as launch_graph.
int launch_graph_incremental(const Shape& sh, const Buffers& b, int64_t Q, const int32_t* touched,
                             const int32_t* n_touched, const int32_t* res_knn, const int64_t* rst,
                             const int32_t* rln, const int32_t* rcol, const float* rval, uint8_t* aff,
                             uint8_t* src, float alpha, int aggregator, long long* status, cudaStream_t s);
// Rows of a layer whose output is known elsewhere are copied instead of
// recomputed (serving: the resident gallery's own layer rows, whose inputs a
// request left unchanged).  Row i >= shift with changed[i] == 0 copies row
// i - shift of the compact CSR (rstart, rlen, rcol, rval), columns + shift.
struct LayerReuse {
  const uint8_t* changed = nullptr;
  const int64_t* rstart = nullptr;
  const int32_t* rlen = nullptr;
  const int32_t* rcol = nullptr;
  const float* rval = nullptr;
  int64_t shift = 0;
};
// Compact copy of a padded-CSR layer (rows 0 .. n-1): cstart = exclusive scan
// of len (n + 1 entries), then the rows packed into ccol / cval.
int launch_layer_compact(int64_t n, const int64_t* start, const int32_t* len, const int32_t* col, const float* val,
                         const int64_t* cstart, int32_t* ccol, float* cval, cudaStream_t s);
int launch_propagate(const Shape& sh, const Buffers& b, int src, int dst, int aggregator,
                      long long* status, int sm_count, const Tuning& t, cudaStream_t s,
                      const LayerReuse* reuse = nullptr, long long* nnz_slot = nullptr);
// rows_sel (nullable): only rows with rows_sel[i] != 0 get their norm.
int launch_row_norms(const Shape& sh, const Buffers& b, int src, const long long* status, cudaStream_t s,
                     const uint8_t* rows_sel = nullptr);
int launch_rank(const Shape& sh, const Buffers& b, int src, int32_t* out_idx, float* out_dist,
                 long long* status, int sm_count, const Tuning& t, cudaStream_t s);
// Gallery column lists known elsewhere (serving: the gallery graph's own final
// layer as CSC, gallery-local rows and columns, values scaled by row norms).
// Column c >= shift of the union maps to resident column c - shift; entries of
// gallery rows g with changed[g] != 0 are skipped (those rows are in the
// request's own lists).
struct RankReuse {
  const int64_t* colptr = nullptr;
  const int32_t* row = nullptr;
  const float* val = nullptr;
  const uint8_t* changed = nullptr;
  int64_t shift = 0;
};
// The same in two parts: the gallery's column lists once, then queries [q0, q1)
// (out_idx / out_dist still address the whole nq x topk output).  rows_sel
// (per union row, nullable): only gallery rows with rows_sel[r] != 0 enter the lists.
int launch_rank_prep(const Shape& sh, const Buffers& b, int src, long long* status, cudaStream_t s,
                     const uint8_t* rows_sel = nullptr);
int launch_rank_queries(const Shape& sh, const Buffers& b, int src, int32_t* out_idx, float* out_dist, int64_t q0,
                        int64_t q1, long long* status, int sm_count, const Tuning& t, cudaStream_t s,
                        const RankReuse* reuse = nullptr);

// Dense initial features (RERANK_FEAT_X): one propagation layer hin -> hout
// (np x dp rows, Eq. 13-14 with the graph's message lists), the final cosines
// of every query row with every gallery row into S (nq x ng), and their
// ranking (one query per CTA, sort scratch rank_scratch_words(ng) per CTA).
int launch_dense_layer(const Shape& sh, const float* hin, float* hout, const int32_t* nbr, const float* nbr_w,
                       const int32_t* nbr_n, int aggregator, cudaStream_t s);
int launch_dense_scores(const Shape& sh, const float* h, double* inv, float* S, cudaStream_t s);
int launch_rank_dense(const Shape& sh, const float* S, int32_t* out_idx, float* out_dist, uint32_t* scratch,
                      long long* status, cudaStream_t s);

size_t rank_smem_bytes(int64_t ng, int threads);
// 32-bit words of global scratch per ranking CTA for a gallery of ng.
int64_t rank_scratch_words(int64_t ng);

// ---- pipeline pieces shared by the single, batched and serving entry points ----
// One pipeline instance: its shape, its buffers and its device status block.
struct JobRun {
  Shape sh;
  Buffers b;
  long long* st = nullptr;
  const void* xq = nullptr;
  const void* xg = nullptr;
  int32_t* out_idx = nullptr;
  float* out_dist = nullptr;
};
bool is_host_ptr(const void* p);
size_t type_size(int dtype);
int choose_chunks(int64_t row_blocks, int64_t col_tiles, int sm_count, int forced);
size_t carve(Carver& c, const Shape& sh, Buffers& b, int sm_count, int precision);
rerank_status plan_shape(const rerank_ctx* ctx, int64_t nq, int64_t ng, int d, int dtype, int k1, int k2,
                         int layers, int64_t topk, bool knn_only, bool host_in, bool host_out, int64_t cap_hint,
                         Shape* out, const Tuning* tune = nullptr);  // tune: override of the table lookup
// copy_overlap: host outputs are copied back in parts while later queries are
// ranked (single calls only; batched instances copy on their own stream).
// phases: which parts to enqueue (status reset, copies in and normalisation /
// the similarity stage / everything after it).
enum { kPhasePre = 1, kPhaseSim = 2, kPhasePost = 4, kPhaseAll = 7 };
rerank_status enqueue_job(rerank_ctx* ctx, const JobRun& j, cudaStream_t s, StageTimer* tm, int64_t* launches,
                          bool copy_overlap = false, int phases = kPhaseAll);
rerank_status map_status(const long long* h, int precision, rerank_info* info, int64_t* need);
int launch_status_reset(long long* st, cudaStream_t s);
// Tuning of an instance: the table entry for (precision, d, bucket of n), else defaults.
Tuning lookup_tuning(const rerank_ctx* ctx, int precision, int64_t n, int d);
bool read_tune_file(const std::string& path, std::vector<TuneEntry>* out);
bool write_tune_file(const std::string& path, const std::vector<TuneEntry>& entries);
// Stop the request loop of a loaded gallery and free it (no-op without one).
rerank_status serve_stop(rerank_ctx* ctx);
int propagate_warp_slots();

}  // namespace rr

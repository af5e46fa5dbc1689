/*
 * rerank.h -- C ABI of the GB300 GNN re-ranking library.
 *
 * The operation is Algorithm 1 of Zhang et al., "Understanding Image Retrieval
 * Re-Ranking: A Graph Neural Network Perspective" (arXiv 2012.07620, Sec. 3.3):
 *   1. S_ij = cos(x_i, x_j) over X_u = X_q u X_g                     (Eq. 7)
 *   2. N(i, k1) = the k1 most similar vertices of row i of S            (Eq. 8)
 *   3. A* = (A + A^T) / 2: 1 for reciprocal neighbours, 1/2 one-way     (Eq. 9, 10)
 *   4. h_i^(0) = row i of A*; edges e_ij = S_ij for j in N(i, k2)       (Eq. 11, 12)
 *   5. L layers of h_i <- h_i + sum_{j in N(i,k2)} e_ij^alpha h_j, then
 *      every h_i is scaled to unit L2 norm                              (Eq. 13, 14)
 *   6. each query's gallery list sorted by cos(h_q, h_g)                (Alg. 1 step 7)
 *
 * Conventions shared by every call:
 *   - Vertex (union) index: queries first, i = 0 .. nq-1, then the gallery,
 *     i = nq + g.  Self is a member of its own neighbourhood with S_ii = 1.
 *   - Every ordering (neighbour lists, final lists) is by score descending,
 *     ties to the lower index.
 *   - Buffers are row-major and contiguous.  Unless a call says otherwise a
 *     buffer may be device memory or host memory; calls that receive any
 *     host buffer copy through the context's device workspace and return only
 *     after the results are in the host buffers.  With device buffers only,
 *     work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) and the call returns once the error word has been read back
 *     (one stream synchronisation at the end of the call).
 *   - The caller owns every buffer it passes; the library never frees them.
 *     The context owns its device workspace, which grows on demand up to
 *     `hbm_budget` and is reused by later calls.
 *   - Every call returns a status and never aborts the process.  A context
 *     must not be used by two host threads at once.
 */
#ifndef RERANK_H
#define RERANK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rerank_ctx rerank_ctx;

typedef enum {
  RERANK_OK = 0,
  RERANK_EINVAL = 1,       /* invalid argument, or an input row that is non-finite or all zero */
  RERANK_ENOMEM = 2,       /* a device or pinned-host allocation failed */
  RERANK_EBUDGET = 3,      /* the workspace for this call would exceed cfg.hbm_budget */
  RERANK_ECUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  RERANK_ETIMEOUT = 5,     /* a bounded device-side wait ran out */
  RERANK_EINTERNAL = 6,    /* an internal consistency check failed (see rerank_last_info) */
  RERANK_EUNSUPPORTED = 7, /* a valid combination that this build does not implement */
  RERANK_EAGAIN = 8        /* serving: no result yet, or the admission queue is full */
} rerank_status;

/* Similarity precision of step 1 (the one dense contraction). */
enum { RERANK_PREC_FP32 = 0, RERANK_PREC_BF16 = 1, RERANK_PREC_FP8 = 2 };
/* Element type of the caller's feature buffers. */
enum { RERANK_DTYPE_F32 = 0, RERANK_DTYPE_BF16 = 1 };
/* The aggregate of Eq. 13. */
enum { RERANK_AGG_SUM = 0, RERANK_AGG_MEAN = 1, RERANK_AGG_MAX = 2 };
/* Initial vertex feature (Sec. 4.2, Table 1): A*_i (Eq. 11), A_i, or x_i. */
enum { RERANK_FEAT_ASTAR = 0, RERANK_FEAT_A = 1, RERANK_FEAT_X = 2 };

typedef struct {
  int device;                /* CUDA device ordinal */
  int precision;             /* RERANK_PREC_*; default FP32 */
  int rescore_m;             /* extra candidates kept per row before exact rescoring; default 16
                                (an autotuner table entry may override it per instance size) */
  float alpha;               /* exponent of Eq. 14; default 2 */
  int aggregator;            /* RERANK_AGG_*; default SUM (Sec. 4.1); MEAN divides the k2 messages'
                                weights by k2; MAX takes their element-wise max (Eq. 13 variants) */
  int feature_mode;          /* RERANK_FEAT_*; default ASTAR.  X: h^(0) = x_i / ||x_i|| (dense
                                d-dimensional rows), propagated densely, final cosines over d;
                                rerank_run only (rerank_run_batch and serving return EUNSUPPORTED) */
  size_t hbm_budget;         /* workspace cap in bytes; 0 = no cap */
  const char* autotune_path; /* JSON tuning table to read (and to write from rerank_autotune); NULL = built-in */
  int stage_timing;          /* nonzero: record CUDA events around every stage (rerank_stage_times) */
} rerank_config;

/* Fill `cfg` with the defaults listed above. */
void rerank_config_init(rerank_config* cfg);

/* Create a context on cfg->device.  *out receives the handle.
 * Errors: EINVAL (null pointers, bad enum values), ECUDA (no usable device,
 * or not a compute capability 10.3 GPU), ENOMEM. */
rerank_status rerank_create(rerank_ctx** out, const rerank_config* cfg);

/* Release the context and its workspace.  Accepts NULL. */
rerank_status rerank_destroy(rerank_ctx* ctx);

/* Static text for a status code. */
const char* rerank_strerror(rerank_status status);

/* The CUDA call and CUDA error text behind the calling thread's last ECUDA or
 * ENOMEM status ("" when there was none).  The string belongs to the library
 * and stays valid until the thread's next failing call. */
const char* rerank_last_cuda_error(void);

/* Host-only validation of the size arguments of rerank_run (no GPU needed):
 * EINVAL unless nq >= 1, ng >= 1, d >= 1, dtype valid, 1 <= k2 <= k1 <= nq+ng,
 * layers >= 0 and 0 <= topk_out <= ng. */
rerank_status rerank_check_args(int64_t nq, int64_t ng, int d, int dtype, int k1, int k2,
                                int layers, int64_t topk_out);

/* Algorithm 1 end to end (steps 1-6 above).
 *   xq        nq x d features of the queries (dtype), raw: the call normalises them
 *   xg        ng x d features of the gallery
 *   k1, k2    neighbourhood sizes of Eq. 8 and Eq. 12
 *   layers    number of propagation layers L (Eq. 14)
 *   topk_out  length of each output list; 0 = the whole gallery (ng)
 *   out_idx   nq x topk_out int32: gallery indices (0 .. ng-1), best first
 *   out_dist  nq x topk_out float: 1 - cos(h_q, h_g) in the same order
 *   stream    cudaStream_t for the enqueued work (NULL = default stream)
 * Errors: EINVAL (as rerank_check_args, null pointers, or an input row that
 * is non-finite or has zero norm), EBUDGET, ENOMEM, ECUDA, EINTERNAL;
 * EUNSUPPORTED when k1 > RERANK_MAX_K1.  Each row's candidate list holds 64
 * entries; capping k1 at 48 keeps 16 of them beyond the k1-th, so that the
 * exact last-resort scan can always bound the columns it leaves out. */
#define RERANK_MAX_K1 48
rerank_status rerank_run(rerank_ctx* ctx, const void* xq, int64_t nq, const void* xg, int64_t ng,
                         int d, int dtype, int k1, int k2, int layers, int64_t topk_out,
                         int32_t* out_idx, float* out_dist, void* stream);

/* One independent instance of Algorithm 1 for rerank_run_batch.  Fields as
 * the arguments of rerank_run; `status` is written by the call. */
typedef struct {
  const void* xq;
  int64_t nq;
  const void* xg;
  int64_t ng;
  int d;
  int dtype;
  int k1, k2, layers;
  int64_t topk_out;
  int32_t* out_idx;
  float* out_dist;
  rerank_status status; /* out: this instance's result code */
} rerank_job;

/* Many independent instances of Algorithm 1 (each exactly as rerank_run would
 * compute it; the paper defines one instance at a time, Sec. 3.3) in one call.
 * The instances share one workspace block and run concurrently on the GPU:
 * their stages are enqueued on internal streams forked from `stream` and
 * joined back into it, largest instances first.  With the BF16 / FP8
 * precisions the similarity + top-K stage of up to 64 instances runs as one
 * persistent tensor-core launch whose CTAs walk the work items of all of
 * them.  A call whose inputs and outputs are all device or pinned host memory
 * is captured as a CUDA graph the second time its pointers and shapes occur
 * and replayed by later calls with the same ones (the context keeps the 4
 * most recently used graphs).
 * The call reads every instance's status with one synchronisation; an
 * instance whose propagation buffers overflowed is rerun alone.
 *   jobs    array of njobs instances; inputs and outputs may be host or device
 *           memory, as for rerank_run
 * Returns OK when every instance succeeded, else the first failing status
 * (each jobs[i].status holds its own).  Argument errors of any instance
 * return EINVAL before anything runs. */
rerank_status rerank_run_batch(rerank_ctx* ctx, rerank_job* jobs, int njobs, void* stream);

/* ---- Serving: a resident gallery and a request loop ----
 *
 * Each request brings nq new query vectors and is answered exactly as
 * Algorithm 1 on X_u = (its queries) u (the resident gallery), queries first
 * (Sec. 3.3): no other request's queries take part.  What depends on the
 * gallery alone is computed once at load and kept on the device: the unit
 * rows and their BF16/FP8 copies, every gallery row's candidate list and its
 * exact top-k1 list.  Per request the library scores the queries against
 * X_u and the gallery against the queries (tensor cores), re-derives the
 * exact top-k1 list of every gallery row that a query can enter (the others
 * keep their resident lists, which stay exact), and runs the graph,
 * propagation and ranking stages on X_u.
 *
 * Requests are admitted into slots: each slot owns a stream and the device
 * buffers of one request of up to max_query queries.  The slot count is set
 * at load by the context's hbm_budget (every slot must fit, beside the
 * resident gallery) and by `slots`.  A request submitted while every slot is
 * busy waits in a host queue and starts as soon as a slot frees, while the
 * other slots' work is still on the GPU; slots run concurrently.  Results
 * depend only on the request and the gallery, never on which other requests
 * share the GPU.  Tensor-core precision only (cfg.precision BF16 or FP8).
 * One thread waits on a ticket at a time.  The caller keeps a request's buffers
 * alive and unchanged until rerank_wait has returned its final status. */
typedef struct {
  int64_t max_query; /* largest nq of a request, 1 .. 1024 */
  int slots;         /* concurrent requests on the GPU; 0 = as many as hbm_budget allows, at most 8 */
  int k1, k2, layers;
} rerank_serve_config;

typedef struct {
  const void* xq;   /* nq x d query features (host or device memory), the gallery's dtype */
  int64_t nq;       /* 1 .. max_query */
  int64_t topk_out; /* length of each output list; 0 = the whole gallery */
  int32_t* out_idx; /* nq x topk_out (host or device), gallery indices best first */
  float* out_dist;  /* nq x topk_out, 1 - cos(h_q, h_g) */
  void* stream;     /* cudaStream_t on which the caller produced xq (NULL = legacy default stream):
                       the request reads xq only after the work queued there before the submit */
} rerank_request;

typedef struct {
  rerank_status status; /* the request's result code */
  double queue_ms;      /* submit -> its work enqueued on a slot */
  double total_ms;      /* submit -> results in the output buffers (host clock) */
  int slot;             /* slot that ran it */
} rerank_ticket_info;

/* Load the resident gallery (ng x d, host or device memory; copied) and start
 * the request loop.  Synchronous.  Errors: EINVAL (sizes, k2 > k1, ng <
 * k1 + rescore_m, max_query < 1), EUNSUPPORTED (FP32 precision, or a gallery
 * already loaded), EBUDGET (the resident data and one slot exceed hbm_budget),
 * ENOMEM, ECUDA, and any status of the gallery's own neighbour lists. */
rerank_status rerank_gallery_load(rerank_ctx* ctx, const void* xg, int64_t ng, int d, int dtype,
                                  const rerank_serve_config* sc);

/* Queue one request; *ticket identifies it.  The caller keeps the request's
 * buffers alive and untouched until rerank_wait reports it finished.
 * Errors: EINVAL (null pointers, nq outside 1 .. max_query, topk_out > ng),
 * EUNSUPPORTED (no gallery loaded). */
rerank_status rerank_submit(rerank_ctx* ctx, const rerank_request* req, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: without limit) for a request.  Returns EAGAIN
 * if it is still running (the ticket stays valid), else the request's status;
 * *info (may be NULL) receives its timings.  A finished ticket is released by
 * this call.  EINVAL for an unknown ticket. */
rerank_status rerank_wait(rerank_ctx* ctx, uint64_t ticket, int timeout_ms, rerank_ticket_info* info);

/* Counters of the request loop. */
typedef struct {
  int slots;                 /* slots admitted by the budget */
  int max_in_flight;         /* most requests on the GPU at once so far */
  int64_t completed;
  int64_t touched_rows;      /* gallery rows re-derived, summed over requests */
  int64_t resident_bytes;    /* gallery data kept on the device */
  int64_t slot_bytes;        /* device memory of one slot */
  int reuse_layers;          /* 1: the gallery's own graph and layers are kept, and a request
                                recomputes only the layer rows whose inputs it changes */
  int64_t recomputed_rows;   /* layer rows recomputed, summed over layers and requests (the
                                rest were taken from the gallery's own layers) */
} rerank_serve_info;
rerank_status rerank_serve_info_get(const rerank_ctx* ctx, rerank_serve_info* info);

/* Finish every queued and running request, stop the loop and free the
 * gallery and the slots.  Also done by rerank_destroy. */
rerank_status rerank_gallery_unload(rerank_ctx* ctx);

/* ---- Autotuner ----
 * Launch shapes per (precision, d, bucket of N = nq + ng; buckets are half
 * octaves, floor(2 log2 N)).  None of them changes a result, only the work
 * decomposition (the paper fixes no schedule; these are GPU choices):
 *   sim_chunks    column chunks of the similarity top-K kernel (0 = SM-count heuristic)
 *   prop_warps    warps per CTA of the propagation kernel
 *   refine_order  1 = refine rows cluster by cluster, 0 = in index order
 *   rescore_m     candidates kept beyond k1 (-1 = cfg.rescore_m); the lists
 *                 stay exact for any value, only the work moves between stages.
 *                 Serving always uses cfg.rescore_m. */
typedef struct {
  int sim_chunks;
  int prop_warps;
  int refine_order;
  int rescore_m;
  int n_bucket;
  double ms; /* pipeline time measured with this choice */
} rerank_tuning;

/* Time the pipeline on the caller's instance under candidate launch shapes
 * (coordinate descent, median of three runs per candidate), store the best
 * for this (precision, d, N bucket) in the context, and, when
 * cfg.autotune_path was set, rewrite that JSON file with the context's whole
 * table.  Later calls of this context (and contexts created with the same
 * path) use the entry for every instance in the bucket.  Synchronous; runs
 * the instance about 60 times.  *out (may be NULL) receives the choice.
 * Errors: as rerank_run; EINVAL if the table file cannot be written. */
rerank_status rerank_autotune(rerank_ctx* ctx, const void* xq, int64_t nq, const void* xg, int64_t ng, int d,
                              int dtype, int k1, int k2, int layers, rerank_tuning* out, void* stream);

/* Host only: the entry of a tuning table file for (precision, n, d).
 * EINVAL if the file is missing or unreadable, EAGAIN if it has no entry. */
rerank_status rerank_tuning_lookup(const char* path, int precision, int64_t n, int d, rerank_tuning* out);

/* Steps 1-2 only: the exact top-k neighbour lists of every vertex of X (Eq. 7-8).
 *   x          n x d features (dtype)
 *   out_idx    n x k int32, sorted by (S desc, index asc); out_idx[i*k] == i
 *              unless a lower-indexed vertex has exactly the same direction
 *   out_score  n x k float: S of each listed pair, the FP32 dot product of the
 *              unit rows: |out_score - S| <= (d_p/32 + 10) * 2^-24 * 1.01 with
 *              d_p = d rounded up to 64 (pairs near a tie are recomputed in FP64)
 * Errors: as rerank_run. */
rerank_status rerank_knn(rerank_ctx* ctx, const void* x, int64_t n, int d, int dtype, int k,
                         int32_t* out_idx, float* out_score, void* stream);

/* rerank_knn without a context and without allocating anything.
 *
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: code running inside a framework whose memory
 * pool owns the whole GPU, real-time loops that cannot afford an allocation,
 * and code that must not grow its footprint at run time.  Instead of a
 * workspace, it uses one fixed scratch area compiled into the library
 * (RERANK_KNN_NOALLOC_SCRATCH_BYTES = 13 MiB) that every GPU which loads the
 * library keeps until the process exits.
 *
 *   x, out_idx, out_score, n, d, dtype, k: as rerank_knn, but all three buffers
 *   must be device memory of the current device, or managed memory (EINVAL
 *   otherwise: host memory, or memory of another GPU).
 * Limits: n <= RERANK_KNN_NOALLOC_MAX_N, d <= RERANK_KNN_NOALLOC_MAX_D,
 * k <= RERANK_KNN_NOALLOC_MAX_K; larger sizes return EBUDGET and nothing runs.
 * The first call on a device looks up the scratch area's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept for the life of the process: do not call this entry
 * point again on a device after cudaDeviceReset of that device.
 * All calls share the one scratch area: two calls whose work overlaps on the
 * GPU (for instance on two streams, or from two host threads) race and give
 * wrong results.  Calls on one stream, one after another, are safe.  The call
 * returns after a stream synchronisation, with the status of the device work.
 * Errors: EINVAL (arguments, host or foreign-device buffers, non-finite or
 * zero rows), EBUDGET (sizes over the limits), ECUDA (a CUDA call failed),
 * ETIMEOUT (a bounded device wait ran out), EUNSUPPORTED (device index 64 or
 * higher), EINTERNAL (a result could not be certified). */
#define RERANK_KNN_NOALLOC_SCRATCH_BYTES (13u << 20)
#define RERANK_KNN_NOALLOC_MAX_N 4096
#define RERANK_KNN_NOALLOC_MAX_D 256
#define RERANK_KNN_NOALLOC_MAX_K 48
rerank_status rerank_knn_noalloc(const void* x, int64_t n, int d, int dtype, int k, int32_t* out_idx,
                                 float* out_score, void* stream);

/* Counters of the last rerank_run / rerank_knn call on this context. */
typedef struct {
  int64_t n_vertices;
  int64_t candidates_per_row;  /* K = min(k1 + m, n), m = rescore_m or the tuned margin */
  int64_t fp64_rescored;       /* candidate scores recomputed in FP64 near a tie */
  int64_t fallback_rows;       /* rows whose first candidate list could not be certified */
  int64_t exact_scan_rows;     /* rows finally redone by the exact FP32 scan of all columns */
  int64_t h_nnz[9];            /* nnz of h^(0) .. h^(min(L,8)); zero after a batched call */
  int64_t workspace_bytes;     /* device workspace held by the context */
  int64_t kernel_launches;     /* kernels of this library launched by the call (last attempt) */
  int32_t error_bits;          /* device error word of the last call (0 = clean) */
  int32_t bad_row;             /* first offending input row for EINVAL from the device, else -1 */
} rerank_info;

rerank_status rerank_last_info(const rerank_ctx* ctx, rerank_info* info);

/* Per-stage device times (ms) of the last call, when cfg.stage_timing was set.
 * Writes up to `cap` entries and the number of stages to *count; names[i]
 * (static strings) label them.  EINVAL when timing was not enabled. */
rerank_status rerank_stage_times(const rerank_ctx* ctx, float* ms, const char** names, int cap,
                                 int* count);

/* Copy an intermediate array of the last call into `dst` (device or host).
 * `what` selects it; *bytes receives the array's size.  With dst == NULL only
 * the size is returned.  ECUDA/EINVAL on failure, EINVAL if cap is too small. */
enum {
  RERANK_DBG_KNN_IDX = 0,    /* n x k1 int32 */
  RERANK_DBG_KNN_SCORE = 1,  /* n x k1 float */
  RERANK_DBG_H0_ROWPTR = 2,  /* n+1 int32: CSR of h^(0) = A* rows, columns ascending */
  RERANK_DBG_H0_COL = 3,     /* nnz int32 */
  RERANK_DBG_H0_VAL = 4,     /* nnz float */
  RERANK_DBG_HL_START = 5,   /* n int64: row start of h^(L) in the padded CSR */
  RERANK_DBG_HL_LEN = 6,     /* n int32: row length of h^(L) */
  RERANK_DBG_HL_COL = 7,     /* capacity int32 (read rows through START/LEN; columns in no set order) */
  RERANK_DBG_HL_VAL = 8,     /* capacity float */
  RERANK_DBG_PART_S = 9,     /* n x P x K float: per-chunk candidate scores of the similarity kernel */
  RERANK_DBG_PART_I = 10,    /* n x P x K int32: their column indices (0x7fffffff = empty slot) */
  RERANK_DBG_QERR = 11,      /* n_pad float: per-row bound on ||unit row - its BF16/FP8 copy|| (tensor-core path) */
  RERANK_DBG_HL_DENSE = 12   /* n x d_p float (d_p = d rounded up to 64, zero padded): h^(L) of a
                                RERANK_FEAT_X run */
};
rerank_status rerank_debug_copy(const rerank_ctx* ctx, int what, void* dst, size_t cap,
                                size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* RERANK_H */

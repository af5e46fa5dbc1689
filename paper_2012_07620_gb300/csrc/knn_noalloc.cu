// rerank_knn_noalloc: the exact neighbour lists of rerank_knn for callers
// that may not allocate device memory (a framework's memory pool owns the
// GPU, a latency-bound loop cannot wait for an allocation, or the process
// must keep a fixed footprint).  All temporaries live in one file-scope
// __device__ array of fixed size; the stages are the same kernels that
// rerank_knn launches, given pointers into that array.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "internal.hpp"

namespace rr {

double rescore_eps(int dp);
int fallback_warps();

namespace {

constexpr int64_t kMaxN = RERANK_KNN_NOALLOC_MAX_N;
constexpr int kMaxD = RERANK_KNN_NOALLOC_MAX_D;
constexpr int kMaxK = 64;  // candidate list capacity (k + 16 for the largest k)
static_assert(RERANK_KNN_NOALLOC_MAX_K + 16 <= kMaxK, "candidate lists of the largest k");
constexpr int kChunks = 4;      // column chunks of the similarity kernel
constexpr int kFbCtas = 16;     // CTAs of the exact fallback kernel
constexpr int kFbWarps = 32;    // warps per fallback CTA (as the fallback kernel uses)
constexpr int64_t kMaxNp = (kMaxN + 127) / 128 * 128;
constexpr int64_t kMaxDp = (kMaxD + 63) / 64 * 64;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
// Byte offsets of every temporary inside the scratch array.
constexpr size_t kOffStatus = 0;
constexpr size_t kOffFbCount = al(kOffStatus + sizeof(long long) * kStCount);
constexpr size_t kOffXhat = al(kOffFbCount + sizeof(int32_t) * 4);
constexpr size_t kOffNorm = al(kOffXhat + sizeof(float) * kMaxNp * kMaxDp);
constexpr size_t kOffPartS = al(kOffNorm + sizeof(double) * kMaxNp);
constexpr size_t kOffPartI = al(kOffPartS + sizeof(float) * kMaxN * kChunks * kMaxK);
constexpr size_t kOffFbRows = al(kOffPartI + sizeof(int32_t) * kMaxN * kChunks * kMaxK);
constexpr size_t kOffFbS = al(kOffFbRows + sizeof(int32_t) * kMaxN);
constexpr size_t kOffFbI = al(kOffFbS + sizeof(float) * kFbCtas * kFbWarps * kMaxK);
constexpr size_t kOffFloor = al(kOffFbI + sizeof(int32_t) * kFbCtas * kFbWarps * kMaxK);
constexpr size_t kTotal = al(kOffFloor + sizeof(int32_t) * kMaxN);
static_assert(kTotal <= RERANK_KNN_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

// The scratch area.  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[RERANK_KNN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

__global__ void noalloc_reset(long long* st, int32_t* fb_count) {
  const int t = threadIdx.x;
  if (t < kStCount) st[t] = (t == kStBadRow) ? LLONG_MAX : 0;
  if (t == 0) *fb_count = 0;
}

// Device address of the scratch area on the current device (looked up once per device).
rerank_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return RERANK_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return RERANK_OK;
}

// Device memory of device `dev` (or managed memory): a buffer on another GPU
// would be a peer access from these kernels, which faults without peer access.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace rr

using namespace rr;

extern "C" rerank_status rerank_knn_noalloc(const void* x, int64_t n, int d, int dtype, int k, int32_t* out_idx,
                                            float* out_score, void* stream) {
  if (!x || !out_idx || !out_score) return RERANK_EINVAL;
  if (n < 1 || d < 1 || k < 1 || k > n || (dtype != RERANK_DTYPE_F32 && dtype != RERANK_DTYPE_BF16))
    return RERANK_EINVAL;
  if (n > kMaxN || d > kMaxD || k > RERANK_KNN_NOALLOC_MAX_K) return RERANK_EBUDGET;
  int dev = 0;
  RR_CUDA(cudaGetDevice(&dev));
  if (!on_device(x, dev) || !on_device(out_idx, dev) || !on_device(out_score, dev)) return RERANK_EINVAL;
  if (fallback_warps() != kFbWarps) return RERANK_EINTERNAL;
  unsigned char* base = nullptr;
  rerank_status st = scratch_address(dev, &base);
  if (st != RERANK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  Shape sh;
  sh.nq = n;
  sh.ng = 0;
  sh.n = n;
  sh.np = (n + 127) / 128 * 128;
  sh.d = d;
  sh.dp = (d + 63) / 64 * 64;
  sh.dtype = dtype;
  sh.k1 = k;
  sh.k2 = 1;
  sh.knn_only = true;
  sh.K = int(std::min<int64_t>(std::min<int64_t>(int64_t(k) + 16, n), kMaxK));
  sh.P = int(std::min<int64_t>(kChunks, sh.np / 128));

  long long* status = reinterpret_cast<long long*>(base + kOffStatus);
  int32_t* fb_count = reinterpret_cast<int32_t*>(base + kOffFbCount);
  float* xhat = reinterpret_cast<float*>(base + kOffXhat);
  double* norm = reinterpret_cast<double*>(base + kOffNorm);
  float* part_s = reinterpret_cast<float*>(base + kOffPartS);
  int32_t* part_i = reinterpret_cast<int32_t*>(base + kOffPartI);
  int32_t* fb_rows = reinterpret_cast<int32_t*>(base + kOffFbRows);
  float* fb_s = reinterpret_cast<float*>(base + kOffFbS);
  int32_t* fb_i = reinterpret_cast<int32_t*>(base + kOffFbI);

  noalloc_reset<<<1, 64, 0, s>>>(status, fb_count);
  launch_normalize(sh, x, x, xhat, norm, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, RERANK_PREC_FP32,
                   status, s);
  launch_sim_fp32_topk(sh, xhat, reinterpret_cast<int*>(base + kOffFloor), part_s, part_i, kFbCtas, s);
  ErrModel em;
  em.kind = 0;
  em.eps = (sh.dp + 10) * kU32 * 1.01;
  launch_refine(sh, x, x, xhat, norm, part_s, part_i, sh.P, em, nullptr, nullptr, false, out_idx, out_score, fb_rows,
                fb_count, status, s);
  launch_refine_fallback(sh, x, x, xhat, norm, out_idx, out_score, fb_rows, fb_count, fb_s, fb_i, status, kFbCtas,
                         s);
  RR_CUDA(cudaGetLastError());
  long long h[kStCount];
  RR_CUDA(cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  const int e = int(h[kStErr]);
  if (e & (kErrNonFinite | kErrZeroNorm)) return RERANK_EINVAL;
  if (e & kErrTimeout) return RERANK_ETIMEOUT;
  if (e & (kErrCertify | kErrInternal | kErrOverflow)) return RERANK_EINTERNAL;
  return RERANK_OK;
}

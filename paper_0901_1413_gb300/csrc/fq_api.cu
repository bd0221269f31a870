// The C ABI of include/fq.h: argument checks, the per-device status word and
// dispatch to the kernels.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fq_common.cuh"
#include "fq_internal.h"

namespace fqk {

namespace {

// Errors kernels detect while running; read and cleared by fq_status().
__device__ unsigned g_status;

thread_local char t_last_cuda_error[256] = "no CUDA error";

constexpr int kMaxDevices = 64;
unsigned *g_status_ptr[kMaxDevices];
std::mutex g_mu;

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// The wait limit later Four-Russians launches carry (fq_debug_wait_limit).
std::atomic<uint64_t> g_wait_limit_ns{kWaitLimitNs};
// The block of the injected wait that nothing completes (fq_debug_stall_block).
std::atomic<int64_t> g_stall_block{-1};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Fields with their own kernels: F_2, F_3, F_5, F_7 and GF(4).
bool base_q(int q) { return q == 2 || q == 3 || q == 4 || q == 5 || q == 7; }
// ... and the extension fields built on them (fq_ext.cu).
bool valid_q(int q) { return base_q(q) || ext_field(q) != nullptr; }

}  // namespace

uint64_t wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }
int64_t stall_block() { return g_stall_block.load(std::memory_order_relaxed); }

int record_cuda_error(cudaError_t e) {
  snprintf(t_last_cuda_error, sizeof(t_last_cuda_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return FQ_ECUDA;
}

int status_word(unsigned **out) {
  int dev = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FQ_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_status_ptr[dev]) {
    void *p = nullptr;
    FQ_CUDA_TRY(cudaGetSymbolAddress(&p, g_status));
    g_status_ptr[dev] = static_cast<unsigned *>(p);
  }
  *out = g_status_ptr[dev];
  return FQ_OK;
}

// The library's scratch pool on each device: stream-ordered allocations that
// keep their memory between products (release threshold: unlimited), so a
// product that needs scratch does not map fresh memory after every
// synchronisation.  fq_release_scratch trims it.
cudaMemPool_t g_pool[kMaxDevices];

int scratch_pool(cudaMemPool_t *out) {
  int dev = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FQ_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    FQ_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = ~uint64_t(0);
    FQ_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return FQ_OK;
}

int scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = nullptr;
  if (int rc = scratch_pool(&pool)) return rc;
  FQ_CUDA_TRY(cudaMallocFromPoolAsync(p, bytes, pool, s));
  return FQ_OK;
}

int scratch_free(void *p, cudaStream_t s) {
  FQ_CUDA_TRY(cudaFreeAsync(p, s));
  return FQ_OK;
}

int tensor_map_encoder(PFN_cuTensorMapEncodeTiled_v12000 *out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    FQ_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return FQ_ENOTSUP;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return FQ_OK;
}

}  // namespace fqk

using fqk::aligned16;
using fqk::base_q;
using fqk::valid_q;

extern "C" {

int fq_planes(int q) {
  switch (q) {
    case 2: return 1;
    case 3: case 4: return 2;
    case 5: case 7: return 3;
    default: {
      const fqk::ExtField *f = fqk::ext_field(q);
      return f ? f->n * fq_planes(f->p) : 0;
    }
  }
}

int64_t fq_pitch_words(int64_t cols) {
  if (cols < 0) return -1;
  const int64_t words = (cols + 63) / 64;
  return (words + 15) / 16 * 16;
}

int64_t fq_planes_words(int q, int64_t rows, int64_t cols) {
  if (!valid_q(q) || rows < 0 || cols < 0) return -1;
  return int64_t(fq_planes(q)) * rows * fq_pitch_words(cols);
}

int fq_pack(int q, int64_t rows, int64_t cols, const uint8_t *res, int64_t ld, uint64_t *planes, void *stream) {
  if (!valid_q(q) || rows < 0 || cols < 0 || ld < cols) return FQ_EINVAL;
  if (rows == 0) return FQ_OK;
  if (!planes || !aligned16(planes) || (cols > 0 && !res)) return FQ_EINVAL;
  return fqk::launch_pack(q, rows, cols, res, ld, planes, static_cast<cudaStream_t>(stream));
}

int fq_unpack(int q, int64_t rows, int64_t cols, const uint64_t *planes, uint8_t *res, int64_t ld, void *stream) {
  if (!valid_q(q) || rows < 0 || cols < 0 || ld < cols) return FQ_EINVAL;
  if (rows == 0 || cols == 0) return FQ_OK;
  if (!planes || !res || !aligned16(planes)) return FQ_EINVAL;
  return fqk::launch_unpack(q, rows, cols, planes, res, ld, static_cast<cudaStream_t>(stream));
}

int fq_add(int q, int64_t rows, int64_t cols, const uint64_t *X, const uint64_t *Y, uint64_t *Z, int sub,
           void *stream) {
  if (!valid_q(q) || rows < 0 || cols < 0 || (sub != 0 && sub != 1)) return FQ_EINVAL;
  if (rows == 0) return FQ_OK;
  if (!X || !Y || !Z || !aligned16(X) || !aligned16(Y) || !aligned16(Z)) return FQ_EINVAL;
  if (base_q(q)) return fqk::launch_add(q, rows, cols, X, Y, Z, sub, static_cast<cudaStream_t>(stream));
  // extension field: coefficientwise over the base field
  const fqk::ExtField *f = fqk::ext_field(q);
  const int64_t block = int64_t(fq_planes(f->p)) * rows * fq_pitch_words(cols);
  for (int j = 0; j < f->n; ++j)
    if (int rc = fqk::launch_add(f->p, rows, cols, X + j * block, Y + j * block, Z + j * block, sub,
                                 static_cast<cudaStream_t>(stream)))
      return rc;
  return FQ_OK;
}

fqk::ProdOptions prod_options(const fq_options &o) {
  fqk::ProdOptions p;
  p.path = o.path;
  p.k = o.k;
  p.variant = o.variant;
  p.kernel = o.kernel;
  p.chunk = o.chunk;
  p.strassen = o.strassen;
  return p;
}

int fq_auto_choice(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel) {
  if (!valid_q(q) || m < 0 || l < 0 || n < 0 || !path || !kernel) return FQ_EINVAL;
  *path = base_q(q) ? FQ_PATH_M4RM : FQ_PATH_KARATSUBA;
  *kernel = 0;
  if (!base_q(q)) return FQ_OK;
  if (fqk::tuned_choice(q, m, l, n, path, kernel)) return FQ_OK;
  if (m == 0 || l == 0 || n == 0) return FQ_OK;
  // no measurement for this shape: the cheaper path by the time model
  int dev = 0, sms = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  FQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (fqk::mma_estimate(q, m, l, n, sms) < fqk::m4rm_estimate(q, m, l, n, sms)) *path = FQ_PATH_MMA;
  return FQ_OK;
}

int fq_matmul_ex(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                 void *stream, const fq_options *opt) {
  if (!valid_q(q) || m < 0 || l < 0 || n < 0) return FQ_EINVAL;
  if (m == 0 || n == 0) return FQ_OK;
  if (!C || !aligned16(C)) return FQ_EINVAL;
  if (l > 0 && (!A || !B || !aligned16(A) || !aligned16(B))) return FQ_EINVAL;
  if (l > 0 && (A == C || B == C)) return FQ_EINVAL;
  if (l >= (int64_t(1) << 31) || m >= (int64_t(1) << 40) || n >= (int64_t(1) << 36)) return FQ_ENOTSUP;
  fq_options o;
  memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  if (o.path < FQ_PATH_AUTO || o.path > FQ_PATH_KARATSUBA) return FQ_EINVAL;
  if (o.path == FQ_PATH_KARATSUBA && base_q(q) && q != 4) return FQ_EINVAL;
  if (o.k != 0 && (o.k < 6 || o.k > 10)) return FQ_EINVAL;
  if (o.chunk < 0 || o.variant < 0) return FQ_EINVAL;
  if (o.kernel < 0 || o.strassen < -1) return FQ_EINVAL;
  return fqk::product(q, m, l, n, A, B, C, prod_options(o), static_cast<cudaStream_t>(stream));
}

int64_t fq_tc_workspace_bytes(int q, int64_t m, int64_t l, int64_t n) {
  if (!base_q(q) || m < 0 || l < 0 || n < 0) return -1;
  return fqk::tc_workspace_bytes(q, m, l, n);
}

int fq_tc_form(int q, int64_t m, int64_t l, int64_t n) {
  if (fq_tc_workspace_bytes(q, m, l, n) < 0) return base_q(q) && m >= 0 && l >= 0 && n >= 0 ? -FQ_ENOTSUP : -FQ_EINVAL;
  return fqk::tc_form(m, l);
}

int fq_tc_prepare(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, void *workspace,
                  void *stream) {
  if (fq_tc_workspace_bytes(q, m, l, n) < 0) return base_q(q) && m >= 0 && l >= 0 && n >= 0 ? FQ_ENOTSUP : FQ_EINVAL;
  if (m == 0 || n == 0 || l == 0) return FQ_OK;
  if (!A || !B || !workspace || !aligned16(A) || !aligned16(B) || !aligned16(workspace)) return FQ_EINVAL;
  return fqk::tc_prepare(q, m, l, n, A, B, workspace, static_cast<cudaStream_t>(stream));
}

int fq_tc_multiply(int q, int64_t m, int64_t l, int64_t n, const void *workspace, uint64_t *C, void *stream) {
  if (fq_tc_workspace_bytes(q, m, l, n) < 0) return base_q(q) && m >= 0 && l >= 0 && n >= 0 ? FQ_ENOTSUP : FQ_EINVAL;
  if (m == 0 || n == 0) return FQ_OK;
  if (!C || !aligned16(C) || (l > 0 && (!workspace || !aligned16(workspace)))) return FQ_EINVAL;
  if (m >= (int64_t(1) << 31) / 2 || n >= (int64_t(1) << 36)) return FQ_ENOTSUP;
  return fqk::tc_multiply(q, m, l, n, workspace, C, static_cast<cudaStream_t>(stream));
}

int fq_planned_kernel(int q, int64_t m, int64_t l, int64_t n, const fq_options *opt) {
  if (!base_q(q) || m <= 0 || l <= 0 || n <= 0) return -FQ_EINVAL;
  fq_options o;
  memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  if (o.k != 0 && (o.k < 6 || o.k > 10)) return -FQ_EINVAL;
  if (o.kernel > 0) return o.kernel <= fq_kernel_count(q) ? o.kernel : -FQ_EINVAL;
  if (o.path == FQ_PATH_AUTO && o.k == 0 && o.variant == 0) {
    int path = 0, kernel = 0;
    if (fqk::tuned_choice(q, m, l, n, &path, &kernel) && path == FQ_PATH_M4RM && kernel > 0) return kernel;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -fqk::record_cuda_error(cudaGetLastError());
  const int i = fqk::m4rm_planned(q, m, l, n, o.k, o.variant, sms);
  return i < 0 ? -FQ_ENOTSUP : i + 1;
}

int fq_strassen_levels(int q, int64_t m, int64_t l, int64_t n, const fq_options *opt) {
  if (!valid_q(q) || m < 0 || l < 0 || n < 0) return -FQ_EINVAL;
  fq_options o;
  memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  if (o.path < FQ_PATH_AUTO || o.path > FQ_PATH_KARATSUBA || o.strassen < -1) return -FQ_EINVAL;
  if (!base_q(q) || m == 0 || l == 0 || n == 0) return 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -fqk::record_cuda_error(cudaGetLastError());
  return fqk::strassen_levels(q, m, l, n, prod_options(o), sms);
}

int fq_matmul(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
              void *stream) {
  return fq_matmul_ex(q, m, l, n, A, B, C, stream, nullptr);
}

int fq_kernel_count(int q) {
  int count = 0;
  fqk::m4rm_variants(q, &count);
  return count;
}

int fq_kernel_info(int q, int idx, int *k, int *max_rows, int *cols, int *warps) {
  int count = 0;
  const fqk::Variant *vs = fqk::m4rm_variants(q, &count);
  if (!vs || idx < 0 || idx >= count) return FQ_EINVAL;
  if (k) *k = vs[idx].k;
  if (max_rows) *max_rows = vs[idx].rs * vs[idx].rows_per_slot;
  if (cols) *cols = vs[idx].cols;
  if (warps) *warps = vs[idx].warps;
  return FQ_OK;
}

int fq_release_scratch(void) {
  int dev = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= fqk::kMaxDevices) return FQ_ENOTSUP;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(fqk::g_mu);
    pool = fqk::g_pool[dev];
  }
  if (!pool) return FQ_OK;
  FQ_CUDA_TRY(cudaDeviceSynchronize());
  FQ_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
  return FQ_OK;
}

int fq_status(void *stream) {
  unsigned *err = nullptr;
  if (int rc = fqk::status_word(&err)) return rc;
  FQ_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned h = 0;
  FQ_CUDA_TRY(cudaMemcpy(&h, err, sizeof(h), cudaMemcpyDeviceToHost));
  if (h != 0) {
    const unsigned zero = 0;
    FQ_CUDA_TRY(cudaMemcpy(err, &zero, sizeof(zero), cudaMemcpyHostToDevice));
  }
  return int(h);
}

const char *fq_error_string(int status) {
  switch (status) {
    case FQ_OK: return "ok";
    case FQ_EINVAL: return "invalid argument";
    case FQ_EVALUE: return "residue out of range for the field";
    case FQ_ECUDA: return "CUDA error";
    case FQ_ETIMEOUT: return "bounded device wait timed out";
    case FQ_ENOTSUP: return "not supported";
    case FQ_ENOMEM: return "out of host memory";
    case FQ_EBOUNDS: return "bounds check failed (debug build)";
    default: return "unknown status";
  }
}

const char *fq_last_cuda_error(void) { return fqk::t_last_cuda_error; }

int fq_debug_wait_limit(int64_t ns) {
  fqk::g_wait_limit_ns.store(ns > 0 ? uint64_t(ns) : fqk::kWaitLimitNs, std::memory_order_relaxed);
  return FQ_OK;
}

int fq_debug_stall_block(int64_t block) {
  fqk::g_stall_block.store(block >= 0 ? block : -1, std::memory_order_relaxed);
  return FQ_OK;
}

}  // extern "C"

// Shared device and host helpers for the fq library (sm_103a only).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fq.h"

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ != 1030)
#error "this library is built for sm_103a only"
#endif

namespace fqk {

// ----------------------------------------------------------------- host side --

// Records the CUDA error text for fq_last_cuda_error() and maps it to FQ_ECUDA.
int record_cuda_error(cudaError_t e);

#define FQ_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t fq_e_ = (expr);                            \
    if (fq_e_ != cudaSuccess) return fqk::record_cuda_error(fq_e_); \
  } while (0)

#define FQ_LAUNCH_CHECK() FQ_CUDA_TRY(cudaGetLastError())

// Device address of the per-device status word kernels record errors in.
int status_word(unsigned **out);

// Encoder for TMA tensor maps, fetched from the driver once.
int tensor_map_encoder(PFN_cuTensorMapEncodeTiled_v12000 *out);

// How long a bounded device wait lasts before it gives up, in nanoseconds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
// The limit the Four-Russians kernels are launched with: kWaitLimitNs unless
// fq_debug_wait_limit set another (process-wide).
uint64_t wait_limit_ns();
// The k-row block at which the Four-Russians kernels launched next make their
// injected wait (fq_debug_stall_block), or -1 for none.
int64_t stall_block();

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// --------------------------------------------------------------- device side --

// First error wins; later ones are dropped.
__device__ __forceinline__ void record_error(unsigned *err, unsigned code) {
  atomicCAS(err, 0u, code);
}

// Bounds checks of the FQ_DEBUG build: `ok` is the condition an access needs;
// a failed check records FQ_EBOUNDS and returns false so that the caller can
// skip (or redirect) the access.  In the release build every check is true
// and compiles away.
#ifdef FQ_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif
__device__ __forceinline__ bool debug_ok(bool ok, unsigned *err) {
  if constexpr (kDebug) {
    if (!ok) record_error(err, FQ_EBOUNDS);
    return ok;
  }
  return true;
}

// Three-input logic op.  LUT bytes: a -> 0xF0, b -> 0xCC, c -> 0xAA.
template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of the mbarrier to complete.  Gives up after
// `limit_ns` of wall time (about two seconds by default) and returns false; the
// caller records FQ_ETIMEOUT and leaves the kernel.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
  uint32_t done = 0;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  if (done) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

}  // namespace fqk

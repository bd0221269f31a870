// Issue rates of tcgen05.mma from operands resident in shared memory: one
// thread issues 4096 x 4 MMAs back to back (no TMA, no waits inside the loop)
// on one SM (M = 128) and on an SM pair (cta_group::2, M = 256), N = 256 and
// 128; the time is clock64 from the first issue to the completion of the
// last (one commit, one bounded wait).  Two kinds:
//   kind::f8f6f4, e4m3 operands, K = 32 per MMA (32 bytes of each row);
//   kind::mxf4.block_scale.scale_vec::2X, packed e2m1 operands, K = 64 per MMA
//   (the same 32 bytes), ue8m0 block scale factors read from TMEM columns
//   256..511, all set to 1.0 (0x7F).
// Every operand element is 1.0 (e4m3 0x38, e2m1 0x2), so each accumulator
// entry must end at K x 4 x 4096 exactly; the probe checks entry (0, 0) of
// every lane it owns.  Each CTA asks for 120 KB of shared memory, so that the
// two CTAs of a pair sit on different SMs.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}
__device__ __forceinline__ uint64_t gtime() { uint64_t t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t; }
template <int PAIR, int N, int FP4>
__global__ void __launch_bounds__(128, 1) mma_rate(int iters, unsigned *err, unsigned long long *cyc,
                                                     float *d00) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t slot;
  __shared__ __align__(8) uint64_t bar;
  const uint32_t base = (su32(sm) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5;
  uint32_t rank = 0;
  if (PAIR) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 48 * 1024 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t *>(sm + (base - su32(sm)))[i] = FP4 ? 0x22222222u : 0x38383838u;
  if (warp == 0) {
    if (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&slot)) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&slot)) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = slot;
  if (FP4) {  // scale factors 1.0 in columns 256..511 of this warp's 32 lanes
    for (int c = 256; c < 512; c += 32)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
                   "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(
                       tmem + (uint32_t(warp * 32) << 16) + uint32_t(c)),
                   "r"(0x7F7F7F7Fu)
                   : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (PAIR) asm volatile("barrier.cluster.arrive.release.aligned; barrier.cluster.wait.acquire.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t M = PAIR ? 256 : 128;
  // f8f6f4: fp32 accumulator (bits 4-5), e4m3 A and B (0); mxf4: E2M1 A and B
  // (1 in bits 7-9 and 10-12), ue8m0 scale factors (bit 23); N >> 3, M >> 4
  const uint32_t idesc = FP4 ? ((1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (1u << 23) | (uint32_t(M >> 4) << 24))
                             : ((1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24));
  const uint32_t sf = tmem + 256u;
  if (threadIdx.x == 0 && rank == 0) {
    const uint32_t a = base, b = base + 16384;
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (PAIR && FP4)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}\n" ::"r"(tmem), "l"(desc(a + 32 * kk)), "l"(desc(b + 32 * kk)), "r"(idesc), "r"(i | kk), "r"(sf), "r"(sf + 128u) : "memory");
        else if (FP4)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}\n" ::"r"(tmem), "l"(desc(a + 32 * kk)), "l"(desc(b + 32 * kk)), "r"(idesc), "r"(i | kk), "r"(sf), "r"(sf + 128u) : "memory");
        else if (PAIR)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem), "l"(desc(a + 32 * kk)), "l"(desc(b + 32 * kk)), "r"(idesc), "r"(i | kk) : "memory");
        else
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem), "l"(desc(a + 32 * kk)), "l"(desc(b + 32 * kk)), "r"(idesc), "r"(i | kk) : "memory");
      }
    }
    if (PAIR)
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(su32(&bar)), "h"((uint16_t)3) : "memory");
    else
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar)) : "memory");
    const uint64_t g0 = gtime();
    uint32_t done = 0;
    while (!done) {
      asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }" : "=r"(done) : "r"(su32(&bar)) : "memory");
      if (gtime() - g0 > 2000000000ull) { atomicOr(err, 1u); break; }
    }
    cyc[blockIdx.x] = clock64() - t0;
  } else if (PAIR && threadIdx.x == 0) {
    const uint64_t g0 = gtime();
    uint32_t done = 0;
    while (!done) {
      asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }" : "=r"(done) : "r"(su32(&bar)) : "memory");
      if (gtime() - g0 > 2000000000ull) { atomicOr(err, 2u); break; }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  {  // accumulator column 0 of this thread's lane (every entry is the same sum)
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(tmem + (uint32_t(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const float want = float((FP4 ? 64 : 32) * 4) * float(iters);
    if (__uint_as_float(v) != want) atomicOr(err, 4u);
    if (threadIdx.x == 0 && rank == 0) d00[0] = __uint_as_float(v);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (PAIR) asm volatile("barrier.cluster.arrive.release.aligned; barrier.cluster.wait.acquire.aligned;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (PAIR) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    else asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}
template <int PAIR, int N, int FP4> void run(const char *name, unsigned *err, unsigned long long *cyc, float *d00) {
  auto k = mma_rate<PAIR, N, FP4>;
  const int smem = 120 * 1024;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaMemset(err, 0, 4);
  if (PAIR) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2); cfg.blockDim = dim3(128); cfg.dynamicSmemBytes = smem; cfg.attrs = at; cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, 4096, err, cyc, d00);
  } else {
    k<<<1, 128, smem>>>(4096, err, cyc, d00);
  }
  cudaError_t e = cudaDeviceSynchronize();
  unsigned h_err = 0; unsigned long long h_cyc = 0; float h_d = 0.f;
  cudaMemcpy(&h_err, err, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&h_cyc, cyc, 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(&h_d, d00, 4, cudaMemcpyDeviceToHost);
  const double flops_per_sm = 2.0 * 128 * N * (FP4 ? 64 : 32) * 4 * 4096;
  printf("{\"probe\": \"tcgen05.mma %s %s\", \"status\": \"%s\", \"timeouts\": %u, \"sum_exact\": %s, "
         "\"d00\": %.1f, \"cycles\": %llu, \"ops_per_clk_per_sm\": %.1f}\n",
         FP4 ? "kind::mxf4 (e2m1, scales 1.0)" : "kind::f8f6f4 (e4m3)", name, cudaGetErrorString(e), h_err & 3u,
         (h_err & 4u) ? "false" : "true", h_d, h_cyc, flops_per_sm / double(h_cyc));
}
int main() {
  unsigned *err; unsigned long long *cyc; float *d00;
  cudaMalloc(&err, 4); cudaMalloc(&cyc, 64); cudaMalloc(&d00, 4);
  run<0, 256, 0>("single SM M=128 N=256", err, cyc, d00);
  run<1, 256, 0>("SM pair  M=256 N=256", err, cyc, d00);
  run<0, 128, 0>("single SM M=128 N=128", err, cyc, d00);
  run<0, 256, 1>("single SM M=128 N=256", err, cyc, d00);
  run<1, 256, 1>("SM pair  M=256 N=256", err, cyc, d00);
  run<0, 128, 1>("single SM M=128 N=128", err, cyc, d00);
  return 0;
}

// Per-SM issue rates of the instructions the product paths are built from:
// LOP3 (the bitsliced field formulas), warp-uniform shared-memory gathers of
// 4, 8 and 16 bytes per lane (table lookups), a LOP3 F_3-add lookup loop, and
// the warp-level integer tensor-core forms mma.sync s8 (m16n8k32) and b1
// and.popc (m16n8k256).  One CTA of 1024 threads per SM; rates are per clock
// per SM from clock64, plus whole-GPU rates from CUDA events.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA error %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__device__ __forceinline__ uint32_t lop3_96(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}

__global__ void k_lop3(uint32_t* out, long long* cyc, int iters) {
  uint32_t a0 = threadIdx.x, a1 = a0 * 3, a2 = a0 * 5, a3 = a0 * 7, a4 = a0 * 11, a5 = a0 * 13, a6 = a0 * 17, a7 = a0 * 19;
  uint32_t b = blockIdx.x * 0x9e3779b9u, c = ~b;
  __syncthreads();
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    a0 = lop3_96(a0, b, c); a1 = lop3_96(a1, b, c); a2 = lop3_96(a2, b, c); a3 = lop3_96(a3, b, c);
    a4 = lop3_96(a4, b, c); a5 = lop3_96(a5, b, c); a6 = lop3_96(a6, b, c); a7 = lop3_96(a7, b, c);
  }
  __syncthreads();
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}

// Warp-uniform gather: every lane of a warp reads the same table entry (index uniform),
// consecutive 8-byte words -> conflict-free. Table: 256 entries x 32 lanes x 8 B = 64 KiB.
template <int VEC>
__global__ void k_lds(uint32_t* out, long long* cyc, int iters) {
  extern __shared__ uint4 smem4[];
  uint32_t* T = reinterpret_cast<uint32_t*>(smem4);
  const int words = 256 * 32 * VEC;  // 32-bit words
  for (int i = threadIdx.x; i < words; i += blockDim.x) T[i] = i * 2654435761u;
  __syncthreads();
  uint32_t acc[VEC];
  for (int v = 0; v < VEC; ++v) acc[v] = 0;
  uint32_t state = (threadIdx.x >> 5) * 0x9e3779b9u + 12345u;  // warp-uniform
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    state = state * 1664525u + 1013904223u;
    uint32_t idx = state >> 24;  // 0..255, warp-uniform
    const uint32_t* e = T + (idx * 32 + (threadIdx.x & 31)) * VEC;
    if (VEC == 1) { acc[0] ^= e[0]; }
    if (VEC == 2) { uint2 w = *reinterpret_cast<const uint2*>(e); acc[0] ^= w.x; acc[1 % VEC] ^= w.y; }
    if (VEC == 4) { uint4 w = *reinterpret_cast<const uint4*>(e); acc[0] ^= w.x; acc[1 % VEC] ^= w.y; acc[2 % VEC] ^= w.z; acc[3 % VEC] ^= w.w; }
  }
  __syncthreads();
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
  uint32_t r = 0; for (int v = 0; v < VEC; ++v) r ^= acc[v];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// F_3 lookup loop prototype: LDS.64 of (plane0, plane1) + 4-LOP3 F_3 add (two rows per iteration,
// so the warp-uniform index math is shared).
__device__ __forceinline__ void f3_add(uint32_t& x0, uint32_t& x1, uint32_t y0, uint32_t y1) {
  uint32_t u, t;
  u = x0 ^ y1;
  t = (x1 ^ y0 ^ y1);
  x0 = (u ^ x1) | t; x1 = u & (x1 ^ y0);
}
__global__ void k_f3loop(uint32_t* out, long long* cyc, int iters) {
  extern __shared__ uint4 smem4[];
  uint2* T = reinterpret_cast<uint2*>(smem4);
  for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) T[i] = make_uint2(i * 2654435761u, i * 40503u);
  __syncthreads();
  uint32_t a0[8], a1[8];
  for (int r = 0; r < 8; ++r) { a0[r] = 0; a1[r] = 0; }
  uint32_t state = (threadIdx.x >> 5) * 0x9e3779b9u + 12345u;
  const uint2* Tl = T + (threadIdx.x & 31);
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    state = state * 1664525u + 1013904223u;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      uint32_t idx = (state >> (r * 4)) & 255u;
      uint2 w = Tl[idx * 32];
      f3_add(a0[r], a1[r], w.x, w.y);
    }
  }
  __syncthreads();
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
  uint32_t r = 0; for (int v = 0; v < 8; ++v) r ^= a0[v] ^ a1[v];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_mma_s8(uint32_t* out, long long* cyc, int iters) {
  uint32_t a[4] = {threadIdx.x, threadIdx.x * 3u, threadIdx.x * 5u, 7u};
  uint32_t b[2] = {blockIdx.x * 11u + 1u, 0x01010101u};
  int d[8][4];
  for (int j = 0; j < 8; ++j) for (int q = 0; q < 4; ++q) d[j][q] = 0;
  __syncthreads();
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+r"(d[j][0]), "+r"(d[j][1]), "+r"(d[j][2]), "+r"(d[j][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
  }
  __syncthreads();
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
  int r = 0; for (int j = 0; j < 8; ++j) for (int q = 0; q < 4; ++q) r ^= d[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_mma_b1(uint32_t* out, long long* cyc, int iters) {
  uint32_t a[4] = {threadIdx.x, threadIdx.x * 3u, threadIdx.x * 5u, 7u};
  uint32_t b[2] = {blockIdx.x * 11u + 1u, 0x01010101u};
  int d[8][4];
  for (int j = 0; j < 8; ++j) for (int q = 0; q < 4; ++q) d[j][q] = 0;
  __syncthreads();
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      asm volatile("mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+r"(d[j][0]), "+r"(d[j][1]), "+r"(d[j][2]), "+r"(d[j][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
  }
  __syncthreads();
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
  int r = 0; for (int j = 0; j < 8; ++j) for (int q = 0; q < 4; ++q) r ^= d[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

static int report(const char* name, long long* dcyc, int blocks, double ops_per_block, float ms, double unit_ops) {
  long long* h = new long long[blocks];
  if (cudaMemcpy(h, dcyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  double mx = 0, sum = 0; for (int i = 0; i < blocks; ++i) { sum += h[i]; if (h[i] > mx) mx = h[i]; }
  double avg = sum / blocks;
  // blocks are 1 per SM (grid = SM count, 1024 threads)
  printf("{\"probe\":\"%s\",\"ops_per_clk_per_sm\":%.2f,\"avg_cycles\":%.0f,\"ms\":%.4f,\"ops_per_s\":%.4e,\"implied_mhz\":%.0f}\n",
         name, ops_per_block / avg, avg, ms, ops_per_block * blocks / (ms * 1e-3) / unit_ops, avg / (ms * 1e3));
  delete[] h; return 0;
}

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int sms = p.multiProcessorCount;
  printf("{\"gpu\":\"%s\",\"sms\":%d,\"cc\":\"%d.%d\",\"smem_optin\":%zu}\n", p.name, sms, p.major, p.minor, p.sharedMemPerBlockOptin);
  const int threads = 1024, blocks = sms;
  uint32_t* out; long long* cyc;
  CK(cudaMalloc(&out, (size_t)blocks * threads * 4)); CK(cudaMalloc(&cyc, blocks * 8));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  float ms;
  for (int rep = 0; rep < 2; ++rep) {
    int it = 20000;
    CK(cudaEventRecord(e0)); k_lop3<<<blocks, threads>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("lop3 lane-ops", cyc, blocks, (double)threads * it * 8, ms, 1.0);
  }
  {
    int it = 20000;
    CK(cudaFuncSetAttribute(k_lds<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 32 * 4));
    CK(cudaEventRecord(e0)); k_lds<1><<<blocks, threads, 256 * 32 * 4>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("lds32 bytes (uniform idx)", cyc, blocks, (double)threads * it * 4, ms, 1.0);
    CK(cudaFuncSetAttribute(k_lds<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 32 * 8));
    CK(cudaEventRecord(e0)); k_lds<2><<<blocks, threads, 256 * 32 * 8>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("lds64 bytes (uniform idx)", cyc, blocks, (double)threads * it * 8, ms, 1.0);
    CK(cudaFuncSetAttribute(k_lds<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 32 * 16));
    CK(cudaEventRecord(e0)); k_lds<4><<<blocks, threads, 256 * 32 * 16>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("lds128 bytes (uniform idx)", cyc, blocks, (double)threads * it * 16, ms, 1.0);
  }
  {
    int it = 5000;
    CK(cudaFuncSetAttribute(k_f3loop, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 32 * 8));
    CK(cudaEventRecord(e0)); k_f3loop<<<blocks, threads, 256 * 32 * 8>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("f3 lookups (warp x 1024 cols)", cyc, blocks, (double)(threads / 32) * it * 8, ms, 1.0);
  }
  {
    int it = 2000;
    CK(cudaEventRecord(e0)); k_mma_s8<<<blocks, threads>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("mma.sync s8 m16n8k32 (int ops)", cyc, blocks, (double)(threads / 32) * it * 8 * 2.0 * 16 * 8 * 32, ms, 1e12);
    CK(cudaEventRecord(e0)); k_mma_b1<<<blocks, threads>>>(out, cyc, it); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    CK(cudaEventElapsedTime(&ms, e0, e1)); report("mma.sync b1 m16n8k256 and.popc (bit ops)", cyc, blocks, (double)(threads / 32) * it * 8 * 2.0 * 16 * 8 * 256, ms, 1e12);
  }
  CK(cudaFree(out)); CK(cudaFree(cyc));
  return 0;
}

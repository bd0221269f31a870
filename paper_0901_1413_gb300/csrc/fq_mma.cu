// Exact F_q product on the integer tensor cores (fq_matmul path FQ_PATH_MMA).
//
// The same product C = A B as the Four-Russians path, as a dense integer
// contraction: residues of A and B enter warp-level mma.sync.m16n8k32 s8 x s8
// -> s32 as balanced int8 (F_2: {0, 1}; F_3: {-1, 0, 1}; F_5: {-2..2}; F_7:
// {-3..3}), the int32 accumulators are reduced mod p every `chunk` columns of
// A, and the result is packed back into bit-planes.  GF(4) follows Section 4.3 at matrix
// level: with A = A0 + alpha A1, B = B0 + alpha B1,
//   AB = (A0 B0 + A1 B1) + alpha ((A0 + A1)(B0 + B1) + A0 B0),
// three integer products of 0/1 matrices, each read mod 2.
//
// No scratch memory: every 128 x 64 slice of A and 64 x BN slice of B is turned
// from bit-planes into int8 tiles in shared memory by the CTA (A by spreading
// code bits to bytes; B, which the tensor core wants k-contiguous per column,
// by a warp-ballot bit transpose).  One CTA of 8 warps owns a 128 x BN tile of
// C; each warp a 32 x BN/2 sub-tile.
#include "fq_codes.cuh"
#include "fq_fields.cuh"
#include "fq_internal.h"

namespace fqk {

namespace {

template <int Q>
struct MmaSpec {
  static constexpr int P = (Q == 5 || Q == 7) ? 3 : (Q == 2 ? 1 : 2);
  static constexpr int NPROD = Q == 4 ? 3 : 1;  // integer products per tile
  static constexpr int MOD = Q == 4 ? 2 : Q;
  static constexpr int BM = 128, BK = 64, BN = Q == 4 ? 64 : 128;
  static constexpr int WN = BN / 2;             // columns per warp (warps 4 x 2)
  static constexpr int NT8 = WN / 8;            // n8 tiles per warp
  static constexpr int LDA = BK + 16;           // bytes per smem row (bank spread)
  static constexpr int A_BYTES = BM * LDA, B_BYTES = BN * LDA;
  static constexpr int SMEM = NPROD * (A_BYTES + B_BYTES);
  static constexpr int LDC = BN + 16;
  static_assert(BM * LDC <= SMEM, "C tile reuses the operand tiles");
  // largest |balanced residue|
  static constexpr int BMAX = (Q == 2 || Q == 4) ? 1 : (Q - 1) / 2;
};

// Canonical codes for the three-plane fields (any 3-bit code is accepted).
template <int Q, int P>
__device__ __forceinline__ void canon_words(uint32_t (&w)[P]) {
  if constexpr (Q == 5) {
    F5::canon(w);
  } else if constexpr (Q == 7) {
    F7::canon(w);
  }
}

// 32 elements (one 32-bit word per plane, canonical codes) -> 32 int8
// operands of product j (8 words, 4 elements each, element 0 in byte 0).
template <int Q, int P>
__device__ __forceinline__ void to_i8(const uint32_t (&w)[P], int j, uint32_t (&out)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t x[P];
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] = spread_nibble((w[p] >> (4 * i)) & 0xFu);
    uint32_t v;
    if constexpr (Q == 2) {                         // 0/1 operands, read mod 2
      v = x[0];
    } else if constexpr (Q == 3) {                  // unit, sign -> 0, 1, -1
      v = (x[0] & ~x[1]) | ((x[0] & x[1]) * 0xFFu);
    } else if constexpr (Q == 4) {                  // a0, a1, a0 + a1 as 0/1
      v = j == 0 ? x[0] : (j == 1 ? x[1] : (x[0] ^ x[1]));
    } else {
      const uint32_t code = x[0] | (x[1] << 1) | (x[2] << 2);
      if constexpr (Q == 5) {                       // 3, 4 -> -2, -1
        v = code + (((code + 5u * kLsb) >> 3) & kLsb) * 251u;
      } else {                                      // 4, 5, 6 -> -3, -2, -1
        v = code + (((code + 4u * kLsb) >> 3) & kLsb) * 249u;
      }
    }
    out[i] = v;
  }
}

__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct MmaParams {
  const uint64_t *A, *B;
  uint64_t *C;
  int64_t m, l, n;
  int64_t pa, pc;
  int64_t chunk_steps;  // k-steps of 64 between reductions
};

template <int Q>
__global__ void __launch_bounds__(256, 1) mma_kernel(const MmaParams prm) {
  using S = MmaSpec<Q>;
  constexpr int P = S::P, NPROD = S::NPROD;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *As = smem;                        // [NPROD][BM][LDA]
  unsigned char *Bs = smem + NPROD * S::A_BYTES;   // [NPROD][BN][LDA]  (k contiguous per column)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 3, wn = warp >> 2;
  const int64_t row0 = int64_t(blockIdx.y) * S::BM;
  const int64_t col0 = int64_t(blockIdx.x) * S::BN;

  int acc[NPROD][2][S::NT8][4];
#pragma unroll
  for (int j = 0; j < NPROD; ++j)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < S::NT8; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][mi][ni][e] = 0;

  const int64_t ksteps = (prm.l + S::BK - 1) / S::BK;
  int64_t since = 0;
  for (int64_t ks = 0; ks < ksteps; ++ks) {
    const int64_t k0 = ks * S::BK;
    // ---- A: row tid / 2, elements k0 + 32 h .. + 31
    {
      const int r = tid >> 1, h = tid & 1;
      const int64_t row = row0 + r;
      uint32_t w[P];
#pragma unroll
      for (int p = 0; p < P; ++p)
        w[p] = row < prm.m ? uint32_t(prm.A[(p * prm.m + row) * prm.pa + (k0 >> 6)] >> (32 * h)) : 0u;
      canon_words<Q, P>(w);
#pragma unroll
      for (int j = 0; j < NPROD; ++j) {
        uint32_t v[8];
        to_i8<Q, P>(w, j, v);
        uint4 *dst = reinterpret_cast<uint4 *>(As + j * S::A_BYTES + r * S::LDA + 32 * h);
        dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
        dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
      }
    }
    // ---- B: warp (kg, cq) transposes k rows k0 + 32 kg .. + 31 x columns 32 cq .. + 31
    {
      const int kg = warp & 1, cq = warp >> 1;
      if (cq * 32 < S::BN) {
        const int64_t kr = k0 + 32 * kg + lane;
        const int64_t c = col0 + 32 * cq;
        uint32_t w[P];
#pragma unroll
        for (int p = 0; p < P; ++p)
          w[p] = kr < prm.l ? uint32_t(prm.B[(p * prm.l + kr) * prm.pc + (c >> 6)] >> (32 * ((c >> 5) & 1))) : 0u;
        canon_words<Q, P>(w);
        uint32_t col[P];
#pragma unroll
        for (int p = 0; p < P; ++p) col[p] = 0u;
#pragma unroll
        for (int b = 0; b < 32; ++b) {
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (w[p] >> b) & 1u);
            col[p] = lane == b ? bal : col[p];
          }
        }
#pragma unroll
        for (int j = 0; j < NPROD; ++j) {
          uint32_t v[8];
          to_i8<Q, P>(col, j, v);
          uint4 *dst = reinterpret_cast<uint4 *>(Bs + j * S::B_BYTES + (32 * cq + lane) * S::LDA + 32 * kg);
          dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
          dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
        }
      }
    }
    __syncthreads();
    // ---- tensor cores: two k32 steps
#pragma unroll
    for (int kk = 0; kk < S::BK; kk += 32) {
#pragma unroll
      for (int j = 0; j < NPROD; ++j) {
        uint32_t a[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
          const unsigned char *ar = As + j * S::A_BYTES + (wm * 32 + mi * 16 + g) * S::LDA + kk + 4 * t;
          a[mi][0] = *reinterpret_cast<const uint32_t *>(ar);
          a[mi][1] = *reinterpret_cast<const uint32_t *>(ar + 8 * S::LDA);
          a[mi][2] = *reinterpret_cast<const uint32_t *>(ar + 16);
          a[mi][3] = *reinterpret_cast<const uint32_t *>(ar + 8 * S::LDA + 16);
        }
#pragma unroll
        for (int ni = 0; ni < S::NT8; ++ni) {
          const unsigned char *br = Bs + j * S::B_BYTES + (wn * S::WN + ni * 8 + g) * S::LDA + kk + 4 * t;
          const uint32_t b[2] = {*reinterpret_cast<const uint32_t *>(br),
                                 *reinterpret_cast<const uint32_t *>(br + 16)};
#pragma unroll
          for (int mi = 0; mi < 2; ++mi) mma_s8(acc[j][mi][ni], a[mi], b);
        }
      }
    }
    // ---- reduce between l-chunks
    if (++since == prm.chunk_steps) {
      since = 0;
#pragma unroll
      for (int j = 0; j < NPROD; ++j)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
          for (int ni = 0; ni < S::NT8; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[j][mi][ni][e] %= S::MOD;
    }
    __syncthreads();
  }

  // ---- epilogue: residues into a byte tile, then pack 64-column words
  unsigned char *Cs = smem;  // [BM][LDC]
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < S::NT8; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = wm * 32 + mi * 16 + g + (e >= 2 ? 8 : 0);
        const int c = wn * S::WN + ni * 8 + 2 * t + (e & 1);
        int v;
        if constexpr (Q == 4) {
          const int c0 = (acc[0][mi][ni][e] + acc[1][mi][ni][e]) & 1;   // A0 B0 + A1 B1
          const int c1 = (acc[2][mi][ni][e] + acc[0][mi][ni][e]) & 1;   // (A0+A1)(B0+B1) + A0 B0
          v = c0 | (c1 << 1);
        } else {
          v = acc[0][mi][ni][e] % Q;
          v += v < 0 ? Q : 0;
        }
        Cs[r * S::LDC + c] = static_cast<unsigned char>(v);
      }
  __syncthreads();
  for (int it = tid; it < S::BM * (S::BN / 64); it += 256) {
    const int r = it / (S::BN / 64), wd = it % (S::BN / 64);
    const int64_t row = row0 + r;
    if (row >= prm.m) continue;
    uint64_t out[P];
#pragma unroll
    for (int p = 0; p < P; ++p) out[p] = 0;
    uint32_t bad = 0;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(Cs + r * S::LDC + 64 * wd);
#pragma unroll
    for (int e = 0; e < 16; ++e) encode4<Q, P>(src[e], out, 4 * e, bad);
#pragma unroll
    for (int p = 0; p < P; ++p) prm.C[(p * prm.m + row) * prm.pc + (col0 >> 6) + wd] = out[p];
  }
}

template <int Q>
int launch_q(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t chunk,
             cudaStream_t s) {
  using S = MmaSpec<Q>;
  MmaParams prm;
  prm.A = A;
  prm.B = B;
  prm.C = C;
  prm.m = m;
  prm.l = l;
  prm.n = n;
  prm.pa = fq_pitch_words(l);
  prm.pc = fq_pitch_words(n);
  // longest exact chunk: |sum| <= chunk * BMAX^2 + (MOD - 1) < 2^31
  const int64_t safe = ((int64_t(1) << 31) - 1 - S::MOD) / (int64_t(S::BMAX) * S::BMAX) / S::BK;
  int64_t steps = chunk > 0 ? cdiv(chunk, S::BK) : safe;
  if (steps > safe) steps = safe;
  if (steps < 1) steps = 1;
  prm.chunk_steps = steps;
  FQ_CUDA_TRY(cudaFuncSetAttribute(mma_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
  const dim3 grid(unsigned(prm.pc * 64 / S::BN), unsigned(cdiv(m, S::BM)));
  if (grid.y > 65535u) return FQ_ENOTSUP;
  mma_kernel<Q><<<grid, 256, S::SMEM, s>>>(prm);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

}  // namespace

// Modelled time (SM cycles) of the tensor-core path: the tcgen05 form where l
// is in its exact range (fq_tc.cu), else this mma.sync form: waves of CTAs
// (one per SM) times 64-column k-steps times the measured cycles of one
// k-step, plus a constant for launch, the first loads and the epilogue (fitted
// on GB300).
double mma_estimate(int q, int64_t m, int64_t l, int64_t n, int sms) {
  if (l <= tc_max_l(q)) return tc_estimate(q, m, l, n, sms);
  const int bn = q == 4 ? MmaSpec<4>::BN : 128;
  const double per_step = (q == 2 || q == 3) ? 4800.0 : (q == 4 ? 8670.0 : 8040.0);
  const int64_t ctas = (fq_pitch_words(n) * 64 / bn) * cdiv(m, 128);
  return double(cdiv(ctas, sms)) * double(cdiv(l, 64)) * per_step + 52000.0;
}

int launch_mma(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
               int64_t chunk, cudaStream_t s) {
  switch (q) {
    case 2: return launch_q<2>(m, l, n, A, B, C, chunk, s);
    case 3: return launch_q<3>(m, l, n, A, B, C, chunk, s);
    case 4: return launch_q<4>(m, l, n, A, B, C, chunk, s);
    case 5: return launch_q<5>(m, l, n, A, B, C, chunk, s);
    case 7: return launch_q<7>(m, l, n, A, B, C, chunk, s);
    default: return FQ_EINVAL;
  }
}

}  // namespace fqk

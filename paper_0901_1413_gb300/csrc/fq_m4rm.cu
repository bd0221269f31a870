// The Method of Four Russians over bitsliced F_q matrices (Section 2 of Boothby
// & Bradshaw), C = A B:
//
//   C_i = sum_s sum_d alpha_d T_s[ phi_d(a_{i,sk}) ... phi_d(a_{i,sk+k-1}) ],
//   T_s[b] = sum_{t<k} b_t B_{sk+t}    (binary combinations of block s of B).
//
// One CTA owns a tile of C: MT rows x CT columns.  For every k-row block s of B
// it builds T_s for its CT columns in shared memory (each builder walks a run of
// entries, every entry one bitsliced add from its parent), then every row of
// the tile gathers D table entries and adds them into register accumulators with
// the LOP3 formulas of fq_fields.cuh.
//
// Shared-memory layout of one table entry: CH chunks of 128 bytes; chunk c holds
// 16 bytes for each of the LPR = 8 lanes that share a row.  A group of 8 lanes
// reading one entry therefore touches one full 128-byte smem row per chunk, and
// the four groups of a warp (four different rows, four different entries) read
// four full rows: no bank conflicts whatever the indices are.
//
// B blocks arrive by TMA (3-D box: CTW words x k rows x P planes; rows past l
// read as zero), double-buffered on two mbarriers.  The k-bit indices
// phi_d(A_i, block s) are computed once per chunk of NB blocks for all MT rows
// and stored as byte offsets into the table.
#include <cstring>
#include <type_traits>

#include "fq_fields.cuh"
#include "fq_internal.h"

namespace fqk {

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }
__host__ __device__ constexpr int popc(int x) { return x == 0 ? 0 : (x & 1) + popc(x >> 1); }
__host__ __device__ constexpr int ctz(int x) { return (x & 1) ? 0 : 1 + ctz(x >> 1); }
constexpr int round128(int x) { return (x + 127) / 128 * 128; }

template <class F, int K_, int WPL_, int RS_, int NW_>
struct M4rmCfg {
  using Field = F;
  static constexpr int K = K_;      // block size (bits per table index)
  static constexpr int WPL = WPL_;  // 32-bit column words per lane and plane
  static constexpr int RS = RS_;    // row slots per warp (each slot: one row per lane group)
  static constexpr int NW = NW_;    // warps per CTA
  static constexpr int P = F::P, D = F::D;
  static constexpr int LPR = 8;
  static constexpr int GPW = 32 / LPR;
  static constexpr int NT = NW * 32;
  static constexpr int PW = P * WPL;
  static_assert(PW % 4 == 0, "lane data must be whole 16-byte chunks");
  static constexpr int CH = PW / 4;
  static constexpr int ENTRY = CH * LPR * 16;
  static constexpr int ENTRIES = 1 << K;
  static constexpr int CT = LPR * 32 * WPL;
  static constexpr int CTW = CT / 64;
  static constexpr int MT = NW * GPW * RS;
  static constexpr int NBUILD = NW * GPW;
  static_assert((NBUILD & (NBUILD - 1)) == 0 && ENTRIES >= NBUILD, "builders must split the table");
  static constexpr int LB = K - ilog2(NBUILD);
  static constexpr int HB = K - LB;
  static constexpr int EPB = 1 << LB;
  static constexpr int NB = 8;
  using Off = std::conditional_t<(D == 3), uint4, uint2>;
  static constexpr int STAGE_BYTES = P * K * CTW * 8;
  static constexpr int STAGE_STRIDE = round128(STAGE_BYTES);
  static constexpr int TABLE_OFF = 0;
  static constexpr int STAGE_OFF = ENTRIES * ENTRY;
  static constexpr int OFFS_OFF = STAGE_OFF + 2 * STAGE_STRIDE;
  static constexpr int BAR_OFF = OFFS_OFF + NB * MT * int(sizeof(Off));
  static constexpr int ABORT_OFF = BAR_OFF + 16;
  static constexpr int SMEM = ABORT_OFF + 16;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(K <= 10 && (D < 3 || K <= 10), "index width");
};

struct M4rmParams {
  const uint64_t *A;
  uint64_t *C;
  int64_t m, l;
  int64_t pa;       // A row pitch (words)
  int64_t pc;       // B and C row pitch (words)
  int64_t nblocks;  // ceil(l / K)
  unsigned *err;
};

template <class Off, int D>
__device__ __forceinline__ Off make_off(const uint32_t (&o)[D]) {
  static_assert(D == 2 || D == 3, "basis of two or three elements");
  if constexpr (D == 3) {
    return make_uint4(o[0], o[1], o[2], 0u);
  } else {
    return make_uint2(o[0], o[1]);
  }
}

// Table byte offsets of phi_d(A_row, block c0 + b) for b < nb and every row of the
// tile (rows past m get offset 0, the zero entry).
template <class Cfg>
__device__ __forceinline__ void build_offsets(const M4rmParams &prm, typename Cfg::Off *offs, int64_t row0,
                                              int64_t c0, int nb, int tid) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, D = Cfg::D, K = Cfg::K;
  const int64_t bit0 = c0 * K;
  const int64_t wlo = bit0 >> 6;
  const int sh = int(bit0 & 63);
  for (int r = tid; r < Cfg::MT; r += Cfg::NT) {
    const int64_t row = row0 + r;
    uint64_t ph[D][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint64_t a[P];
      const int64_t w = wlo + j;
      const bool in = row < prm.m && w < prm.pa;
#pragma unroll
      for (int p = 0; p < P; ++p) a[p] = in ? __ldg(prm.A + (p * prm.m + row) * prm.pa + w) : 0ull;
      uint64_t f[D];
      F::phi(a, f);
#pragma unroll
      for (int d = 0; d < D; ++d) ph[d][j] = f[d];
    }
#pragma unroll
    for (int b = 0; b < Cfg::NB; ++b) {
      if (b < nb) {
        const int o = sh + b * K;
        const int wi = o >> 6, bo = o & 63;
        uint32_t off[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const uint64_t lo = wi == 0 ? ph[d][0] : (wi == 1 ? ph[d][1] : ph[d][2]);
          const uint64_t hi = wi == 0 ? ph[d][1] : ph[d][2];
          uint64_t v = lo >> bo;
          if (bo != 0) v |= hi << (64 - bo);
          off[d] = uint32_t(v & ((1u << K) - 1u)) * uint32_t(Cfg::ENTRY);
        }
        offs[b * Cfg::MT + r] = make_off<typename Cfg::Off, D>(off);
      }
    }
  }
}

// Lane gl's words of row t of the staged B block: plane p, words gl*WPL ...
template <class Cfg>
__device__ __forceinline__ void load_brow(const unsigned char *stage, int t, int gl,
                                          uint32_t (&v)[Cfg::PW]) {
  constexpr int WPL = Cfg::WPL, RW = Cfg::CT / 32;
#pragma unroll
  for (int p = 0; p < Cfg::P; ++p) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(stage) + (p * Cfg::K + t) * RW + gl * WPL;
    if constexpr (WPL == 4) {
      const uint4 x = *reinterpret_cast<const uint4 *>(src);
      v[p * 4 + 0] = x.x; v[p * 4 + 1] = x.y; v[p * 4 + 2] = x.z; v[p * 4 + 3] = x.w;
    } else if constexpr (WPL == 2) {
      const uint2 x = *reinterpret_cast<const uint2 *>(src);
      v[p * 2 + 0] = x.x; v[p * 2 + 1] = x.y;
    } else {
#pragma unroll
      for (int w = 0; w < WPL; ++w) v[p * WPL + w] = src[w];
    }
  }
}

// x += y on every column word of a lane's slice.
template <class Cfg>
__device__ __forceinline__ void add_slice(uint32_t (&x)[Cfg::PW], const uint32_t (&y)[Cfg::PW]) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, WPL = Cfg::WPL;
#pragma unroll
  for (int w = 0; w < WPL; ++w) {
    uint32_t a[P], b[P];
#pragma unroll
    for (int p = 0; p < P; ++p) { a[p] = x[p * WPL + w]; b[p] = y[p * WPL + w]; }
    F::add(a, b);
#pragma unroll
    for (int p = 0; p < P; ++p) x[p * WPL + w] = a[p];
  }
}

template <class Cfg>
__device__ __forceinline__ void store_entry(unsigned char *table, int e, int gl, const uint32_t (&v)[Cfg::PW]) {
#pragma unroll
  for (int c = 0; c < Cfg::CH; ++c) {
    *reinterpret_cast<uint4 *>(table + e * Cfg::ENTRY + c * (Cfg::LPR * 16) + gl * 16) =
        make_uint4(v[4 * c + 0], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  }
}

// One step of a builder's walk: entry e0 + X is entry e0 + (X & (X - 1)) plus
// row ctz(X) of the block.  In increasing X that parent is the last entry
// visited with popcount(X) - 1 bits, kept in S[popcount(X) - 1].
template <class Cfg, int X>
__device__ __forceinline__ void build_walk(uint32_t (&S)[Cfg::LB + 1][Cfg::PW], unsigned char *table,
                                           const unsigned char *stage, int e0, int gl) {
  if constexpr (X < Cfg::EPB) {
    constexpr int pc = popc(X), tz = ctz(X);
    uint32_t r[Cfg::PW];
    load_brow<Cfg>(stage, tz, gl, r);
#pragma unroll
    for (int j = 0; j < Cfg::PW; ++j) S[pc][j] = S[pc - 1][j];
    add_slice<Cfg>(S[pc], r);
    store_entry<Cfg>(table, e0 + X, gl, S[pc]);
    build_walk<Cfg, X + 1>(S, table, stage, e0, gl);
  }
}

// Builder j fills entries [j EPB, (j+1) EPB): their high index bits are j
// (rows LB.. of the block), summed once; the low LB bits are walked by
// build_walk, one bitsliced add per entry.
template <class Cfg>
__device__ __forceinline__ void build_table(unsigned char *table, const unsigned char *stage, int builder,
                                            int gl) {
  constexpr int PW = Cfg::PW, LB = Cfg::LB;
  uint32_t S[LB + 1][PW];
  uint32_t r[PW];
#pragma unroll
  for (int j = 0; j < PW; ++j) S[0][j] = 0u;
#pragma unroll
  for (int t = 0; t < Cfg::HB; ++t) {
    if ((builder >> t) & 1) {
      load_brow<Cfg>(stage, LB + t, gl, r);
      add_slice<Cfg>(S[0], r);
    }
  }
  const int e0 = builder * Cfg::EPB;
  store_entry<Cfg>(table, e0, gl, S[0]);
  build_walk<Cfg, 1>(S, table, stage, e0, gl);
}

template <class Cfg>
__device__ __forceinline__ void lookup_block(uint32_t (&acc)[Cfg::RS][Cfg::PW], const unsigned char *table,
                                             const typename Cfg::Off *offs_b, int warp, int grp, int gl) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, D = Cfg::D, WPL = Cfg::WPL, PW = Cfg::PW, CH = Cfg::CH;
  const unsigned char *tl = table + gl * 16;
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i) {
    const int r = warp * (Cfg::GPW * Cfg::RS) + i * Cfg::GPW + grp;
    const typename Cfg::Off o = offs_b[r];
    uint32_t od[D];
    if constexpr (D == 3) {
      od[0] = o.x; od[1] = o.y; od[2] = o.z;
    } else {
      od[0] = o.x; od[1] = o.y;
    }
    uint32_t t[D][PW];
#pragma unroll
    for (int d = 0; d < D; ++d) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const uint4 v = *reinterpret_cast<const uint4 *>(tl + od[d] + c * (Cfg::LPR * 16));
        t[d][4 * c + 0] = v.x; t[d][4 * c + 1] = v.y; t[d][4 * c + 2] = v.z; t[d][4 * c + 3] = v.w;
      }
    }
#pragma unroll
    for (int w = 0; w < WPL; ++w) {
      uint32_t a[P], tt[D][P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        a[p] = acc[i][p * WPL + w];
#pragma unroll
        for (int d = 0; d < D; ++d) tt[d][p] = t[d][p * WPL + w];
      }
      F::accumulate(a, tt);
#pragma unroll
      for (int p = 0; p < P; ++p) acc[i][p * WPL + w] = a[p];
    }
  }
}

template <class Cfg>
__device__ __forceinline__ void store_tile(uint32_t (&acc)[Cfg::RS][Cfg::PW], const M4rmParams &prm,
                                           int64_t row0, int64_t w0, int warp, int grp, int gl) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, WPL = Cfg::WPL;
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i) {
    const int64_t row = row0 + warp * (Cfg::GPW * Cfg::RS) + i * Cfg::GPW + grp;
    if (row < prm.m) {
#pragma unroll
      for (int w = 0; w < WPL; ++w) {
        uint32_t a[P];
#pragma unroll
        for (int p = 0; p < P; ++p) a[p] = acc[i][p * WPL + w];
        F::canon(a);
#pragma unroll
        for (int p = 0; p < P; ++p) acc[i][p * WPL + w] = a[p];
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        uint64_t *dst = prm.C + (p * prm.m + row) * prm.pc + w0 + gl * (WPL / 2);
        if constexpr (WPL == 4) {
          *reinterpret_cast<uint4 *>(dst) =
              make_uint4(acc[i][p * 4 + 0], acc[i][p * 4 + 1], acc[i][p * 4 + 2], acc[i][p * 4 + 3]);
        } else {
          static_assert(WPL == 2, "lane slice of one or two 64-bit words");
          *reinterpret_cast<uint2 *>(dst) = make_uint2(acc[i][p * 2 + 0], acc[i][p * 2 + 1]);
        }
      }
    }
  }
}

template <class Cfg>
__global__ void __launch_bounds__(Cfg::NT, 1)
    m4rm_kernel(const __grid_constant__ CUtensorMap tmB, const M4rmParams prm) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = lane / Cfg::LPR, gl = lane % Cfg::LPR;
  const int64_t row0 = int64_t(blockIdx.y) * Cfg::MT;
  const int64_t w0 = int64_t(blockIdx.x) * Cfg::CTW;

  unsigned char *table = smem + Cfg::TABLE_OFF;
  typename Cfg::Off *offs = reinterpret_cast<typename Cfg::Off *>(smem + Cfg::OFFS_OFF);
  const uint32_t stage_s = smem_u32(smem + Cfg::STAGE_OFF);
  const uint32_t bar_s = smem_u32(smem + Cfg::BAR_OFF);
  volatile int &s_abort = *reinterpret_cast<int *>(smem + Cfg::ABORT_OFF);

  if (tid == 0) {
    s_abort = 0;
    mbar_init(bar_s, 1);
    mbar_init(bar_s + 8, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && prm.nblocks > 0) {
    mbar_expect_tx(bar_s, Cfg::STAGE_BYTES);
    tma_load_3d(stage_s, &tmB, bar_s, int(w0), 0, 0);
  }

  uint32_t acc[Cfg::RS][Cfg::PW];
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i)
#pragma unroll
    for (int j = 0; j < Cfg::PW; ++j) acc[i][j] = 0u;

  for (int64_t c0 = 0; c0 < prm.nblocks; c0 += Cfg::NB) {
    const int nb = int(prm.nblocks - c0 < Cfg::NB ? prm.nblocks - c0 : Cfg::NB);
    __syncthreads();  // the previous chunk's lookups are done with `offs`
    build_offsets<Cfg>(prm, offs, row0, c0, nb, tid);
    for (int b = 0; b < nb; ++b) {
      const int64_t s = c0 + b;
      const int buf = int(s & 1);
      if (!mbar_wait_bounded(bar_s + 8 * buf, uint32_t((s >> 1) & 1))) s_abort = 1;
      __syncthreads();  // table free; offsets and this block's B rows visible
      if (s_abort) {
        if (tid == 0) record_error(prm.err, FQ_ETIMEOUT);
        return;
      }
      if (tid == 0 && s + 1 < prm.nblocks) {
        fence_proxy_async_smem();
        const uint32_t nbar = bar_s + 8 * (buf ^ 1);
        mbar_expect_tx(nbar, Cfg::STAGE_BYTES);
        tma_load_3d(stage_s + (buf ^ 1) * Cfg::STAGE_STRIDE, &tmB, nbar, int(w0), int((s + 1) * Cfg::K), 0);
      }
      build_table<Cfg>(table, smem + Cfg::STAGE_OFF + buf * Cfg::STAGE_STRIDE, warp * Cfg::GPW + grp, gl);
      __syncthreads();  // table complete
      lookup_block<Cfg>(acc, table, offs + b * Cfg::MT, warp, grp, gl);
    }
  }
  store_tile<Cfg>(acc, prm, row0, w0, warp, grp, gl);
}

template <class Cfg>
static int launch_cfg(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                      cudaStream_t s) {
  (void)n;
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  M4rmParams prm;
  prm.A = A;
  prm.C = C;
  prm.m = m;
  prm.l = l;
  prm.pa = fq_pitch_words(l);
  prm.pc = fq_pitch_words(n);
  prm.nblocks = cdiv(l, Cfg::K);
  prm.err = err;

  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  if (l > 0) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (int rc = tensor_map_encoder(&encode)) return rc;
    const cuuint64_t dims[3] = {cuuint64_t(prm.pc), cuuint64_t(l), cuuint64_t(Cfg::P)};
    const cuuint64_t strides[2] = {cuuint64_t(prm.pc) * 8u, cuuint64_t(prm.pc) * 8u * cuuint64_t(l)};
    const cuuint32_t box[3] = {cuuint32_t(Cfg::CTW), cuuint32_t(Cfg::K), cuuint32_t(Cfg::P)};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<uint64_t *>(B), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return FQ_EINVAL;
  }
  FQ_CUDA_TRY(cudaFuncSetAttribute(m4rm_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
  const dim3 grid(unsigned(prm.pc / Cfg::CTW), unsigned(cdiv(m, Cfg::MT)));
  if (grid.y > 65535u) return FQ_ENOTSUP;
  m4rm_kernel<Cfg><<<grid, Cfg::NT, Cfg::SMEM, s>>>(map, prm);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

int launch_m4rm(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                int k, int variant, cudaStream_t s) {
  (void)variant;
  if (k != 0 && k != 8) return FQ_ENOTSUP;
  switch (q) {
    case 3: return launch_cfg<M4rmCfg<F3, 8, 2, 16, 8>>(m, l, n, A, B, C, s);
    case 4: return launch_cfg<M4rmCfg<GF4, 8, 2, 16, 8>>(m, l, n, A, B, C, s);
    case 5: return launch_cfg<M4rmCfg<F5, 8, 4, 8, 8>>(m, l, n, A, B, C, s);
    case 7: return launch_cfg<M4rmCfg<F7, 8, 4, 8, 8>>(m, l, n, A, B, C, s);
    default: return FQ_EINVAL;
  }
}

}  // namespace fqk

// The Method of Four Russians over bitsliced F_q matrices (Section 2 of Boothby
// & Bradshaw), C = A B:
//
//   C_i = sum_s sum_d alpha_d T_s[ phi_d(a_{i,sk}) ... phi_d(a_{i,sk+k-1}) ],
//   T_s[b] = sum_{t<k} b_t B_{sk+t}    (binary combinations of block s of B).
//
// One CTA owns a tile of C: `mt` rows (chosen per launch, at most MT) by CT
// columns.  For every k-row block s of B it builds T_s for its CT columns in
// shared memory, then every row of the tile gathers D table entries and adds
// them into register accumulators with the LOP3 formulas of fq_fields.cuh.
//
// Lane groups.  LPR lanes share one row; each lane owns WPL 32-bit words of
// every plane (32 WPL columns).  One table entry is CH chunks of 128 bytes; a
// chunk holds VB = 128 / LPR bytes for each lane of a group, so a group reading
// an entry reads whole 128-byte shared-memory rows and the GPW = 32 / LPR groups
// of a warp (different rows, arbitrary entries) never conflict on banks.
//
// Table build.  32 builder groups each own 2^(k-5) consecutive entries: their 5
// high index bits select rows of the block that are summed once, then the low
// k-5 bits are walked so that every further entry is one bitsliced add of a
// register-resident B row to an earlier entry.
//
// Data movement.  B blocks (CTW words x k rows x P planes, rows past l read as
// zero) arrive by TMA, double-buffered on two mbarriers.  For each chunk of NB
// blocks, the A words covering them are staged with cp.async, and the indices
// phi_d(A_i, block s) are turned once into table byte offsets for all rows.
#pragma once

#include <cstring>
#include <type_traits>

#include "fq_fields.cuh"
#include "fq_internal.h"

namespace fqk {

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }
constexpr int round128(int x) { return (x + 127) / 128 * 128; }
__host__ __device__ constexpr int popc(int x) { return x == 0 ? 0 : (x & 1) + popc(x >> 1); }
__host__ __device__ constexpr int ctz(int x) { return (x & 1) ? 0 : 1 + ctz(x >> 1); }

template <class F, int K_, int LPR_, int WPL_, int RS_, int NW_>
struct M4rmCfg {
  using Field = F;
  static constexpr int K = K_;      // block size: bits per table index
  static constexpr int LPR = LPR_;  // lanes per row group
  static constexpr int WPL = WPL_;  // 32-bit column words per lane and plane
  static constexpr int RS = RS_;    // row slots per warp
  static constexpr int NW = NW_;    // warps per CTA
  static constexpr int P = F::P, D = F::D;
  static constexpr int AP = F::AP;            // accumulator planes (F_5: four, mod 15)
  static constexpr int GPW = 32 / LPR;
  static constexpr int NT = NW * 32;
  static constexpr int PW = P * WPL;          // 32-bit words per lane per entry
  static constexpr int APW = AP * WPL;        // 32-bit accumulator words per lane and row slot
  static constexpr int VB = 128 / LPR;        // bytes per lane per load
  static constexpr int VW = VB / 4;           // 32-bit words per lane per load
  static_assert(PW % VW == 0, "lane data must be whole vector loads");
  static constexpr int CH = PW / VW;          // 128-byte chunks per entry
  static constexpr int ENTRY = CH * 128;
  static constexpr int ENTRIES = 1 << K;
  static constexpr int CT = LPR * 32 * WPL;   // columns per tile
  static_assert(CT % 64 == 0, "tile is whole 64-bit words");
  static constexpr int CTW = CT / 64;
  static constexpr int ROWS_PER_SLOT = NW * GPW;
  static constexpr int MT = RS * ROWS_PER_SLOT;  // most rows a CTA holds
  static constexpr int NBUILD = 32;              // builder groups
  static constexpr int NBW = NBUILD / GPW;       // builder warps
  static_assert(NW >= NBW, "enough warps to build");
  static constexpr int LB = K - 5, HB = 5, EPB = 1 << LB;
  static_assert(K >= 6 && K <= 10, "k in 6..10");
  static constexpr int NB = 64 / K;              // blocks per A chunk (<= 64 bits)
  // table byte offsets of one row and block: one per basis element
  using Off = std::conditional_t<(D >= 3), uint4, std::conditional_t<(D == 2), uint2, uint32_t>>;
  static_assert(D <= 4, "at most four basis elements");
  static constexpr int STAGE_BYTES = P * K * CTW * 8;
  static constexpr int STAGE_STRIDE = round128(STAGE_BYTES);
  static constexpr int TABLE_OFF = 0;
  static constexpr int BSTAGE_OFF = ENTRIES * ENTRY;
  static constexpr int ASTAGE_OFF = BSTAGE_OFF + 2 * STAGE_STRIDE;  // [p][r][2] uint64
  static constexpr int ASTAGE_BYTES = P * MT * 16;
  static constexpr int OFFS_OFF = ASTAGE_OFF + ASTAGE_BYTES;
  static constexpr int BAR_OFF = OFFS_OFF + NB * MT * int(sizeof(Off));  // B stages [2], stall
  static constexpr int ABORT_OFF = BAR_OFF + 24;
  static constexpr int SMEM = ABORT_OFF + 16;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

struct M4rmParams {
  const uint64_t *A;
  uint64_t *C;
  int64_t m, l;
  int64_t pa;       // A row pitch (words)
  int64_t pc;       // B and C row pitch (words)
  int64_t nblocks;  // ceil(l / K)
  int mt;           // rows per CTA (== MT except in tests)
  uint32_t one;     // the constant 1, as data (keeps address arithmetic on IMAD)
  unsigned *err;
  uint64_t wait_ns; // bound of the builders' waits for B blocks
  int64_t stall;    // block of the injected wait that nothing completes (-1: none)
};

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int VW>
__device__ __forceinline__ void lds_vec(uint32_t addr, uint32_t *v) {
  if constexpr (VW == 4) {
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(addr));
  } else if constexpr (VW == 2) {
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(addr));
  } else {
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v[0]) : "r"(addr));
  }
}

template <int VW>
__device__ __forceinline__ void sts_vec(uint32_t addr, const uint32_t *v) {
  if constexpr (VW == 4) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]),
                 "r"(v[3]) : "memory");
  } else if constexpr (VW == 2) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(v[0]), "r"(v[1]) : "memory");
  } else {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v[0]) : "memory");
  }
}

// Stages words wlo, wlo + 1 of every plane of the tile's rows (cp.async),
// layout [p][r][2].
template <class Cfg>
__device__ __forceinline__ void stage_a(const M4rmParams &prm, uint32_t astage, int64_t row0, int rows_here,
                                        int64_t wlo, int tid) {
  constexpr int P = Cfg::P;
  for (int e = tid; e < P * Cfg::MT * 2; e += Cfg::NT) {
    const int j = e & 1;
    const int r = (e >> 1) % Cfg::MT;
    const int p = (e >> 1) / Cfg::MT;
    const int64_t w = wlo + j;
    if (r < rows_here && w < prm.pa)
      cp_async8(astage + uint32_t(e) * 8u, prm.A + (p * prm.m + row0 + r) * prm.pa + w);
  }
  cp_async_commit();
}

// Table byte offsets of phi_d(A_row, block c0 + b), b < nb, for every row slot
// of the tile (rows past the tile get offset 0, the zero entry).
template <class Cfg>
__device__ __forceinline__ void build_offsets(const M4rmParams &prm, const unsigned char *astage,
                                              typename Cfg::Off *offs, int rows_here, int64_t c0, int nb,
                                              int tid) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, D = Cfg::D, K = Cfg::K;
  const int64_t wlo = (c0 * K) >> 6;
  const int sh = int((c0 * K) & 63);
  const uint64_t *as = reinterpret_cast<const uint64_t *>(astage);
  for (int r = tid; r < Cfg::MT; r += Cfg::NT) {
    uint64_t lo[D], hi[D];
    if (r < rows_here) {
      uint64_t a0[P], a1[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        a0[p] = wlo < prm.pa ? as[(p * Cfg::MT + r) * 2 + 0] : 0ull;
        a1[p] = wlo + 1 < prm.pa ? as[(p * Cfg::MT + r) * 2 + 1] : 0ull;
      }
      F::phi(a0, lo);
      F::phi(a1, hi);
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d) lo[d] = hi[d] = 0ull;
    }
    // the 64 bits starting at bit sh of word wlo
    uint64_t win[D];
#pragma unroll
    for (int d = 0; d < D; ++d) win[d] = sh ? (lo[d] >> sh) | (hi[d] << (64 - sh)) : lo[d];
#pragma unroll
    for (int b = 0; b < Cfg::NB; ++b) {
      if (b < nb) {
        uint32_t off[D];
#pragma unroll
        for (int d = 0; d < D; ++d)
          off[d] = uint32_t((win[d] >> (b * K)) & ((1u << K) - 1u)) * uint32_t(Cfg::ENTRY);
        typename Cfg::Off o;
        if constexpr (D == 4) {
          o = make_uint4(off[0], off[1], off[2], off[3]);
        } else if constexpr (D == 3) {
          o = make_uint4(off[0], off[1], off[2], 0u);
        } else if constexpr (D == 2) {
          o = make_uint2(off[0], off[1]);
        } else {
          o = off[0];
        }
        offs[b * Cfg::MT + r] = o;
      }
    }
  }
}

// Lane gl's words of row t of the staged B block (layout [plane][row][CT/32]).
template <class Cfg>
__device__ __forceinline__ void load_brow(uint32_t stage, int t, int gl, uint32_t (&v)[Cfg::PW]) {
  constexpr int WPL = Cfg::WPL, RW = Cfg::CT / 32;
  constexpr int V = WPL >= 4 ? 4 : WPL;
#pragma unroll
  for (int p = 0; p < Cfg::P; ++p) {
    const uint32_t addr = stage + uint32_t(((p * Cfg::K + t) * RW + gl * WPL) * 4);
#pragma unroll
    for (int w = 0; w < WPL; w += V) lds_vec<V>(addr + w * 4, &v[p * WPL + w]);
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
    for (int p = 0; p < P; ++p) {
      a[p] = x[p * WPL + w];
      b[p] = y[p * WPL + w];
    }
    F::add(a, b);
#pragma unroll
    for (int p = 0; p < P; ++p) x[p * WPL + w] = a[p];
  }
}

template <class Cfg>
__device__ __forceinline__ void store_entry(uint32_t tbl_lane, int e, const uint32_t (&v)[Cfg::PW]) {
#pragma unroll
  for (int c = 0; c < Cfg::CH; ++c)
    sts_vec<Cfg::VW>(tbl_lane + uint32_t(e * Cfg::ENTRY + c * 128), &v[c * Cfg::VW]);
}

// One step of a builder's walk: entry e0 + X is entry e0 + (X & (X - 1)) plus
// block row ctz(X).  In increasing X that parent is the last entry visited with
// popcount(X) - 1 bits, held in S[popcount(X) - 1].
template <class Cfg, int X>
__device__ __forceinline__ void build_walk(uint32_t (&S)[Cfg::LB + 1][Cfg::PW],
                                           const uint32_t (&rows)[Cfg::LB][Cfg::PW], uint32_t tbl_lane, int e0) {
  if constexpr (X < Cfg::EPB) {
    constexpr int pc = popc(X), tz = ctz(X);
#pragma unroll
    for (int j = 0; j < Cfg::PW; ++j) S[pc][j] = S[pc - 1][j];
    add_slice<Cfg>(S[pc], rows[tz]);
    store_entry<Cfg>(tbl_lane, e0 + X, S[pc]);
    build_walk<Cfg, X + 1>(S, rows, tbl_lane, e0);
  }
}

template <class Cfg>
__device__ __forceinline__ void build_table(uint32_t tbl_lane, uint32_t stage, int builder, int gl) {
  constexpr int PW = Cfg::PW, LB = Cfg::LB;
  uint32_t rows[LB][PW];
#pragma unroll
  for (int t = 0; t < LB; ++t) load_brow<Cfg>(stage, t, gl, rows[t]);
  uint32_t S[LB + 1][PW];
#pragma unroll
  for (int j = 0; j < PW; ++j) S[0][j] = 0u;
#pragma unroll
  for (int t = 0; t < Cfg::HB; ++t) {
    if ((builder >> t) & 1) {
      uint32_t r[PW];
      load_brow<Cfg>(stage, LB + t, gl, r);
      add_slice<Cfg>(S[0], r);
    }
  }
  const int e0 = builder * Cfg::EPB;
  store_entry<Cfg>(tbl_lane, e0, S[0]);
  build_walk<Cfg, 1>(S, rows, tbl_lane, e0);
}

// PARTIAL = false: every slot is processed (rows past the tile have offset 0,
// the zero entry), so the unrolled loop is one basic block the scheduler can
// pipeline.  PARTIAL = true: slots from `slots` on hold no row of the tile and
// are skipped (tiles much shorter than the kernel's height).
template <class Cfg, bool PARTIAL = false>
__device__ __forceinline__ void lookup_block(uint32_t (&acc)[Cfg::RS][Cfg::APW], uint32_t tbl_lane,
                                             const typename Cfg::Off *offs_b, int warp, int grp, uint32_t one,
                                             unsigned *err, int slots = Cfg::RS) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, D = Cfg::D, AP = Cfg::AP, WPL = Cfg::WPL, PW = Cfg::PW, CH = Cfg::CH, VW = Cfg::VW;
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i) {
    if (!PARTIAL || i < slots) {
      const int r = i * Cfg::ROWS_PER_SLOT + warp * Cfg::GPW + grp;
      const typename Cfg::Off o = offs_b[r];
      uint32_t od[D];
      if constexpr (D == 4) {
        od[0] = o.x; od[1] = o.y; od[2] = o.z; od[3] = o.w;
      } else if constexpr (D == 3) {
        od[0] = o.x; od[1] = o.y; od[2] = o.z;
      } else if constexpr (D == 2) {
        od[0] = o.x; od[1] = o.y;
      } else {
        od[0] = o;
      }
      uint32_t t[D][PW];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if constexpr (kDebug)  // every offset is a table entry (idx < 2^k): else entry 0
          if (!debug_ok(od[d] < uint32_t(Cfg::ENTRIES * Cfg::ENTRY), err)) od[d] = 0u;
        const uint32_t addr = imad(od[d], one, tbl_lane);
#pragma unroll
        for (int c = 0; c < CH; ++c) lds_vec<VW>(addr + c * 128, &t[d][c * VW]);
      }
#pragma unroll
      for (int w = 0; w < WPL; ++w) {
        uint32_t a[AP], tt[D][P];
#pragma unroll
        for (int p = 0; p < AP; ++p) a[p] = acc[i][p * WPL + w];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int d = 0; d < D; ++d) tt[d][p] = t[d][p * WPL + w];
        F::accumulate(a, tt);
#pragma unroll
        for (int p = 0; p < AP; ++p) acc[i][p * WPL + w] = a[p];
      }
    }
  }
}

template <class Cfg>
__device__ __forceinline__ void store_tile(uint32_t (&acc)[Cfg::RS][Cfg::APW], const M4rmParams &prm,
                                           int64_t row0, int rows_here, int64_t w0, int warp, int grp, int gl) {
  using F = typename Cfg::Field;
  constexpr int P = Cfg::P, AP = Cfg::AP, WPL = Cfg::WPL;
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i) {
    const int r = i * Cfg::ROWS_PER_SLOT + warp * Cfg::GPW + grp;
    if (r < rows_here && debug_ok(row0 + r < prm.m && w0 + Cfg::CTW <= prm.pc, prm.err)) {
      const int64_t row = row0 + r;
      uint32_t out[P * WPL];  // canonical codes, plane-major like the accumulator
#pragma unroll
      for (int w = 0; w < WPL; ++w) {
        uint32_t a[AP], x[P];
#pragma unroll
        for (int p = 0; p < AP; ++p) a[p] = acc[i][p * WPL + w];
        F::finish(a, x);
#pragma unroll
        for (int p = 0; p < P; ++p) out[p * WPL + w] = x[p];
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        uint32_t *dst = reinterpret_cast<uint32_t *>(prm.C + (p * prm.m + row) * prm.pc + w0) + gl * WPL;
        if constexpr (WPL == 4) {
          *reinterpret_cast<uint4 *>(dst) = make_uint4(out[p * 4 + 0], out[p * 4 + 1], out[p * 4 + 2], out[p * 4 + 3]);
        } else if constexpr (WPL == 2) {
          *reinterpret_cast<uint2 *>(dst) = make_uint2(out[p * 2 + 0], out[p * 2 + 1]);
        } else {
          static_assert(WPL == 1, "lane slice of one, two or four words");
          dst[0] = out[p];
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
  const int64_t row0 = int64_t(blockIdx.y) * prm.mt;
  const int rows_here = int(prm.m - row0 < prm.mt ? prm.m - row0 : prm.mt);
  const int64_t w0 = int64_t(blockIdx.x) * Cfg::CTW;

  const uint32_t table_s = smem_u32(smem + Cfg::TABLE_OFF);
  const uint32_t tbl_lane = table_s + uint32_t(gl * Cfg::VB);
  const uint32_t bstage_s = smem_u32(smem + Cfg::BSTAGE_OFF);
  const uint32_t astage_s = smem_u32(smem + Cfg::ASTAGE_OFF);
  typename Cfg::Off *offs = reinterpret_cast<typename Cfg::Off *>(smem + Cfg::OFFS_OFF);
  const uint32_t bar_s = smem_u32(smem + Cfg::BAR_OFF);
  volatile int &s_abort = *reinterpret_cast<int *>(smem + Cfg::ABORT_OFF);
  const bool builder = warp < Cfg::NBW;

  if (tid == 0) {
    s_abort = 0;
    mbar_init(bar_s, 1);
    mbar_init(bar_s + 8, 1);
    mbar_init(bar_s + 16, 1);  // never arrived on
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && prm.nblocks > 0) {
    mbar_expect_tx(bar_s, Cfg::STAGE_BYTES);
    tma_load_3d(bstage_s, &tmB, bar_s, int(w0), 0, 0);
  }
  if (prm.nblocks > 0) stage_a<Cfg>(prm, astage_s, row0, rows_here, 0, tid);

  uint32_t acc[Cfg::RS][Cfg::APW];
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i)
#pragma unroll
    for (int j = 0; j < Cfg::APW; ++j) acc[i][j] = 0u;

  for (int64_t c0 = 0; c0 < prm.nblocks; c0 += Cfg::NB) {
    const int nb = int(prm.nblocks - c0 < Cfg::NB ? prm.nblocks - c0 : Cfg::NB);
    cp_async_wait_all();
    __syncthreads();  // A words of this chunk staged; previous lookups done with `offs`
    build_offsets<Cfg>(prm, smem + Cfg::ASTAGE_OFF, offs, rows_here, c0, nb, tid);
    __syncthreads();  // A stage consumed
    if (c0 + Cfg::NB < prm.nblocks)
      stage_a<Cfg>(prm, astage_s, row0, rows_here, ((c0 + Cfg::NB) * Cfg::K) >> 6, tid);
    for (int b = 0; b < nb; ++b) {
      const int64_t s = c0 + b;
      const int buf = int(s & 1);
      if (builder && !mbar_wait_bounded(bar_s + 8 * buf, uint32_t((s >> 1) & 1), prm.wait_ns)) s_abort = 1;
      if (warp == 0 && s == prm.stall) {  // injected failure: the whole warp waits in lockstep
        if (!mbar_wait_bounded(bar_s + 16, 0, prm.wait_ns)) s_abort = 1;
        __syncwarp();
      }
      __syncthreads();  // table free; this block's B rows visible to the builders
      if (s_abort) {
        // Block s's copy is the only one in flight (block s + 1's is issued
        // below): wait for it with the default bound before the CTA exits.
        if (tid == 0) {
          record_error(prm.err, FQ_ETIMEOUT);
          mbar_wait_bounded(bar_s + 8 * buf, uint32_t((s >> 1) & 1));
        }
        cp_async_wait_all();
        return;
      }
      if (tid == 0 && s + 1 < prm.nblocks) {
        fence_proxy_async_smem();
        const uint32_t nbar = bar_s + 8 * (buf ^ 1);
        mbar_expect_tx(nbar, Cfg::STAGE_BYTES);
        tma_load_3d(bstage_s + (buf ^ 1) * Cfg::STAGE_STRIDE, &tmB, nbar, int(w0), int((s + 1) * Cfg::K), 0);
      }
      if (builder) build_table<Cfg>(tbl_lane, bstage_s + buf * Cfg::STAGE_STRIDE, warp * Cfg::GPW + grp, gl);
      __syncthreads();  // table complete
      if (rows_here == Cfg::MT)
        lookup_block<Cfg>(acc, tbl_lane, offs + b * Cfg::MT, warp, grp, prm.one, prm.err);
      else
        lookup_block<Cfg, true>(acc, tbl_lane, offs + b * Cfg::MT, warp, grp, prm.one, prm.err,
                                (rows_here + Cfg::ROWS_PER_SLOT - 1) / Cfg::ROWS_PER_SLOT);
    }
  }
  store_tile<Cfg>(acc, prm, row0, rows_here, w0, warp, grp, gl);
}

// ------------------------------------------------------------------ host --

template <class Cfg>
int launch_cfg(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int mt,
               cudaStream_t s) {
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  if (mt < 1 || mt > Cfg::MT) return FQ_EINVAL;
  M4rmParams prm;
  prm.A = A;
  prm.C = C;
  prm.m = m;
  prm.l = l;
  prm.pa = fq_pitch_words(l);
  prm.pc = fq_pitch_words(n);
  prm.nblocks = cdiv(l, Cfg::K);
  prm.mt = mt;
  prm.one = 1u;
  prm.err = err;
  prm.wait_ns = wait_limit_ns();
  prm.stall = stall_block();

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
  const dim3 grid(unsigned(prm.pc / Cfg::CTW), unsigned(cdiv(m, mt)));
  if (grid.y > 65535u) return FQ_ENOTSUP;
  m4rm_kernel<Cfg><<<grid, Cfg::NT, Cfg::SMEM, s>>>(map, prm);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

// Picks (k, rows per CTA) for a product: the index of the variant, or -1.
// Without a request, every compiled variant is costed: one CTA per SM, waves
// of CTAs, and per CTA ceil(l/k) blocks of (about 1.2 * 2^k table adds + D adds
// per row).  A requested k narrows the choice; a requested height (tests) takes
// the tallest variant of that k, to run with `mt` rows per CTA.
inline int plan_pick(const Variant *vs, int nv, int d, int64_t m, int64_t l, int64_t n, int k, int mt, int sms) {
  int pick = -1;
  if (mt > 0) {
    for (int i = 0; i < nv; ++i)
      if ((k == 0 ? vs[i].k == 8 : vs[i].k == k) && (pick < 0 || vs[i].rs > vs[pick].rs)) pick = i;
    return pick;
  }
  double best = 1e300;
  for (int i = 0; i < nv; ++i) {
    if (k != 0 && vs[i].k != k) continue;
    const int64_t rows = int64_t(vs[i].rs) * vs[i].rows_per_slot;
    const int64_t ctas = cdiv(m, rows) * (fq_pitch_words(n) / (vs[i].cols / 64));
    const int64_t waves = cdiv(ctas, sms);
    const double cost =
        double(waves) * double(cdiv(l, vs[i].k)) * (1.2 * double(1 << vs[i].k) + double(rows) * d);
    if (cost < best * 0.999) {
      best = cost;
      pick = i;
    }
  }
  return pick;
}

inline int plan_and_launch(const Variant *vs, int nv, int d, int64_t m, int64_t l, int64_t n,
                           const uint64_t *A, const uint64_t *B, uint64_t *C, int k, int mt, int kernel,
                           cudaStream_t s) {
  if (kernel > 0) {
    if (kernel > nv) return FQ_EINVAL;
    const Variant &v = vs[kernel - 1];
    if (k != 0 && k != v.k) return FQ_EINVAL;
    return v.launch(m, l, n, A, B, C, mt > 0 ? mt : v.rs * v.rows_per_slot, s);
  }
  int dev = 0, sms = 152;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  FQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int i = plan_pick(vs, nv, d, m, l, n, k, mt, sms);
  if (i < 0) return FQ_ENOTSUP;
  return vs[i].launch(m, l, n, A, B, C, mt > 0 ? mt : vs[i].rs * vs[i].rows_per_slot, s);
}

}  // namespace fqk

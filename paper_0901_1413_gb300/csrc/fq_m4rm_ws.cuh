// Warp-specialised Four-Russians kernel for the two-plane fields (F_3, GF(4))
// and F_2.
//
// Same product as fq_m4rm.cuh (Section 2 of Boothby & Bradshaw):
//   C_i = sum_s sum_d alpha_d T_s[phi_d(A_i, block s)],  T_s[b] = sum_t b_t B_{sk+t},
// but the work of one block is split between two kinds of warps so that the
// lookups -- the part that scales with the rows -- never wait for the rest:
//
//  * NPW = 4 or 8 producer warps (one or two warpgroups, few registers): stage A's words one chunk
//    of NB blocks ahead (TMA boxes of 4 words x 96 rows x 2 planes), turn the k-bit fields phi_d(A_i, block s) of
//    a whole chunk into table byte offsets for every row of the tile (two 16-bit
//    offsets per word), and build T_s in shared memory from the TMA-loaded B
//    block (16 builder groups, each walking 2^(k-4) entries with one bitsliced
//    add per entry).
//  * 16 - NPW consumer warps (the other warpgroups, most registers): for every block,
//    gather D table entries per row and add them into register accumulators.
//
// Tables are double- or triple-buffered by block (NBUF), B blocks are staged
// NSTAGE blocks ahead (enough for fast consumers: an F_2 block is short next
// to a TMA round trip) and offsets double-buffered by chunk: while consumers
// read table s mod NBUF, producers
// fill the next ones, and the offsets of chunk c + 1 are written while chunk c
// is consumed.  Hand-over is by mbarriers (tfull: 128
// producer arrivals; tempty: 384 consumer arrivals).  Every wait is bounded
// (Params::wait_ns); on a timeout the CTA records FQ_ETIMEOUT and runs out its
// loops without waiting again: consumers make no further lookups (so every
// shared-memory address stays valid), the TMA thread issues no further copies
// and, before the CTA exits, waits for the copies it had issued.
#pragma once

#include <cstring>

#include "fq_fields.cuh"
#include "fq_internal.h"

namespace fqk {

namespace ws {

__host__ __device__ constexpr int popc(int x) { return x == 0 ? 0 : (x & 1) + popc(x >> 1); }
__host__ __device__ constexpr int ctz(int x) { return (x & 1) ? 0 : 1 + ctz(x >> 1); }
constexpr int round128(int x) { return (x + 127) / 128 * 128; }

template <class F, int K_, int RS_, int NPW_ = 4, int NBUF_ = 2, int NSTAGE_ = (NBUF_ == 3 ? 3 : 4)>
struct Cfg {
  using Field = F;
  static_assert((F::P == 2 && F::D == 2) || (F::P == 1 && F::D == 1), "two planes and two basis elements, or F_2");
  static constexpr int K = K_;        // block size
  static constexpr int RS = RS_;      // row slots per consumer warp (even)
  static_assert(RS % 2 == 0, "slots are read in pairs");
  static constexpr int P = F::P, D = F::D;
  // 8-lane groups; a lane holds 16 bytes of an entry: WPL words of each plane
  static constexpr int LPR = 8, GPW = 4, PW = 4, WPL = PW / P;
  static constexpr int NPW = NPW_, NCW = 16 - NPW;         // producer / consumer warps
  static constexpr int NBUF = NBUF_;                        // table buffers
  static_assert(NBUF >= 2 && NBUF <= 4, "two to four table buffers");
  static constexpr int NSTAGE = NSTAGE_;                    // B block stages
  static_assert(NSTAGE >= NBUF && NSTAGE <= 16, "B stages");
  static_assert(NPW == 4 || NPW == 8, "one or two producer warpgroups");
  static constexpr int NT = (NPW + NCW) * 32;
  static constexpr int NPT = NPW * 32;                      // producer threads
  static constexpr int PREG = NPW == 4 ? 80 : 64;           // registers after setmaxnreg
  static constexpr int CREG = NPW == 4 ? 144 : 192;
  static_assert(NPT * PREG + NCW * 32 * CREG == 65536, "register split");
  static constexpr int ENTRY = 128;                         // bytes per table entry (idx * 128 below)
  static constexpr int ENTRIES = 1 << K;
  static constexpr int CT = 32 * LPR * WPL, CTW = CT / 64;  // columns (words) per tile: 512, F_2 1024
  static constexpr int ROWS_PER_SLOT = NCW * GPW;
  static constexpr int MT = RS * ROWS_PER_SLOT;             // rows per CTA
  static constexpr int NBUILD = NPW * GPW;                  // builder groups
  static constexpr int HB = NPW == 4 ? 4 : 5, LB = K - HB, EPB = 1 << LB;
  static_assert(K >= 6 && K <= 9, "k in 6..9 (offsets idx * 128 fit 16 bits)");
  static constexpr int NB = 64 / K;                         // blocks per A chunk
  static constexpr int STAGE_BYTES = P * K * CTW * 8;
  static constexpr int STAGE_STRIDE = round128(STAGE_BYTES);
  static constexpr int TABLE_BYTES = ENTRIES * ENTRY;
  static constexpr int OFFS_BYTES = NB * MT * 4;            // one chunk: [b][pair][rows/slot][2] uint32
  static constexpr int ABOX_ROWS = 2 * ROWS_PER_SLOT;       // TMA box rows for A
  static constexpr int ABOX_WORDS = 4;
  static constexpr int ABOXES = MT / ABOX_ROWS;
  static_assert(MT % ABOX_ROWS == 0, "whole A boxes");
  static constexpr int ABOX_BYTES = ABOX_WORDS * ABOX_ROWS * P * 8;
  static constexpr int ASTAGE_BYTES = ABOXES * ABOX_BYTES;  // [box][p][rows][4] uint64
  static constexpr int TABLE_OFF = 0;
  static constexpr int OFFS_OFF = NBUF * TABLE_BYTES;
  static constexpr int BSTAGE_OFF = OFFS_OFF + 2 * OFFS_BYTES;
  static constexpr int ASTAGE_OFF = BSTAGE_OFF + NSTAGE * STAGE_STRIDE;
  static constexpr int BAR_OFF = ASTAGE_OFF + ASTAGE_BYTES;  // bfull[NSTAGE], tfull[NBUF], tempty[NBUF], afull, stall
  static constexpr int ABORT_OFF = BAR_OFF + 8 * (NSTAGE + 2 * NBUF + 2);
  static constexpr int SMEM = ABORT_OFF + 16;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

struct Params {
  const uint64_t *A;
  uint64_t *C;
  int64_t m, l;
  int64_t pa, pc;   // row pitches (words) of A and of B, C
  int64_t nblocks;  // ceil(l / K)
  int mt;           // rows per CTA (<= MT)
  uint32_t one;     // the constant 1 as data: address adds stay on IMAD
  unsigned *err;
  uint64_t wait_ns; // bound of each hand-over wait
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
__device__ __forceinline__ int64_t cdiv_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }
template <int N>
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void lds128(uint32_t addr, uint32_t (&v)[4]) {
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(addr));
}
__device__ __forceinline__ void sts128(uint32_t addr, const uint32_t (&v)[4]) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

// Bounded wait that also gives up at once when the CTA has aborted.  A phase
// that is already complete returns without reading the shared abort flag.
// True when the phase completed, false when the CTA has given up.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int &abort_flag,
                                              unsigned *err, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  if (abort_flag) return false;
  if (!mbar_wait_bounded(bar, parity, limit_ns)) {
    abort_flag = 1;
    record_error(err, FQ_ETIMEOUT);
    return false;
  }
  return true;
}

// ------------------------------------------------------------- producers --

// Stage A's words x .. x + 3 (x = the chunk's first word rounded down to even,
// so the copy starts on a 16-byte boundary) of both planes of the tile's rows:
// ABOXES TMA boxes completing on `afull`.  Rows past m and words past the
// pitch read as zero.
template <class C>
__device__ __forceinline__ void stage_a(const CUtensorMap *tmA, uint32_t astage, uint32_t afull, int64_t row0,
                                        int64_t c0) {
  const int x = int(((c0 * C::K) >> 6) & ~int64_t(1));
  mbar_expect_tx(afull, C::ASTAGE_BYTES);
  for (int j = 0; j < C::ABOXES; ++j)
    tma_load_3d(astage + uint32_t(j * C::ABOX_BYTES), tmA, afull, x, int(row0 + j * C::ABOX_ROWS), 0);
}

// Offsets of phi_d(A_r, block s) for the blocks s = c0 .. c0 + nb - 1 of a
// chunk and every row of the tile, packed off0 | off1 << 16 (off = idx * 128).
// Layout [b][slot pair][48 rows][2 slots]: a consumer warp reads two slots of
// its four row groups in one wavefront; a producer thread handles the two rows
// of one slot pair and writes them with one 8-byte store.
template <class C>
__device__ __forceinline__ void build_offsets(const Params &prm, const unsigned char *astage, uint32_t *offs,
                                              int rows_here, int64_t c0, int nb, int ptid) {
  using F = typename C::Field;
  const int64_t bit0 = c0 * C::K;
  const int o = int(bit0 - 64 * (((bit0 >> 6)) & ~int64_t(1)));  // 0 .. 127 within the staged words
  const int wi = o >> 6, sh = o & 63;
  const int64_t valid = prm.l - bit0;
  const uint64_t keep = valid < 64 ? (uint64_t(1) << valid) - 1u : ~uint64_t(0);
  const uint32_t mask = (1u << C::K) - 1u;
  const uint64_t *as = reinterpret_cast<const uint64_t *>(astage);
  for (int pr = ptid; pr < C::MT / 2; pr += C::NPT) {
    const int j = pr / C::ROWS_PER_SLOT, rem = pr % C::ROWS_PER_SLOT;  // slots 2j, 2j + 1
    uint32_t packed[2][C::NB];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = (2 * j + h) * C::ROWS_PER_SLOT + rem;
      uint64_t win[C::D];
#pragma unroll
      for (int d = 0; d < C::D; ++d) win[d] = 0ull;
      if (r < rows_here) {
        const uint64_t *rowp = as + (r / C::ABOX_ROWS) * (C::ABOX_BYTES / 8) + (r % C::ABOX_ROWS) * C::ABOX_WORDS;
        uint64_t f[C::P];
#pragma unroll
        for (int p = 0; p < C::P; ++p) {
          const uint64_t *wp = rowp + p * (C::ABOX_ROWS * C::ABOX_WORDS);
          const uint64_t w0 = wi ? wp[1] : wp[0];
          const uint64_t w1 = wi ? wp[2] : wp[1];
          f[p] = sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;   // the chunk's 64 bits
        }
        F::phi(f, win);
#pragma unroll
        for (int d = 0; d < C::D; ++d) win[d] &= keep;
      }
      if constexpr (C::D == 1) {
        // F_2: one offset per row and block
#pragma unroll
        for (int b = 0; b < C::NB; ++b) packed[h][b] = (uint32_t(win[0] >> (b * C::K)) & mask) * uint32_t(C::ENTRY);
      } else if constexpr (C::K == 8) {
        // byte b of each map: one byte permute, then idx * 128 in both halves
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const uint32_t x = uint32_t(win[0] >> (32 * (b >> 2)));
          const uint32_t y = uint32_t(win[1] >> (32 * (b >> 2)));
          const uint32_t r = __byte_perm(x, y, uint32_t(b & 3) | (uint32_t(4 + (b & 3)) << 4));
          packed[h][b] = ((r & 0xFFu) << 7) | ((r & 0xFF00u) << 15);
        }
      } else {
#pragma unroll
        for (int b = 0; b < C::NB; ++b) {
          const uint32_t i0 = uint32_t(win[0] >> (b * C::K)) & mask;
          const uint32_t i1 = uint32_t(win[1] >> (b * C::K)) & mask;
          packed[h][b] = (i0 * uint32_t(C::ENTRY)) | ((i1 * uint32_t(C::ENTRY)) << 16);
        }
      }
    }
    uint2 *dst = reinterpret_cast<uint2 *>(offs) + j * C::ROWS_PER_SLOT + rem;
#pragma unroll
    for (int b = 0; b < C::NB; ++b)
      if (b < nb) dst[b * (C::MT / 2)] = make_uint2(packed[0][b], packed[1][b]);
  }
}

template <class C>
__device__ __forceinline__ void load_brow(uint32_t stage, int t, int gl, uint32_t (&v)[4]) {
  if constexpr (C::P == 1) {
    // stage layout [row][32 x 32-bit]; lane gl's words at gl * 4
    lds128(stage + uint32_t(t * C::CTW * 8 + gl * 16), v);
    return;
  }
  // stage layout [p][row][16 x 32-bit]; lane gl's words of plane p at gl * 2
  const uint32_t a0 = stage + uint32_t((0 * C::K + t) * 64 + gl * 8);
  const uint32_t a1 = stage + uint32_t((1 * C::K + t) * 64 + gl * 8);
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(a0));
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v[2]), "=r"(v[3]) : "r"(a1));
}

// entry layout (per lane, 16 bytes): plane 0 words 0..WPL-1, then plane 1's
template <class F>
__device__ __forceinline__ void add_lane(uint32_t (&x)[4], const uint32_t (&y)[4]) {
  constexpr int P = F::P, WPL = 4 / P;
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

// Entries of a builder's run in breadth-first order: by number of set bits,
// then by value.  Entry x is built from x without its highest bit, which sits
// one level up, so all adds of a level are independent.
__host__ __device__ constexpr int bfs_entry(int lb, int i) {
  int seen = 0;
  for (int pc = 0; pc <= lb; ++pc)
    for (int x = 0; x < (1 << lb); ++x)
      if (popc(x) == pc) {
        if (seen == i) return x;
        ++seen;
      }
  return -1;
}
__host__ __device__ constexpr int top_bit(int x) { return x <= 1 ? 0 : 1 + top_bit(x >> 1); }

template <class C, int I>
__device__ __forceinline__ void build_bfs(uint32_t (&V)[C::EPB][4], const uint32_t (&rows)[C::LB][4],
                                          uint32_t tbl_lane, int e0) {
  if constexpr (I < C::EPB) {
    constexpr int x = bfs_entry(C::LB, I), hb = top_bit(x), parent = x ^ (1 << hb);
#pragma unroll
    for (int j = 0; j < 4; ++j) V[x][j] = V[parent][j];
    add_lane<typename C::Field>(V[x], rows[hb]);
    sts128(tbl_lane + uint32_t((e0 + x) * C::ENTRY), V[x]);
    build_bfs<C, I + 1>(V, rows, tbl_lane, e0);
  }
}

// Builder j (0 .. NBUILD-1) fills entries [j EPB, (j + 1) EPB): its high index
// bits j select rows LB.. of the block, summed as a tree (adding a zero row
// leaves a value unchanged); the LB low rows then build the run breadth-first.
template <class C>
__device__ __forceinline__ void build_table(uint32_t tbl_lane, uint32_t stage, int builder, int gl) {
  using F = typename C::Field;
  uint32_t rows[C::LB][4];
#pragma unroll
  for (int t = 0; t < C::LB; ++t) load_brow<C>(stage, t, gl, rows[t]);
  uint32_t hi[C::HB][4];
#pragma unroll
  for (int t = 0; t < C::HB; ++t) {
    load_brow<C>(stage, C::LB + t, gl, hi[t]);
    const uint32_t keep = ((builder >> t) & 1) ? 0xFFFFFFFFu : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[t][j] &= keep;
  }
#pragma unroll
  for (int w = 1; w < C::HB; w *= 2)
#pragma unroll
    for (int t = 0; t + w < C::HB; t += 2 * w) add_lane<F>(hi[t], hi[t + w]);
  uint32_t V[C::EPB][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) V[0][j] = hi[0][j];
  const int e0 = builder * C::EPB;
  sts128(tbl_lane + uint32_t(e0 * C::ENTRY), V[0]);
  build_bfs<C, 1>(V, rows, tbl_lane, e0);
}

// ------------------------------------------------------------- consumers --

template <class C>
__device__ __forceinline__ void lookup_block(uint32_t (&acc)[C::RS][4], uint32_t tbl_lane, uint32_t offs_s, int cw,
                                             int grp, uint32_t one, unsigned *err) {
  using F = typename C::Field;
#pragma unroll
  for (int j = 0; j < C::RS / 2; ++j) {
    uint32_t o[2];
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                 : "=r"(o[0]), "=r"(o[1]) : "r"(offs_s + uint32_t(((j * C::ROWS_PER_SLOT) + cw * C::GPW + grp) * 8)));
    if constexpr (kDebug) {  // every offset is a table entry (idx < 2^k): else entry 0
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool ok = C::D == 1 ? o[h] < uint32_t(C::TABLE_BYTES)
                                  : ((o[h] & 0xFFFFu) < uint32_t(C::TABLE_BYTES) && (o[h] >> 16) < uint32_t(C::TABLE_BYTES));
        if (!debug_ok(ok, err)) o[h] = 0u;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * j + h;
      if constexpr (C::D == 1) {
        // F_2: one gather, one XOR per word
        uint32_t t0[4];
        lds128(imad(o[h], one, tbl_lane), t0);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          uint32_t a[1] = {acc[i][w]};
          const uint32_t tt[1][1] = {{t0[w]}};
          F::accumulate(a, tt);
          acc[i][w] = a[0];
        }
      } else {
        // off1 = o >> 16 and off0 = o - off1 * 2^16, both as IMADs
        const uint32_t hi = __umulhi(o[h], 65536u);
        const uint32_t a1 = imad(hi, one, tbl_lane);
        const uint32_t a0 = imad(hi, 0xFFFF0000u, imad(o[h], one, tbl_lane));
        uint32_t t0[4], t1[4];
        lds128(a0, t0);
        lds128(a1, t1);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          uint32_t a[2] = {acc[i][w], acc[i][2 + w]};
          const uint32_t tt[2][2] = {{t0[w], t0[2 + w]}, {t1[w], t1[2 + w]}};
          F::accumulate(a, tt);
          acc[i][w] = a[0];
          acc[i][2 + w] = a[1];
        }
      }
    }
  }
}

template <class C>
__global__ void __launch_bounds__(C::NT, 1) m4rm_ws_kernel(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmA,
                                                          const Params prm) {
  using F = typename C::Field;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = lane >> 3, gl = lane & 7;
  const int64_t row0 = int64_t(blockIdx.y) * prm.mt;
  const int rows_here = int(prm.m - row0 < prm.mt ? prm.m - row0 : prm.mt);
  const int64_t w0 = int64_t(blockIdx.x) * C::CTW;

  const uint32_t base = smem_u32(smem);
  const uint32_t bfull = base + C::BAR_OFF, tfull = bfull + 8 * C::NSTAGE, tempty = tfull + 8 * C::NBUF,
                 afull = tempty + 8 * C::NBUF, stall = afull + 8;
  volatile int &abort_flag = *reinterpret_cast<int *>(smem + C::ABORT_OFF);

  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < C::NSTAGE; ++i) mbar_init(bfull + 8 * i, 1);
    for (int i = 0; i < C::NBUF; ++i) {
      mbar_init(tfull + 8 * i, C::NPT);
      mbar_init(tempty + 8 * i, C::NCW * 32);
    }
    mbar_init(afull, 1);
    mbar_init(stall, 1);  // never arrived on
    fence_mbar_init();
  }
  __syncthreads();

  if (warp < C::NPW) {
    // ------------------------------------------------------- producers
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::PREG));
    const int ptid = tid;
    const int builder = warp * C::GPW + grp;
    const uint32_t tbl_lane0 = base + C::TABLE_OFF + uint32_t(gl * 16);
    // copies thread 0 has issued: B blocks 0 .. b_issued - 1 (in order), A chunks 0 .. a_issued - 1
    int64_t b_issued = 0, a_issued = 0;
    if (ptid == 0) {
      for (int64_t s = 0; s < C::NSTAGE && s < prm.nblocks; ++s, ++b_issued) {
        mbar_expect_tx(bfull + 8 * uint32_t(s), C::STAGE_BYTES);
        tma_load_3d(base + C::BSTAGE_OFF + uint32_t(s) * C::STAGE_STRIDE, &tmB, bfull + 8 * uint32_t(s), int(w0),
                    int(s * C::K), 0);
      }
    }
    const uint32_t astage = base + C::ASTAGE_OFF;
    const unsigned char *astage_p = smem + C::ASTAGE_OFF;
    const int64_t nchunks = cdiv_dev(prm.nblocks, C::NB);
    uint32_t *const offs0 = reinterpret_cast<uint32_t *>(smem + C::OFFS_OFF);  // chunk buffers 0, 1
    uint32_t aphase = 0;  // completed uses of afull
    // prologue: offsets of chunk 0, A words of chunk 1 in flight
    if (prm.nblocks > 0) {
      if (ptid == 0) {
        stage_a<C>(&tmA, astage, afull, row0, 0);
        ++a_issued;
      }
      wait_or_abort(afull, aphase & 1, abort_flag, prm.err, prm.wait_ns);
      ++aphase;
      build_offsets<C>(prm, astage_p, offs0, rows_here, 0, int(prm.nblocks < C::NB ? prm.nblocks : C::NB), ptid);
      producer_sync<C::NPT>();  // the A stage is free
      if (ptid == 0 && nchunks > 1 && !abort_flag) {
        fence_proxy_async_smem();
        stage_a<C>(&tmA, astage, afull, row0, C::NB);
        ++a_issued;
      }
    }
    for (int64_t s = 0; s < prm.nblocks; ++s) {
      const int buf = int(s % C::NBUF);
      const uint32_t use = uint32_t(s / C::NBUF);
      if (s == prm.stall && warp == 0) {
        // Injected failure: a wait that nothing completes.  The whole warp
        // waits in lockstep (every lane polls the same barrier and clock), so
        // it does not diverge, and it reconverges before the producers' named
        // barrier, which all 32 lanes of a warp must reach together.
        if (!mbar_wait_bounded(stall, 0, prm.wait_ns)) {
          abort_flag = 1;
          record_error(prm.err, FQ_ETIMEOUT);
        }
        __syncwarp();
      }
      if (s % C::NB == C::NBUF - 1) {
        // block NBUF - 1 of chunk c: write the offsets of chunk c + 1 into the
        // buffer chunk c - 1 used -- consumers are done with it once block
        // s - NBUF is consumed, the same wait the table buffer needs below --
        // then prefetch the A words of chunk c + 2
        const int64_t c = s / C::NB;
        if (c + 1 < nchunks) {
          if (s >= C::NBUF) wait_or_abort(tempty + 8 * buf, (use - 1) & 1, abort_flag, prm.err, prm.wait_ns);
          wait_or_abort(afull, aphase & 1, abort_flag, prm.err, prm.wait_ns);
          ++aphase;
          const int64_t c1 = (c + 1) * C::NB;
          build_offsets<C>(prm, astage_p, offs0 + ((c + 1) & 1) * (C::OFFS_BYTES / 4), rows_here, c1,
                           int(prm.nblocks - c1 < C::NB ? prm.nblocks - c1 : C::NB), ptid);
          producer_sync<C::NPT>();  // the A stage is free
          if (ptid == 0 && c + 2 < nchunks && !abort_flag) {
            fence_proxy_async_smem();
            stage_a<C>(&tmA, astage, afull, row0, (c + 2) * C::NB);
            ++a_issued;
          }
        }
      }
      if (s >= C::NBUF) wait_or_abort(tempty + 8 * buf, (use - 1) & 1, abort_flag, prm.err, prm.wait_ns);
      const int sb = int(s % C::NSTAGE);
      wait_or_abort(bfull + 8 * sb, uint32_t(s / C::NSTAGE) & 1, abort_flag, prm.err, prm.wait_ns);
      build_table<C>(tbl_lane0 + uint32_t(buf * C::TABLE_BYTES), base + C::BSTAGE_OFF + sb * C::STAGE_STRIDE,
                     builder, gl);
      producer_sync<C::NPT>();  // every producer is done with this B stage
      if (ptid == 0 && s + C::NSTAGE < prm.nblocks && !abort_flag) {
        fence_proxy_async_smem();
        mbar_expect_tx(bfull + 8 * sb, C::STAGE_BYTES);
        tma_load_3d(base + C::BSTAGE_OFF + sb * C::STAGE_STRIDE, &tmB, bfull + 8 * sb, int(w0),
                    int((s + C::NSTAGE) * C::K), 0);
        ++b_issued;
      }
      mbar_arrive(tfull + 8 * buf);
    }
    // After a wait gave up, copies thread 0 issued may still be landing in
    // this CTA's shared memory; the CTA must not exit before they have.
    // Thread 0 issues a copy into a stage only after its own wait saw the
    // stage's previous copy complete, so only the last copy of each stage can
    // be outstanding: wait for those (with the default bound -- issued copies
    // always complete).
    if (ptid == 0 && abort_flag) {
      for (int64_t j = b_issued > C::NSTAGE ? b_issued - C::NSTAGE : 0; j < b_issued; ++j)
        mbar_wait_bounded(bfull + 8 * uint32_t(j % C::NSTAGE), uint32_t(j / C::NSTAGE) & 1);
      if (a_issued > 0) mbar_wait_bounded(afull, uint32_t(a_issued - 1) & 1);
    }
  } else {
    // ------------------------------------------------------- consumers
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::CREG));
    const int cw = warp - C::NPW;
    const uint32_t tbl_lane0 = base + C::TABLE_OFF + uint32_t(gl * 16);
    uint32_t acc[C::RS][4];
#pragma unroll
    for (int i = 0; i < C::RS; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0u;
    for (int64_t s = 0; s < prm.nblocks; ++s) {
      const int buf = int(s % C::NBUF);
      // No lookup once the CTA has given up.  A consumer that skipped a wait
      // is ahead of the producers, and a later parity test can then pass on
      // an older phase (waiting for parity 1 passes on a barrier still in
      // phase 0): its offsets may never have been written, and unwritten
      // offsets are not table addresses.  No consumer skips a wait before the
      // flag is set, so while it is clear every completed wait is in order.
      const bool have = wait_or_abort(tfull + 8 * buf, uint32_t(s / C::NBUF) & 1, abort_flag, prm.err, prm.wait_ns) &&
                        !abort_flag;
      const int64_t c = s / C::NB;
      const uint32_t offs_s =
          base + C::OFFS_OFF + uint32_t(c & 1) * C::OFFS_BYTES + uint32_t((s - c * C::NB) * C::MT) * 4u;
      if (have) lookup_block<C>(acc, tbl_lane0 + uint32_t(buf * C::TABLE_BYTES), offs_s, cw, grp, prm.one, prm.err);
      mbar_arrive(tempty + 8 * buf);
    }
    // epilogue: canonical codes (F_3 and GF(4) codes are already canonical)
#pragma unroll
    for (int i = 0; i < C::RS; ++i) {
      const int r = i * C::ROWS_PER_SLOT + cw * C::GPW + grp;
      if (r < rows_here && debug_ok(row0 + r < prm.m && w0 + C::CTW <= prm.pc, prm.err)) {
        const int64_t row = row0 + r;
#pragma unroll
        for (int p = 0; p < C::P; ++p) {
          uint32_t *dst = reinterpret_cast<uint32_t *>(prm.C + (p * prm.m + row) * prm.pc + w0) + gl * C::WPL;
          if constexpr (C::WPL == 4) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
          } else {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(acc[i][2 * p + 0], acc[i][2 * p + 1]);
          }
        }
      }
    }
  }
}

template <class C>
int launch(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *Cm, int mt,
           cudaStream_t s) {
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  if (mt < 1 || mt > C::MT) return FQ_EINVAL;
  Params prm;
  prm.A = A;
  prm.C = Cm;
  prm.m = m;
  prm.l = l;
  prm.pa = fq_pitch_words(l);
  prm.pc = fq_pitch_words(n);
  prm.nblocks = cdiv(l, C::K);
  prm.mt = mt;
  prm.one = 1u;
  prm.err = err;
  prm.wait_ns = wait_limit_ns();
  prm.stall = stall_block();
  CUtensorMap map, amap;
  memset(&map, 0, sizeof(map));
  memset(&amap, 0, sizeof(amap));
  if (l > 0) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (int rc = tensor_map_encoder(&encode)) return rc;
    {
      const cuuint64_t adims[3] = {cuuint64_t(prm.pa), cuuint64_t(m), cuuint64_t(C::P)};
      const cuuint64_t astr[2] = {cuuint64_t(prm.pa) * 8u, cuuint64_t(prm.pa) * 8u * cuuint64_t(m)};
      const cuuint32_t abox[3] = {cuuint32_t(C::ABOX_WORDS), cuuint32_t(C::ABOX_ROWS), cuuint32_t(C::P)};
      const cuuint32_t aestr[3] = {1, 1, 1};
      CUresult cr = encode(&amap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<uint64_t *>(A), adims, astr, abox,
                           aestr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (cr != CUDA_SUCCESS) return FQ_EINVAL;
    }
    const cuuint64_t dims[3] = {cuuint64_t(prm.pc), cuuint64_t(l), cuuint64_t(C::P)};
    const cuuint64_t strides[2] = {cuuint64_t(prm.pc) * 8u, cuuint64_t(prm.pc) * 8u * cuuint64_t(l)};
    const cuuint32_t box[3] = {cuuint32_t(C::CTW), cuuint32_t(C::K), cuuint32_t(C::P)};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<uint64_t *>(B), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return FQ_EINVAL;
  }
  FQ_CUDA_TRY(cudaFuncSetAttribute(m4rm_ws_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  const dim3 grid(unsigned(prm.pc / C::CTW), unsigned(cdiv(m, mt)));
  if (grid.y > 65535u) return FQ_ENOTSUP;
  m4rm_ws_kernel<C><<<grid, C::NT, C::SMEM, s>>>(map, amap, prm);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

}  // namespace ws

}  // namespace fqk

// Exact F_q product on the 5th-generation tensor cores (tcgen05, TMEM).
//
// The same product C = A B as the Four-Russians path, as a dense contraction
// of small integers.  The integer tcgen05 kind is not available on sm_103a, so
// residues enter as balanced small floats with fp32 accumulation, which is
// exact here: balanced residues |a|, |b| <= (p - 1) / 2 <= 3 are exact in e4m3
// (1, 2, 3 = 1.000, 1.000 x 2, 1.100 x 2 in binary) and in e2m1 (0010, 0100,
// 0101), every product is an exact small integer, and every partial sum of l
// of them stays an integer below 2^24 in magnitude (the launcher checks
// l * B^2 < 2^24 and otherwise takes the mma.sync s8 path), so no rounding
// ever happens.  The epilogue reads the fp32 accumulators from TMEM, reduces
// mod p and packs the residues into bit-planes.
//
// GF(4) follows Section 4.3 at matrix level with three F_2 products (the
// Karatsuba form): X = A0 B0, Y = A1 B1, Z = (A0 + A1)(B0 + B1), each read mod
// 2; then C's plane 0 = X + Y and plane 1 = Z + X (= A0 B1 + A1 B0 + A1 B1,
// the coefficient of alpha once alpha^2 = alpha + 1 is folded in).  The first
// product writes X into both planes, the other two add theirs in (XOR).
//
// Layout.  The operands are first converted from planes to K-contiguous rows
// (A as m rows, B transposed to n_pad rows, zero past l), as the tensor core
// reads them, in one of two formats, and persistent product kernels read them
// through TMA (128-byte swizzle) and keep their fp32 sums in TMEM; one thread
// issues the MMAs and a group of warps drains the accumulators (tcgen05.ld)
// and writes the packed codes:
//   - e4m3 bytes, la = roundup(l, 128) per row, kind::f8f6f4:
//     - single SMs (m <= 128): 128 x 256 tiles, two 256-column accumulators,
//       so a tile's epilogue overlaps the next tile's products;
//     - SM pairs (cta_group::2): 256 x 256 tiles, each CTA staging its own
//       halves of A and B^T, also double-buffered;
//     - SM pairs, wide: 256 x 512 tiles, two MMAs per step into one
//       512-column accumulator, for a third more load-latency cover;
//   - packed e2m1, la / 2 bytes per row (la = roundup(l, 256)), kind::mxf4
//     with block scale factors 1.0 held in TMEM, at twice the e4m3 rate: SM
//     pairs, 256 x 448 tiles (the default for m > 128 and l >= 2048).
// The batched form gives whole products to pairs of persistent CTAs (one
// cluster each) whose converter warps write each product's e4m3 operands
// into the pair's two scratch buffers while their tensor-core warps compute
// the previous product's tiles.  Every mbarrier wait is bounded.
#include <cstring>

#include "../../include/fq.h"
#include "fq_common.cuh"
#include "fq_e4m3.cuh"
#include "fq_internal.h"

namespace fqk {

namespace tc {

constexpr int BM = 128, BN = 256, BK = 128, UK = 32, STAGES = 4;  // BK, UK: k per stage, per MMA (bytes)
constexpr int A_BYTES = BM * BK, B_BYTES = BN * BK, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int ACC = 2;                         // TMEM accumulators (epilogue overlaps the next tile)
constexpr int BAR_OFF = STAGES * STAGE_BYTES;  // full[S], empty[S], accfull[ACC], accempty[ACC], drain, tmem slot, abort
constexpr int NBARS = 2 * STAGES + 2 * ACC + 1;
constexpr int SMEM = BAR_OFF + 8 * NBARS + 16 + 1024;  // + alignment slack
constexpr int TMEM_COLS = ACC * BN;
constexpr int THREADS = 256;
constexpr int GROUP_M = 8;                     // tile order: default row blocks per group (L2 reuse)
constexpr int GROUP_M4 = 16;                   // the same for the fp4 form (its operands are half the bytes)
constexpr int THREADS_B = 640;                 // batched kernel: sixteen epilogue warps

// ---------------------------------------------------------- conversions --

// Balanced value of a code (the bits of the element in planes 0, 1, 2).
// F_3: unit | sign << 1 (code 2 is unused); F_5, F_7: any 3-bit code, read mod
// p; F_2 and the GF(4) planes: the bit.
template <int Q>
__host__ __device__ constexpr int code_value(int code) {
  if (Q == 3) return code == 1 ? 1 : (code == 3 ? -1 : 0);
  if (Q == 5 || Q == 7) {
    const int r = code % Q;
    return r > Q / 2 ? r - Q : r;
  }
  return code & 1;
}

// The planes a conversion reads: GF(4) becomes one F_2 plane, `sel` 0, 1 or
// 2 picking plane 0, plane 1 or their sum; other fields pass through.
template <int Q>
struct ConvField {
  static constexpr int Q2 = Q == 4 ? 2 : Q;
  static constexpr int P2 = Q == 2 || Q == 4 ? 1 : (Q == 3 ? 2 : 3);
};
template <int Q, int P>
__device__ __forceinline__ void select_planes(const uint32_t (&t)[P], int sel, uint32_t (&o)[ConvField<Q>::P2]) {
  if constexpr (Q == 4) {
    o[0] = sel == 0 ? t[0] : (sel == 1 ? t[1] : (t[0] ^ t[1]));
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) o[p] = t[p];
  }
}

// Rows of a planes matrix to e4m3 bytes: out[r * ld + off + c] for c < cols,
// cols and off multiples of 16 (cols may run into the planes' zero padding,
// which gives zeros).  One thread per 16 elements (a 16-byte store), so that a
// warp writes 512 contiguous bytes; a thread loads RPT rows' words before it
// converts any of them.
constexpr int RPT = 4;
template <int Q, int P>
__global__ void rows_to_e4m3(const uint64_t *__restrict__ X, int64_t rows, int64_t cols, int64_t pitch,
                             uint8_t *__restrict__ out, int64_t ld, int64_t off, int sel) {
  using CF = ConvField<Q>;
  // grid: x over the 16-byte pieces of a row, y over groups of RPT rows
  // (grid-stride); the next group's words are loaded before this group is
  // converted and stored
  const int64_t piece = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t c0 = piece * 16;
  if (c0 >= cols) return;
  const uint32_t *X32 = reinterpret_cast<const uint32_t *>(X);
  const int64_t word = piece >> 1;    // the 32-bit plane word holding the 16 elements
  const int half = int(piece & 1);
  auto load = [&](int64_t r0, uint32_t (&t)[RPT][P]) {
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int p = 0; p < P; ++p)
        t[i][p] = r0 + i < rows ? __ldg(X32 + (p * rows + r0 + i) * pitch * 2 + word) : 0u;
  };
  const int64_t step = int64_t(gridDim.y) * RPT;
  int64_t r0 = int64_t(blockIdx.y) * RPT;
  uint32_t t[RPT][P], nt[RPT][P];
  if (r0 < rows) load(r0, t);
  for (; r0 < rows; r0 += step) {
    if (r0 + step < rows) load(r0 + step, nt);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      if (r0 + i >= rows) break;
      uint32_t o[CF::P2];
      select_planes<Q, P>(t[i], sel, o);
      *reinterpret_cast<uint4 *>(out + (r0 + i) * ld + off + c0) = e4m3x16<CF::Q2, CF::P2>(o, half);
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int p = 0; p < P; ++p) t[i][p] = nt[i][p];
  }
}

// Launch shape of rows_to_e4m3 for rows x cols (cols a multiple of 16): one
// wave of 256-thread blocks (8 per SM on 152 SMs), each walking row groups.
inline dim3 rows_grid(int64_t rows, int64_t cols) {
  const int64_t pieces = cols / 16, xs = cdiv(pieces, 256), groups = cdiv(rows, RPT);
  const int64_t want = cdiv(int64_t(152) * 8, xs);
  const int64_t ys = groups < want ? groups : want;
  return dim3(unsigned(xs), unsigned(ys < 65535 ? (ys > 0 ? ys : 1) : 65535));
}

// 32 x 32 bit transpose across a warp: afterwards bit i of lane j's word is
// bit j of lane i's word before.  Five stages swap the off-diagonal s x s
// blocks between lanes l and l ^ s (s = 16, 8, 4, 2, 1): a lane keeps its
// bits under `keep` (the mask m of the stage's low blocks, or ~m when bit s of
// the lane is set) and takes the rest from the partner's word rotated left by
// s (or right by s): the bits a rotation wraps around land under `keep`.
struct Transpose32 {
  uint32_t rot[5], keep[5];
  __device__ __forceinline__ explicit Transpose32(int lane) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int s = 16 >> k;
      const uint32_t m = s == 16 ? 0x0000FFFFu : (s == 8 ? 0x00FF00FFu : (s == 4 ? 0x0F0F0F0Fu : (s == 2 ? 0x33333333u : 0x55555555u)));
      rot[k] = (lane & s) ? uint32_t(32 - s) : uint32_t(s);
      keep[k] = (lane & s) ? ~m : m;
    }
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, 16 >> k);
      x = lop3<0xE4>(x, __funnelshift_l(y, y, rot[k]), keep[k]);  // (x & keep) | (rot & ~keep)
    }
    return x;
  }
};

__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) { return Transpose32(lane)(x); }

// B^T as e4m3 bytes straight from B's planes: out[j * ld + off + k] = the byte
// of B[k][j] for every column j of the planes' pitch (n_pad = 64 pitch) and
// k < kcols (a multiple of 16; rows k >= rows read as zero).  A CTA of eight
// warps turns a 128 (k) x 256 (j) block around: warp w loads rows k0 + 32 (w %
// 4) + lane, 128 columns from j0 + 128 (w / 4), transposes each 32 x 32 bit
// block across the warp, converts lane j's 32 bits into 32 bytes and puts
// them in a shared 256 x 128-byte tile (16-byte chunks XOR-swizzled by row, so
// that eight lanes hit eight bank groups); the tile leaves in 128-byte rows.
constexpr int TK = 128, TJ = 256;
// One 128 (k) x 256 (j) block of B^T from B's planes: bytes k0 + 16 c ..
// of column j0 + jl go to out_block + jl * ld + 16 c, for k0 + 16 c < kcols
// and j0 + jl < jcols.
template <int Q, int P>
__device__ __forceinline__ void transpose_block(const uint64_t *__restrict__ X, int64_t rows, int64_t pitch,
                                                uint8_t *__restrict__ out_block, int64_t ld, int64_t kcols,
                                                int64_t jcols, int sel, int64_t k0, int64_t j0, uint4 *tile) {
  using CF = ConvField<Q>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kq = warp & 3, jh = warp >> 2;
  const int64_t k = k0 + 32 * kq + lane;
  const int64_t w0 = (j0 + 128 * jh) / 64;  // first word of the warp's 128 columns (16-byte aligned)
  uint32_t t[4][P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint4 v = k < rows ? __ldg(reinterpret_cast<const uint4 *>(X + (p * rows + k) * pitch + w0)) : make_uint4(0u, 0u, 0u, 0u);
    t[0][p] = v.x;
    t[1][p] = v.y;
    t[2][p] = v.z;
    t[3][p] = v.w;
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    uint32_t o[CF::P2];
    select_planes<Q, P>(t[g], sel, o);
#pragma unroll
    for (int p = 0; p < CF::P2; ++p) o[p] = transpose32(o[p], lane);
    // lane: column jl of the tile, bit i = row k0 + 32 kq + i
    const int jl = 128 * jh + 32 * g + lane, c0 = 2 * kq;
    uint4 lo, hi;
    e4m3x32<CF::Q2, CF::P2>(o, lo, hi);
    tile[jl * 8 + (c0 ^ (jl & 7))] = lo;
    tile[jl * 8 + ((c0 + 1) ^ (jl & 7))] = hi;
  }
  __syncthreads();
#pragma unroll
  for (int i = threadIdx.x; i < TJ * 8; i += 256) {
    const int jl = i >> 3, c = i & 7;
    if (k0 + 16 * c < kcols && j0 + jl < jcols)
      *reinterpret_cast<uint4 *>(out_block + jl * ld + 16 * c) = tile[jl * 8 + (c ^ (jl & 7))];
  }
}

// B^T as e4m3 bytes straight from B's planes: out[j * ld + off + k] = the byte
// of B[k][j] for every column j of the planes' pitch (n_pad = 64 pitch) and
// k < kcols (a multiple of 16; rows k >= rows read as zero).  A CTA of eight
// warps turns a 128 (k) x 256 (j) block around: warp w loads rows k0 + 32 (w %
// 4) + lane, 128 columns from j0 + 128 (w / 4), transposes each 32 x 32 bit
// block across the warp, converts lane j's 32 bits into 32 bytes and puts
// them in a shared 256 x 128-byte tile (16-byte chunks XOR-swizzled by row, so
// that eight lanes hit eight bank groups); the tile leaves in 128-byte rows.
template <int Q, int P>
__global__ void __launch_bounds__(256) planes_to_e4m3_t(const uint64_t *__restrict__ X, int64_t rows, int64_t pitch,
                                                        uint8_t *__restrict__ out, int64_t ld, int64_t off,
                                                        int64_t kcols, int sel) {
  __shared__ uint4 tile[TJ * TK / 16];
  const int64_t k0 = int64_t(blockIdx.x) * TK, j0 = int64_t(blockIdx.y) * TJ;
  transpose_block<Q, P>(X, rows, pitch, out + j0 * ld + off + k0, ld, kcols, int64_t(1) << 62, sel, k0, j0, tile);
}

// ------------------------------------------- packed e2m1 (fp4) operands --
//
// The fp4 form feeds the same balanced residues to tcgen05.mma kind::mxf4
// (packed e2m1, two elements to a byte, block scale factors all 1.0), which
// runs at twice the e4m3 rate and takes half the operand bytes.  e2m1 has a
// sign bit, two exponent bits biased by 1 and one mantissa bit: 0, 1, 2, 3 are
// 0000, 0010, 0100, 0101 and the sign is bit 3, so 0, +-1, +-2, +-3 are exact.
// Both operands are K-major: element k of a row is nibble k of the row (the
// low nibble of byte k / 2 for even k).  Which nibble the tensor core takes
// first does not matter, since A and B pair the same positions.
__host__ __device__ constexpr uint32_t e2m1_nibble(int v) {
  return v == 0 ? 0u : ((v < 0 ? 8u : 0u) | ((v == 1 || v == -1) ? 2u : ((v == 2 || v == -2) ? 4u : 5u)));
}

// Bit b of the e2m1 nibble of a 3-bit code, as a LOP3 truth table of (plane
// 2, plane 1, plane 0): the table's index is then the code itself.
template <int Q>
__host__ __device__ constexpr int nibble_lut(int b) {
  int lut = 0;
  for (int c = 0; c < 8; ++c) lut |= int((e2m1_nibble(code_value<Q>(c)) >> b) & 1u) << c;
  return lut;
}

// Bits 0..7 of x spread to bits 0, 4, ..., 28.
__device__ __forceinline__ uint32_t spread8(uint32_t x) {
  x = (x | (x << 12)) & 0x000F000Fu;
  x = (x | (x << 6)) & 0x03030303u;
  return (x | (x << 3)) & 0x11111111u;
}

// 32 elements (bit i of the plane words t) as 32 packed e2m1 nibbles, element
// i in bits 4 (i % 8) .. of word i / 8.  The nibble's bits are first formed
// 32 elements at a time as bit-planes: F_2 (and a selected GF(4) plane) puts
// the element in bit 1 (1.0); F_3 puts the unit in bit 1 and the sign in bit
// 3 (the unused code 2 gives -0, which adds nothing); F_5 and F_7 take one
// LOP3 per nibble bit over the three code planes.
template <int Q, int P>
__device__ __forceinline__ uint4 e2m1x32(const uint32_t (&t)[P]) {
  uint32_t nb[4];
  if constexpr (Q == 2) {
    nb[0] = 0u; nb[1] = t[0]; nb[2] = 0u; nb[3] = 0u;
  } else if constexpr (Q == 3) {
    nb[0] = 0u; nb[1] = t[0]; nb[2] = 0u; nb[3] = t[1];
  } else {
    nb[0] = lop3<nibble_lut<Q>(0)>(t[2], t[1], t[0]);
    nb[1] = lop3<nibble_lut<Q>(1)>(t[2], t[1], t[0]);
    nb[2] = lop3<nibble_lut<Q>(2)>(t[2], t[1], t[0]);
    nb[3] = lop3<nibble_lut<Q>(3)>(t[2], t[1], t[0]);
  }
  uint32_t o[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    uint32_t x = 0u;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if ((Q == 2 || Q == 3) && (b == 0 || b == 2)) continue;
      if (Q == 2 && b == 3) continue;
      x |= spread8((nb[b] >> (8 * w)) & 0xFFu) << b;
    }
    o[w] = x;
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// Rows of a planes matrix to packed e2m1: byte c / 2 of out[r * ld ..] holds
// elements c and c + 1 of row r, for c < cols (a multiple of 32, which may run
// into the planes' zero padding, giving zeros).  One thread per 32 elements
// (one 32-bit plane word in, a 16-byte store out, so that a warp writes 512
// contiguous bytes); a thread loads the next group of RPT rows' words before
// it converts the current one.
template <int Q, int P>
__global__ void rows_to_fp4(const uint64_t *__restrict__ X, int64_t rows, int64_t cols, int64_t pitch,
                            uint8_t *__restrict__ out, int64_t ld, int sel) {
  using CF = ConvField<Q>;
  const int64_t piece = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;  // the 32-bit word of the row
  if (piece * 32 >= cols) return;
  const uint32_t *X32 = reinterpret_cast<const uint32_t *>(X);
  auto load = [&](int64_t r0, uint32_t (&t)[RPT][P]) {
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int p = 0; p < P; ++p)
        t[i][p] = r0 + i < rows ? __ldg(X32 + (p * rows + r0 + i) * pitch * 2 + piece) : 0u;
  };
  const int64_t step = int64_t(gridDim.y) * RPT;
  int64_t r0 = int64_t(blockIdx.y) * RPT;
  uint32_t t[RPT][P], nt[RPT][P];
  if (r0 < rows) load(r0, t);
  for (; r0 < rows; r0 += step) {
    if (r0 + step < rows) load(r0 + step, nt);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      if (r0 + i >= rows) break;
      uint32_t o[CF::P2];
      select_planes<Q, P>(t[i], sel, o);
      *reinterpret_cast<uint4 *>(out + (r0 + i) * ld + piece * 16) = e2m1x32<CF::Q2, CF::P2>(o);
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int p = 0; p < P; ++p) t[i][p] = nt[i][p];
  }
}

// Launch shape of rows_to_fp4 for rows x cols (cols a multiple of 32): one
// wave of 256-thread blocks (`per_sm` resident per SM, from the occupancy
// calculator), each walking row groups.
inline dim3 rows_grid4(int64_t rows, int64_t cols, int sms, int per_sm) {
  const int64_t pieces = cols / 32, xs = cdiv(pieces, 256), groups = cdiv(rows, RPT);
  const int64_t want = cdiv(int64_t(sms) * per_sm, xs);
  const int64_t ys = groups < want ? groups : want;
  return dim3(unsigned(xs), unsigned(ys < 65535 ? (ys > 0 ? ys : 1) : 65535));
}

// B^T as packed e2m1 straight from B's planes: row j of out (ld bytes) holds
// B[k][j] in nibble k, for every column j of the planes' pitch (n_pad = 64
// pitch) and k < kcols (a multiple of 64; rows k >= rows read as zero).  The
// work is in blocks of 64 (k) x 256 (j), taken by a persistent grid (k
// fastest, so that neighbouring CTAs fill neighbouring bytes of the same
// output rows).  In a block, warp w loads rows k0 + 32 (w % 2) + lane, one
// word (64 columns) j0 / 64 + w / 2 of every plane, transposes its two 32 x 32
// bit blocks across the warp and converts lane j's 32 bits into 16 bytes,
// chunk w % 2 of row j of a shared 256 x 32-byte tile (the chunk index XORed
// with bit 2 of the row, so that the eight lanes of a store phase hit eight
// bank groups); the tile leaves in 32-byte row pieces.
constexpr int TK4 = 64, TJ4 = 256;
template <int Q, int P>
__global__ void __launch_bounds__(256) planes_to_fp4_t(const uint64_t *__restrict__ X, int64_t rows, int64_t pitch,
                                                       uint8_t *__restrict__ out, int64_t ld, int sel,
                                                       int64_t kblocks, int64_t blocks) {
  using CF = ConvField<Q>;
  __shared__ uint4 tile[TJ4 * 2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kq = warp & 1, jq = warp >> 1;
  const Transpose32 tr(lane);
  for (int64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x) {
    const int64_t k0 = (blk % kblocks) * TK4, j0 = (blk / kblocks) * TJ4;
    const int64_t k = k0 + 32 * kq + lane;
    uint32_t t[2][P];  // half g: columns j0 + 64 jq + 32 g .. + 31
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t w = k < rows ? __ldg(X + (p * rows + k) * pitch + j0 / 64 + jq) : 0ull;
      t[0][p] = uint32_t(w);
      t[1][p] = uint32_t(w >> 32);
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      uint32_t o[CF::P2];
      select_planes<Q, P>(t[g], sel, o);
#pragma unroll
      for (int p = 0; p < CF::P2; ++p) o[p] = tr(o[p]);
      const int jl = 64 * jq + 32 * g + lane;  // lane: column j0 + jl, bit i = row k0 + 32 kq + i
      tile[jl * 2 + (kq ^ ((jl >> 2) & 1))] = e2m1x32<CF::Q2, CF::P2>(o);
    }
    __syncthreads();
#pragma unroll
    for (int i = threadIdx.x; i < TJ4 * 2; i += 256) {
      const int jl = i >> 1, c = i & 1;
      *reinterpret_cast<uint4 *>(out + (j0 + jl) * ld + k0 / 2 + 16 * c) = tile[jl * 2 + (c ^ ((jl >> 2) & 1))];
    }
    __syncthreads();
  }
}

// Resident 256-thread blocks per SM of a kernel (the occupancy calculator).
template <class K>
int occupancy256(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 256, 0) != cudaSuccess || n < 1) n = 1;
  return n;
}

// The fp4 conversions' resident blocks per SM, computed once per field.
template <int Q, int P>
struct Fp4Occupancy {
  static int rows() {
    static const int n = occupancy256(rows_to_fp4<Q, P>);
    return n;
  }
  static int transpose() {
    static const int n = occupancy256(planes_to_fp4_t<Q, P>);
    return n;
  }
};

// ------------------------------------------------------------------ GEMM --

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows
// and the 128-byte swizzle: start address, leading byte offset 16 (unused by
// this layout), stride 1024 bytes between 8-row groups, descriptor version 1,
// layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;                 // leading byte offset 16 B
  d |= uint64_t(1024 >> 4) << 32;         // stride byte offset 1024 B
  d |= uint64_t(1) << 46;                 // version
  d |= uint64_t(2) << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f8f6f4: fp32 accumulator (bits 4-5 = 1), e4m3
// A and B (bits 7-9, 10-12 = 0), both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait that gives up at once when the CTA has aborted.
__device__ __forceinline__ void wait_bar(uint32_t bar, uint32_t parity, volatile int *abort_flag, unsigned *err) {
  if (*abort_flag) return;
  if (!mbar_wait_bounded(bar, parity)) {
    *abort_flag = 1;
    record_error(err, FQ_ETIMEOUT);
  }
}

// Exit path after a wait gave up.  Copies the producer issued land in this
// CTA's shared memory and MMAs the issuing thread started read it and write
// TMEM, so neither may outlive the CTA or its TMEM allocation.
//  * drain_copies: the producer issues a stage's next copy only after its
//    wait saw the stage consumed (and so its previous copy landed), so only
//    the last `stages` copies can be in flight: wait for their full phases.
//  * drain_mmas: one commit after all the thread's MMAs, waited for.
// Both wait with the default bound and ignore the abort flag.
__device__ __forceinline__ void drain_copies(uint32_t full, int issued, int stages) {
  for (int j = issued > stages ? issued - stages : 0; j < issued; ++j)
    mbar_wait_bounded(full + 8 * uint32_t(j % stages), uint32_t((j / stages) & 1));
}

struct GemmParams {
  uint64_t *C;
  int64_t m, pc;   // rows of C, pitch words of C
  int ksteps;      // la / 128
  int mblocks, nblocks, tiles;
  int group;       // row blocks per group of the tile order
  int plane;       // GF(4): -1 writes both planes, 0 or 1 adds into that plane
  bool small;      // every sum's magnitude is at most kSmallSum (l B^2 <= 2^22 - 8)
  unsigned *err;
};

// Tile t in grouped order: prm.group row blocks at a time, all column blocks
// of the group, so that a wave of tiles reuses a few rows of A and columns
// of B from L2.
__device__ __forceinline__ void tile_coords(const GemmParams &prm, int t, int &mb, int &nb) {
  const int per_group = prm.group * prm.nblocks;
  const int g = t / per_group, first = g * prm.group;
  const int rows = prm.mblocks - first < prm.group ? prm.mblocks - first : prm.group;
  const int in = t - g * per_group;
  mb = first + in % rows;
  nb = in / rows;
}

// Bits 0, 2, ..., 30 of x gathered into bits 0..15.
__device__ __forceinline__ uint32_t even16(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  return (x | (x >> 8)) & 0x0000FFFFu;
}

// Bits 0, 4, ..., 28 of x gathered into bits 0..7.
__device__ __forceinline__ uint32_t nib8(uint32_t x) {
  x &= 0x11111111u;
  x = (x | (x >> 3)) & 0x03030303u;
  x = (x | (x >> 6)) & 0x000F000Fu;
  return (x | (x >> 12)) & 0x000000FFu;
}

// Sums of magnitude at most kSmallSum leave the fp32 accumulator through one
// add: for an integer x with |x| <= 2^22 - 8, residue_magic<p>() + x is exact
// and lies in [2^23, 2^24), so its bit pattern is 0x4B000000 + (the constant
// - 2^23) + x; the constant is 1.5 2^23 + d, d (0, 2, 1, 0 for p = 2, 3, 5, 7)
// making that pattern congruent to x mod p.
constexpr int64_t kSmallSum = (int64_t(1) << 22) - 8;
template <int MOD>
__device__ __forceinline__ float residue_magic() {
  return MOD == 3 ? 12582914.0f : (MOD == 5 ? 12582913.0f : 12582912.0f);
}

// 32 accumulator values of one row (exact integers in fp32, |x| < 2^24)
// reduced mod p and packed into one 32-bit word per plane (value i at bit i).
// Each value first becomes a non-negative 32-bit integer y with x's residue:
// the bits of x + residue_magic (one add) when the caller knows |x| <=
// kSmallSum (`small`), else the truncated integer plus p 2^25.  Then q =
// floor(y / p) by a multiply-high (0x55555556 is exact for y < 2^31 at p =
// 3, 0x24924925 for y < 2^32 / 3 at p = 7, 0xCCCCCCCD with a shift at p = 5),
// and r = y - p q is added into 2-bit (p = 3) or 4-bit (p = 5, 7) fields,
// whose bit-planes are gathered 16 or 8 values at a time.  p = 2 takes y's
// low bit.  v is overwritten.
template <int Q, int P>
__device__ __forceinline__ void pack32(uint32_t (&v)[32], uint32_t (&h)[P], bool small) {
  constexpr int mod = Q == 4 ? 2 : Q;
  if (small) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) + residue_magic<mod>());
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = uint32_t(__float2int_rz(__uint_as_float(v[i])) + mod * (1 << 25));
  }
  if constexpr (mod == 2) {
    uint32_t part[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 32; ++i) part[i & 3] += (v[i] & 1u) << i;
    h[0] = (part[0] | part[1]) | (part[2] | part[3]);
  } else if constexpr (mod == 3) {
    uint32_t f[2] = {0u, 0u};  // value i in bits 2 (i % 16) .. of f[i / 16]
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const uint32_t q = __umulhi(v[i], 0x55555556u);
      f[i >> 4] += (v[i] - 3u * q) << (2 * (i & 15));
    }
    // unit: r != 0 (either bit of the field); sign: r == 2 (its high bit)
    h[0] = even16(f[0] | (f[0] >> 1)) | (even16(f[1] | (f[1] >> 1)) << 16);
    h[1] = even16(f[0] >> 1) | (even16(f[1] >> 1) << 16);
  } else {
    uint32_t f[4] = {0u, 0u, 0u, 0u};  // value i in bits 4 (i % 8) .. of f[i / 8]
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const uint32_t q = mod == 5 ? (__umulhi(v[i], 0xCCCCCCCDu) >> 2) : __umulhi(v[i], 0x24924925u);
      f[i >> 3] += (v[i] - uint32_t(mod) * q) << (4 * (i & 7));
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
      h[p] = nib8(f[0] >> p) | (nib8(f[1] >> p) << 8) | (nib8(f[2] >> p) << 16) | (nib8(f[3] >> p) << 24);
  }
}

// NW 64-column words of one accumulator row (this lane's TMEM lane, from
// column address taddr), reduced mod p and packed into plane words (pack32
// per 32-value load).
template <int Q, int P, int NW = BN / 64>
__device__ __forceinline__ void drain_accumulator(uint32_t taddr, uint64_t (&words)[P][NW], bool small,
                                                  int live = 2 * NW) {
#pragma unroll
  for (int c = 0; c < 2 * NW; ++c) {
    if (c >= live) {  // columns past the product's n (warp-uniform): nothing to read
#pragma unroll
      for (int p = 0; p < P; ++p) {
        if (c & 1)
          words[p][c >> 1] &= 0xFFFFFFFFull;
        else
          words[p][c >> 1] = 0ull;
      }
      continue;
    }
    uint32_t v[32], hw[P];
    tmem_ld32(taddr + uint32_t(c * 32), v);
    pack32<Q, P>(v, hw, small);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t h = hw[p];
      if (c & 1)
        words[p][c >> 1] |= h << 32;
      else
        words[p][c >> 1] = h;
    }
  }
}

// Store one row's packed words at word w0 of C's row.  GF(4): plane < 0
// writes the F_2 result into both planes, else XORs it into that plane.
template <int Q, int P, int NW = BN / 64>
__device__ __forceinline__ void store_words(const GemmParams &prm, int64_t row, int64_t w0,
                                            const uint64_t (&words)[P][NW]) {
  if (!debug_ok(row < prm.m && w0 + NW <= prm.pc, prm.err)) return;
  if constexpr (Q == 4) {
    if (prm.plane < 0) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        uint64_t *dst = prm.C + (int64_t(p) * prm.m + row) * prm.pc + w0;
#pragma unroll
        for (int w = 0; w < NW; ++w) dst[w] = words[0][w];
      }
    } else {
      uint64_t *dst = prm.C + (int64_t(prm.plane) * prm.m + row) * prm.pc + w0;
#pragma unroll
      for (int w = 0; w < NW; ++w) dst[w] ^= words[0][w];
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      uint64_t *dst = prm.C + (int64_t(p) * prm.m + row) * prm.pc + w0;
#pragma unroll
      for (int w = 0; w < NW; ++w) dst[w] = words[p][w];
    }
  }
}

// Persistent: CTA b takes tiles b, b + grid, ...  Warp 0 streams A and B
// slices through the stage ring, warp 1 issues the MMAs of each tile into one
// of two TMEM accumulators, warps 4..7 drain the other accumulator (TMEM
// lanes 32 (warp - 4) .. + 31 are rows of the tile) and store the codes.
template <int Q, int P>
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const GemmParams prm) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned (128-byte swizzle atoms)
  unsigned char *smem = smem_raw + (base - raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full = base + BAR_OFF, empty = full + 8 * STAGES, accfull = empty + 8 * STAGES,
                 accempty = accfull + 8 * ACC;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + BAR_OFF + 8 * NBARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + BAR_OFF + 8 * NBARS + 8);

  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + 8 * s, 1);
      mbar_init(empty + 8 * s, 1);
    }
    for (int b = 0; b < ACC; ++b) {
      mbar_init(accfull + 8 * b, 1);
      mbar_init(accempty + 8 * b, 4);  // one arrival per epilogue warp
    }
    mbar_init(accempty + 8 * ACC, 1);  // the MMA drain
    fence_mbar_init();
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int it = 0;
    for (int t = blockIdx.x; t < prm.tiles && !*abort_flag; t += gridDim.x) {
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      for (int ks = 0; ks < prm.ksteps; ++ks, ++it) {
        const int s = it % STAGES;
        if (it >= STAGES) wait_bar(empty + 8 * s, uint32_t((it / STAGES - 1) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        const uint32_t a_dst = base + uint32_t(s * STAGE_BYTES), b_dst = a_dst + A_BYTES;
        mbar_expect_tx(full + 8 * s, STAGE_BYTES);
        tma_load_2d(a_dst, &tmA, full + 8 * s, ks * BK, mb * BM);
        tma_load_2d(b_dst, &tmB, full + 8 * s, ks * BK, nb * BN);
      }
    }
    if (*abort_flag) drain_copies(full, it, STAGES);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    int it = 0, li = 0;
    for (int t = blockIdx.x; t < prm.tiles && !*abort_flag; t += gridDim.x, ++li) {
      const int b = li % ACC;
      if (li >= ACC) wait_bar(accempty + 8 * b, uint32_t((li / ACC - 1) & 1), abort_flag, prm.err);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + uint32_t(b * BN);
      for (int ks = 0; ks < prm.ksteps; ++ks, ++it) {
        const int s = it % STAGES;
        wait_bar(full + 8 * s, uint32_t((it / STAGES) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_src = base + uint32_t(s * STAGE_BYTES), b_src = a_src + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk)
          mma_e4m3(d, smem_desc(a_src + UK * kk), smem_desc(b_src + UK * kk), (ks | kk) != 0);
        mma_commit(empty + 8 * s);  // the stage is free once these MMAs have read it
      }
      mma_commit(accfull + 8 * b);  // this tile's accumulator is complete
    }
    if (*abort_flag) {  // the MMAs issued so far complete before TMEM is freed
      mma_commit(accempty + 8 * ACC);
      mbar_wait_bounded(accempty + 8 * ACC, 0);
    }
  } else if (warp >= 4) {
    // ---- epilogue
    const int ew = warp - 4;
    int li = 0;
    for (int t = blockIdx.x; t < prm.tiles; t += gridDim.x, ++li) {
      const int b = li % ACC;
      wait_bar(accfull + 8 * b, uint32_t((li / ACC) & 1), abort_flag, prm.err);
      if (*abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      const int64_t row = int64_t(mb) * BM + ew * 32 + lane;
      uint64_t words[P][BN / 64];
      drain_accumulator<Q, P>(tmem + (uint32_t(ew * 32) << 16) + uint32_t(b * BN), words, prm.small);
      // the accumulator has been read: hand it back to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(accempty + 8 * b);
      if (row < prm.m) store_words<Q, P>(prm, row, int64_t(nb) * (BN / 64), words);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------- CTA-pair product --
//
// The same product on SM pairs (cta_group::2): a cluster of two CTAs owns a
// 256 x 256 tile of C.  Each CTA stages its own 128 rows of A and its own 128
// rows of B^T (a 6-stage ring of 32 KB stages), and the TMA loads of both
// count on the leader CTA's full barrier.  The leader's MMA thread issues
// tcgen05.mma.cta_group::2 (M = 256, N = 256, K = 32), which reads A and B^T
// from both CTAs' shared memory and writes rows 128 r .. 128 r + 127 of the
// tile into CTA r's TMEM; its commits arrive on the stage and accumulator
// barriers of both CTAs.  Both epilogues hand an accumulator back on the
// leader's barrier.  Per flop, each SM moves two thirds of the operand bytes
// of the single-CTA kernel.

constexpr int A2_BYTES = 128 * BK, B2_BYTES = 128 * BK;  // a CTA's 128 rows of A, or of one B^T block
constexpr int kWideKsteps = 32;  // k-slices from which the wide pair form runs (l > 3968)

// Geometry of the SM-pair kernels.  The standard form owns 256 x 256 tiles
// with two 256-column accumulators (the epilogue overlaps the next tile); the
// wide form owns 256 x 512 tiles with one 512-column accumulator: each CTA
// stages two 128-row B^T blocks per k-slice and the leader issues two MMAs
// (N = 256 each) per 32-deep step, so a k-slice brings 48 KB for 1024 MMA
// cycles instead of 32 KB for 512 (a third more time to cover a load's
// latency with the same 192 KB ring), at the price of an epilogue that no
// MMA overlaps.
template <bool WIDE>
struct PairGeo {
  static constexpr int NB = WIDE ? 512 : 256;       // columns of C per pair tile
  static constexpr int BBLK = NB / 256;             // 128-row B^T blocks per CTA per stage
  static constexpr int STAGE = A2_BYTES + BBLK * B2_BYTES;
  static constexpr int STAGES = WIDE ? 4 : 6;
  static constexpr int NACC = WIDE ? 1 : 2;         // accumulators of NB columns (NB * NACC = 512)
  static constexpr int BAR_OFF = STAGES * STAGE;
  static constexpr int NBARS = 2 * STAGES + 2 * NACC + 1;  // + the MMA drain barrier
  static constexpr int SMEM = BAR_OFF + 8 * NBARS + 16 + 1024;
  static constexpr int EPI = WIDE ? 8 : 4;          // epilogue warps (the wide form's is exposed: twice as many)
  static constexpr int THREADS = 128 + 32 * EPI;
};
// kind::f8f6f4, fp32 accumulator, e4m3 A and B, K-major, N = 256, M = 256
constexpr uint32_t kIdesc2 = (1u << 4) | (uint32_t(BN >> 3) << 17) | (uint32_t(256 >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// The shared::cluster address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA load into this CTA's shared memory whose bytes count on an mbarrier of
// either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void mma_e4m3_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc2), "r"(accumulate)
      : "memory");
}

// Arrive on the mbarrier at this offset in both CTAs once the pair's issued
// MMAs have completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(static_cast<uint16_t>(3))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

// Bounded wait with cluster-scope acquire (arrivals from the peer CTA).
__device__ __forceinline__ void wait_bar_cluster(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                                 unsigned *err) {
  if (*abort_flag) return;
  uint32_t done = 0;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return;
    if (globaltimer_ns() - t0 > 2000000000ull) {
      *abort_flag = 1;
      record_error(err, FQ_ETIMEOUT);
      return;
    }
  }
}

template <int Q, int P, bool WIDE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PairGeo<WIDE>::THREADS, 1)
    tc_gemm2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const GemmParams prm) {
  using G = PairGeo<WIDE>;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned (128-byte swizzle atoms)
  unsigned char *smem = smem_raw + (base - raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t full = base + G::BAR_OFF, empty = full + 8 * G::STAGES, accfull = empty + 8 * G::STAGES,
                 accempty = accfull + 8 * G::NACC;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G::BAR_OFF + 8 * G::NBARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G::BAR_OFF + 8 * G::NBARS + 8);

  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < G::STAGES; ++s) {
      mbar_init(full + 8 * s, 1);   // the leader's producer arrives; both CTAs' bytes complete it
      mbar_init(empty + 8 * s, 1);  // one multicast commit
    }
    for (int b = 0; b < G::NACC; ++b) {
      mbar_init(accfull + 8 * b, 1);
      mbar_init(accempty + 8 * b, 2 * G::EPI);  // the epilogue warps of both CTAs (the leader's barrier)
    }
    mbar_init(accempty + 8 * G::NACC, 1);  // the leader's MMA drain
    fence_mbar_init();
  }
  if (warp == 2) {  // one warp of each CTA allocates the pair's columns together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised, the columns allocated
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int cl = int(blockIdx.x >> 1), ncl = int(gridDim.x >> 1);

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (both CTAs): this CTA's rows of A and of each B^T block
    int it = 0;
    for (int t = cl; t < prm.tiles && !*abort_flag; t += ncl) {
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      for (int ks = 0; ks < prm.ksteps; ++ks, ++it) {
        const int s = it % G::STAGES;
        if (it >= G::STAGES) wait_bar(empty + 8 * s, uint32_t((it / G::STAGES - 1) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        if (leader) mbar_expect_tx(full + 8 * s, 2 * G::STAGE);
        const uint32_t bar = map_to_rank(full + 8 * s, 0);
        const uint32_t a_dst = base + uint32_t(s * G::STAGE), b_dst = a_dst + A2_BYTES;
        tma_load_2d_pair(a_dst, &tmA, bar, ks * BK, mb * 256 + 128 * int(rank));
#pragma unroll
        for (int j = 0; j < G::BBLK; ++j)
          tma_load_2d_pair(b_dst + uint32_t(j * B2_BYTES), &tmB, bar, ks * BK, nb * G::NB + 256 * j + 128 * int(rank));
      }
    }
    // The last commits to this CTA's stage barriers have landed before it
    // exits.  After a wait gave up these waits still run (default bound): this
    // CTA's copies count on the leader's full barrier, which it cannot watch,
    // but a stage's commit comes only after its copies have landed, and a
    // copy that never gets one was issued at least the whole bound earlier.
    for (int j = it > G::STAGES ? it - G::STAGES : 0; j < it; ++j)
      mbar_wait_bounded(empty + 8 * uint32_t(j % G::STAGES), uint32_t((j / G::STAGES) & 1));
  } else if (warp == 1 && lane == 0 && leader) {
    // ---- MMA issuer (the leader CTA only)
    int it = 0, li = 0;
    for (int t = cl; t < prm.tiles && !*abort_flag; t += ncl, ++li) {
      const int b = li % G::NACC;
      if (li >= G::NACC)
        wait_bar_cluster(accempty + 8 * b, uint32_t((li / G::NACC - 1) & 1), abort_flag, prm.err);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + uint32_t(b * G::NB);
      for (int ks = 0; ks < prm.ksteps; ++ks, ++it) {
        const int s = it % G::STAGES;
        wait_bar(full + 8 * s, uint32_t((it / G::STAGES) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_src = base + uint32_t(s * G::STAGE), b_src = a_src + A2_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk)
#pragma unroll
          for (int j = 0; j < G::BBLK; ++j)  // B^T block j -> accumulator columns 256 j ..
            mma_e4m3_pair(d + uint32_t(256 * j), smem_desc(a_src + UK * kk),
                          smem_desc(b_src + uint32_t(j * B2_BYTES) + UK * kk), (ks | kk) != 0);
        mma_commit_pair(empty + 8 * s);  // both CTAs' stage s is free once these MMAs have read it
      }
      mma_commit_pair(accfull + 8 * b);  // this tile's accumulators are complete in both CTAs
    }
    if (*abort_flag) {  // the pair's MMAs complete before either CTA frees its TMEM
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       accempty + 8 * G::NACC)
                   : "memory");
      mbar_wait_bounded(accempty + 8 * G::NACC, 0);
    }
  } else if (warp >= 4) {
    // ---- epilogue (both CTAs): rows 128 rank + 32 (warp % 4) + lane of the
    // tile; with eight epilogue warps, group (warp - 4) / 4 takes 128 of
    // every 256 columns
    constexpr int CW = 256 / (G::EPI / 4);  // columns per warp per 256-column block
    const int ew = warp & 3, grp = (warp - 4) >> 2;
    const uint32_t back = leader ? accempty : map_to_rank(accempty, 0);
    int li = 0;
    for (int t = cl; t < prm.tiles; t += ncl, ++li) {
      const int b = li % G::NACC;
      wait_bar(accfull + 8 * b, uint32_t((li / G::NACC) & 1), abort_flag, prm.err);
      if (*abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      const int64_t row = int64_t(mb) * 256 + 128 * int(rank) + ew * 32 + lane;
#pragma unroll 1
      for (int j = 0; j < G::BBLK; ++j) {  // one 256-column block at a time
        uint64_t words[P][CW / 64];
        drain_accumulator<Q, P, CW / 64>(
            tmem + (uint32_t(ew * 32) << 16) + uint32_t(b * G::NB + 256 * j + CW * grp), words, prm.small);
        if (row < prm.m)
          store_words<Q, P, CW / 64>(prm, row, int64_t(nb) * (G::NB / 64) + 4 * j + (CW / 64) * grp, words);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if (leader)
          mbar_arrive_cta(accempty + 8 * b);
        else
          mbar_arrive_cluster(back + 8 * b);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // neither CTA touches the other's memory any more
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------- fp4 CTA-pair product --
//
// The product on SM pairs from packed e2m1 operands (tcgen05.mma.cta_group::2
// kind::mxf4, twice the e4m3 rate).  A 128-byte k-slice is 256 elements deep
// and feeds four MMAs of K = 64, the same 32 bytes per MMA as the e4m3 form,
// so the descriptors, the swizzle and the stage layout do not change.  The
// block-scaled kind reads scale factors from TMEM: columns 448..511 of both
// CTAs are filled once with ue8m0 1.0 (0x7F) in every byte, so whichever
// bytes the hardware takes, every block is scaled by 1.0 and the sums stay
// the exact integers of the e4m3 form.  That leaves 448 columns for the
// accumulator: a pair owns 256 x 448 tiles (7 words of C), computed as two
// MMAs of N = 224 per 64-deep step, each CTA staging its 128 rows of A and
// 112 rows of each of the two B^T halves (44 KB a stage, 5 stages).  The
// last column tile of a product is narrower (w = 64 pitch - 448 nb, a
// multiple of 64): its halves take N_j = min(w - 224 j, 224) columns, and
// CTA r loads B^T rows 224 j + r N_j / 2 .., so that accumulator column c is
// always tile column c.  The accumulator is not double-buffered; twice as
// many epilogue warps as in the 256 x 256 pair form drain it, each a
// quarter of the row's words.
namespace f4 {
constexpr int NB = 448, HALF = 224, BROWS = HALF / 2;  // tile columns, per MMA, B^T rows per CTA per half
constexpr int B_BYTES = BROWS * BK;                     // 14 KB (a whole number of 1 KB swizzle atoms)
constexpr int STAGE = A2_BYTES + 2 * B_BYTES;
constexpr int STAGES = 5;
constexpr int BAR_OFF = STAGES * STAGE;
constexpr int NBARS = 2 * STAGES + 2 + 1;  // full, empty, accfull, accempty, the MMA drain
constexpr int SMEM = BAR_OFF + 8 * NBARS + 16 + 1024;
constexpr int EPI = 16;                     // epilogue warps: lane quadrant warp % 4, column group (warp - 4) / 4
constexpr int THREADS = 128 + 32 * EPI;
constexpr int WORDS = NB / 64;              // 64-column words of C per tile row
constexpr int GROUPS = EPI / 4, WPG = (WORDS + GROUPS - 1) / GROUPS;  // column groups, words per group
constexpr uint32_t SF_COL = NB;             // scale factors: columns 448 .. 511
static_assert(SMEM <= 232448, "shared memory per CTA");
}  // namespace f4

// kind::mxf4 instruction descriptor: E2M1 A and B (format 1, bits 7-9 and
// 10-12), both K-major, N >> 3 (bits 17-22), ue8m0 scale factors (bit 23),
// M = 256 (bits 24-28), scale-factor ids 0, dense K = 64.
__host__ __device__ constexpr uint32_t idesc_mxf4_pair(int n) {
  return (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (1u << 23) | (uint32_t(256 >> 4) << 24);
}

__device__ __forceinline__ void mma_fp4_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t accumulate, uint32_t sf) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate), "r"(sf), "r"(sf + 32u)
      : "memory");
}

// 32 TMEM columns of this warp's lane quadrant set to v.
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(v)
      : "memory");
}

// Columns of tile nb of the fp4 pair form: 448, or what is left of the pitch.
__device__ __forceinline__ int f4_width(const GemmParams &prm, int nb) {
  const int64_t left = 64 * prm.pc - int64_t(f4::NB) * nb;
  return left < f4::NB ? int(left) : f4::NB;
}

// Two 32-column TMEM loads (columns taddr .. + 63 of this warp's lanes), one
// wait for both.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[2][32]) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[h][0]), "=r"(v[h][1]), "=r"(v[h][2]), "=r"(v[h][3]), "=r"(v[h][4]), "=r"(v[h][5]), "=r"(v[h][6]),
          "=r"(v[h][7]), "=r"(v[h][8]), "=r"(v[h][9]), "=r"(v[h][10]), "=r"(v[h][11]), "=r"(v[h][12]),
          "=r"(v[h][13]), "=r"(v[h][14]), "=r"(v[h][15]), "=r"(v[h][16]), "=r"(v[h][17]), "=r"(v[h][18]),
          "=r"(v[h][19]), "=r"(v[h][20]), "=r"(v[h][21]), "=r"(v[h][22]), "=r"(v[h][23]), "=r"(v[h][24]),
          "=r"(v[h][25]), "=r"(v[h][26]), "=r"(v[h][27]), "=r"(v[h][28]), "=r"(v[h][29]), "=r"(v[h][30]),
          "=r"(v[h][31])
        : "r"(taddr + uint32_t(32 * h)));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int Q, int P>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(f4::THREADS, 1)
    tc_gemm4_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const GemmParams prm) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned (128-byte swizzle atoms)
  unsigned char *smem = smem_raw + (base - raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t full = base + f4::BAR_OFF, empty = full + 8 * f4::STAGES, accfull = empty + 8 * f4::STAGES,
                 accempty = accfull + 8, drain = accempty + 8;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + f4::BAR_OFF + 8 * f4::NBARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + f4::BAR_OFF + 8 * f4::NBARS + 8);

  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < f4::STAGES; ++s) {
      mbar_init(full + 8 * s, 1);   // the leader's producer arrives; both CTAs' bytes complete it
      mbar_init(empty + 8 * s, 1);  // one multicast commit
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, 2 * f4::EPI);  // the epilogue warps of both CTAs (the leader's barrier)
    mbar_init(drain, 1);               // the leader's MMA drain
    fence_mbar_init();
  }
  if (warp == 2) {  // one warp of each CTA allocates the pair's columns together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised, the columns allocated
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (warp >= 4 && warp < 8) {  // scale factors 1.0 (ue8m0 0x7F) in columns 448..511 of every lane
    const uint32_t q0 = tmem + (uint32_t((warp & 3) * 32) << 16) + f4::SF_COL;
    tmem_fill32(q0, 0x7F7F7F7Fu);
    tmem_fill32(q0 + 32u, 0x7F7F7F7Fu);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // both CTAs' scale factors are in place before the first MMA
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int cl = int(blockIdx.x >> 1), ncl = int(gridDim.x >> 1);

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (both CTAs): this CTA's rows of A and of each B^T half
    int it = 0;
    for (int t = cl; t < prm.tiles && !*abort_flag; t += ncl) {
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      const int w = f4_width(prm, nb);
      const int n0 = w < f4::HALF ? w : f4::HALF, n1 = w - n0;
      const int halves = n1 > 0 ? 2 : 1;
      for (int ks = 0; ks < prm.ksteps; ++ks, ++it) {
        const int s = it % f4::STAGES;
        if (it >= f4::STAGES) wait_bar(empty + 8 * s, uint32_t((it / f4::STAGES - 1) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        if (leader) mbar_expect_tx(full + 8 * s, 2 * (A2_BYTES + halves * f4::B_BYTES));
        const uint32_t bar = map_to_rank(full + 8 * s, 0);
        const uint32_t a_dst = base + uint32_t(s * f4::STAGE), b_dst = a_dst + A2_BYTES;
        tma_load_2d_pair(a_dst, &tmA, bar, ks * BK, mb * 256 + 128 * int(rank));
        tma_load_2d_pair(b_dst, &tmB, bar, ks * BK, nb * f4::NB + int(rank) * (n0 / 2));
        if (halves == 2)
          tma_load_2d_pair(b_dst + uint32_t(f4::B_BYTES), &tmB, bar, ks * BK,
                           nb * f4::NB + f4::HALF + int(rank) * (n1 / 2));
      }
    }
    // The last commits to this CTA's stage barriers have landed before it
    // exits (see tc_gemm2_kernel: a stage is committed only after its copies
    // have landed, and these waits run with the default bound).
    for (int j = it > f4::STAGES ? it - f4::STAGES : 0; j < it; ++j)
      mbar_wait_bounded(empty + 8 * uint32_t(j % f4::STAGES), uint32_t((j / f4::STAGES) & 1));
  } else if (warp == 1 && lane == 0 && leader) {
    // ---- MMA issuer (the leader CTA only)
    int it = 0, li = 0;
    const uint32_t sf = tmem + f4::SF_COL;
    for (int t = cl; t < prm.tiles && !*abort_flag; t += ncl, ++li) {
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      const int w = f4_width(prm, nb);
      const int n0 = w < f4::HALF ? w : f4::HALF, n1 = w - n0;
      const uint32_t id0 = idesc_mxf4_pair(n0), id1 = idesc_mxf4_pair(n1 > 0 ? n1 : 32);
      if (li >= 1) wait_bar_cluster(accempty, uint32_t((li - 1) & 1), abort_flag, prm.err);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int ks = 0; ks < prm.ksteps; ++ks, ++it) {
        const int s = it % f4::STAGES;
        wait_bar(full + 8 * s, uint32_t((it / f4::STAGES) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_src = base + uint32_t(s * f4::STAGE), b_src = a_src + A2_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk) {
          mma_fp4_pair(tmem, smem_desc(a_src + UK * kk), smem_desc(b_src + UK * kk), id0, (ks | kk) != 0, sf);
          if (n1 > 0)
            mma_fp4_pair(tmem + uint32_t(f4::HALF), smem_desc(a_src + UK * kk),
                         smem_desc(b_src + uint32_t(f4::B_BYTES) + UK * kk), id1, (ks | kk) != 0, sf);
        }
        mma_commit_pair(empty + 8 * s);  // both CTAs' stage s is free once these MMAs have read it
      }
      mma_commit_pair(accfull);  // this tile's accumulator is complete in both CTAs
    }
    if (*abort_flag) {  // the pair's MMAs complete before either CTA frees its TMEM
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain)
                   : "memory");
      mbar_wait_bounded(drain, 0);
    }
  } else if (warp >= 4) {
    // ---- epilogue (both CTAs): row 128 rank + 32 (warp % 4) + lane of the
    // tile; column group g = (warp - 4) / 4 drains words [WPG g, WPG (g + 1))
    // of the tile's seven (those inside its width)
    const int ew = warp & 3, grp = (warp - 4) >> 2;
    const int w_lo = f4::WPG * grp, w_hi = w_lo + f4::WPG < f4::WORDS ? w_lo + f4::WPG : f4::WORDS;
    const uint32_t back = leader ? accempty : map_to_rank(accempty, 0);
    int li = 0;
    for (int t = cl; t < prm.tiles; t += ncl, ++li) {
      wait_bar(accfull, uint32_t(li & 1), abort_flag, prm.err);
      if (*abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int mb, nb;
      tile_coords(prm, t, mb, nb);
      const int w = f4_width(prm, nb);
      const int64_t row = int64_t(mb) * 256 + 128 * int(rank) + ew * 32 + lane;
#pragma unroll 1
      for (int wd = w_lo; wd < w_hi && 64 * wd < w; ++wd) {
        uint32_t v[2][32], h0[P], h1[P];
        tmem_ld64(tmem + (uint32_t(ew * 32) << 16) + uint32_t(64 * wd), v);
        pack32<Q, P>(v[0], h0, prm.small);
        pack32<Q, P>(v[1], h1, prm.small);
        uint64_t words[P][1];
#pragma unroll
        for (int p = 0; p < P; ++p) words[p][0] = uint64_t(h0[p]) | (uint64_t(h1[p]) << 32);
        if (row < prm.m) store_words<Q, P, 1>(prm, row, int64_t(nb) * f4::WORDS + wd, words);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if (leader)
          mbar_arrive_cta(accempty);
        else
          mbar_arrive_cluster(back);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // neither CTA touches the other's memory any more
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------- batched products --
//
// The persistent CTAs work in groups of kTcGroup (one thread-block cluster);
// each group works through its own products, in the order the plan lists
// them, and the group's CTAs share every product: all of them convert parts
// of its operands into the group's scratch buffer, and CTA r of the group
// computes the product's tiles r, r + kTcGroup, ...  Sharing halves the
// operand bytes the GPU keeps live at a time (two products per group instead
// of two per SM), so that more of the converted operands are read back from
// L2 rather than DRAM.  Product i of a group uses the group's scratch buffer
// i mod 2, rows of 128 bytes, both operands K-blocked in 128-row blocks:
//   A (K-major): the 128-element chunk c of k of row r at row
//       ((r / 128) * kb + c) * 128 + r % 128        (kb = la / 128 k-slices);
//   B (N-major, B as it is, no transpose): the 128-element chunk c of n of
//       row k at row (c * kb + k / 128) * 128 + k % 128, after A's rows;
//       rows k in [l, la) are zero (the depth padding).
// A stage of the tile kernel is one 128-row block of A and two of B (the two
// 128-column halves of a 256-column tile), 16 KB each, so every TMA copy is
// one contiguous 16 KB block.  Converter warps fill one buffer while the
// TMA, MMA and epilogue warps compute the previous product from the other.
//
// Warps: 0 (one thread) TMA loads, 1 (one thread) MMAs, 2 TMEM allocation,
// 4..11 epilogue (TMEM lane quadrant warp % 4, 128-column half (warp - 4) /
// 4), 12..27 and, once the TMEM is allocated, 2 and 3 converters.
// Hand-overs, on mbarriers in every CTA of the group with cluster-scope
// release and acquire:
//   conv_full[b]   converters -> TMA threads: the product's operands are in
//                  buffer b (each converter thread orders its global writes
//                  before the async proxy's reads, then arrives on every
//                  CTA's barrier);
//   conv_empty[b]  MMA threads -> converters: every copy out of buffer b has
//                  landed in shared memory (each MMA thread arrives on every
//                  CTA's barrier after its last full-stage wait of the
//                  product), so the buffer may be refilled.
// A group's CTAs leave together (a cluster barrier), so no arrival reaches a
// CTA that has exited.
constexpr int EPI_WARPS_B = 8;
constexpr int CONV_WARPS = 16;                  // warps 12..27
constexpr int FIRST_CONV_WARP = 4 + EPI_WARPS_B;
constexpr int THREADS_F = 32 * FIRST_CONV_WARP + 32 * CONV_WARPS;
constexpr int CONV_THREADS = 32 * (CONV_WARPS + 2);  // and warps 2, 3 once the TMEM is allocated
constexpr int NBARS_F = NBARS + 4;  // + conv_full[2], conv_empty[2]
constexpr int SMEM_F = BAR_OFF + 8 * NBARS_F + 16 + 1024;
// kind::f8f6f4, fp32 accumulator, e4m3 A (K-major) and B (N-major), N = 256, M = 128
constexpr uint32_t kIdescMn = kIdesc | (1u << 16);

// Shared-memory descriptor of an N-major operand with the 128-byte swizzle:
// 128-column atoms (128 bytes wide, one per 16 KB block of 128 k-rows),
// leading byte offset 16 KB between the atoms along N, stride byte offset
// 1024 bytes between groups of 8 k-rows.
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t(16384 >> 4) << 16;        // leading byte offset: the next 128 columns
  d |= uint64_t(1024 >> 4) << 32;         // stride byte offset: the next 8 k-rows
  d |= uint64_t(1) << 46;                 // version
  d |= uint64_t(2) << 61;                 // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_e4m3_mn(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdescMn), "r"(accumulate)
      : "memory");
}

// A planes matrix of `rows_valid` rows (pitch words, P planes; rows up to
// `rows` read as zero) as e4m3 bytes in 128-element chunks: chunk c of row r
// (c < chunks) becomes the 128-byte scratch row row_of(r, c).  The work is
// split in 16-element pieces, eight to a chunk, so that eight consecutive
// threads write one 128-byte row (a warp's 16-byte stores cover four whole
// rows).  Converter thread ct of the nct converting threads takes the pieces
// ct, ct + nct, ... (row-major), UNR at a time with all their words loaded
// first; a thread's (row, piece) advances by the stride's quotient and
// remainder, so no division runs per piece.
template <int Q, int P, class RowOf>
__device__ __forceinline__ void convert_rows(const uint64_t *__restrict__ X, int rows_valid, int rows, int64_t pitch,
                                             int chunks, uint8_t *buf, int ct, int nct, RowOf row_of) {
  using CF = ConvField<Q>;
  constexpr int UNR = P == 2 ? 8 : 4;  // pieces whose loads are in flight together (registers allow 8 for two planes)
  const int per_row = 8 * chunks;
  const int radv = nct / per_row, padv = nct % per_row;
  const uint32_t *X32 = reinterpret_cast<const uint32_t *>(X);
  int r = ct / per_row, piece = ct % per_row;
  while (r < rows) {
    uint32_t t[UNR][P];
    int rr[UNR], pp[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      rr[u] = r;
      pp[u] = piece;
#pragma unroll
      for (int p = 0; p < P; ++p)
        t[u][p] = r < rows_valid ? __ldg(X32 + (p * int64_t(rows_valid) + r) * pitch * 2 + (piece >> 1)) : 0u;
      r += radv;
      piece += padv;
      if (piece >= per_row) {
        piece -= per_row;
        ++r;
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (rr[u] >= rows) break;
      uint32_t o[CF::P2];
      select_planes<Q, P>(t[u], 0, o);
      *reinterpret_cast<uint4 *>(buf + row_of(rr[u], pp[u] >> 3) * 128 + (pp[u] & 7) * 16) =
          e4m3x16<CF::Q2, CF::P2>(o, pp[u] & 1);
    }
  }
}

// Starts copying `bytes` at `p` (16-byte aligned, a multiple of 16) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, int64_t bytes) {
  const char *c = static_cast<const char *>(p);
  for (int64_t off = 0; off < bytes; off += 65536) {
    const int64_t n = bytes - off < 65536 ? bytes - off : 65536;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(uint32_t(n)) : "memory");
  }
}

struct BatchParams {
  const BatchProd *prods;
  const int32_t *cta_begin, *cta_list;  // products of group g: cta_list[cta_begin[g] .. cta_begin[g + 1])
  const int64_t *cta_rows;              // kTcGroups x 2: first tensor-map row of each group's buffer 0 and buffer 1
  uint8_t *scratch;
  const uint64_t *const *A;
  const uint64_t *const *B;
  uint64_t *const *C;
  unsigned *err;
};

// One row's words of a batched tile, columns past n cleared; the last column
// tile also clears C's padding words up to the pitch.
struct BatchOut {  // what an epilogue thread needs of its tile's product
  uint64_t *C;
  int64_t m, n, nr, pc;
};

template <int Q, int P>
__device__ __forceinline__ void store_batched(const BatchOut &bp, uint64_t *C, int64_t row, int64_t w0, int half,
                                              uint64_t (&words)[P][2], unsigned *err) {
  // this thread's words w0 + 2 half, + 1 of a 256-column tile
  const int64_t wa = w0 + 2 * half;
  const bool last = (w0 + BN / 64) * 64 >= bp.nr;
  if (!debug_ok(row < bp.m && wa + 1 < bp.pc, err)) return;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    uint64_t *dst = C + (int64_t(p) * bp.m + row) * bp.pc;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int64_t keep = bp.n - (wa + w) * 64;
      const uint64_t mask = keep >= 64 ? ~0ull : (keep <= 0 ? 0ull : ((1ull << keep) - 1));
      dst[wa + w] = words[p][w] & mask;
    }
    if (last)  // C's padding words past the last tile, split between the two halves
      for (int64_t w = w0 + BN / 64 + half; w < bp.pc; w += 2) dst[w] = 0ull;
  }
}

// Row block and column block of tile t of a product with mbs x nbs tiles.
// The operand that the tile walk streams again and again should be the
// smaller one: row blocks outer (A's block stays while all of B streams)
// when A is the larger operand, column blocks outer otherwise.
__device__ __forceinline__ void batch_tile(int t, int mbs, int nbs, int nr, int &mb, int &nb) {
  if (mbs * BM < nr) {  // A (mbs 128 rows) smaller than B (nr columns), per k-slice
    nb = t / mbs;
    mb = t - nb * mbs;
  } else {
    mb = t / nbs;
    nb = t - mb * nbs;
  }
}

// The persistent batched kernel: group g (cluster g) computes the products of
// its list, one after another, 128 x 256 tiles each (in batch_tile's order),
// from the e4m3 operands its converter warps write into its two scratch
// buffers; CTA r of the group takes tiles r, r + kTcGroup, ... of each.
template <int Q, int P>
__global__ void __cluster_dims__(kTcGroup, 1, 1) __launch_bounds__(THREADS_F, 1)
    tc_batched_kernel(const __grid_constant__ CUtensorMap tmA, const BatchParams prm) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *smem = smem_raw + (base - raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full = base + BAR_OFF, empty = full + 8 * STAGES, accfull = empty + 8 * STAGES,
                 accempty = accfull + 8 * ACC, drain = accempty + 8 * ACC, conv_full = drain + 8,
                 conv_empty = conv_full + 16;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + BAR_OFF + 8 * NBARS_F);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + BAR_OFF + 8 * NBARS_F + 8);
  const int rank = int(cluster_rank());

  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + 8 * s, 1);
      mbar_init(empty + 8 * s, 1);
    }
    for (int b = 0; b < ACC; ++b) {
      mbar_init(accfull + 8 * b, 1);
      mbar_init(accempty + 8 * b, EPI_WARPS_B);
    }
    mbar_init(drain, 1);  // the MMA drain
    for (int b = 0; b < 2; ++b) {
      mbar_init(conv_full + 8 * b, kTcGroup * CONV_THREADS);  // every converter thread of the group
      mbar_init(conv_empty + 8 * b, kTcGroup);                // every MMA thread of the group
    }
    fence_mbar_init();
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  cluster_sync();  // every CTA's barriers initialised before any arrival from another CTA
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int grp = blockIdx.x / kTcGroup;
  const int first = prm.cta_begin[grp], count = prm.cta_begin[grp + 1] - first;
  const int64_t row_buf[2] = {prm.cta_rows[2 * grp], prm.cta_rows[2 * grp + 1]};

  if (warp == 0 && lane == 0) {
    // ---- TMA: this CTA's tiles of each product, from its buffer once it is filled
    int it = 0;
    for (int i = 0; i < count && !*abort_flag; ++i) {
      const int b = i & 1;
      wait_bar_cluster(conv_full + 8 * b, uint32_t((i >> 1) & 1), abort_flag, prm.err);
      if (*abort_flag) break;
      const BatchProd bp = prm.prods[prm.cta_list[first + i]];
      const int kb = bp.la >> 7, nbs = bp.nr >> 8, tiles = ((bp.m + 127) >> 7) * nbs;
      const int ya = int(row_buf[b]), yb = int(row_buf[b] + batch_a_rows(bp.m, bp.la));
      for (int t = rank; t < tiles && !*abort_flag; t += kTcGroup) {
        int mb, nb;
        batch_tile(t, (bp.m + 127) >> 7, nbs, bp.nr, mb, nb);
        for (int ks = 0; ks < kb; ++ks, ++it) {
          const int s = it % STAGES;
          if (it >= STAGES) wait_bar(empty + 8 * s, uint32_t((it / STAGES - 1) & 1), abort_flag, prm.err);
          if (*abort_flag) break;
          const uint32_t a_dst = base + uint32_t(s * STAGE_BYTES), b_dst = a_dst + A_BYTES;
          mbar_expect_tx(full + 8 * s, STAGE_BYTES);
          // three contiguous 16 KB blocks: A's rows, then B's two 128-column halves
          tma_load_2d(a_dst, &tmA, full + 8 * s, 0, ya + (mb * kb + ks) * 128);
          tma_load_2d(b_dst, &tmA, full + 8 * s, 0, yb + ((2 * nb) * kb + ks) * 128);
          tma_load_2d(b_dst + 16384, &tmA, full + 8 * s, 0, yb + ((2 * nb + 1) * kb + ks) * 128);
        }
      }
    }
    if (*abort_flag) drain_copies(full, it, STAGES);
  } else if (warp == 1 && lane == 0) {
    // ---- MMAs; after this CTA's last stage of a product has landed, its part
    // of the buffer is free (arrivals on every CTA of the group).  The thread
    // first waits for the product's operands, as the TMA thread does: a CTA
    // with no tiles in two products of the same buffer would otherwise arrive
    // twice in one phase of conv_empty, before another CTA had read the first.
    int it = 0, li = 0;
    bool issued = false;
    for (int i = 0; i < count && !*abort_flag; ++i) {
      wait_bar_cluster(conv_full + 8 * (i & 1), uint32_t((i >> 1) & 1), abort_flag, prm.err);
      if (*abort_flag) break;
      const BatchProd bp = prm.prods[prm.cta_list[first + i]];
      const int kb = bp.la >> 7, tiles = ((bp.m + 127) >> 7) * (bp.nr >> 8);
      for (int t = rank; t < tiles && !*abort_flag; t += kTcGroup, ++li) {
        const int ab = li % ACC;
        if (li >= ACC) wait_bar(accempty + 8 * ab, uint32_t((li / ACC - 1) & 1), abort_flag, prm.err);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + uint32_t(ab * BN);
        for (int ks = 0; ks < kb; ++ks, ++it) {
          const int s = it % STAGES;
          wait_bar(full + 8 * s, uint32_t((it / STAGES) & 1), abort_flag, prm.err);
          if (*abort_flag) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_src = base + uint32_t(s * STAGE_BYTES), b_src = a_src + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / UK; ++kk)  // B: 32 k-rows of 128 bytes per step
            mma_e4m3_mn(d, smem_desc(a_src + UK * kk), smem_desc_mn(b_src + 128 * UK * kk), (ks | kk) != 0);
          mma_commit(empty + 8 * s);
          issued = true;
        }
        mma_commit(accfull + 8 * ab);
      }
      if (!*abort_flag)
        for (int r = 0; r < kTcGroup; ++r) mbar_arrive_cluster(map_to_rank(conv_empty + 8 * (i & 1), uint32_t(r)));
    }
    if (*abort_flag && issued) {  // the MMAs issued so far complete before TMEM is freed
      mma_commit(drain);
      mbar_wait_bounded(drain, 0);
    }
  } else if (warp >= 4 && warp < FIRST_CONV_WARP) {
    // ---- epilogue: TMEM lane quadrant warp % 4, columns 128 half .. + 127
    const int ew = warp & 3, half = (warp - 4) >> 2;
    int li = 0;
    for (int i = 0; i < count && !*abort_flag; ++i) {
      const BatchProd bp = prm.prods[prm.cta_list[first + i]];
      BatchOut bo;
      bo.m = bp.m;
      bo.n = bp.n;
      bo.nr = bp.nr;
      bo.pc = bp.pc;
      bo.C = prm.C[bp.p];
      const int nbs = bp.nr >> 8, tiles = ((bp.m + 127) >> 7) * nbs;
      for (int t = rank; t < tiles; t += kTcGroup, ++li) {
        const int ab = li % ACC;
        wait_bar(accfull + 8 * ab, uint32_t((li / ACC) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int mb, nb;
        batch_tile(t, (bp.m + 127) >> 7, nbs, bp.nr, mb, nb);
        const int64_t row = int64_t(mb) * BM + ew * 32 + lane;
        const int64_t w0 = int64_t(nb) * (BN / 64);
        const int64_t col0 = (w0 + 2 * half) * 64;
        // 32-column chunks holding columns < n
        const int64_t rest = bo.n - col0;
        const int live = rest <= 0 ? 0 : (rest >= 128 ? 4 : int((rest + 31) / 32));
        uint64_t words[P][2];
        constexpr int64_t bb = Q == 4 || Q == 2 ? 1 : (Q - 1) / 2;  // the largest balanced magnitude
        drain_accumulator<Q, P, 2>(tmem + (uint32_t(ew * 32) << 16) + uint32_t(ab * BN + half * 128), words,
                                   int64_t(bp.l) * bb * bb <= kSmallSum, live);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(accempty + 8 * ab);
        if (row < bo.m) store_batched<Q, P>(bo, bo.C, row, w0, half, words, prm.err);
      }
    }
  } else if (warp >= FIRST_CONV_WARP || warp == 2 || warp == 3) {
    // ---- converters: product i into buffer i mod 2, once every CTA of the
    // group has finished reading the product two before it from that buffer;
    // the group's converter threads share each product's pieces, and the
    // next product's planes are fetched into L2 meanwhile (A by CTA 0, B by
    // the last CTA of the group)
    const int ct = warp >= FIRST_CONV_WARP ? tid - 32 * FIRST_CONV_WARP : 32 * CONV_WARPS + tid - 64;
    const int gct = rank * CONV_THREADS + ct;
    constexpr int nct = kTcGroup * CONV_THREADS;
    for (int i = 0; i < count && !*abort_flag; ++i) {
      const int b = i & 1;
      if (i >= 2) {
        wait_bar_cluster(conv_empty + 8 * b, uint32_t(((i - 2) >> 1) & 1), abort_flag, prm.err);
        if (*abort_flag) break;
      }
      const BatchProd bp = prm.prods[prm.cta_list[first + i]];
      if (ct == 0 && i + 1 < count) {
        const BatchProd nx = prm.prods[prm.cta_list[first + i + 1]];
        if (rank == 0) prefetch_l2(prm.A[nx.p], int64_t(P) * nx.m * nx.pa * 8);
        if (rank == kTcGroup - 1) prefetch_l2(prm.B[nx.p], int64_t(P) * nx.l * nx.pb * 8);
      }
      uint8_t *buf = prm.scratch + row_buf[b] * 128;
      const int kb = bp.la >> 7;
      convert_rows<Q, P>(prm.A[bp.p], bp.m, bp.m, bp.pa, kb, buf, gct, nct, [kb](int r, int c) {
        return int64_t((r >> 7) * kb + c) * 128 + (r & 127);
      });
      convert_rows<Q, P>(prm.B[bp.p], bp.l, bp.la, bp.pb, bp.nr >> 7, buf + batch_a_rows(bp.m, bp.la) * 128, gct,
                         nct, [kb](int r, int c) { return int64_t(c * kb + (r >> 7)) * 128 + (r & 127); });
      // this thread's writes are visible to the TMA loads that follow the hand-over
      asm volatile("fence.proxy.async.global;" ::: "memory");
      for (int r = 0; r < kTcGroup; ++r) mbar_arrive_cluster(map_to_rank(conv_full + 8 * b, uint32_t(r)));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  cluster_sync();  // no CTA leaves while another may still arrive on its barriers
}

// ------------------------------------------------------------------ host --

int make_map(CUtensorMap *map, const uint8_t *ptr, int64_t inner, int64_t rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (int rc = tensor_map_encoder(&encode)) return rc;
  memset(map, 0, sizeof(*map));
  const cuuint64_t dims[2] = {cuuint64_t(inner), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(inner)};
  const cuuint32_t box[2] = {cuuint32_t(BK), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(ptr), dims, strides,
                             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS ? FQ_OK : FQ_EINVAL;
}


// Product forms: 2 single SMs (128 x 256 tiles), 3 SM pairs (256 x 256), 4
// SM pairs (256 x 512), all from e4m3 operands; 5 SM pairs (256 x 448) from
// packed e2m1 operands.  By shape: a product of at most 128 rows would leave
// half of every pair idle, so it runs on single SMs; products at least
// kFp4MinL deep take the fp4 form (twice the tensor rate, half the operand
// bytes), whose unoverlapped epilogue a shallower product would not amortise;
// the rest take the 256 x 256 pair form (or, from kWideKsteps k-slices, the
// wide one).
constexpr int64_t kFp4MinL = 2048;
inline int form_for(int64_t m, int64_t l, const TcOptions &to) {
  if (to.form) return to.form;
  if (m <= BM) return 2;
  if (l >= kFp4MinL) return 5;
  return cdiv(l, BK) >= kWideKsteps ? 4 : 3;
}

// Prepared operands in a workspace: per product (GF(4) has three, the other
// fields one) A as m rows, then B transposed as npad rows, each row `row`
// bytes: la e4m3 bytes (la = l rounded up to 128), or la / 2 bytes of packed
// e2m1 (la = l rounded up to 256) for the fp4 form.
struct Layout {
  int rounds;
  bool fp4;
  bool small;  // l B^2 <= kSmallSum: every partial sum leaves the accumulator through one add
  int64_t la, row, npad, pc, a_bytes, b_bytes;
};

inline Layout layout_for(int q, int64_t m, int64_t l, int64_t n, int form) {
  Layout lo;
  lo.rounds = q == 4 ? 3 : 1;
  lo.fp4 = form == 5;
  const int64_t b = q == 2 || q == 4 ? 1 : (q - 1) / 2;  // the largest balanced magnitude
  lo.small = l * b * b <= kSmallSum;
  lo.la = cdiv(l, lo.fp4 ? 2 * BK : BK) * (lo.fp4 ? 2 * BK : BK);
  lo.row = lo.fp4 ? lo.la / 2 : lo.la;
  lo.pc = fq_pitch_words(n);
  lo.npad = lo.pc * 64;
  lo.a_bytes = m * lo.row;
  lo.b_bytes = lo.npad * lo.row;
  return lo;
}

template <int Q, int P>
int gemm(const uint8_t *Ab, const uint8_t *Bt, uint64_t *C, int64_t m, const Layout &lo, int form, int plane,
         const TcOptions &to, cudaStream_t s) {
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  const bool pair = form == 3 || form == 4 || form == 5, wide = form == 4, fp4 = form == 5;
  const int rows = pair ? 2 * BM : BM;
  CUtensorMap ma, mb;
  if (int rc = make_map(&ma, Ab, lo.row, m, BM)) return rc;
  if (int rc = make_map(&mb, Bt, lo.row, lo.npad, fp4 ? f4::BROWS : (pair ? BM : BN))) return rc;
  GemmParams prm;
  prm.C = C;
  prm.m = m;
  prm.pc = lo.pc;
  prm.ksteps = int(lo.row / BK);
  prm.mblocks = int(cdiv(m, rows));
  prm.nblocks = int(fp4 ? cdiv(lo.npad, f4::NB) : lo.npad / (wide ? 2 * BN : BN));
  const int64_t tiles = int64_t(prm.mblocks) * prm.nblocks;
  if (tiles >= (int64_t(1) << 31)) return FQ_ENOTSUP;
  prm.tiles = int(tiles);
  prm.plane = plane;
  prm.small = lo.small;
  prm.err = err;
  prm.group = to.group > 0 ? to.group : (fp4 ? GROUP_M4 : GROUP_M);
  int dev = 0, sms = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  FQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (pair) {
    const int64_t pairs = sms / 2 > 0 ? sms / 2 : 1;
    const int grid = 2 * int(tiles < pairs ? tiles : pairs);
    if (fp4) {
      FQ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm4_kernel<Q, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, f4::SMEM));
      tc_gemm4_kernel<Q, P><<<grid, f4::THREADS, f4::SMEM, s>>>(ma, mb, prm);
    } else if (wide) {
      FQ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm2_kernel<Q, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PairGeo<true>::SMEM));
      tc_gemm2_kernel<Q, P, true><<<grid, PairGeo<true>::THREADS, PairGeo<true>::SMEM, s>>>(ma, mb, prm);
    } else {
      FQ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm2_kernel<Q, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PairGeo<false>::SMEM));
      tc_gemm2_kernel<Q, P, false><<<grid, PairGeo<false>::THREADS, PairGeo<false>::SMEM, s>>>(ma, mb, prm);
    }
  } else {
    FQ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<Q, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    const int grid = int(tiles < sms ? tiles : sms);
    tc_gemm_kernel<Q, P><<<grid, THREADS, SMEM, s>>>(ma, mb, prm);
  }
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

// B^T (npad x ld bytes from offset off) from B's planes, k < kcols.
template <int Q, int P>
void transpose_to(const uint64_t *B, int64_t l, int64_t pitch, int64_t npad, uint8_t *out, int64_t ld, int64_t off,
                  int64_t kcols, int sel, cudaStream_t s) {
  const dim3 grid(unsigned(cdiv(kcols, TK)), unsigned(npad / TJ));
  planes_to_e4m3_t<Q, P><<<grid, 256, 0, s>>>(B, l, pitch, out, ld, off, kcols, sel);
}

template <int Q, int P>
int prepare(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint8_t *ws, int form,
            cudaStream_t s) {
  const Layout lo = layout_for(Q, m, l, n, form);
  if (lo.npad / TJ > 65535) return FQ_ENOTSUP;
  const int64_t pa = fq_pitch_words(l);
  int dev = 0, sms = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  FQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // GF(4): the operands of X, Y, Z are A0, A1, A0 + A1 and B0, B1, B0 + B1 (sel 0, 1, 2)
  for (int r = 0; r < lo.rounds; ++r) {
    uint8_t *a = ws + r * (lo.a_bytes + lo.b_bytes), *b = a + lo.a_bytes;
    if (lo.fp4) {
      const int per_a = Fp4Occupancy<Q, P>::rows(), per_b = Fp4Occupancy<Q, P>::transpose();
      rows_to_fp4<Q, P><<<rows_grid4(m, lo.la, sms, per_a), 256, 0, s>>>(A, m, lo.la, pa, a, lo.row, r);
      const int64_t kblocks = lo.la / TK4, blocks = kblocks * (lo.npad / TJ4);
      const int64_t grid = blocks < int64_t(sms) * per_b ? blocks : int64_t(sms) * per_b;
      planes_to_fp4_t<Q, P><<<unsigned(grid), 256, 0, s>>>(B, l, lo.pc, b, lo.row, r, kblocks, blocks);
    } else {
      rows_to_e4m3<Q, P><<<rows_grid(m, lo.la), 256, 0, s>>>(A, m, lo.la, pa, a, lo.la, 0, r);
      transpose_to<Q, P>(B, l, lo.pc, lo.npad, b, lo.la, 0, lo.la, r, s);
    }
  }
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

template <int Q, int P>
int multiply(int64_t m, int64_t l, int64_t n, const uint8_t *ws, uint64_t *C, int form, const TcOptions &to,
             cudaStream_t s) {
  const Layout lo = layout_for(Q, m, l, n, form);
  // GF(4): X into both planes, then Y added into plane 0 and Z into plane 1
  const int plane[3] = {-1, 0, 1};
  for (int r = 0; r < lo.rounds; ++r) {
    const uint8_t *a = ws + r * (lo.a_bytes + lo.b_bytes), *b = a + lo.a_bytes;
    if (int rc = gemm<Q, P>(a, b, C, m, lo, form, plane[r], to, s)) return rc;
  }
  return FQ_OK;
}

template <int Q, int P>
int batched(const TcBatch &b, const uint64_t *const *A, const uint64_t *const *B, uint64_t *const *C,
            cudaStream_t s) {
  if (b.nprod == 0) return FQ_OK;
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  CUtensorMap ma;  // 128-row blocks of 128 bytes: A's and B's alike
  if (int rc = make_map(&ma, b.scratch, BK, b.scratch_rows, BM)) return rc;
  BatchParams prm;
  prm.prods = b.prods;
  prm.cta_begin = b.cta_begin;
  prm.cta_list = b.cta_list;
  prm.cta_rows = b.cta_rows;
  prm.scratch = b.scratch;
  prm.A = A;
  prm.B = B;
  prm.C = C;
  prm.err = err;
  FQ_CUDA_TRY(cudaFuncSetAttribute(tc_batched_kernel<Q, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_F));
  tc_batched_kernel<Q, P><<<kTcCtas, THREADS_F, SMEM_F, s>>>(ma, prm);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

}  // namespace tc

// Largest l for which every partial sum stays below 2^24 in magnitude.
int64_t tc_max_l(int q) {
  const int64_t b = q == 2 || q == 4 ? 1 : (q - 1) / 2;
  return ((int64_t(1) << 24) - 1) / (b * b);
}

// Modelled time (SM cycles), fitted on GB300.  e4m3 forms: the busiest CTA's
// tiles (ceil(tiles / SMs) of 128 x 256, one persistent CTA per SM) times
// 128-deep k-steps at about 760 cycles each.  fp4 form: the busiest pair's
// 256 x 448 tiles, each 256-deep k-step about 1120 cycles plus about 6000 for
// the tile's epilogue.  Per product (GF(4) runs three), plus the operand
// conversion's bytes at about 2.8 TB/s (1.7 TB/s for the three-plane fields)
// and about 30 us of launches and set-up.
double tc_estimate(int q, int64_t m, int64_t l, int64_t n, int sms) {
  const int form = tc::form_for(m, l, TcOptions());
  const tc::Layout lo = tc::layout_for(q, m, l, n, form);
  const int64_t units = sms > 0 ? sms : 1;
  double gemm;
  if (lo.fp4) {
    const int64_t tiles = cdiv(lo.npad, tc::f4::NB) * cdiv(m, 2 * tc::BM);
    const int64_t pairs = units / 2 > 0 ? units / 2 : 1;
    gemm = double(cdiv(tiles, pairs)) * (double(lo.row / tc::BK) * 1120.0 + 6000.0);
  } else {
    const int64_t tiles = (lo.npad / tc::BN) * cdiv(m, tc::BM);
    gemm = double(cdiv(tiles, units)) * double(lo.la / tc::BK) * 760.0;
  }
  const double bytes = double(lo.rounds) * double(lo.a_bytes + lo.b_bytes);
  const double rate = (q == 5 || q == 7) ? 1.7e12 : 2.8e12;
  return double(lo.rounds) * gemm + bytes * 2.07e9 / rate + 62000.0;
}

int tc_form(int64_t m, int64_t l) { return tc::form_for(m, l, TcOptions()); }

int64_t tc_workspace_bytes(int q, int64_t m, int64_t l, int64_t n, const TcOptions &to) {
  if (!(q == 2 || q == 3 || q == 4 || q == 5 || q == 7) || m < 0 || l < 0 || n < 0 || l > tc_max_l(q)) return -1;
  const tc::Layout lo = tc::layout_for(q, m, l, n, tc::form_for(m, l, to));
  return int64_t(lo.rounds) * (lo.a_bytes + lo.b_bytes);
}

int tc_prepare(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, void *ws,
               cudaStream_t s, const TcOptions &to) {
  if (l == 0 || m == 0 || n == 0) return FQ_OK;
  uint8_t *w = static_cast<uint8_t *>(ws);
  const int form = tc::form_for(m, l, to);
  switch (q) {
    case 2: return tc::prepare<2, 1>(m, l, n, A, B, w, form, s);
    case 3: return tc::prepare<3, 2>(m, l, n, A, B, w, form, s);
    case 4: return tc::prepare<4, 2>(m, l, n, A, B, w, form, s);
    case 5: return tc::prepare<5, 3>(m, l, n, A, B, w, form, s);
    case 7: return tc::prepare<7, 3>(m, l, n, A, B, w, form, s);
    default: return FQ_EINVAL;
  }
}

int tc_multiply(int q, int64_t m, int64_t l, int64_t n, const void *ws, uint64_t *C, cudaStream_t s,
                const TcOptions &to) {
  if (m == 0 || n == 0) return FQ_OK;
  if (l == 0) {
    FQ_CUDA_TRY(cudaMemsetAsync(C, 0, size_t(fq_planes(q)) * size_t(m) * size_t(fq_pitch_words(n)) * 8u, s));
    return FQ_OK;
  }
  const uint8_t *w = static_cast<const uint8_t *>(ws);
  const int form = tc::form_for(m, l, to);
  switch (q) {
    case 2: return tc::multiply<2, 1>(m, l, n, w, C, form, to, s);
    case 3: return tc::multiply<3, 2>(m, l, n, w, C, form, to, s);
    case 4: return tc::multiply<4, 2>(m, l, n, w, C, form, to, s);
    case 5: return tc::multiply<5, 3>(m, l, n, w, C, form, to, s);
    case 7: return tc::multiply<7, 3>(m, l, n, w, C, form, to, s);
    default: return FQ_EINVAL;
  }
}

int launch_tc(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
              cudaStream_t s, const TcOptions &to) {
  const int64_t bytes = tc_workspace_bytes(q, m, l, n, to);
  if (bytes < 0) return FQ_ENOTSUP;
  if (l == 0) return tc_multiply(q, m, l, n, nullptr, C, s, to);
  void *mem = nullptr;
  if (int rc = scratch_alloc(&mem, size_t(bytes), s)) return rc;
  int rc = tc_prepare(q, m, l, n, A, B, mem, s, to);
  if (rc == FQ_OK) rc = tc_multiply(q, m, l, n, mem, C, s, to);
  const int fr = scratch_free(mem, s);
  return rc ? rc : fr;
}

int tc_batched(const TcBatch &b, const uint64_t *const *A, const uint64_t *const *B, uint64_t *const *C,
               cudaStream_t s) {
  if (b.scratch_rows >= (int64_t(1) << 31)) return FQ_ENOTSUP;
  switch (b.q) {
    case 3: return tc::batched<3, 2>(b, A, B, C, s);
    case 5: return tc::batched<5, 3>(b, A, B, C, s);
    case 7: return tc::batched<7, 3>(b, A, B, C, s);
    default: return FQ_EINVAL;
  }
}

}  // namespace fqk

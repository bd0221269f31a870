// Residue <-> code-bit conversions, four elements (bytes of a 32-bit word) at a
// time, shared by fq_pack/fq_unpack and the tensor-core path's epilogue.
// Codes: Section 4.1 (F_3), 4.2 (F_5, F_7), 4.3 (GF(4)); F_2 is one bit.
#pragma once

#include "fq_common.cuh"

namespace fqk {

constexpr uint32_t kLsb = 0x01010101u;

// Gathers bit 0 of each byte of x (bits 0, 8, 16, 24) into bits 0..3.  The
// partial products of x * 0x204081 land on distinct bit positions, so bits
// 21..24 are exactly those four bits.
__device__ __forceinline__ uint32_t gather_nibble(uint32_t x) { return ((x * 0x204081u) >> 21) & 0xFu; }

// Inverse: bits 0..3 of n spread to bit 0 of each byte.
__device__ __forceinline__ uint32_t spread_nibble(uint32_t n) { return (n * 0x204081u) & kLsb; }

// Encodes 4 residues (bytes of v, element e at byte 0) into the plane words.
template <int Q, int P>
__device__ __forceinline__ void encode4(uint32_t v, uint64_t (&out)[P], int e, uint32_t &bad) {
  // bytes >= Q: bit 7 of the byte set in m
  const uint32_t m = (v & 0x80808080u) | (((v | 0x80808080u) - uint32_t(Q) * kLsb) & 0x80808080u);
  bad |= m;
  v &= ~((m >> 7) * 0xFFu);  // invalid residues are stored as 0
  if constexpr (Q == 3) {
    const uint32_t unit = (v | (v >> 1)) & kLsb;
    const uint32_t sign = (v >> 1) & kLsb;
    out[0] |= uint64_t(gather_nibble(unit)) << e;
    out[1] |= uint64_t(gather_nibble(sign)) << e;
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) out[p] |= uint64_t(gather_nibble((v >> p) & kLsb)) << e;
  }
}

// Residues of 4 elements (bytes) from the four code bits starting at element e.
template <int Q, int P>
__device__ __forceinline__ uint32_t decode4(const uint64_t (&in)[P], int e) {
  uint32_t x[P];
#pragma unroll
  for (int p = 0; p < P; ++p) x[p] = spread_nibble(uint32_t(in[p] >> e) & 0xFu);
  if constexpr (Q == 2) {
    return x[0];
  } else if constexpr (Q == 3) {
    return x[0] + (x[0] & x[1]);                    // (1,0) -> 1, (1,1) -> 2
  } else if constexpr (Q == 4) {
    return x[0] | (x[1] << 1);                      // a0 + 2 a1
  } else {
    const uint32_t code = x[0] | (x[1] << 1) | (x[2] << 2);
    if constexpr (Q == 7) {
      const uint32_t seven = ((code + kLsb) >> 3) & kLsb;      // code == 7
      return code - 7u * seven;
    } else {
      const uint32_t ge5 = ((code + 3u * kLsb) >> 3) & kLsb;   // code >= 5
      return code - 5u * ge5;
    }
  }
}

}  // namespace fqk

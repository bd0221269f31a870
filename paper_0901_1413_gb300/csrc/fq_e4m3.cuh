// Plane words to e4m3 bytes, 16 or 32 elements at a time, for the tensor-core
// operands of the F_3, F_5 and F_7 products (and of F_2 products, such as the
// three of GF(4)).  Host and device: the host build is what the CPU tests
// check byte for byte against the e4m3 format.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fqk {

// Byte j (0..3) of x, zero-extended.
__host__ __device__ __forceinline__ uint32_t byte_of(uint32_t x, int j) {
#ifdef __CUDA_ARCH__
  return __byte_perm(x, 0u, 0x4440u | uint32_t(j));
#else
  return (x >> (8 * j)) & 0xFFu;
#endif
}

// Elements 0 .. 4 G - 1 of one 32-bit word per plane (element i at bit i) as
// e4m3 bytes, four to an output word (element 4 g + i in byte i of w[g]).
// The codes are first sorted into magnitude classes bitsliced, for all the
// elements at once (F_5: |v| = 1, |v| = 2; F_7: |v| = 1, |v| >= 2, |v| = 3;
// and the sign), each class plane is split into its even and odd nibbles, and
// then every four elements take one nibble of each class, spread to the
// bytes' low bits by a multiply (the four shifted copies of a nibble by 1 +
// 2^7 + 2^14 + 2^21 cannot overlap), and masked into the byte value: 1 ->
// 0x38, 2 -> 0x40, 3 -> 0x44, the sign 0x80.  Q = 2: one plane, 1 -> 0x38.
template <int Q, int P, int G>
__host__ __device__ __forceinline__ void e4m3_groups(const uint32_t (&t)[P], uint32_t (&w)[G]) {
  static_assert(Q == 2 || Q == 3 || Q == 5 || Q == 7, "F_2 (one plane), F_3, F_5, F_7");
  constexpr int NC = Q == 2 ? 1 : (Q == 3 ? 2 : (Q == 5 ? 3 : 4));  // class planes: unit class first, sign last
  uint32_t cls[NC];
  if constexpr (Q == 2) {
    cls[0] = t[0];
  } else if constexpr (Q == 3) {
    cls[0] = t[0];  // unit (code 2, a sign without the unit, gives -0)
    cls[1] = t[1];  // sign
  } else {
    const uint32_t c0 = t[0], c1 = t[1], c2 = t[2];  // code = c0 + 2 c1 + 4 c2, read mod p
    if constexpr (Q == 5) {
      cls[0] = (~c2 & ~c1 & c0) | (c2 & ~c1 & ~c0) | (c2 & c1 & ~c0);  // codes 1, 4, 6: |v| = 1
      cls[1] = (~c2 & c1) | (c2 & c1 & c0);                            // codes 2, 3, 7: |v| = 2
      cls[2] = (~c2 & c1 & c0) | (c2 & ~c1 & ~c0);                     // codes 3, 4: negative
    } else {
      cls[0] = (~c2 & ~c1 & c0) | (c2 & c1 & ~c0);                     // codes 1, 6: |v| = 1
      cls[1] = (~c2 & c1) | (c2 & ~c1);                                // codes 2..5: |v| >= 2
      cls[2] = (~c2 & c1 & c0) | (c2 & ~c1 & ~c0);                     // codes 3, 4: |v| = 3
      cls[3] = (c2 & ~c1) | (c2 & c1 & ~c0);                           // codes 4, 5, 6: negative
    }
  }
  constexpr uint32_t kSpread = 0x204081u;
  uint32_t even[NC], odd[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    even[c] = cls[c] & 0x0F0F0F0Fu;
    odd[c] = (cls[c] >> 4) & 0x0F0F0F0Fu;
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {  // elements 4 g .. 4 g + 3: nibble g
    uint32_t n[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) n[c] = byte_of((g & 1) ? odd[c] : even[c], g >> 1);
    uint32_t v = ((n[0] * kSpread) & 0x01010101u) * 0x38u;             // |v| = 1
    if constexpr (Q == 5) v |= (n[1] * (kSpread << 6)) & 0x40404040u;  // |v| = 2
    if constexpr (Q == 7) {
      v |= (n[1] * (kSpread << 6)) & 0x40404040u;                      // |v| >= 2
      v |= (n[2] * (kSpread << 2)) & 0x04040404u;                      // |v| = 3
    }
    if constexpr (Q != 2) v |= (n[NC - 1] * (kSpread << 7)) & 0x80808080u;  // sign
    w[g] = v;
  }
}

// All 32 elements: 0..15 in lo, 16..31 in hi.
template <int Q, int P>
__host__ __device__ __forceinline__ void e4m3x32(const uint32_t (&t)[P], uint4 &lo, uint4 &hi) {
  uint32_t w[8];
  e4m3_groups<Q, P, 8>(t, w);
  lo = make_uint4(w[0], w[1], w[2], w[3]);
  hi = make_uint4(w[4], w[5], w[6], w[7]);
}

// Elements 16 half .. 16 half + 15 (half 0 or 1), for writers whose threads
// store 16 bytes each.
template <int Q, int P>
__host__ __device__ __forceinline__ uint4 e4m3x16(const uint32_t (&t)[P], int half) {
  uint32_t h[P], w[4];
#pragma unroll
  for (int p = 0; p < P; ++p) h[p] = t[p] >> (16 * half);
  e4m3_groups<Q, P, 4>(h, w);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace fqk

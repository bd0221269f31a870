// Bitsliced field arithmetic on 32-bit plane words (Sections 3-4 of Boothby &
// Bradshaw).  One call works on 32 elements: bit b of word p is bit p of the
// code of element b.
//
// Each field type gives P (planes), D (size of the additive basis, Section 2),
// AP (planes of the Four-Russians accumulator: P, or 4 for F_5), add / sub on
// one column word, `accumulate` (acc += sum_d alpha_d t_d, the Four-Russians
// inner step), `finish` (the accumulator to canonical codes), `canon`
// (canonical codes) and `phi` (the binary maps phi_d of Section 2 on 64-bit
// words of A's planes).
#pragma once

#include "fq_common.cuh"

namespace fqk {

// ------------------------------------------------------------------ F_2 ----
// One plane; the binary Four-Russians case of Section 2 (basis {1}, phi_0 = the
// element itself); addition is XOR.  The base field of GF(4) and F_8 in the
// matrix-level products of Section 4.3.
struct F2 {
  static constexpr int Q = 2, P = 1, D = 1, AP = P;
  __device__ __forceinline__ static void add(uint32_t (&x)[P], const uint32_t (&y)[P]) { x[0] ^= y[0]; }
  __device__ __forceinline__ static void sub(uint32_t (&x)[P], const uint32_t (&y)[P]) { x[0] ^= y[0]; }
  __device__ __forceinline__ static void accumulate(uint32_t (&acc)[P], const uint32_t (&t)[D][P]) {
    acc[0] ^= t[0][0];
  }
  __device__ __forceinline__ static void canon(uint32_t (&)[P]) {}
  __device__ __forceinline__ static void finish(const uint32_t (&acc)[AP], uint32_t (&x)[P]) { x[0] = acc[0]; }
  __device__ __forceinline__ static void phi(const uint64_t (&a)[P], uint64_t (&ph)[D]) { ph[0] = a[0]; }
};

// ------------------------------------------------------------------ F_3 ----
// Codes (x0, x1): 0 = (0,0), 1 = (1,0), -1 = (1,1) (Section 4.1); basis {1, -1},
// phi_0(a) = [a = 1], phi_1(a) = [a = -1].
struct F3 {
  static constexpr int Q = 3, P = 2, D = 2, AP = P;

  // x += y.  Section 4.1's six-gate add, with its outputs in the order that
  // makes it exact (x0 = unit, x1 = sign), fused into four LOP3s:
  //   u = x0 ^ y1, t = x1 ^ y0 ^ y1, x0' = (u ^ x1) | t, x1' = u & (x1 ^ y0).
  __device__ __forceinline__ static void add(uint32_t &x0, uint32_t &x1, uint32_t y0, uint32_t y1) {
    const uint32_t u = x0 ^ y1;
    const uint32_t t = lop3<0x96>(x1, y0, y1);
    const uint32_t r0 = lop3<0xBE>(u, x1, t);
    const uint32_t r1 = lop3<0x60>(u, x1, y0);
    x0 = r0;
    x1 = r1;
  }
  // x -= y: the add above applied to -y = (y0, y0 ^ y1) (Section 4.1 negation),
  // still four LOP3s.
  __device__ __forceinline__ static void sub(uint32_t &x0, uint32_t &x1, uint32_t y0, uint32_t y1) {
    const uint32_t u = lop3<0x96>(x0, y0, y1);
    const uint32_t t = x1 ^ y1;
    const uint32_t r0 = lop3<0xBE>(u, x1, t);
    const uint32_t r1 = lop3<0x60>(u, x1, y0);
    x0 = r0;
    x1 = r1;
  }
  __device__ __forceinline__ static void add(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    add(x[0], x[1], y[0], y[1]);
  }
  __device__ __forceinline__ static void sub(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    sub(x[0], x[1], y[0], y[1]);
  }
  // acc += 1 * t[0] + (-1) * t[1]
  __device__ __forceinline__ static void accumulate(uint32_t (&acc)[P], const uint32_t (&t)[D][P]) {
    add(acc[0], acc[1], t[0][0], t[0][1]);
    sub(acc[0], acc[1], t[1][0], t[1][1]);
  }
  __device__ __forceinline__ static void canon(uint32_t (&)[P]) {}
  __device__ __forceinline__ static void finish(const uint32_t (&acc)[AP], uint32_t (&x)[P]) {
    x[0] = acc[0];
    x[1] = acc[1];
  }
  __device__ __forceinline__ static void phi(const uint64_t (&a)[P], uint64_t (&ph)[D]) {
    ph[0] = a[0] & ~a[1];
    ph[1] = a[0] & a[1];
  }
};

// ---------------------------------------------------------------- GF(4) ----
// GF(4) = F_2[x]/(x^2+x+1), element a0 + alpha a1, codes (a0, a1) (Section 4.3);
// basis {1, alpha}, phi_d(a) = a_d; addition is XOR.
struct GF4 {
  static constexpr int Q = 4, P = 2, D = 2, AP = P;
  __device__ __forceinline__ static void add(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    x[0] ^= y[0];
    x[1] ^= y[1];
  }
  __device__ __forceinline__ static void sub(uint32_t (&x)[P], const uint32_t (&y)[P]) { add(x, y); }
  // acc += t[0] + alpha * t[1], alpha (b0 + alpha b1) = b1 + alpha (b0 + b1).
  __device__ __forceinline__ static void accumulate(uint32_t (&acc)[P], const uint32_t (&t)[D][P]) {
    acc[0] = lop3<0x96>(acc[0], t[0][0], t[1][1]);
    acc[1] = lop3<0x96>(acc[1], t[0][1], t[1][0]) ^ t[1][1];
  }
  __device__ __forceinline__ static void canon(uint32_t (&)[P]) {}
  __device__ __forceinline__ static void finish(const uint32_t (&acc)[AP], uint32_t (&x)[P]) {
    x[0] = acc[0];
    x[1] = acc[1];
  }
  __device__ __forceinline__ static void phi(const uint64_t (&a)[P], uint64_t (&ph)[D]) {
    ph[0] = a[0];
    ph[1] = a[1];
  }
};

// ------------------------------------------------------- F_5 and F_7 shared --
// Plain binary codes a2 a1 a0 read mod p, not unique (Section 4.2); basis {1,2,4}.

// Grade-school add of two 3-bit codes into s3 s2 s1 s0 (Section 4.2's `add`).
__device__ __forceinline__ void ripple3(const uint32_t (&x)[3], const uint32_t (&y)[3], uint32_t &s0,
                                        uint32_t &s1, uint32_t &s2, uint32_t &s3) {
  s0 = x[0] ^ y[0];
  const uint32_t c0 = x[0] & y[0];
  s1 = x[1] ^ y[1] ^ c0;
  const uint32_t c1 = (x[1] & y[1]) | (c0 & (x[1] ^ y[1]));
  s2 = x[2] ^ y[2] ^ c1;
  s3 = (x[2] & y[2]) | (c1 & (x[2] ^ y[2]));
}

// ------------------------------------------------------------------ F_7 ----
struct F7 {
  static constexpr int Q = 7, P = 3, D = 3, AP = P;
  // x += y: s = add(x, y); x = add(s2 s1 s0, s3) -- the carry out of bit 2 is the
  // unit bit mod 7 (Section 4.2); the second add never carries out.
  __device__ __forceinline__ static void add(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    uint32_t s0, s1, s2, s3;
    ripple3(x, y, s0, s1, s2, s3);
    const uint32_t d0 = s0 & s3;
    x[0] = s0 ^ s3;
    x[1] = s1 ^ d0;
    x[2] = s2 ^ (s1 & d0);
  }
  // x -= y: add the complement (negation is plane-wise NOT, Section 4.2).
  __device__ __forceinline__ static void sub(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    const uint32_t n[P] = {~y[0], ~y[1], ~y[2]};
    add(x, n);
  }
  // acc += t0 + 2 t1 + 4 t2.  Doubling is a rotation of the planes (Section
  // 4.2); because 8 = 1 mod 7 a carry-save adder works mod 7 too (its carry
  // vector rotates instead of shifting), so the four operands are compressed
  // to two with two carry-save adders and finished with one add.
  __device__ __forceinline__ static void csa(const uint32_t (&x)[P], const uint32_t (&y)[P], const uint32_t (&z)[P],
                                             uint32_t (&s)[P], uint32_t (&c)[P]) {
    uint32_t m[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      s[i] = lop3<0x96>(x[i], y[i], z[i]);
      m[i] = lop3<0xE8>(x[i], y[i], z[i]);
    }
    c[0] = m[2];  // carry out of bit 2 has weight 8 = 1 mod 7
    c[1] = m[0];
    c[2] = m[1];
  }
  __device__ __forceinline__ static void accumulate(uint32_t (&acc)[P], const uint32_t (&t)[D][P]) {
    const uint32_t d1[P] = {t[1][2], t[1][0], t[1][1]};
    const uint32_t d2[P] = {t[2][1], t[2][2], t[2][0]};
    uint32_t s1[P], c1[P], s2[P], c2[P];
    csa(t[0], d1, d2, s1, c1);
    csa(acc, s1, c1, s2, c2);
#pragma unroll
    for (int i = 0; i < P; ++i) acc[i] = s2[i];
    add(acc, c2);
  }
  // Canonical code: 7 (111) -> 0, others unchanged (Section 4.2's reduce with the
  // common term read as a0 & a1 & a2).
  __device__ __forceinline__ static void canon(uint32_t (&x)[P]) {
    const uint32_t c = x[0] & x[1] & x[2];
    x[0] ^= c;
    x[1] ^= c;
    x[2] ^= c;
  }
  __device__ __forceinline__ static void finish(const uint32_t (&acc)[AP], uint32_t (&x)[P]) {
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] = acc[p];
    canon(x);
  }
  __device__ __forceinline__ static void phi(const uint64_t (&a)[P], uint64_t (&ph)[D]) {
    const uint64_t c = a[0] & a[1] & a[2];
    ph[0] = a[0] ^ c;
    ph[1] = a[1] ^ c;
    ph[2] = a[2] ^ c;
  }
};

// ------------------------------------------------------------------ F_5 ----
struct F5 {
  // the accumulator is a four-bit value mod 15 (= 3 x 5), folded to a code once
  static constexpr int Q = 5, P = 3, D = 3, AP = 4;
  // fold5: the 4-bit s3 s2 s1 s0 folded to three bits with the same value mod 5
  // (Section 4.2, its eight-operation form).
  __device__ __forceinline__ static void fold5(uint32_t s0, uint32_t s1, uint32_t s2, uint32_t s3,
                                               uint32_t (&r)[P]) {
    const uint32_t t = s2 | s1;
    const uint32_t r2 = s0 ^ t;
    const uint32_t r1 = (r2 & s0) ^ (s3 ^ s1);
    r[0] = (t ^ s2) | (r1 & s3);
    r[1] = r1;
    r[2] = r2;
  }
  __device__ __forceinline__ static void add(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    uint32_t s0, s1, s2, s3;
    ripple3(x, y, s0, s1, s2, s3);
    fold5(s0, s1, s2, s3, x);
  }
  // 2x = fold5(x2 x1 x0 0)
  __device__ __forceinline__ static void dbl(const uint32_t (&x)[P], uint32_t (&r)[P]) {
    fold5(0u, x[0], x[1], x[2], r);
  }
  // -x = 4x = fold5(x1 x0 0 x2)
  __device__ __forceinline__ static void neg(const uint32_t (&x)[P], uint32_t (&r)[P]) {
    fold5(x[2], 0u, x[0], x[1], r);
  }
  __device__ __forceinline__ static void sub(uint32_t (&x)[P], const uint32_t (&y)[P]) {
    uint32_t n[P];
    neg(y, n);
    add(x, n);
  }
  // acc += t0 + 2 t1 + 4 t2 for a four-bit accumulator mod 15 = 3 * 5 (its
  // value mod 5 is the F_5 element).  Mod 15 (16 = 1) doubling a 4-bit number
  // rotates it and carry-save adders wrap their carry, as for F_7 mod 7:
  // 2 t1 = (0, t1_0, t1_1, t1_2) and 4 t2 = (t2_2, 0, t2_0, t2_1) as 4-bit
  // numbers.  Two carry-save adders take acc, t0, 2 t1, 4 t2 to two 4-bit
  // numbers and one end-around add to one (at most 15: u + w <= 30, so the
  // carry added back at bit 0 cannot carry out again).  No fold per step:
  // `finish` applies Section 4.2's fold5 once, when the product is stored.
  __device__ __forceinline__ static void accumulate(uint32_t (&acc)[AP], const uint32_t (&t)[D][P]) {
    // first carry-save adder on x = t0, y = 2 t1, z = 4 t2 (zero bits dropped)
    uint32_t s[4], m[4];
    s[0] = t[0][0] ^ t[2][2];
    m[0] = t[0][0] & t[2][2];
    s[1] = t[0][1] ^ t[1][0];
    m[1] = t[0][1] & t[1][0];
    s[2] = lop3<0x96>(t[0][2], t[1][1], t[2][0]);
    m[2] = lop3<0xE8>(t[0][2], t[1][1], t[2][0]);
    s[3] = t[1][2] ^ t[2][1];
    m[3] = t[1][2] & t[2][1];
    // carry vector rotated: weight 16 = 1 mod 15
    const uint32_t c[4] = {m[3], m[0], m[1], m[2]};
    // second carry-save adder with acc (4 bits)
    uint32_t u[4], v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      u[i] = lop3<0x96>(acc[i], s[i], c[i]);
      v[i] = lop3<0xE8>(acc[i], s[i], c[i]);
    }
    const uint32_t w[4] = {v[3], v[0], v[1], v[2]};
    // u + w mod 15: 4-bit add, then the carry out added back at bit 0
    uint32_t r[4];
    r[0] = u[0] ^ w[0];
    uint32_t k = u[0] & w[0];
#pragma unroll
    for (int i = 1; i < 4; ++i) {
      r[i] = lop3<0x96>(u[i], w[i], k);
      k = lop3<0xE8>(u[i], w[i], k);
    }
    const uint32_t a0 = r[0] & k;
    const uint32_t b0 = r[1] & a0;
    acc[0] = r[0] ^ k;
    acc[1] = r[1] ^ a0;
    acc[2] = r[2] ^ b0;
    acc[3] = r[3] ^ (r[2] & b0);
  }
  // The accumulator (mod 15) to a canonical F_5 code: fold5, then canon.
  __device__ __forceinline__ static void finish(const uint32_t (&acc)[AP], uint32_t (&x)[P]) {
    fold5(acc[0], acc[1], acc[2], acc[3], x);
    canon(x);
  }
  // Canonical code: 5, 6, 7 -> 0, 1, 2 (c marks codes >= 5).  Section 4.2's
  // printed reduce is not a reduction; this one is derived from the code table.
  __device__ __forceinline__ static void canon(uint32_t (&x)[P]) {
    const uint32_t c = x[2] & (x[0] | x[1]);
    const uint32_t r0 = (x[0] & ~c) | (c & x[1] & ~x[0]);
    const uint32_t r1 = x[1] & (~c | x[0]);
    const uint32_t r2 = x[2] & ~c;
    x[0] = r0;
    x[1] = r1;
    x[2] = r2;
  }
  __device__ __forceinline__ static void phi(const uint64_t (&a)[P], uint64_t (&ph)[D]) {
    const uint64_t c = a[2] & (a[0] | a[1]);
    ph[0] = (a[0] & ~c) | (c & a[1] & ~a[0]);
    ph[1] = a[1] & (~c | a[0]);
    ph[2] = a[2] & ~c;
  }
};

}  // namespace fqk

/*
 * Context baseline: the paper's own method, bitsliced Four Russians (Sections
 * 2-4 of Boothby & Bradshaw), on the host's CPU cores with 64-element words --
 * the setting of the paper's Table 1, run on this machine for comparison.
 *
 * NOT part of the product path: the GPU library never calls it (there is no
 * CPU fallback), and it shares no code with the CUDA kernels or the oracle.
 * Inputs and outputs are residue matrices (one uint8 per element, row-major);
 * packing to planes and unpacking are outside the timed multiplication.
 *
 * Codes (Section 4): F_2 one plane; F_3 (unit, sign) with 0 = 00, 1 = 10,
 * -1 = 11; F_5 and F_7 the binary digits of the residue (not unique after
 * additions); GF(4) = F_2[x]/(x^2 + x + 1) as (a0, a1).  Basis (Section 2):
 * F_3 {1, -1}; F_5, F_7 {1, 2, 4} combined by Horner's rule; GF(4) {1, x}.
 * Table of a k-row block: T[b] = sum_t b_t B_{sk+t}, each entry one add from
 * entry b & (b - 1).  OpenMP splits the rows of C; every thread builds its own
 * tables (no synchronisation inside the product).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t word;

/* ---- element formulas on 64-element words ------------------------------- */

/* F_3 add, Section 4.1 with its outputs in the order that makes it exact:
 * unit = s | t, sign = (x0 ^ y1) & (x1 ^ y0). */
static inline void f3_add(word *x0, word *x1, word y0, word y1) {
  const word s = *x0 ^ y1 ^ *x1, t = *x1 ^ y0 ^ y1;
  const word sign = (*x0 ^ y1) & (*x1 ^ y0);
  *x0 = s | t;
  *x1 = sign;
}
/* F_3 subtract, Section 4.1 as printed. */
static inline void f3_sub(word *x0, word *x1, word y0, word y1) {
  const word t = *x0 ^ y0;
  const word r0 = t | (*x1 ^ y1), r1 = (t ^ y1) & (y0 ^ *x1);
  *x0 = r0;
  *x1 = r1;
}
/* grade-school add of two 3-bit codes into four bits */
static inline void add3(const word *a, const word *b, word *s) {
  const word c0 = a[0] & b[0];
  s[0] = a[0] ^ b[0];
  const word c1 = (a[1] & b[1]) | (c0 & (a[1] ^ b[1]));
  s[1] = a[1] ^ b[1] ^ c0;
  s[2] = a[2] ^ b[2] ^ c1;
  s[3] = (a[2] & b[2]) | (c1 & (a[2] ^ b[2]));
}
/* F_7 (Section 4.2): the carry of the 3-bit add is the unit bit mod 7 */
static inline void f7_add(word *x, const word *y) {
  word s[4];
  add3(x, y, s);
  const word c0 = s[0] & s[3];
  x[0] = s[0] ^ s[3];
  const word c1 = s[1] & c0;
  x[1] = s[1] ^ c0;
  x[2] = s[2] ^ c1;
}
static inline void f7_dbl(word *x) {  /* a rotation of the planes */
  const word t = x[2];
  x[2] = x[1];
  x[1] = x[0];
  x[0] = t;
}
/* F_5 (Section 4.2): fold5, the eight-operation form */
static inline void fold5(word s0, word s1, word s2, word s3, word *r) {
  const word t = s2 | s1;
  const word r2 = s0 ^ t;
  const word r1 = (r2 & s0) ^ (s3 ^ s1);
  r[0] = (t ^ s2) | (r1 & s3);
  r[1] = r1;
  r[2] = r2;
}
static inline void f5_add(word *x, const word *y) {
  word s[4];
  add3(x, y, s);
  fold5(s[0], s[1], s[2], s[3], x);
}
static inline void f5_dbl(word *x) { fold5(0, x[0], x[1], x[2], x); }

/* ---- packing ------------------------------------------------------------- */

static int planes_of(int q) { return q == 2 ? 1 : (q == 3 || q == 4) ? 2 : 3; }

static void pack(int q, int64_t rows, int64_t cols, const uint8_t *R, word *out, int64_t W) {
  const int P = planes_of(q);
  memset(out, 0, (size_t)P * (size_t)rows * (size_t)W * sizeof(word));
  for (int64_t r = 0; r < rows; ++r)
    for (int64_t c = 0; c < cols; ++c) {
      const unsigned v = R[r * cols + c];
      unsigned code = v;
      if (q == 3) code = v == 0 ? 0u : (v == 1 ? 1u : 3u);
      for (int p = 0; p < P; ++p)
        if ((code >> p) & 1u) out[((int64_t)p * rows + r) * W + c / 64] |= (word)1 << (c % 64);
    }
}

static void unpack(int q, int64_t rows, int64_t cols, const word *in, int64_t W, uint8_t *R) {
  const int P = planes_of(q);
  for (int64_t r = 0; r < rows; ++r)
    for (int64_t c = 0; c < cols; ++c) {
      unsigned code = 0;
      for (int p = 0; p < P; ++p) code |= (unsigned)((in[((int64_t)p * rows + r) * W + c / 64] >> (c % 64)) & 1u) << p;
      unsigned v = code;
      if (q == 3) v = code == 0 ? 0u : (code == 1 ? 1u : 2u);
      else if (q == 5 || q == 7) v = code % (unsigned)q;
      R[r * cols + c] = (uint8_t)v;
    }
}

/* k bits of plane p of row i of A starting at column c0 (zero past l) */
static inline unsigned bits_at(const word *A, int64_t m, int64_t W, int p, int64_t i, int64_t c0, int k,
                               int64_t l) {
  const word *row = A + ((int64_t)p * m + i) * W;
  const int64_t w = c0 / 64;
  const int sh = (int)(c0 % 64);
  word v = row[w] >> sh;
  if (sh + k > 64 && w + 1 < W) v |= row[w + 1] << (64 - sh);
  int valid = (int)(l - c0 < k ? l - c0 : k);
  return (unsigned)(v & (((word)1 << valid) - 1));
}

/* the binary maps phi_d of Section 2 on one row's k-bit fields */
static void phi_indices(int q, const word *A, int64_t m, int64_t W, int64_t i, int64_t c0, int k, int64_t l,
                        unsigned *idx) {
  if (q == 3) {
    const unsigned u = bits_at(A, m, W, 0, i, c0, k, l), s = bits_at(A, m, W, 1, i, c0, k, l);
    idx[0] = u & ~s;  /* a = 1 */
    idx[1] = u & s;   /* a = -1 */
  } else {
    for (int p = 0; p < planes_of(q); ++p) idx[p] = bits_at(A, m, W, p, i, c0, k, l);
  }
}

static void add_rows(int q, word *x, const word *y, int64_t W) {
  /* x += y on one row of P planes (each W words, plane stride W) */
  switch (q) {
    case 2: for (int64_t w = 0; w < W; ++w) x[w] ^= y[w]; break;
    case 4: for (int64_t w = 0; w < 2 * W; ++w) x[w] ^= y[w]; break;
    case 3: for (int64_t w = 0; w < W; ++w) f3_add(&x[w], &x[W + w], y[w], y[W + w]); break;
    default:
      for (int64_t w = 0; w < W; ++w) {
        word a[3] = {x[w], x[W + w], x[2 * W + w]};
        const word b[3] = {y[w], y[W + w], y[2 * W + w]};
        if (q == 5) f5_add(a, b); else f7_add(a, b);
        x[w] = a[0];
        x[W + w] = a[1];
        x[2 * W + w] = a[2];
      }
  }
}

/* acc += sum_d alpha_d T[idx_d] on one row */
static void accumulate(int q, word *acc, const word *T, const unsigned *idx, int64_t W) {
  const int P = planes_of(q);
  const int64_t E = (int64_t)P * W;  /* words per table entry */
  switch (q) {
    case 2: {
      const word *t = T + idx[0] * E;
      for (int64_t w = 0; w < W; ++w) acc[w] ^= t[w];
      break;
    }
    case 3: {
      const word *t0 = T + idx[0] * E, *t1 = T + idx[1] * E;
      for (int64_t w = 0; w < W; ++w) {
        f3_add(&acc[w], &acc[W + w], t0[w], t0[W + w]);
        f3_sub(&acc[w], &acc[W + w], t1[w], t1[W + w]);
      }
      break;
    }
    case 4: {  /* acc += t0 + x t1, x (b0 + b1 x) = b1 + (b0 + b1) x */
      const word *t0 = T + idx[0] * E, *t1 = T + idx[1] * E;
      for (int64_t w = 0; w < W; ++w) {
        acc[w] ^= t0[w] ^ t1[W + w];
        acc[W + w] ^= t0[W + w] ^ t1[w] ^ t1[W + w];
      }
      break;
    }
    default: {  /* acc += t0 + 2 (t1 + 2 t2) by Horner's rule */
      const word *t0 = T + idx[0] * E, *t1 = T + idx[1] * E, *t2 = T + idx[2] * E;
      for (int64_t w = 0; w < W; ++w) {
        word h[3] = {t2[w], t2[W + w], t2[2 * W + w]};
        const word b1[3] = {t1[w], t1[W + w], t1[2 * W + w]};
        const word b0[3] = {t0[w], t0[W + w], t0[2 * W + w]};
        word a[3] = {acc[w], acc[W + w], acc[2 * W + w]};
        if (q == 5) {
          f5_dbl(h); f5_add(h, b1); f5_dbl(h); f5_add(h, b0); f5_add(a, h);
        } else {
          f7_dbl(h); f7_add(h, b1); f7_dbl(h); f7_add(h, b0); f7_add(a, h);
        }
        acc[w] = a[0];
        acc[W + w] = a[1];
        acc[2 * W + w] = a[2];
      }
    }
  }
}

static int threads_for(int threads) {
#ifdef _OPENMP
  return threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

/* C = A B on packed planes; returns 0, or 1 on bad arguments, 2 if out of memory */
static int m4rm(int q, int64_t m, int64_t l, const word *A, int64_t Wa, const word *B, word *C,
                int64_t W, int k, int threads) {
  const int P = planes_of(q);
  const int nt = threads_for(threads);
  int status = 0;
  memset(C, 0, (size_t)P * (size_t)m * (size_t)W * sizeof(word));
#pragma omp parallel num_threads(nt)
  {
    int me = 0, team = 1;
#ifdef _OPENMP
    me = omp_get_thread_num();
    team = omp_get_num_threads();
#endif
    const int64_t r0 = m * me / team, r1 = m * (me + 1) / team;
    const int64_t E = (int64_t)P * W;
    word *T = (word *)malloc(((size_t)1 << k) * (size_t)E * sizeof(word));
    word *acc = (word *)malloc((size_t)(r1 - r0 > 0 ? r1 - r0 : 1) * (size_t)E * sizeof(word));
    word *brow = (word *)malloc((size_t)E * sizeof(word));
    if (!T || !acc || !brow) {
#pragma omp atomic write
      status = 2;
    } else if (r1 > r0) {
      memset(acc, 0, (size_t)(r1 - r0) * (size_t)E * sizeof(word));
      for (int64_t c0 = 0; c0 < l; c0 += k) {
        /* table of block c0 .. c0 + k - 1 */
        memset(T, 0, (size_t)E * sizeof(word));
        for (unsigned b = 1; b < (1u << k); ++b) {
          const unsigned parent = b & (b - 1);
          const int t = __builtin_ctz(b);
          memcpy(T + (int64_t)b * E, T + (int64_t)parent * E, (size_t)E * sizeof(word));
          if (c0 + t < l) {
            for (int p = 0; p < P; ++p) memcpy(brow + (int64_t)p * W, B + ((int64_t)p * l + c0 + t) * W, (size_t)W * sizeof(word));
            add_rows(q, T + (int64_t)b * E, brow, W);
          }
        }
        for (int64_t i = r0; i < r1; ++i) {
          unsigned idx[3] = {0, 0, 0};
          phi_indices(q, A, m, Wa, i, c0, k, l, idx);
          accumulate(q, acc + (i - r0) * E, T, idx, W);
        }
      }
      for (int64_t i = r0; i < r1; ++i)
        for (int p = 0; p < P; ++p)
          memcpy(C + ((int64_t)p * m + i) * W, acc + (i - r0) * E + (int64_t)p * W, (size_t)W * sizeof(word));
    }
    free(T);
    free(acc);
    free(brow);
  }
  return status;
}

static double now_ms(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec * 1e3 + (double)ts.tv_nsec * 1e-6;
}

/* C = A B over field q (2, 3, 4, 5, 7) with block size k (1..12); residues in
 * and out.  *ms receives the time of the multiplication on packed planes
 * (packing excluded).  Returns 0, 1 for bad arguments, 2 if out of memory. */
int fq_cpu_m4rm(int q, int64_t m, int64_t l, int64_t n, const uint8_t *A, const uint8_t *B, uint8_t *C, int k,
                int threads, double *ms) {
  if (!(q == 2 || q == 3 || q == 4 || q == 5 || q == 7) || m < 0 || l < 0 || n < 0 || k < 1 || k > 12) return 1;
  if (m == 0 || n == 0) return 0;
  const int P = planes_of(q);
  const int64_t Wa = (l + 63) / 64 > 0 ? (l + 63) / 64 : 1, W = (n + 63) / 64;
  word *pa = (word *)calloc((size_t)P * (size_t)m * (size_t)Wa, sizeof(word));
  word *pb = (word *)calloc((size_t)P * (size_t)(l > 0 ? l : 1) * (size_t)W, sizeof(word));
  word *pc = (word *)calloc((size_t)P * (size_t)m * (size_t)W, sizeof(word));
  int status = 2;
  if (pa && pb && pc) {
    pack(q, m, l, A, pa, Wa);
    pack(q, l, n, B, pb, W);
    const double t0 = now_ms();
    status = m4rm(q, m, l, pa, Wa, pb, pc, W, k, threads);
    if (ms) *ms = now_ms() - t0;
    if (status == 0) unpack(q, m, n, pc, W, C);
  }
  free(pa);
  free(pb);
  free(pc);
  return status;
}

int fq_cpu_threads(int threads) { return threads_for(threads); }

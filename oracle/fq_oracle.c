/*
 * TEST INFRASTRUCTURE ONLY -- the CPU oracle for C = AB over F_p and GF(4).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code.  It shares nothing with the CUDA path: no headers, no helpers,
 * no tables.  Inputs and outputs are plain residue matrices (one uint8 per
 * element, row-major, leading dimensions in elements).
 *
 * What it computes is the plain definition of the product, written the way
 * Section 2 of Boothby & Bradshaw states it before any Four-Russians step:
 * row i of C is a linear combination of the rows of B with the coefficients of
 * row i of A,   C_i = A_i B = sum_{j<l} a_ij B_j   (Section 2, first display).
 *
 *  - F_p (p = 2, 3, 5, 7): every term a_ij * b_jt is an integer in [0, (p-1)^2];
 *    the row sum is accumulated exactly in int64 and reduced mod p once at the
 *    end, so the result is the product over the integers reduced mod p.
 *  - GF(4) = F_2[x]/(x^2 + x + 1) (Section 4.3): element code c = c0 + 2*c1 is
 *    the polynomial c0 + c1*x; a product is polynomial multiplication over F_2
 *    followed by the substitution x^2 = x + 1; addition is XOR of codes.
 *
 * Rows are independent, so an OpenMP loop over i is the only parallelism; it
 * changes no arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

static int set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) return threads;
  return omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

/* Number of threads the next call with this request will use. */
int fq_oracle_threads(int threads) { return set_threads(threads); }

/* C (m x n) = A (m x l) * B (l x n) over F_p, entries of A and B in [0, p). */
int fq_oracle_matmul_fp(int p, int64_t m, int64_t l, int64_t n,
                        const uint8_t *A, int64_t lda,
                        const uint8_t *B, int64_t ldb,
                        uint8_t *C, int64_t ldc, int threads) {
  if (p < 2 || m < 0 || l < 0 || n < 0) return ORACLE_EINVAL;
  if (m == 0 || n == 0) return ORACLE_OK;
  if (!A || !B || !C || lda < l || ldb < n || ldc < n) return ORACLE_EINVAL;
  int nt = set_threads(threads);
  int status = ORACLE_OK;
#pragma omp parallel num_threads(nt)
  {
    int64_t *acc = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!acc) {
#pragma omp atomic write
      status = ORACLE_ENOMEM;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
      if (!acc) continue;
      memset(acc, 0, (size_t)n * sizeof(int64_t));
      const uint8_t *Ai = A + i * lda;
      for (int64_t j = 0; j < l; ++j) {          /* C_i += a_ij * B_j */
        const int64_t a = Ai[j];
        const uint8_t *Bj = B + j * ldb;
        for (int64_t t = 0; t < n; ++t) acc[t] += a * (int64_t)Bj[t];
      }
      uint8_t *Ci = C + i * ldc;
      for (int64_t t = 0; t < n; ++t) Ci[t] = (uint8_t)(acc[t] % p);
    }
    free(acc);
  }
  return status;
}

/* Product of two GF(4) elements given as codes c0 + 2*c1 <-> c0 + c1*x. */
static unsigned gf4_mul(unsigned a, unsigned b) {
  const unsigned a0 = a & 1u, a1 = (a >> 1) & 1u;
  const unsigned b0 = b & 1u, b1 = (b >> 1) & 1u;
  /* (a0 + a1 x)(b0 + b1 x) = e0 + e1 x + e2 x^2 over F_2 */
  unsigned e0 = a0 & b0;
  unsigned e1 = (a0 & b1) ^ (a1 & b0);
  const unsigned e2 = a1 & b1;
  /* reduce modulo x^2 + x + 1:  x^2 = x + 1 */
  e0 ^= e2;
  e1 ^= e2;
  return e0 | (e1 << 1);
}

/* C = A * B over GF(4), entries are codes in [0, 4). */
int fq_oracle_matmul_gf4(int64_t m, int64_t l, int64_t n,
                         const uint8_t *A, int64_t lda,
                         const uint8_t *B, int64_t ldb,
                         uint8_t *C, int64_t ldc, int threads) {
  if (m < 0 || l < 0 || n < 0) return ORACLE_EINVAL;
  if (m == 0 || n == 0) return ORACLE_OK;
  if (!A || !B || !C || lda < l || ldb < n || ldc < n) return ORACLE_EINVAL;
  int nt = set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) {
    uint8_t *Ci = C + i * ldc;
    memset(Ci, 0, (size_t)n);
    const uint8_t *Ai = A + i * lda;
    for (int64_t j = 0; j < l; ++j) {            /* C_i += a_ij * B_j */
      const unsigned a = Ai[j] & 3u;
      const uint8_t *Bj = B + j * ldb;
      for (int64_t t = 0; t < n; ++t) Ci[t] ^= (uint8_t)gf4_mul(a, Bj[t] & 3u);
    }
  }
  return ORACLE_OK;
}

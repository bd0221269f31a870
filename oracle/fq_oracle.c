/*
 * TEST INFRASTRUCTURE ONLY -- the CPU oracle for C = AB over F_p, GF(4) and
 * the extension fields F_{p^n}.
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
 *  - F_{p^n} = F_p[x]/(f) for a monic f of degree n (Section 4.3, "non-prime
 *    fields"): element code c = sum_j c_j p^j is the polynomial sum_j c_j x^j.
 *    Addition is coefficientwise mod p; a product is schoolbook polynomial
 *    multiplication followed by the substitution x^n = r_0 + r_1 x + ... +
 *    r_{n-1} x^{n-1} (f = x^n - sum_j r_j x^j), highest degree first.  Both
 *    operations are tabulated once per call from that definition; the row
 *    combination then reads the tables.
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

/* Coefficients (base p digits) of an F_{p^n} code. */
static void ext_digits(int p, int n, unsigned c, int *d) {
  for (int j = 0; j < n; ++j) {
    d[j] = (int)(c % (unsigned)p);
    c /= (unsigned)p;
  }
}

static unsigned ext_code(int p, int n, const int *d) {
  unsigned c = 0;
  for (int j = n - 1; j >= 0; --j) c = c * (unsigned)p + (unsigned)d[j];
  return c;
}

/* a * b in F_p[x]/(x^n - sum_j r_j x^j): schoolbook product, then each x^k with
 * k >= n (highest first) replaced by x^(k-n) * sum_j r_j x^j. */
static unsigned ext_mul(int p, int n, const int *r, unsigned a, unsigned b) {
  int da[8], db[8];
  int64_t e[16];
  ext_digits(p, n, a, da);
  ext_digits(p, n, b, db);
  for (int k = 0; k < 2 * n - 1; ++k) e[k] = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) e[i + j] += (int64_t)da[i] * db[j];
  for (int k = 2 * n - 2; k >= n; --k) {
    for (int j = 0; j < n; ++j) e[k - n + j] += e[k] * r[j];
    e[k] = 0;
  }
  int d[8];
  for (int j = 0; j < n; ++j) d[j] = (int)(e[j] % p);
  return ext_code(p, n, d);
}

static unsigned ext_add(int p, int n, unsigned a, unsigned b) {
  int da[8], db[8], d[8];
  ext_digits(p, n, a, da);
  ext_digits(p, n, b, db);
  for (int j = 0; j < n; ++j) d[j] = (da[j] + db[j]) % p;
  return ext_code(p, n, d);
}

/* C = A * B over F_{p^n} with x^n = sum_j r[j] x^j, codes in [0, p^n) <= 255. */
int fq_oracle_matmul_ext(int p, int n, const int *r, int64_t m, int64_t l, int64_t nn,
                         const uint8_t *A, int64_t lda,
                         const uint8_t *B, int64_t ldb,
                         uint8_t *C, int64_t ldc, int threads) {
  if (p < 2 || n < 1 || n > 7 || !r || m < 0 || l < 0 || nn < 0) return ORACLE_EINVAL;
  int q = 1;
  for (int j = 0; j < n; ++j) q *= p;
  if (q > 256) return ORACLE_EINVAL;
  for (int j = 0; j < n; ++j)
    if (r[j] < 0 || r[j] >= p) return ORACLE_EINVAL;
  if (m == 0 || nn == 0) return ORACLE_OK;
  if (!A || !B || !C || lda < l || ldb < nn || ldc < nn) return ORACLE_EINVAL;
  uint8_t *mul = (uint8_t *)malloc((size_t)q * (size_t)q);
  uint8_t *add = (uint8_t *)malloc((size_t)q * (size_t)q);
  if (!mul || !add) {
    free(mul);
    free(add);
    return ORACLE_ENOMEM;
  }
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) {
      mul[a * q + b] = (uint8_t)ext_mul(p, n, r, (unsigned)a, (unsigned)b);
      add[a * q + b] = (uint8_t)ext_add(p, n, (unsigned)a, (unsigned)b);
    }
  int status = ORACLE_OK;
  for (int64_t i = 0; i < m && status == ORACLE_OK; ++i)
    for (int64_t j = 0; j < l; ++j)
      if (A[i * lda + j] >= q) status = ORACLE_EINVAL;
  for (int64_t j = 0; j < l && status == ORACLE_OK; ++j)
    for (int64_t t = 0; t < nn; ++t)
      if (B[j * ldb + t] >= q) status = ORACLE_EINVAL;
  if (status == ORACLE_OK) {
    int nt = set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t i = 0; i < m; ++i) {
      uint8_t *Ci = C + i * ldc;
      memset(Ci, 0, (size_t)nn);
      const uint8_t *Ai = A + i * lda;
      for (int64_t j = 0; j < l; ++j) {          /* C_i += a_ij * B_j */
        const uint8_t *mrow = mul + (size_t)Ai[j] * (size_t)q;
        const uint8_t *Bj = B + j * ldb;
        for (int64_t t = 0; t < nn; ++t) Ci[t] = add[(size_t)Ci[t] * (size_t)q + mrow[Bj[t]]];
      }
    }
  }
  free(mul);
  free(add);
  return status;
}

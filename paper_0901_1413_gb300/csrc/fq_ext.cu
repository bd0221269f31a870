// Products over extension fields F_{p^n} by Section 4.3's matrix-level method.
//
// A matrix over F_{p^n} = F_p[x]/(f) is stored as its coefficient matrices,
// A = A_0 + A_1 x + ... + A_{n-1} x^{n-1} with every A_j a packed F_p matrix
// (the planes of A_0, then those of A_1, ...).  The product's polynomial
// coefficients come from few base-field products:
//   n = 2 (Karatsuba):  c_0 = A_0 B_0, c_2 = A_1 B_1,
//                       c_1 = (A_0 + A_1)(B_0 + B_1) - c_0 - c_2;
//   n = 3 (the paper's trinomial formula, six products):
//     c_0 = A_0 B_0, c_4 = A_2 B_2,
//     c_1 = (A_0 + A_1)(B_0 + B_1) - A_0 B_0 - A_1 B_1,
//     c_2 = (A_0 + A_2)(B_0 + B_2) - A_0 B_0 - A_2 B_2 + A_1 B_1,
//     c_3 = (A_2 + A_1)(B_2 + B_1) - A_2 B_2 - A_1 B_1,
// and f = x^n - (r_0 + r_1 x + ...) folds c_k, k >= n, into the low
// coefficients.  Every output coefficient is thus a fixed F_p combination of
// the products, computed on the host once and applied by one bitsliced
// elementwise kernel.
//
// The base-field products are ordinary products (Four Russians or the
// tensor-core path, with Strassen-Winograd levels where they pay); the operand
// sums use the base field's bitsliced add.  The
// first n products (A_j B_j) are written straight into C's coefficient slots;
// the others, and the operand sums, live in stream-ordered scratch from the
// library's pool, released on the same stream.
#include "../../include/fq.h"
#include "fq_fields.cuh"
#include "fq_internal.h"

namespace fqk {

namespace {

// x^n = r_0 + r_1 x + ... + r_{n-1} x^{n-1}; every f is monic, irreducible and
// primitive.  GF(4) uses the paper's x^2 + x + 1.
const ExtField kExt[] = {
    {4, 2, 2, {1, 1, 0}},      // x^2 + x + 1
    {8, 2, 3, {1, 1, 0}},      // x^3 + x + 1
    {9, 3, 2, {1, 1, 0}},      // x^2 + 2x + 2
    {25, 5, 2, {3, 1, 0}},     // x^2 + 4x + 2
    {27, 3, 3, {2, 1, 0}},     // x^3 + 2x + 1
    {49, 7, 2, {4, 1, 0}},     // x^2 + 6x + 3
    {125, 5, 3, {2, 2, 0}},    // x^3 + 3x + 3
};

constexpr int kMaxProducts = 6;

// Products of the plan: the coefficient indices summed on each side.
struct Product {
  int a0, a1;  // A side: A_a0 (+ A_a1 when a1 >= 0)
};
const Product kQuadratic[3] = {{0, -1}, {1, -1}, {0, 1}};
const Product kCubic[6] = {{0, -1}, {1, -1}, {2, -1}, {0, 1}, {0, 2}, {1, 2}};

struct Weights {
  int w[3][kMaxProducts];  // output coefficient j = sum_k w[j][k] product_k (mod p)
};

// The combination weights of a field's products.
Weights plan_weights(const ExtField &f) {
  const int n = f.n, np = n == 2 ? 3 : 6;
  int c[5][kMaxProducts] = {};
  if (n == 2) {
    c[0][0] = 1;                                  // A0 B0
    c[2][1] = 1;                                  // A1 B1
    c[1][2] = 1, c[1][0] = -1, c[1][1] = -1;      // (A0 + A1)(B0 + B1) - A0 B0 - A1 B1
  } else {
    c[0][0] = 1;
    c[4][2] = 1;
    c[1][3] = 1, c[1][0] = -1, c[1][1] = -1;
    c[2][4] = 1, c[2][0] = -1, c[2][2] = -1, c[2][1] = 1;
    c[3][5] = 1, c[3][2] = -1, c[3][1] = -1;
  }
  for (int k = 2 * n - 2; k >= n; --k) {          // x^k = x^(k-n) (r_0 + r_1 x + ...)
    for (int j = 0; j < n; ++j)
      for (int t = 0; t < np; ++t) c[k - n + j][t] += f.r[j] * c[k][t];
    for (int t = 0; t < np; ++t) c[k][t] = 0;
  }
  Weights W = {};
  for (int j = 0; j < n; ++j)
    for (int t = 0; t < np; ++t) W.w[j][t] = ((c[j][t] % f.p) + f.p) % f.p;
  return W;
}

// acc += w * x for a small non-negative w (double and add).
template <class F>
__device__ __forceinline__ void add_multiple(uint32_t (&acc)[F::P], const uint32_t (&x)[F::P], int w) {
  uint32_t d[F::P];
#pragma unroll
  for (int p = 0; p < F::P; ++p) d[p] = x[p];
  while (w > 0) {
    if (w & 1) F::add(acc, d);
    w >>= 1;
    if (w > 0) F::add(d, d);
  }
}

// C_j = sum_k w[j][k] product_k, elementwise over `words` 64-bit words per plane.
// Products 0 .. N-1 sit in C's coefficient slots, the rest in T; every thread
// reads all of its word's inputs before it writes, so C is updated in place.
template <class F, int N, int NP>
__global__ void combine_kernel(int64_t words, uint64_t *C, const uint64_t *T, const Weights W) {
  constexpr int P = F::P;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < words;
       i += int64_t(gridDim.x) * blockDim.x) {
    uint32_t x[NP][2][P];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint64_t v = k < N ? C[(int64_t(k) * P + p) * words + i] : T[(int64_t(k - N) * P + p) * words + i];
        x[k][0][p] = uint32_t(v);
        x[k][1][p] = uint32_t(v >> 32);
      }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      uint32_t acc[2][P];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int p = 0; p < P; ++p) acc[h][p] = 0u;
#pragma unroll
        for (int k = 0; k < NP; ++k) add_multiple<F>(acc[h], x[k][h], W.w[j][k]);
        F::canon(acc[h]);
      }
#pragma unroll
      for (int p = 0; p < P; ++p)
        C[(int64_t(j) * P + p) * words + i] = uint64_t(acc[0][p]) | (uint64_t(acc[1][p]) << 32);
    }
  }
}

template <class F, int N>
int launch_combine(int64_t words, uint64_t *C, const uint64_t *T, const Weights &W, cudaStream_t s) {
  constexpr int NP = N == 2 ? 3 : 6;
  if (words == 0) return FQ_OK;
  const int th = 256;
  const int64_t want = cdiv(words, th), cap = 152 * 16;
  combine_kernel<F, N, NP><<<unsigned(want < cap ? want : cap), th, 0, s>>>(words, C, T, W);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

int combine(const ExtField &f, int64_t words, uint64_t *C, const uint64_t *T, const Weights &W, cudaStream_t s) {
  const bool quad = f.n == 2;
  switch (f.p) {
    case 2: return quad ? launch_combine<F2, 2>(words, C, T, W, s) : launch_combine<F2, 3>(words, C, T, W, s);
    case 3: return quad ? launch_combine<F3, 2>(words, C, T, W, s) : launch_combine<F3, 3>(words, C, T, W, s);
    case 5: return quad ? launch_combine<F5, 2>(words, C, T, W, s) : launch_combine<F5, 3>(words, C, T, W, s);
    case 7: return quad ? launch_combine<F7, 2>(words, C, T, W, s) : launch_combine<F7, 3>(words, C, T, W, s);
    default: return FQ_EINVAL;
  }
}

int base_planes(int p) { return p == 2 ? 1 : (p == 3 ? 2 : 3); }

int run(const ExtField &f, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
        uint64_t *ws, const ProdOptions &o, cudaStream_t s) {
  const int N = f.n, NP = N == 2 ? 3 : 6, PP = base_planes(f.p);
  const Product *prods = N == 2 ? kQuadratic : kCubic;
  const int64_t pa = fq_pitch_words(l), pc = fq_pitch_words(n);
  const int64_t a_words = PP * m * pa, b_words = PP * l * pc, c_words = PP * m * pc;
  // scratch: [sum products: A sum, B sum][products beyond the first N]
  uint64_t *T = ws + (NP - N) * (a_words + b_words);
  for (int k = 0; k < NP; ++k) {
    const Product &pr = prods[k];
    const uint64_t *a = A + pr.a0 * a_words, *b = B + pr.a0 * b_words;
    if (pr.a1 >= 0) {
      uint64_t *sa = ws + (k - N) * (a_words + b_words), *sb = sa + a_words;
      if (int rc = launch_add(f.p, m, l, A + pr.a0 * a_words, A + pr.a1 * a_words, sa, 0, s)) return rc;
      if (int rc = launch_add(f.p, l, n, B + pr.a0 * b_words, B + pr.a1 * b_words, sb, 0, s)) return rc;
      a = sa;
      b = sb;
    }
    uint64_t *dst = k < N ? C + k * c_words : T + (k - N) * c_words;
    if (int rc = product(f.p, m, l, n, a, b, dst, o, s)) return rc;
  }
  return combine(f, m * pc, C, T, plan_weights(f), s);
}

}  // namespace

const ExtField *ext_field(int q) {
  for (const ExtField &f : kExt)
    if (f.q == q) return &f;
  return nullptr;
}

int64_t ext_workspace_words(int q, int64_t m, int64_t l, int64_t n) {
  const ExtField *f = ext_field(q);
  if (!f) return -1;
  const int N = f->n, NP = N == 2 ? 3 : 6, PP = base_planes(f->p);
  const int64_t pa = fq_pitch_words(l), pc = fq_pitch_words(n);
  return (NP - N) * (PP * m * pa + PP * l * pc + PP * m * pc);
}

int launch_ext(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
               const ProdOptions &o, cudaStream_t s) {
  const ExtField *f = ext_field(q);
  if (!f) return FQ_EINVAL;
  const int64_t words = ext_workspace_words(q, m, l, n);
  void *ws = nullptr;
  if (int rc = scratch_alloc(&ws, size_t(words > 0 ? words : 1) * 8u, s)) return rc;
  ProdOptions base = o;
  if (base.path == FQ_PATH_KARATSUBA) base.path = FQ_PATH_AUTO;
  const int rc = run(*f, m, l, n, A, B, C, static_cast<uint64_t *>(ws), base, s);
  const int fr = scratch_free(ws, s);
  return rc ? rc : fr;
}

}  // namespace fqk

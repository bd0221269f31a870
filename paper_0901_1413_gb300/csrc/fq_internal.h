// Internal launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fqk {

int launch_pack(int q, int64_t rows, int64_t cols, const uint8_t *res, int64_t ld, uint64_t *planes,
                cudaStream_t s);
int launch_unpack(int q, int64_t rows, int64_t cols, const uint64_t *planes, uint8_t *res, int64_t ld,
                  cudaStream_t s);
int launch_add(int q, int64_t rows, int64_t cols, const uint64_t *X, const uint64_t *Y, uint64_t *Z, int sub,
               cudaStream_t s);
// Canonical codes in place (F_5, F_7; a no-op for the other fields).
int launch_canon(int q, int64_t rows, int64_t cols, uint64_t *Z, cudaStream_t s);
int launch_m4rm(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                int k, int variant, int kernel, cudaStream_t s);

int launch_mma(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
               int64_t chunk, cudaStream_t s);
// The tcgen05 form of the tensor-core path (fq_tc.cu): FQ_ENOTSUP when l is
// beyond the exact fp32 range of the field (tc_max_l).
struct TcOptions {
  int form = 0;   // 0: by shape; 2: single SMs; 3: SM pairs, 256-column tiles; 4: SM pairs, 512-column tiles
                  // (these three from e4m3 operands); 5: SM pairs, 448-column tiles from packed e2m1 (fp4)
  int group = 0;  // row blocks per group of the tile order (0: 8)
};
int launch_tc(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
              cudaStream_t s, const TcOptions &to = TcOptions());
int64_t tc_max_l(int q);
// Its two stages on a caller's workspace (bytes: tc_workspace_bytes, -1 if
// the product is outside the tcgen05 form): operands to e4m3 or packed e2m1
// (by the form, which both stages must be given alike), then the product.
int64_t tc_workspace_bytes(int q, int64_t m, int64_t l, int64_t n, const TcOptions &to = TcOptions());
int tc_prepare(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, void *ws,
               cudaStream_t s, const TcOptions &to = TcOptions());
int tc_multiply(int q, int64_t m, int64_t l, int64_t n, const void *ws, uint64_t *C, cudaStream_t s,
                const TcOptions &to = TcOptions());
double tc_estimate(int q, int64_t m, int64_t l, int64_t n, int sms);
// The tcgen05 product form a shape takes by default (2 .. 5, as TcOptions::form).
int tc_form(int64_t m, int64_t l);

// Batched products on the tcgen05 path.  The kTcCtas persistent CTAs work in
// groups of kTcGroup (one thread-block cluster), and the plan gives every
// product to one group (longest first, each to the least-loaded group).  A
// group works through its products in turn: its converter warps (of all its
// CTAs) write a product's A and B as e4m3 bytes into one of the group's two
// scratch buffers (K-blocked rows of 128 bytes: a 128-row block of A, or a
// 128-column block of B, holds its 128-deep k-slices one after another) while
// its TMA, MMA and epilogue warps compute the previous product's 128 x 256
// tiles from the other, CTA r of the group taking tiles r, r + kTcGroup, ...
constexpr int kTcCtas = 152;
constexpr int kTcGroup = 2;
constexpr int kTcGroups = kTcCtas / kTcGroup;
static_assert(kTcCtas % kTcGroup == 0, "whole groups");
struct BatchProd {
  int32_t p;              // index into the caller's pointer arrays
  int32_t m, l, n;
  int32_t la;             // l rounded up to 128 (bytes of an arena row used)
  int32_t nr;             // n rounded up to 256 (B^T rows reserved)
  int64_t pa, pb, pc;     // pitch words of A, B, C
  int64_t a_row0, b_row0; // unused (kept for the record layout)
};
struct TcBatch {
  int q = 0;
  int nprod = 0;
  int64_t scratch_rows = 0;            // rows of 128 bytes of all groups' buffers together
  const BatchProd *prods = nullptr;    // device
  const int32_t *cta_begin = nullptr;  // device, kTcGroups + 1: products of group g are cta_list[begin[g] .. begin[g+1])
  const int32_t *cta_list = nullptr;   // device, nprod product indices, each group's in the order it computes them
  const int64_t *cta_rows = nullptr;   // device, kTcGroups x 2: first scratch row of each group's buffers 0 and 1
  uint8_t *scratch = nullptr;          // device, scratch_rows x 128 bytes (1024-byte aligned)
};
// Rows of 128 bytes a product's operands take in a scratch buffer: A, then B^T.
__host__ __device__ inline int64_t batch_a_rows(int m, int la) { return int64_t((m + 127) / 128) * la; }
__host__ __device__ inline int64_t batch_bt_rows(int nr, int la) { return int64_t(nr) * (la / 128); }
int tc_batched(const TcBatch &b, const uint64_t *const *A, const uint64_t *const *B, uint64_t *const *C,
               cudaStream_t s);

// One compiled M4RM kernel shape of a field (the planner's candidates).
struct Variant {
  int k, rs;
  int (*launch)(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, cudaStream_t);
  int rows_per_slot;
  int cols, warps;
};
// The variant table of field q (nullptr and 0 for a bad q).
const Variant *m4rm_variants(int q, int *count);
// The variant index the M4RM planner picks for a product (-1 if none).
int m4rm_planned(int q, int64_t m, int64_t l, int64_t n, int k, int mt, int sms);

// Modelled times (SM cycles) of the two paths for a product, for the
// FQ_PATH_AUTO choice when no measured choice exists.
double m4rm_estimate(int q, int64_t m, int64_t l, int64_t n, int sms);
double mma_estimate(int q, int64_t m, int64_t l, int64_t n, int sms);

// Extension fields F_{p^n} = F_p[x]/(f), f = x^n - (r_0 + r_1 x + r_2 x^2)
// (fq_ext.cu): the field of code size q, or nullptr.
struct ExtField {
  int q, p, n;
  int r[3];
};
const ExtField *ext_field(int q);
// Stream-ordered scratch from the library's per-device pool (fq_api.cu).
int scratch_alloc(void **p, size_t bytes, cudaStream_t s);
int scratch_free(void *p, cudaStream_t s);

// Options of one product (fq_options without the ABI padding).
struct ProdOptions {
  int path, k, variant, kernel;
  int64_t chunk;
  int strassen;  // 0 = time model, -1 = never, L > 0 = exactly L levels where the shape allows
};
int64_t ext_workspace_words(int q, int64_t m, int64_t l, int64_t n);
int launch_ext(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
               const ProdOptions &o, cudaStream_t s);

// C = A B over field q by the options (fq_strassen.cu): the matrix-level
// products of an extension field, Strassen-Winograd levels over a base field,
// then the Four-Russians or tensor-core kernels.
int product(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
            const ProdOptions &o, cudaStream_t s);
// Strassen-Winograd levels `product` takes for a base-field product.
int strassen_levels(int q, int64_t m, int64_t l, int64_t n, const ProdOptions &o, int sms);

// The autotuned (path, kernel) for a shape, if fq_autotune measured one.
bool tuned_choice(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel);

}  // namespace fqk

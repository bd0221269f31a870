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
int launch_m4rm(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                int k, int variant, int kernel, cudaStream_t s);

int launch_mma(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
               int64_t chunk, cudaStream_t s);

// One compiled M4RM kernel shape of a field (the planner's candidates).
struct Variant {
  int k, rs;
  int (*launch)(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, cudaStream_t);
  int rows_per_slot;
  int cols, warps;
};
// The variant table of field q (nullptr and 0 for a bad q).
const Variant *m4rm_variants(int q, int *count);

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
// Base-product options of an extension-field product.
struct ExtOptions {
  int path, k, variant, kernel;
  int64_t chunk;
};
int64_t ext_workspace_words(int q, int64_t m, int64_t l, int64_t n);
int launch_ext(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
               const ExtOptions &o, cudaStream_t s);

// The autotuned (path, kernel) for a shape, if fq_autotune measured one.
bool tuned_choice(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel);

}  // namespace fqk

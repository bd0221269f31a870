// fq_matmul's M4RM path: dispatch by field to the planner of each field's
// compiled kernel variants.
#include "fq_internal.h"
#include "../../include/fq.h"

namespace fqk {

int launch_m4rm_f3(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, int, cudaStream_t);
int launch_m4rm_gf4(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, int,
                    cudaStream_t);
int launch_m4rm_f5(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, int, cudaStream_t);
int launch_m4rm_f7(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, int, cudaStream_t);

int launch_m4rm(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k,
                int variant, cudaStream_t s) {
  // variant > 0 forces the rows per CTA (tests and tuning)
  switch (q) {
    case 3: return launch_m4rm_f3(m, l, n, A, B, C, k, variant, s);
    case 4: return launch_m4rm_gf4(m, l, n, A, B, C, k, variant, s);
    case 5: return launch_m4rm_f5(m, l, n, A, B, C, k, variant, s);
    case 7: return launch_m4rm_f7(m, l, n, A, B, C, k, variant, s);
    default: return FQ_EINVAL;
  }
}

}  // namespace fqk

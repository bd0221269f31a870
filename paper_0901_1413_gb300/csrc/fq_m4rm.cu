// fq_matmul's M4RM path: dispatch by field to the planner over each field's
// compiled kernel variants.
#include "../../include/fq.h"
#include "fq_internal.h"
#include "fq_m4rm.cuh"

namespace fqk {

#define FQ_FIELD_DECL(name)                                                                                   \
  int launch_m4rm_##name(int64_t, int64_t, int64_t, const uint64_t *, const uint64_t *, uint64_t *, int, int, \
                         int, cudaStream_t);                                                                  \
  const Variant *m4rm_variants_##name(int *count);
FQ_FIELD_DECL(f2)
FQ_FIELD_DECL(f3)
FQ_FIELD_DECL(gf4)
FQ_FIELD_DECL(f5)
FQ_FIELD_DECL(f7)
#undef FQ_FIELD_DECL

int launch_m4rm(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k,
                int variant, int kernel, cudaStream_t s) {
  // variant > 0 forces the rows per CTA, kernel > 0 the compiled kernel
  switch (q) {
    case 2: return launch_m4rm_f2(m, l, n, A, B, C, k, variant, kernel, s);
    case 3: return launch_m4rm_f3(m, l, n, A, B, C, k, variant, kernel, s);
    case 4: return launch_m4rm_gf4(m, l, n, A, B, C, k, variant, kernel, s);
    case 5: return launch_m4rm_f5(m, l, n, A, B, C, k, variant, kernel, s);
    case 7: return launch_m4rm_f7(m, l, n, A, B, C, k, variant, kernel, s);
    default: return FQ_EINVAL;
  }
}

const Variant *m4rm_variants(int q, int *count) {
  *count = 0;
  switch (q) {
    case 2: return m4rm_variants_f2(count);
    case 3: return m4rm_variants_f3(count);
    case 4: return m4rm_variants_gf4(count);
    case 5: return m4rm_variants_f5(count);
    case 7: return m4rm_variants_f7(count);
    default: return nullptr;
  }
}

int m4rm_planned(int q, int64_t m, int64_t l, int64_t n, int k, int mt, int sms) {
  int nv = 0;
  const Variant *vs = m4rm_variants(q, &nv);
  if (!vs) return -1;
  const int d = q == 2 ? 1 : ((q == 5 || q == 7) ? 3 : 2);
  return plan_pick(vs, nv, d, m, l, n, k, mt, sms);
}

}  // namespace fqk

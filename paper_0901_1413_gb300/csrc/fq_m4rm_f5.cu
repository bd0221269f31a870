// M4RM kernel instances for F_5 (three planes, 1024-column tiles, 8 warps) and the planner's variant table.
#include "fq_m4rm.cuh"

namespace fqk {

namespace {
using C_k6_r8 = M4rmCfg<F5, 6, 8, 4, 8, 8>;
using C_k7_r8 = M4rmCfg<F5, 7, 8, 4, 8, 8>;
using C_k8_r8 = M4rmCfg<F5, 8, 8, 4, 8, 8>;
using C_k8_r2 = M4rmCfg<F5, 8, 8, 4, 2, 8>;
using C_k8_r4 = M4rmCfg<F5, 8, 8, 4, 4, 8>;
using C_k8_r6 = M4rmCfg<F5, 8, 8, 4, 6, 8>;
using C_k8_r7 = M4rmCfg<F5, 8, 8, 4, 7, 8>;
using C_k7_r4 = M4rmCfg<F5, 7, 8, 4, 4, 8>;
using C_k7_r6 = M4rmCfg<F5, 7, 8, 4, 6, 8>;
using C_k7_r7 = M4rmCfg<F5, 7, 8, 4, 7, 8>;

template <class Cfg>
int run(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int mt, cudaStream_t s) {
  return launch_cfg<Cfg>(m, l, n, A, B, C, mt, s);
}

const Variant kVariants[] = {
    {6, 8, &run<C_k6_r8>, 32},
    {7, 8, &run<C_k7_r8>, 32},
    {8, 8, &run<C_k8_r8>, 32},
    {8, 2, &run<C_k8_r2>, 32},
    {8, 4, &run<C_k8_r4>, 32},
    {8, 6, &run<C_k8_r6>, 32},
    {8, 7, &run<C_k8_r7>, 32},
    {7, 4, &run<C_k7_r4>, 32},
    {7, 6, &run<C_k7_r6>, 32},
    {7, 7, &run<C_k7_r7>, 32}
};
}  // namespace

int launch_m4rm_f5(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k,
                   int mt, cudaStream_t s) {
  return plan_and_launch(kVariants, int(sizeof(kVariants) / sizeof(kVariants[0])), F5::D, 16, m, l, n, A,
                         B, C, k, mt, s);
}

}  // namespace fqk

// M4RM kernel instances for F_7 (three planes, 1024-column tiles) and the planner's variant table.
#include "fq_m4rm_ws.cuh"
#include "fq_m4rm.cuh"

namespace fqk {

namespace {
template <class W>
int run_ws(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int mt, cudaStream_t s) {
  return ws::launch<W>(m, l, n, A, B, C, mt, s);
}
template <class Cf>
int run(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int mt, cudaStream_t s) {
  return launch_cfg<Cf>(m, l, n, A, B, C, mt, s);
}

// {k, row slots, launcher, rows per slot, columns per CTA, warps per CTA}
const Variant kVariants[] = {
    {8, 8, &run<M4rmCfg<F7, 8, 8, 4, 8, 8>>, 32, 1024, 8},
    {8, 7, &run<M4rmCfg<F7, 8, 8, 4, 7, 8>>, 32, 1024, 8},
    {8, 6, &run<M4rmCfg<F7, 8, 8, 4, 6, 8>>, 32, 1024, 8},
    {8, 4, &run<M4rmCfg<F7, 8, 8, 4, 4, 8>>, 32, 1024, 8},
    {8, 2, &run<M4rmCfg<F7, 8, 8, 4, 2, 8>>, 32, 1024, 8},
    {7, 8, &run<M4rmCfg<F7, 7, 8, 4, 8, 8>>, 32, 1024, 8},
    {7, 7, &run<M4rmCfg<F7, 7, 8, 4, 7, 8>>, 32, 1024, 8},
    {7, 6, &run<M4rmCfg<F7, 7, 8, 4, 6, 8>>, 32, 1024, 8},
    {7, 4, &run<M4rmCfg<F7, 7, 8, 4, 4, 8>>, 32, 1024, 8},
    {6, 8, &run<M4rmCfg<F7, 6, 8, 4, 8, 8>>, 32, 1024, 8},
};
}  // namespace

const Variant *m4rm_variants_f7(int *count) {
  *count = int(sizeof(kVariants) / sizeof(kVariants[0]));
  return kVariants;
}

int launch_m4rm_f7(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k, int mt,
                   int kernel, cudaStream_t s) {
  return plan_and_launch(kVariants, int(sizeof(kVariants) / sizeof(kVariants[0])), F7::D, m, l, n, A, B, C, k,
                         mt, kernel, s);
}

}  // namespace fqk

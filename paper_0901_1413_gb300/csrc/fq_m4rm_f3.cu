// M4RM kernel instances for F_3 (two planes, 512-column tiles) and the planner's variant table.
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
    {8, 20, &run_ws<ws::Cfg<F3, 8, 20, 4, 3>>, 48, 512, 16},
    {8, 16, &run_ws<ws::Cfg<F3, 8, 16, 4, 3>>, 48, 512, 16},
    {8, 12, &run_ws<ws::Cfg<F3, 8, 12, 4, 3>>, 48, 512, 16},
    {8, 8, &run_ws<ws::Cfg<F3, 8, 8, 4, 3>>, 48, 512, 16},
    {8, 4, &run_ws<ws::Cfg<F3, 8, 4, 4, 3>>, 48, 512, 16},
    {8, 24, &run_ws<ws::Cfg<F3, 8, 24, 4, 2>>, 48, 512, 16},
    {7, 24, &run_ws<ws::Cfg<F3, 7, 24, 4, 2>>, 48, 512, 16},
    {6, 24, &run_ws<ws::Cfg<F3, 6, 24, 4, 2>>, 48, 512, 16},
    {9, 16, &run_ws<ws::Cfg<F3, 9, 16, 4, 2>>, 48, 512, 16},
    {8, 32, &run_ws<ws::Cfg<F3, 8, 32, 8, 2>>, 32, 512, 16},
    {8, 24, &run_ws<ws::Cfg<F3, 8, 24, 8, 2>>, 32, 512, 16},
    {8, 16, &run_ws<ws::Cfg<F3, 8, 16, 8, 2>>, 32, 512, 16},
    {8, 8, &run_ws<ws::Cfg<F3, 8, 8, 8, 2>>, 32, 512, 16},
    {7, 32, &run_ws<ws::Cfg<F3, 7, 32, 8, 2>>, 32, 512, 16},
    {6, 32, &run_ws<ws::Cfg<F3, 6, 32, 8, 2>>, 32, 512, 16},
    {9, 16, &run_ws<ws::Cfg<F3, 9, 16, 8, 2>>, 32, 512, 16},
    {10, 16, &run<M4rmCfg<F3, 10, 8, 2, 16, 16>>, 64, 512, 16},
};
}  // namespace

const Variant *m4rm_variants_f3(int *count) {
  *count = int(sizeof(kVariants) / sizeof(kVariants[0]));
  return kVariants;
}

int launch_m4rm_f3(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k, int mt,
                   int kernel, cudaStream_t s) {
  return plan_and_launch(kVariants, int(sizeof(kVariants) / sizeof(kVariants[0])), F3::D, m, l, n, A, B, C, k,
                         mt, kernel, s);
}

}  // namespace fqk

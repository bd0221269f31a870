// M4RM kernel instances for F_3 (warp-specialised, 512-column tiles) and the
// planner's variant table.
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

const Variant kVariants[] = {
    {8, 24, &run_ws<ws::Cfg<F3, 8, 24>>, 48},
    {8, 20, &run_ws<ws::Cfg<F3, 8, 20>>, 48},
    {8, 16, &run_ws<ws::Cfg<F3, 8, 16>>, 48},
    {8, 12, &run_ws<ws::Cfg<F3, 8, 12>>, 48},
    {8, 8, &run_ws<ws::Cfg<F3, 8, 8>>, 48},
    {8, 4, &run_ws<ws::Cfg<F3, 8, 4>>, 48},
    {9, 16, &run_ws<ws::Cfg<F3, 9, 16>>, 48},
    {7, 24, &run_ws<ws::Cfg<F3, 7, 24>>, 48},
    {6, 24, &run_ws<ws::Cfg<F3, 6, 24>>, 48},
    {10, 16, &run<M4rmCfg<F3, 10, 8, 2, 16, 16>>, 64},
};
}  // namespace

int launch_m4rm_f3(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k, int mt,
                   cudaStream_t s) {
  return plan_and_launch(kVariants, int(sizeof(kVariants) / sizeof(kVariants[0])), F3::D, 8, m, l, n, A, B, C, k, mt,
                         s);
}

}  // namespace fqk

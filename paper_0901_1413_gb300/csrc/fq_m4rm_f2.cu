// M4RM kernel instances for F_2 (one plane, 1024-column tiles, 16 warps) and the
// planner's variant table.  F_2 is the binary case of Section 2 and the base
// field of the matrix-level GF(4) and F_8 products of Section 4.3.
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
// Warp-specialised kernels first (4 producer + 12 consumer warps, 48 rows per
// slot), then the all-warps kernels that reach k = 10.
const Variant kVariants[] = {
    {8, 20, &run_ws<ws::Cfg<F2, 8, 20, 4, 3, 16>>, 48, 1024, 16},
    {8, 16, &run_ws<ws::Cfg<F2, 8, 16, 4, 3, 16>>, 48, 1024, 16},
    {8, 12, &run_ws<ws::Cfg<F2, 8, 12, 4, 3, 16>>, 48, 1024, 16},
    {8, 10, &run_ws<ws::Cfg<F2, 8, 10, 4, 3, 16>>, 48, 1024, 16},
    {8, 8, &run_ws<ws::Cfg<F2, 8, 8, 4, 3, 16>>, 48, 1024, 16},
    {8, 4, &run_ws<ws::Cfg<F2, 8, 4, 4, 3, 16>>, 48, 1024, 16},
    {9, 16, &run_ws<ws::Cfg<F2, 9, 16, 4, 2, 16>>, 48, 1024, 16},
    {7, 20, &run_ws<ws::Cfg<F2, 7, 20, 4, 3, 16>>, 48, 1024, 16},
    {6, 20, &run_ws<ws::Cfg<F2, 6, 20, 4, 3, 16>>, 48, 1024, 16},
    {8, 10, &run_ws<ws::Cfg<F2, 8, 10, 4, 4, 16>>, 48, 1024, 16},
    {8, 32, &run_ws<ws::Cfg<F2, 8, 32, 8, 3, 16>>, 32, 1024, 16},
    {8, 24, &run_ws<ws::Cfg<F2, 8, 24, 8, 3, 16>>, 32, 1024, 16},
    {8, 16, &run_ws<ws::Cfg<F2, 8, 16, 8, 3, 16>>, 32, 1024, 16},
    {8, 12, &run_ws<ws::Cfg<F2, 8, 12, 8, 3, 16>>, 32, 1024, 16},
    {7, 32, &run_ws<ws::Cfg<F2, 7, 32, 8, 3, 16>>, 32, 1024, 16},
    {10, 16, &run<M4rmCfg<F2, 10, 8, 4, 16, 16>>, 64, 1024, 16},
    {10, 8, &run<M4rmCfg<F2, 10, 8, 4, 8, 16>>, 64, 1024, 16},
    {8, 16, &run<M4rmCfg<F2, 8, 8, 4, 16, 16>>, 64, 1024, 16},
};
}  // namespace

const Variant *m4rm_variants_f2(int *count) {
  *count = int(sizeof(kVariants) / sizeof(kVariants[0]));
  return kVariants;
}

int launch_m4rm_f2(int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C, int k, int mt,
                   int kernel, cudaStream_t s) {
  return plan_and_launch(kVariants, int(sizeof(kVariants) / sizeof(kVariants[0])), F2::D, m, l, n, A, B, C, k,
                         mt, kernel, s);
}

}  // namespace fqk

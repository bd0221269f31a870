// Many independent products C_p = A_p B_p in one persistent launch.
//
// The host plan splits every product into items (a run of rows x one column
// tile of C) with a block size k chosen per item by the planner's cost model,
// and orders items longest first.  The work list lives in a device workspace
// the caller owns; each launch resets one queue counter and starts as many
// CTAs as fit on the SMs (two per SM for F_3 and GF(4)), and every CTA pops
// items with an atomic until the list is exhausted,
// running the Four-Russians item body of fq_m4rm.cuh on each (B blocks staged
// with cp.async, since the operands' addresses are only known at launch).  A
// launch allocates nothing and never waits on the host, so it can be captured
// in a CUDA graph and replayed.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <new>
#include <vector>

#include "fq_m4rm.cuh"

namespace fqk {

namespace batched {

struct Item {
  int32_t product;
  int32_t row0;
  int32_t rows;
  int32_t col_tile;
  int32_t k;  // block size; 0: the column tile is all padding, store zeros
  int32_t pad[3];
};
static_assert(sizeof(Item) == 32, "item layout");

struct Shape {
  int64_t m, l, n;
};

// Workspace: [header 64 B][shapes: count x 24 B, rounded to 64][items: n x 32 B]
struct Header {
  uint32_t next;      // queue counter, reset by every launch
  uint32_t count;     // products
  uint32_t nitems;
  uint32_t q;
  uint32_t pad[12];
};
static_assert(sizeof(Header) == 64, "header layout");

__host__ __device__ inline int64_t shapes_bytes(int count) { return (int64_t(count) * int64_t(sizeof(Shape)) + 63) / 64 * 64; }

// Stage rows s K .. s K + K - 1 of B's CTW-word column tile, all planes, into
// `stage` ([p][row][CTW words]); rows past l are zero.
template <class Cfg>
__device__ __forceinline__ void stage_b(const uint64_t *B, int64_t l, int64_t pc, uint32_t stage, int64_t w0,
                                        int64_t s, int tid) {
  constexpr int CHUNKS = Cfg::P * Cfg::K * Cfg::CTW / 2;  // 16-byte pieces
  for (int e = tid; e < CHUNKS; e += Cfg::NT) {
    const int c = e % (Cfg::CTW / 2);
    const int t = (e / (Cfg::CTW / 2)) % Cfg::K;
    const int p = e / (Cfg::CTW / 2) / Cfg::K;
    const int64_t row = s * Cfg::K + t;
    const uint32_t dst = stage + uint32_t(e) * 16u;
    if (row < l) {
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                   "l"(B + (p * l + row) * pc + w0 + 2 * c) : "memory");
    } else {
      asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
    }
  }
  cp_async_commit();
}

// One item: rows [row0, row0 + rows) of product C = A B, column tile w0.
template <class Cfg>
__device__ __noinline__ void run_item(const M4rmParams &prm, const uint64_t *B, int64_t w0, int64_t row0,
                                         int rows_here, unsigned char *smem, int tid, int warp, int grp, int gl) {
  const uint32_t table_s = smem_u32(smem + Cfg::TABLE_OFF);
  const uint32_t tbl_lane = table_s + uint32_t(gl * Cfg::VB);
  const uint32_t bstage_s = smem_u32(smem + Cfg::BSTAGE_OFF);
  const uint32_t astage_s = smem_u32(smem + Cfg::ASTAGE_OFF);
  typename Cfg::Off *offs = reinterpret_cast<typename Cfg::Off *>(smem + Cfg::OFFS_OFF);
  const bool builder = warp < Cfg::NBW;
  const int slots = (rows_here + Cfg::ROWS_PER_SLOT - 1) / Cfg::ROWS_PER_SLOT;  // slots holding rows

  uint32_t acc[Cfg::RS][Cfg::PW];
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i)
#pragma unroll
    for (int j = 0; j < Cfg::PW; ++j) acc[i][j] = 0u;

  if (prm.nblocks > 0) {
    stage_b<Cfg>(B, prm.l, prm.pc, bstage_s, w0, 0, tid);
    stage_a<Cfg>(prm, astage_s, row0, rows_here, 0, tid);
  }
  for (int64_t c0 = 0; c0 < prm.nblocks; c0 += Cfg::NB) {
    const int nb = int(prm.nblocks - c0 < Cfg::NB ? prm.nblocks - c0 : Cfg::NB);
    cp_async_wait_all();
    __syncthreads();  // A words of this chunk staged; previous lookups done with `offs`
    build_offsets<Cfg>(prm, smem + Cfg::ASTAGE_OFF, offs, rows_here, c0, nb, tid);
    __syncthreads();  // A stage consumed
    if (c0 + Cfg::NB < prm.nblocks)
      stage_a<Cfg>(prm, astage_s, row0, rows_here, ((c0 + Cfg::NB) * Cfg::K) >> 6, tid);
    for (int b = 0; b < nb; ++b) {
      const int64_t s = c0 + b;
      const int buf = int(s & 1);
      cp_async_wait_all();
      __syncthreads();  // table free; this block's B rows staged
      if (s + 1 < prm.nblocks)
        stage_b<Cfg>(B, prm.l, prm.pc, bstage_s + (buf ^ 1) * Cfg::STAGE_STRIDE, w0, s + 1, tid);
      if (builder) build_table<Cfg>(tbl_lane, bstage_s + buf * Cfg::STAGE_STRIDE, warp * Cfg::GPW + grp, gl);
      __syncthreads();  // table complete
      lookup_block<Cfg, true>(acc, tbl_lane, offs + b * Cfg::MT, warp, grp, prm.one, slots);
    }
  }
  cp_async_wait_all();
  store_tile<Cfg>(acc, prm, row0, rows_here, w0, warp, grp, gl);
}

template <class C6, class C7, class C8>
__global__ void __launch_bounds__(C8::NT, C8::P == 2 ? 2 : 1)
    batched_kernel(unsigned char *ws, const uint64_t *const *Aptr, const uint64_t *const *Bptr, uint64_t *const *Cptr,
                   unsigned *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Item s_item;
  __shared__ int s_idx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = lane / C8::LPR, gl = lane % C8::LPR;
  Header *hdr = reinterpret_cast<Header *>(ws);
  const Shape *shapes = reinterpret_cast<const Shape *>(ws + sizeof(Header));
  const Item *items = reinterpret_cast<const Item *>(ws + sizeof(Header) + shapes_bytes(int(hdr->count)));
  const uint32_t nitems = hdr->nitems;
  while (true) {
    if (tid == 0) {
      const uint32_t i = atomicAdd(&hdr->next, 1u);
      s_idx = int(i < nitems ? i : nitems);
      if (i < nitems) s_item = items[i];
    }
    __syncthreads();
    if (s_idx >= int(nitems)) break;
    const Item it = s_item;
    const Shape sh = shapes[it.product];
    M4rmParams prm;
    prm.A = Aptr[it.product];
    prm.C = Cptr[it.product];
    prm.m = sh.m;
    prm.l = sh.l;
    prm.pa = (((sh.l + 63) / 64) + 15) / 16 * 16;
    prm.pc = (((sh.n + 63) / 64) + 15) / 16 * 16;
    prm.mt = it.rows;
    prm.one = 1u;
    prm.err = err;
    const uint64_t *B = Bptr[it.product];
    const int64_t w0 = int64_t(it.col_tile) * C8::CTW;
    if (it.k == 0) {  // padding columns only: C's words there are zero
      for (int e = tid; e < C8::P * it.rows * C8::CTW; e += C8::NT) {
        const int w = e % C8::CTW, r = (e / C8::CTW) % it.rows, p = e / C8::CTW / it.rows;
        prm.C[(p * prm.m + it.row0 + r) * prm.pc + w0 + w] = 0ull;
      }
      __syncthreads();
      continue;
    }
    switch (it.k) {
      case 6:
        prm.nblocks = (sh.l + 5) / 6;
        run_item<C6>(prm, B, w0, it.row0, it.rows, smem, tid, warp, grp, gl);
        break;
      case 7:
        prm.nblocks = (sh.l + 6) / 7;
        run_item<C7>(prm, B, w0, it.row0, it.rows, smem, tid, warp, grp, gl);
        break;
      default:
        prm.nblocks = (sh.l + 7) / 8;
        run_item<C8>(prm, B, w0, it.row0, it.rows, smem, tid, warp, grp, gl);
        break;
    }
    __syncthreads();  // item done before s_item is overwritten
  }
}

template <class F>
struct Kernels;
// Two-plane fields: 8 warps and 512 rows per CTA, two CTAs per SM, so that one
// CTA's table build overlaps the other's lookups.
template <>
struct Kernels<F3> {
  using C6 = M4rmCfg<F3, 6, 8, 2, 16, 8>;
  using C7 = M4rmCfg<F3, 7, 8, 2, 16, 8>;
  using C8 = M4rmCfg<F3, 8, 8, 2, 16, 8>;
};
template <>
struct Kernels<GF4> {
  using C6 = M4rmCfg<GF4, 6, 8, 2, 16, 8>;
  using C7 = M4rmCfg<GF4, 7, 8, 2, 16, 8>;
  using C8 = M4rmCfg<GF4, 8, 8, 2, 16, 8>;
};
template <>
struct Kernels<F5> {
  using C6 = M4rmCfg<F5, 6, 8, 4, 8, 8>;
  using C7 = M4rmCfg<F5, 7, 8, 4, 8, 8>;
  using C8 = M4rmCfg<F5, 8, 8, 4, 8, 8>;
};
template <>
struct Kernels<F7> {
  using C6 = M4rmCfg<F7, 6, 8, 4, 8, 8>;
  using C7 = M4rmCfg<F7, 7, 8, 4, 8, 8>;
  using C8 = M4rmCfg<F7, 8, 8, 4, 8, 8>;
};

template <class F>
constexpr int smem_for() {
  using K = Kernels<F>;
  int s = K::C6::SMEM;
  s = K::C7::SMEM > s ? K::C7::SMEM : s;
  s = K::C8::SMEM > s ? K::C8::SMEM : s;
  return s;
}

template <class F>
int launch_field(unsigned char *ws, const uint64_t *const *A, const uint64_t *const *B, uint64_t *const *C,
                 cudaStream_t s) {
  using K = Kernels<F>;
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  auto kern = batched_kernel<typename K::C6, typename K::C7, typename K::C8>;
  constexpr int smem = smem_for<F>();
  FQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int dev = 0, sms = 152;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  FQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 1;
  FQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::C8::NT, smem));
  if (per_sm < 1) per_sm = 1;
  FQ_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(uint32_t), s));
  kern<<<sms * per_sm, K::C8::NT, smem, s>>>(ws, A, B, C, err);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

template <class F>
constexpr int max_rows() {
  return Kernels<F>::C8::MT;
}
template <class F>
constexpr int tile_words() {
  return Kernels<F>::C8::CTW;
}

}  // namespace batched

}  // namespace fqk

// ------------------------------------------------------------------ C ABI --

struct fq_batch_plan {
  int q;
  int count;
  std::vector<fqk::batched::Shape> shapes;
  std::vector<fqk::batched::Item> items;
  int64_t workspace_bytes;
  double model_cost;  // sum of modelled item costs (adds)
};

extern "C" {

int fq_batched_plan_create(int q, int count, const int64_t *m, const int64_t *l, const int64_t *n,
                           fq_batch_plan **out) {
  using namespace fqk::batched;
  if (!out) return FQ_EINVAL;
  *out = nullptr;
  if (!(q == 3 || q == 4 || q == 5 || q == 7) || count < 0 || (count > 0 && (!m || !l || !n))) return FQ_EINVAL;
  fq_batch_plan *plan = new (std::nothrow) fq_batch_plan();
  if (!plan) return FQ_ENOMEM;
  plan->q = q;
  plan->count = count;
  const int d = q == 3 || q == 4 ? 2 : 3;
  const int mt_max = (q == 3 || q == 4) ? fqk::batched::max_rows<fqk::F3>() : fqk::batched::max_rows<fqk::F5>();
  const int ctw = (q == 3 || q == 4) ? fqk::batched::tile_words<fqk::F3>() : fqk::batched::tile_words<fqk::F5>();
  std::vector<std::pair<double, Item>> costed;
  plan->model_cost = 0;
  for (int p = 0; p < count; ++p) {
    if (m[p] < 0 || l[p] < 0 || n[p] < 0 || m[p] >= (int64_t(1) << 31) || l[p] >= (int64_t(1) << 31) ||
        n[p] >= (int64_t(1) << 36)) {
      delete plan;
      return FQ_EINVAL;
    }
    plan->shapes.push_back(Shape{m[p], l[p], n[p]});
    if (m[p] == 0 || n[p] == 0) continue;
    const int64_t col_tiles = fq_pitch_words(n[p]) / ctw;
    const int64_t row_tiles = fqk::cdiv(m[p], mt_max);
    const int rows = int(fqk::cdiv(m[p], row_tiles));
    // block size per item: the cheapest of k = 6, 7, 8 by the cost model
    int best_k = 8;
    double best = 1e300;
    for (int k = 6; k <= 8; ++k) {
      const double cost = double(fqk::cdiv(l[p], k)) * (1.2 * double(1 << k) + double(rows) * d) + 2000.0;
      if (cost < best) {
        best = cost;
        best_k = k;
      }
    }
    const int64_t real_tiles = fqk::cdiv(fqk::cdiv(n[p], 64), ctw);  // tiles holding real columns
    for (int64_t rt = 0; rt < row_tiles; ++rt) {
      for (int64_t ct = 0; ct < col_tiles; ++ct) {
        const int64_t r0 = rt * rows;
        const int rr = int(m[p] - r0 < rows ? m[p] - r0 : rows);
        Item it{};
        it.product = p;
        it.row0 = int32_t(r0);
        it.rows = rr;
        it.col_tile = int32_t(ct);
        it.k = ct < real_tiles ? best_k : 0;
        const double cost = ct < real_tiles ? best : 1.0;
        costed.push_back({cost, it});
        plan->model_cost += cost;
      }
    }
  }
  // longest first
  std::stable_sort(costed.begin(), costed.end(),
                   [](const std::pair<double, Item> &a, const std::pair<double, Item> &b) { return a.first > b.first; });
  for (auto &c : costed) plan->items.push_back(c.second);
  plan->workspace_bytes =
      int64_t(sizeof(Header)) + shapes_bytes(count) + int64_t(plan->items.size()) * int64_t(sizeof(Item));
  *out = plan;
  return FQ_OK;
}

int64_t fq_batched_workspace_bytes(const fq_batch_plan *plan) { return plan ? plan->workspace_bytes : -1; }

int64_t fq_batched_items(const fq_batch_plan *plan) { return plan ? int64_t(plan->items.size()) : -1; }

int fq_batched_plan_upload(const fq_batch_plan *plan, void *workspace, void *stream) {
  using namespace fqk::batched;
  if (!plan || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 63u) != 0) return FQ_EINVAL;
  std::vector<unsigned char> host(size_t(plan->workspace_bytes), 0);
  Header h{};
  h.next = 0;
  h.count = uint32_t(plan->count);
  h.nitems = uint32_t(plan->items.size());
  h.q = uint32_t(plan->q);
  memcpy(host.data(), &h, sizeof(h));
  if (plan->count) memcpy(host.data() + sizeof(Header), plan->shapes.data(), plan->shapes.size() * sizeof(Shape));
  if (!plan->items.empty())
    memcpy(host.data() + sizeof(Header) + shapes_bytes(plan->count), plan->items.data(),
           plan->items.size() * sizeof(Item));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FQ_CUDA_TRY(cudaMemcpyAsync(workspace, host.data(), host.size(), cudaMemcpyHostToDevice, s));
  FQ_CUDA_TRY(cudaStreamSynchronize(s));
  return FQ_OK;
}

int fq_matmul_batched(const fq_batch_plan *plan, const uint64_t *const *A, const uint64_t *const *B,
                      uint64_t *const *C, void *workspace, void *stream) {
  if (!plan || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 63u) != 0) return FQ_EINVAL;
  if (plan->items.empty()) return FQ_OK;
  if (!A || !B || !C) return FQ_EINVAL;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (plan->q) {
    case 3: return fqk::batched::launch_field<fqk::F3>(ws, A, B, C, s);
    case 4: return fqk::batched::launch_field<fqk::GF4>(ws, A, B, C, s);
    case 5: return fqk::batched::launch_field<fqk::F5>(ws, A, B, C, s);
    case 7: return fqk::batched::launch_field<fqk::F7>(ws, A, B, C, s);
    default: return FQ_EINVAL;
  }
}

int fq_batched_plan_destroy(fq_batch_plan *plan) {
  delete plan;
  return FQ_OK;
}

}  // extern "C"

// ------------------------------------------- batched products without allocation --
//
// fq_matmul_batched_static runs the same persistent kernel as fq_matmul_batched,
// but its work list and queue counter live in this file-scope device array
// instead of a workspace the caller allocates.  The array exists once per GPU
// that loads the library and stays until the process exits.

namespace {

constexpr int64_t kStaticScratchBytes = FQ_BATCH_STATIC_BYTES;
static __device__ __align__(256) unsigned char g_batch_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
unsigned char *g_scratch_addr[kMaxStaticDevices];
std::mutex g_scratch_mu;

// Device address of g_batch_scratch on the current device.  In host code the
// array's name is only a host-side handle, so the address is looked up once per
// device (with that device current) and reused.
int static_scratch(unsigned char **out) {
  int dev = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxStaticDevices) return FQ_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_batch_scratch);
    if (e != cudaSuccess) return fqk::record_cuda_error(e);
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[dev];
  return FQ_OK;
}

}  // namespace

extern "C" int fq_matmul_batched_static(const fq_batch_plan *plan, const uint64_t *const *A,
                                        const uint64_t *const *B, uint64_t *const *C, void *stream) {
  using namespace fqk::batched;
  if (!plan) return FQ_EINVAL;
  if (plan->items.empty()) return FQ_OK;
  if (!A || !B || !C) return FQ_EINVAL;
  if (plan->workspace_bytes > kStaticScratchBytes) return FQ_ENOTSUP;  // does not fit the fixed array
  unsigned char *ws = nullptr;
  if (int rc = static_scratch(&ws)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The array holds whatever the previous call left: write this plan's header
  // (queue counter 0), shapes and items before the launch, in stream order.
  Header h{};
  h.next = 0;
  h.count = uint32_t(plan->count);
  h.nitems = uint32_t(plan->items.size());
  h.q = uint32_t(plan->q);
  FQ_CUDA_TRY(cudaMemcpyAsync(ws, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  if (plan->count)
    FQ_CUDA_TRY(cudaMemcpyAsync(ws + sizeof(Header), plan->shapes.data(), plan->shapes.size() * sizeof(Shape),
                                cudaMemcpyHostToDevice, s));
  FQ_CUDA_TRY(cudaMemcpyAsync(ws + sizeof(Header) + shapes_bytes(plan->count), plan->items.data(),
                              plan->items.size() * sizeof(Item), cudaMemcpyHostToDevice, s));
  switch (plan->q) {
    case 3: return launch_field<fqk::F3>(ws, A, B, C, s);
    case 4: return launch_field<fqk::GF4>(ws, A, B, C, s);
    case 5: return launch_field<fqk::F5>(ws, A, B, C, s);
    case 7: return launch_field<fqk::F7>(ws, A, B, C, s);
    default: return FQ_EINVAL;
  }
}

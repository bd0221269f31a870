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
#include <atomic>
#include <exception>
#include <memory>
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

  uint32_t acc[Cfg::RS][Cfg::APW];
#pragma unroll
  for (int i = 0; i < Cfg::RS; ++i)
#pragma unroll
    for (int j = 0; j < Cfg::APW; ++j) acc[i][j] = 0u;

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
      lookup_block<Cfg, true>(acc, tbl_lane, offs + b * Cfg::MT, warp, grp, prm.one, prm.err, slots);
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
    prm.wait_ns = kWaitLimitNs;  // the item body stages B with cp.async: no mbarrier waits
    prm.stall = -1;
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
  std::vector<fqk::batched::Item> items;      // Four-Russians items
  std::vector<fqk::BatchProd> tc_prods;       // products on the tcgen05 path
  std::vector<int32_t> tc_cta_begin;          // kTcGroups + 1
  std::vector<int32_t> tc_cta_list;           // product indices, each group's in the order it computes them
  std::vector<int64_t> tc_cta_rows;           // kTcGroups x 2: first scratch row of each group's buffers
  int64_t tc_tiles = 0;                       // 128 x 256 tiles of the tcgen05 products
  int64_t scratch_rows = 0;                   // 128-byte rows of all groups' buffers
  int64_t off_prods = 0, off_cta_begin = 0, off_cta_list = 0, off_cta_rows = 0, off_scratch = 0;
  int64_t table_bytes = 0;      // header .. CTA rows (uploaded)
  int64_t workspace_bytes = 0;  // plus the scratch buffers
  double model_cost = 0;        // modelled SM-cycles of the whole plan
};

namespace {

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// fq_debug_fail_host_alloc: the countdown of host allocation points before
// one fails (-1: none armed).
std::atomic<int64_t> g_fail_alloc{-1};

// A host allocation point of plan building: throws std::bad_alloc, as a
// failed allocation would, when the armed countdown reaches it.
void host_alloc_point() {
  int64_t left = g_fail_alloc.load(std::memory_order_relaxed);
  while (left >= 0) {
    if (g_fail_alloc.compare_exchange_weak(left, left - 1, std::memory_order_relaxed)) {
      if (left == 0) throw std::bad_alloc();
      return;
    }
  }
}

// Modelled SM-cycles per unit of the batched Four-Russians item cost (table
// entries + rows x basis size per block), fitted to the 4096-product batch
// on GB300: F_3 and GF(4) run two CTAs per SM.
double m4rm_unit_cycles(int q) { return q == 3 || q == 4 ? 2.1 : (q == 5 ? 8.5 : 8.0); }

// Modelled SM-cycles of one product on the tcgen05 path: tiles x 128-deep
// k-steps at ~760 cycles, and the conversion's bytes at ~3 TB/s shared by
// 152 SMs at 2.07 GHz.
double tc_product_cycles(int64_t m, int64_t l, int64_t n) {
  const int64_t la = fqk::cdiv(l, 128) * 128, nr = fqk::cdiv(n, 256) * 256;
  const double tiles = double(fqk::cdiv(m, 128)) * double(nr / 256);
  const double bytes = double(m + n) * double(la);
  return tiles * double(la / 128) * 760.0 + bytes * (2.07e9 * 152.0 / 3.0e12);
}

int plan_create(int q, int count, const int64_t *m, const int64_t *l, const int64_t *n, int path,
                fq_batch_plan **out) {
  using namespace fqk::batched;
  if (!out) return FQ_EINVAL;
  *out = nullptr;
  if (!(q == 3 || q == 4 || q == 5 || q == 7) || count < 0 || (count > 0 && (!m || !l || !n))) return FQ_EINVAL;
  if (!(path == FQ_PATH_AUTO || path == FQ_PATH_M4RM || path == FQ_PATH_MMA)) return FQ_EINVAL;
  host_alloc_point();
  std::unique_ptr<fq_batch_plan> plan(new (std::nothrow) fq_batch_plan());
  if (!plan) return FQ_ENOMEM;
  plan->q = q;
  plan->count = count;
  const int d = q == 3 || q == 4 ? 2 : 3;
  const int mt_max = (q == 3 || q == 4) ? fqk::batched::max_rows<fqk::F3>() : fqk::batched::max_rows<fqk::F5>();
  const int ctw = (q == 3 || q == 4) ? fqk::batched::tile_words<fqk::F3>() : fqk::batched::tile_words<fqk::F5>();
  std::vector<std::pair<double, Item>> costed;
  // AUTO's products that the per-product models gave to Four Russians but the
  // tcgen05 form could take (with their costs), for the whole-plan check below
  struct Alt {
    int p;
    double m4rm, tc, longest;
  };
  std::vector<Alt> alts;
  auto add_tc = [&](int p) {
    fqk::BatchProd bp{};
    bp.p = p;
    bp.m = int32_t(m[p]);
    bp.l = int32_t(l[p]);
    bp.n = int32_t(n[p]);
    bp.la = int32_t(fqk::cdiv(l[p], 128) * 128);
    bp.nr = int32_t(fqk::cdiv(n[p], 256) * 256);
    bp.pa = fq_pitch_words(l[p]);
    bp.pb = fq_pitch_words(n[p]);
    bp.pc = fq_pitch_words(n[p]);
    bp.a_row0 = 0;
    bp.b_row0 = 0;
    host_alloc_point();
    plan->tc_prods.push_back(bp);
  };
  for (int p = 0; p < count; ++p) {
    if (m[p] < 0 || l[p] < 0 || n[p] < 0 || m[p] >= (int64_t(1) << 31) || l[p] >= (int64_t(1) << 31) ||
        n[p] >= (int64_t(1) << 31))
      return FQ_EINVAL;
    host_alloc_point();
    plan->shapes.push_back(Shape{m[p], l[p], n[p]});
    if (m[p] == 0 || n[p] == 0) continue;
    // Four-Russians items of this product and their modelled cost
    std::vector<std::pair<double, Item>> mine;
    double m4rm = 0;
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
        mine.push_back({cost, it});
        m4rm += cost * m4rm_unit_cycles(q);
      }
    }
    // the path: the tcgen05 form takes F_3, F_5 and F_7 products with 0 < l
    // within its exact range (and n <= 2^30, so that n rounded up to 256 stays
    // a 32-bit count), when asked to or when its model is cheaper
    const bool tc_ok = (q == 3 || q == 5 || q == 7) && l[p] > 0 && l[p] <= fqk::tc_max_l(q) &&
                       n[p] <= (int64_t(1) << 30);
    const double tc = tc_ok ? tc_product_cycles(m[p], l[p], n[p]) : 1e300;
    const bool use_tc = tc_ok && (path == FQ_PATH_MMA || (path == FQ_PATH_AUTO && tc < m4rm));
    if (!use_tc) {
      if (tc_ok && path == FQ_PATH_AUTO) {
        double longest = 0;
        for (auto &c : mine) longest = c.first > longest ? c.first : longest;
        alts.push_back(Alt{p, m4rm, tc, longest * m4rm_unit_cycles(q)});
      }
      for (auto &c : mine) costed.push_back(c);
      plan->model_cost += m4rm;
      continue;
    }
    add_tc(p);
    plan->model_cost += tc;
  }
  // Whole plan: a Four-Russians launch for a few products cannot fill the GPU
  // (its time is at least its longest item, plus ~20 us of launch); if the
  // tcgen05 launch would absorb them in less time, they go there too.
  if (!alts.empty() && !plan->tc_prods.empty()) {
    double m4rm = 0, tc = 0, longest = 0;
    for (const Alt &a : alts) {
      m4rm += a.m4rm;
      tc += a.tc;
      longest = a.longest > longest ? a.longest : longest;
    }
    const double sms = 152.0;
    const double m4rm_wall = (m4rm / sms > longest ? m4rm / sms : longest) + 40000.0;
    if (tc / sms < m4rm_wall) {
      std::vector<char> moved(size_t(count), 0);
      for (const Alt &a : alts) moved[size_t(a.p)] = 1;
      std::vector<std::pair<double, Item>> keep;
      for (auto &c : costed)
        if (!moved[size_t(c.second.product)]) keep.push_back(c);
      costed.swap(keep);
      for (const Alt &a : alts) {
        add_tc(a.p);
        plan->model_cost += a.tc - a.m4rm;
      }
    }
  }
  // The Four-Russians kernel numbers items with a 32-bit queue counter: larger
  // plans are refused.
  constexpr int64_t kMax32 = (int64_t(1) << 31) - 1;
  if (int64_t(costed.size()) > kMax32) return FQ_ENOTSUP;
  // longest first
  std::stable_sort(costed.begin(), costed.end(),
                   [](const std::pair<double, Item> &a, const std::pair<double, Item> &b) { return a.first > b.first; });
  for (auto &c : costed) {
    host_alloc_point();
    plan->items.push_back(c.second);
  }
  // tcgen05 work: whole products to the kTcGroups groups of persistent CTAs
  // (kTcGroup CTAs, one cluster, share each product), longest first, each to
  // the least-loaded group by the modelled cost; a group then takes its
  // products smallest first (the first one's conversion is the only one no
  // MMA overlaps).  Each group owns two scratch buffers, buffer b sized for
  // the largest of its products b, b + 2, ...
  const int T = int(plan->tc_prods.size());
  constexpr int NC = fqk::kTcGroups;
  plan->tc_cta_begin.assign(NC + 1, 0);
  plan->tc_cta_rows.assign(2 * NC, 0);
  if (T > 0) {
    std::vector<double> cost(size_t(T), 0.0);
    std::vector<int> order(size_t(T), 0);
    for (int i = 0; i < T; ++i) {
      const fqk::BatchProd &bp = plan->tc_prods[size_t(i)];
      cost[size_t(i)] = tc_product_cycles(bp.m, bp.l, bp.n);
      order[size_t(i)] = i;
      plan->tc_tiles += fqk::cdiv(bp.m, 128) * (bp.nr / 256);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[size_t(x)] > cost[size_t(y)]; });
    std::vector<double> load(NC, 0.0);
    std::vector<std::vector<int32_t>> per(NC);
    for (int i : order) {
      int c = 0;
      for (int k = 1; k < NC; ++k)
        if (load[size_t(k)] < load[size_t(c)]) c = k;
      per[size_t(c)].push_back(int32_t(i));
      load[size_t(c)] += cost[size_t(i)];
    }
    int64_t rows = 0;
    for (int c = 0; c < NC; ++c) {
      std::vector<int32_t> &list = per[size_t(c)];
      std::reverse(list.begin(), list.end());
      int64_t size[2] = {0, 0};
      for (size_t j = 0; j < list.size(); ++j) {
        const fqk::BatchProd &bp = plan->tc_prods[size_t(list[j])];
        const int64_t need = fqk::batch_a_rows(bp.m, bp.la) + fqk::batch_bt_rows(bp.nr, bp.la);
        size[j & 1] = need > size[j & 1] ? need : size[j & 1];
      }
      plan->tc_cta_begin[size_t(c) + 1] = plan->tc_cta_begin[size_t(c)] + int32_t(list.size());
      plan->tc_cta_list.insert(plan->tc_cta_list.end(), list.begin(), list.end());
      plan->tc_cta_rows[2 * size_t(c)] = rows;
      plan->tc_cta_rows[2 * size_t(c) + 1] = rows + size[0];
      rows += size[0] + size[1];
    }
    plan->scratch_rows = rows;
  }
  // the kernel's TMA coordinates are 32-bit scratch rows
  if (plan->scratch_rows > kMax32) return FQ_ENOTSUP;
  // workspace: [header][shapes][items][products][CTA begins][CTA lists][CTA
  // rows] | [scratch buffers]
  int64_t off = int64_t(sizeof(Header)) + shapes_bytes(count) + int64_t(plan->items.size()) * int64_t(sizeof(Item));
  if (T > 0) {
    plan->off_prods = off = align_up(off, 64);
    off += int64_t(T) * int64_t(sizeof(fqk::BatchProd));
    plan->off_cta_begin = off = align_up(off, 64);
    off += int64_t(NC + 1) * 4;
    plan->off_cta_list = off = align_up(off, 64);
    off += int64_t(T) * 4;
    plan->off_cta_rows = off = align_up(off, 64);
    off += int64_t(2 * NC) * 8;
  }
  plan->table_bytes = off;
  if (T > 0) {
    plan->off_scratch = off = align_up(off, 1024);
    off += plan->scratch_rows * 128;
  }
  plan->workspace_bytes = off;
  *out = plan.release();
  return FQ_OK;
}

// The C entry points return status codes: host allocation failures of the
// plan's tables (std::bad_alloc, std::length_error) become FQ_ENOMEM.
template <class Fn>
int host_guard(Fn &&fn) {
  try {
    return fn();
  } catch (const std::exception &) {
    return FQ_ENOMEM;
  }
}

// The host image of a plan's tables (header .. tile list).
std::vector<unsigned char> plan_tables(const fq_batch_plan *plan) {
  using namespace fqk::batched;
  host_alloc_point();
  std::vector<unsigned char> host(size_t(plan->table_bytes), 0);
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
  if (!plan->tc_prods.empty()) {
    memcpy(host.data() + plan->off_prods, plan->tc_prods.data(), plan->tc_prods.size() * sizeof(fqk::BatchProd));
    memcpy(host.data() + plan->off_cta_begin, plan->tc_cta_begin.data(), plan->tc_cta_begin.size() * 4);
    memcpy(host.data() + plan->off_cta_list, plan->tc_cta_list.data(), plan->tc_cta_list.size() * 4);
    memcpy(host.data() + plan->off_cta_rows, plan->tc_cta_rows.data(), plan->tc_cta_rows.size() * 8);
  }
  return host;
}

// The tcgen05 part of a plan in the workspace `ws`.
fqk::TcBatch tc_view(const fq_batch_plan *plan, unsigned char *ws) {
  fqk::TcBatch b;
  b.q = plan->q;
  b.nprod = int(plan->tc_prods.size());
  b.scratch_rows = plan->scratch_rows;
  b.prods = reinterpret_cast<const fqk::BatchProd *>(ws + plan->off_prods);
  b.cta_begin = reinterpret_cast<const int32_t *>(ws + plan->off_cta_begin);
  b.cta_list = reinterpret_cast<const int32_t *>(ws + plan->off_cta_list);
  b.cta_rows = reinterpret_cast<const int64_t *>(ws + plan->off_cta_rows);
  b.scratch = ws + plan->off_scratch;
  return b;
}

}  // namespace

extern "C" {

int fq_batched_plan_create(int q, int count, const int64_t *m, const int64_t *l, const int64_t *n,
                           fq_batch_plan **out) {
  return host_guard([&] { return plan_create(q, count, m, l, n, FQ_PATH_AUTO, out); });
}

int fq_batched_plan_create_ex(int q, int count, const int64_t *m, const int64_t *l, const int64_t *n, int path,
                              fq_batch_plan **out) {
  return host_guard([&] { return plan_create(q, count, m, l, n, path, out); });
}

int64_t fq_batched_workspace_bytes(const fq_batch_plan *plan) { return plan ? plan->workspace_bytes : -1; }

int64_t fq_batched_items(const fq_batch_plan *plan) { return plan ? int64_t(plan->items.size()) : -1; }

int64_t fq_batched_tc_products(const fq_batch_plan *plan) { return plan ? int64_t(plan->tc_prods.size()) : -1; }

int64_t fq_batched_tc_tiles(const fq_batch_plan *plan) { return plan ? plan->tc_tiles : -1; }

int fq_batched_plan_upload(const fq_batch_plan *plan, void *workspace, void *stream) {
  if (!plan || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 63u) != 0) return FQ_EINVAL;
  return host_guard([&] {
    const std::vector<unsigned char> host = plan_tables(plan);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FQ_CUDA_TRY(cudaMemcpyAsync(workspace, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    FQ_CUDA_TRY(cudaStreamSynchronize(s));
    return FQ_OK;
  });
}

int fq_matmul_batched_stages(const fq_batch_plan *plan, const uint64_t *const *A, const uint64_t *const *B,
                             uint64_t *const *C, void *workspace, void *stream, int stages) {
  if (!plan || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 63u) != 0) return FQ_EINVAL;
  if (stages < 0 || stages > FQ_BATCH_STAGE_ALL) return FQ_EINVAL;
  if (plan->items.empty() && plan->tc_prods.empty()) return FQ_OK;
  if (!A || !B || !C) return FQ_EINVAL;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!plan->tc_prods.empty() && (stages & FQ_BATCH_STAGE_TC))
    if (int rc = fqk::tc_batched(tc_view(plan, ws), A, B, C, s)) return rc;
  if (plan->items.empty() || !(stages & FQ_BATCH_STAGE_M4RM)) return FQ_OK;
  switch (plan->q) {
    case 3: return fqk::batched::launch_field<fqk::F3>(ws, A, B, C, s);
    case 4: return fqk::batched::launch_field<fqk::GF4>(ws, A, B, C, s);
    case 5: return fqk::batched::launch_field<fqk::F5>(ws, A, B, C, s);
    case 7: return fqk::batched::launch_field<fqk::F7>(ws, A, B, C, s);
    default: return FQ_EINVAL;
  }
}

int fq_matmul_batched(const fq_batch_plan *plan, const uint64_t *const *A, const uint64_t *const *B,
                      uint64_t *const *C, void *workspace, void *stream) {
  return fq_matmul_batched_stages(plan, A, B, C, workspace, stream, FQ_BATCH_STAGE_ALL);
}

int fq_batched_product_path(const fq_batch_plan *plan, int p) {
  if (!plan || p < 0 || p >= plan->count) return -FQ_EINVAL;
  for (const fqk::BatchProd &bp : plan->tc_prods)
    if (bp.p == p) return FQ_PATH_MMA;
  return FQ_PATH_M4RM;
}

int fq_debug_fail_host_alloc(int64_t after) {
  g_fail_alloc.store(after >= 0 ? after : -1, std::memory_order_relaxed);
  return FQ_OK;
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
  if (plan->items.empty() && plan->tc_prods.empty()) return FQ_OK;
  if (!A || !B || !C) return FQ_EINVAL;
  // tcgen05 products need their arenas; the fixed array holds work lists only
  if (!plan->tc_prods.empty() || plan->workspace_bytes > kStaticScratchBytes) return FQ_ENOTSUP;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the work list is copied from host memory at every call, which a captured
  // graph could not repeat
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  FQ_CUDA_TRY(cudaStreamIsCapturing(s, &capture));
  if (capture != cudaStreamCaptureStatusNone) return FQ_ENOTSUP;
  unsigned char *ws = nullptr;
  if (int rc = static_scratch(&ws)) return rc;
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

// Product dispatch and Strassen-Winograd levels over the base-field kernels.
//
// The paper notes that the Method of Four Russians serves well as the base case
// of an asymptotically faster algorithm (Section 2).  One Strassen-Winograd
// level splits A, B and C into quadrants and forms C from seven half-size
// products and fifteen additions:
//   S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2,
//   T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21,
//   P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4,
//   P5 = S1 T1,   P6 = S2 T2,   P7 = S3 T3,
//   C11 = P1 + P2,  U2 = P1 + P6,  U3 = U2 + P7,  C22 = U3 + P5,
//   C12 = U2 + P5 + P3,  C21 = U3 - P4.
// Additions are the bitsliced elementwise formulas (fq_add); quadrants are
// copied out of and back into the packed matrices by a 16-byte copy kernel.  A level is taken where the time model says seven half-size products
// plus the additions and copies beat the direct product, and only for shapes
// whose halves are whole 1024-column pitches (m, l, n multiples of 2048).
#include "../../include/fq.h"
#include "fq_common.cuh"
#include "fq_internal.h"

namespace fqk {

namespace {

constexpr int64_t kStrassenAlign = 2048;

int planes_of(int q) { return q == 2 ? 1 : ((q == 5 || q == 7) ? 3 : 2); }

bool base_field(int q) { return q == 2 || q == 3 || q == 4 || q == 5 || q == 7; }

bool splittable(int64_t m, int64_t l, int64_t n) {
  return m >= kStrassenAlign && l >= kStrassenAlign && n >= kStrassenAlign && m % kStrassenAlign == 0 &&
         l % kStrassenAlign == 0 && n % kStrassenAlign == 0;
}

// Modelled cycles of the direct product on the options' path.
double direct_cycles(int q, int64_t m, int64_t l, int64_t n, const ProdOptions &o, int sms) {
  const double mk = m4rm_estimate(q, m, l, n, sms), mm = mma_estimate(q, m, l, n, sms);
  if (o.path == FQ_PATH_MMA) return mm;
  if (o.path == FQ_PATH_M4RM || o.k || o.kernel || o.variant) return mk;
  return mk < mm ? mk : mm;
}

// Modelled cycles of one level's additions and copies: every byte of the
// quadrant traffic at about 6 TB/s and 2.07 GHz (HBM-bound elementwise work).
double level_overhead_cycles(int q, int64_t m, int64_t l, int64_t n) {
  const double P = planes_of(q);
  const double a = P * double(m) * double(fq_pitch_words(l)) * 8.0;  // bytes of A
  const double b = P * double(l) * double(fq_pitch_words(n)) * 8.0;
  const double c = P * double(m) * double(fq_pitch_words(n)) * 8.0;
  const double bytes = 5.0 * a + 5.0 * b + 7.25 * c;
  return bytes * 2.07e9 / 6.0e12 + 40000.0;  // plus launch gaps of ~60 small launches
}

// Best modelled cycles with up to `depth` levels; `levels` receives the count.
double best_cycles(int q, int64_t m, int64_t l, int64_t n, const ProdOptions &o, int sms, int depth,
                   int *levels) {
  const double direct = direct_cycles(q, m, l, n, o, sms);
  *levels = 0;
  if (depth <= 0 || !splittable(m, l, n)) return direct;
  int sub = 0;
  const double split = 7.0 * best_cycles(q, m / 2, l / 2, n / 2, o, sms, depth - 1, &sub) +
                       level_overhead_cycles(q, m, l, n);
  if (split < 0.97 * direct) {
    *levels = sub + 1;
    return split;
  }
  return direct;
}

// Quadrant (qi, qj) of a packed rows x cols matrix <-> a packed (rows/2) x
// (cols/2) matrix; cols/2 is a multiple of 1024, so neither side has padding.
// One thread per 16-byte piece, grid-stride over planes x rows x pieces.
__global__ void quadrant_kernel(int P, int64_t rows, int64_t pf, int64_t pq, const uint64_t *src, uint64_t *dst,
                                int64_t src_off, int64_t dst_off, bool out_of_full) {
  const int64_t hr = rows / 2, pieces = pq / 2, total = int64_t(P) * hr * pieces;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t w = (i % pieces) * 2, r = (i / pieces) % hr, p = i / pieces / hr;
    const int64_t f = (p * rows + r) * pf + w, h = (p * hr + r) * pq + w;
    const int64_t si = out_of_full ? src_off + f : h, di = out_of_full ? h : dst_off + f;
    *reinterpret_cast<uint4 *>(dst + di) = *reinterpret_cast<const uint4 *>(src + si);
  }
}

int copy_quadrant(int P, int64_t rows, int64_t cols, const uint64_t *full, uint64_t *quad, int qi, int qj,
                  bool out_of_full, cudaStream_t s) {
  const int64_t pf = fq_pitch_words(cols), hr = rows / 2, pq = fq_pitch_words(cols / 2);
  const int64_t off = qi * hr * pf + qj * pq;  // the quadrant's first word within each plane
  const int64_t total = int64_t(P) * hr * (pq / 2);
  const int64_t want = cdiv(total, 256), cap = 152 * 16;
  const unsigned grid = unsigned(want < cap ? want : cap);
  if (out_of_full)
    quadrant_kernel<<<grid, 256, 0, s>>>(P, rows, pf, pq, full, quad, off, 0, true);
  else
    quadrant_kernel<<<grid, 256, 0, s>>>(P, rows, pf, pq, quad, const_cast<uint64_t *>(full), 0, off, false);
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

int direct(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
           const ProdOptions &o, int sms, cudaStream_t s) {
  int path = o.path;
  int kernel = o.kernel;
  if (path == FQ_PATH_AUTO && o.k == 0 && o.kernel == 0 && o.variant == 0) {
    int p = 0, kk = 0;
    if (tuned_choice(q, m, l, n, &p, &kk)) {
      path = p;
      kernel = kk;
    } else if (l > 0 && mma_estimate(q, m, l, n, sms) < m4rm_estimate(q, m, l, n, sms)) {
      path = FQ_PATH_MMA;
    }
  }
  if (path == FQ_PATH_MMA) {
    // tcgen05 (e4m3 or packed e2m1, exact fp32 sums) unless a reduction
    // chunk or the mma.sync s8 form (kernel = 1) is requested, or l is beyond
    // its exact range; kernel = 2, 3, 4 force its single-SM, SM-pair or wide
    // SM-pair e4m3 kernel, 5 the fp4 SM-pair kernel
    if (o.chunk == 0 && o.kernel != 1 && l <= tc_max_l(q)) {
      TcOptions to;
      to.form = o.kernel >= 2 && o.kernel <= 5 ? o.kernel : 0;
      to.group = o.variant;
      return launch_tc(q, m, l, n, A, B, C, s, to);
    }
    return launch_mma(q, m, l, n, A, B, C, o.chunk, s);
  }
  return launch_m4rm(q, m, l, n, A, B, C, o.k, o.variant, kernel, s);
}

int strassen(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
             const ProdOptions &o, cudaStream_t s) {
  const int P = planes_of(q);
  const int64_t hm = m / 2, hl = l / 2, hn = n / 2;
  const int64_t qa = P * hm * fq_pitch_words(hl), qb = P * hl * fq_pitch_words(hn), qc = P * hm * fq_pitch_words(hn);
  // scratch: A11 A12 A21 A22, S1..S4 | B11 B12 B21 B22, T1..T4 | P1..P7
  void *mem = nullptr;
  if (int rc = scratch_alloc(&mem, size_t(8 * qa + 8 * qb + 7 * qc) * 8u, s)) return rc;
  uint64_t *ws = static_cast<uint64_t *>(mem);
  uint64_t *a[4], *S[4], *b[4], *T[4], *Pp[7];
  for (int i = 0; i < 4; ++i) {
    a[i] = ws + i * qa;
    S[i] = ws + (4 + i) * qa;
    b[i] = ws + 8 * qa + i * qb;
    T[i] = ws + 8 * qa + (4 + i) * qb;
  }
  for (int i = 0; i < 7; ++i) Pp[i] = ws + 8 * qa + 8 * qb + i * qc;
  ProdOptions child = o;
  if (o.strassen > 0) child.strassen = o.strassen == 1 ? -1 : o.strassen - 1;

  int rc = FQ_OK;
  auto add = [&](int64_t rows, int64_t cols, const uint64_t *x, const uint64_t *y, uint64_t *z, int sub) {
    if (rc == FQ_OK) rc = launch_add(q, rows, cols, x, y, z, sub, s);
  };
  auto mul = [&](const uint64_t *x, const uint64_t *y, uint64_t *z) {
    if (rc == FQ_OK) rc = product(q, hm, hl, hn, x, y, z, child, s);
  };
  for (int i = 0; i < 4 && rc == FQ_OK; ++i) rc = copy_quadrant(P, m, l, A, a[i], i / 2, i % 2, true, s);
  for (int i = 0; i < 4 && rc == FQ_OK; ++i) rc = copy_quadrant(P, l, n, B, b[i], i / 2, i % 2, true, s);
  // a = {A11, A12, A21, A22}, b = {B11, B12, B21, B22}
  add(hm, hl, a[2], a[3], S[0], 0);  // S1 = A21 + A22
  add(hm, hl, S[0], a[0], S[1], 1);  // S2 = S1 - A11
  add(hm, hl, a[0], a[2], S[2], 1);  // S3 = A11 - A21
  add(hm, hl, a[1], S[1], S[3], 1);  // S4 = A12 - S2
  add(hl, hn, b[1], b[0], T[0], 1);  // T1 = B12 - B11
  add(hl, hn, b[3], T[0], T[1], 1);  // T2 = B22 - T1
  add(hl, hn, b[3], b[1], T[2], 1);  // T3 = B22 - B12
  add(hl, hn, T[1], b[2], T[3], 1);  // T4 = T2 - B21
  mul(a[0], b[0], Pp[0]);            // P1 = A11 B11
  mul(a[1], b[2], Pp[1]);            // P2 = A12 B21
  mul(S[3], b[3], Pp[2]);            // P3 = S4 B22
  mul(a[3], T[3], Pp[3]);            // P4 = A22 T4
  mul(S[0], T[0], Pp[4]);            // P5 = S1 T1
  mul(S[1], T[1], Pp[5]);            // P6 = S2 T2
  mul(S[2], T[2], Pp[6]);            // P7 = S3 T3
  add(hm, hn, Pp[0], Pp[1], Pp[1], 0);  // C11 = P1 + P2            (in P2)
  add(hm, hn, Pp[0], Pp[5], Pp[5], 0);  // U2 = P1 + P6             (in P6)
  add(hm, hn, Pp[5], Pp[6], Pp[6], 0);  // U3 = U2 + P7             (in P7)
  add(hm, hn, Pp[6], Pp[4], Pp[0], 0);  // C22 = U3 + P5            (in P1)
  add(hm, hn, Pp[5], Pp[4], Pp[4], 0);  // U4 = U2 + P5             (in P5)
  add(hm, hn, Pp[4], Pp[2], Pp[2], 0);  // C12 = U4 + P3            (in P3)
  add(hm, hn, Pp[6], Pp[3], Pp[3], 1);  // C21 = U3 - P4            (in P4)
  uint64_t *cq[4] = {Pp[1], Pp[2], Pp[3], Pp[0]};  // C11, C12, C21, C22
  for (int i = 0; i < 4 && rc == FQ_OK; ++i) rc = copy_quadrant(P, m, n, C, cq[i], i / 2, i % 2, false, s);
  // F_5 and F_7 sums leave non-canonical codes; the direct kernels' outputs
  // are canonical, so reduce C's planes the same way.
  if (rc == FQ_OK && (q == 5 || q == 7)) rc = launch_canon(q, m, n, C, s);
  const int fr = scratch_free(mem, s);
  return rc ? rc : fr;
}

}  // namespace

int strassen_levels(int q, int64_t m, int64_t l, int64_t n, const ProdOptions &o, int sms) {
  if (!base_field(q) || o.strassen < 0 || o.path == FQ_PATH_KARATSUBA) return 0;
  if (o.strassen > 0) {
    int lv = 0;
    while (lv < o.strassen && splittable(m >> lv, l >> lv, n >> lv)) ++lv;
    return lv;
  }
  int lv = 0;
  best_cycles(q, m, l, n, o, sms, 4, &lv);
  return lv;
}

int product(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
            const ProdOptions &o, cudaStream_t s) {
  if (!base_field(q) || o.path == FQ_PATH_KARATSUBA) return launch_ext(q, m, l, n, A, B, C, o, s);
  int dev = 0, sms = 0;
  FQ_CUDA_TRY(cudaGetDevice(&dev));
  FQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // with strassen = 0 the time model decides again at every level
  if (m > 0 && n > 0 && l > 0 && strassen_levels(q, m, l, n, o, sms) > 0) return strassen(q, m, l, n, A, B, C, o, s);
  return direct(q, m, l, n, A, B, C, o, sms, s);
}

}  // namespace fqk

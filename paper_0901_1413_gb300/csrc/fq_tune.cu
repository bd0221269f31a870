// Measured autotuning of fq_matmul: time every compiled Four-Russians kernel of
// the field and the tensor-core path on the caller's operands, keep the
// fastest per (q, m, l, n), and let FQ_PATH_AUTO calls of that shape use it.
#include <array>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <exception>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fq_common.cuh"
#include "fq_internal.h"

namespace fqk {

namespace {

struct Choice {
  int path;    // FQ_PATH_M4RM or FQ_PATH_MMA
  int kernel;  // 1-based compiled kernel for M4RM, 0 for the planner
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t>, Choice> g_tuned;

}  // namespace

bool tuned_choice(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(q, m, l, n));
  if (it == g_tuned.end()) return false;
  *path = it->second.path;
  *kernel = it->second.kernel;
  return true;
}

// Modelled time (SM cycles) of the planner's M4RM choice: per wave of one
// CTA per SM and per block of k columns of A, the larger of the table build
// (the producer warps of the F_3 and GF(4) kernels build the next table while
// the consumers look up the current one) and the lookups (a fixed part plus a
// part per row of the tile), plus a constant for launch and the last store.
// The constants are fitted to GB300 measurements of the compiled kernels.
double m4rm_estimate(int q, int64_t m, int64_t l, int64_t n, int sms) {
  double fixed = 300.0, per_row = 2.9, build = 1700.0, hand_off = 0.0;
  if (q == 2) {  // warp-specialised kernels, one 128-byte gather per row and block
    hand_off = 700.0;  // producer/consumer hand-off per block, whatever k
    fixed = 300.0;
    per_row = 1.0;
    build = 0.0;
  } else if (q == 5) {
    fixed = 1500.0;
    per_row = 26.0;
    build = 0.0;
  } else if (q == 7) {
    fixed = 1200.0;
    per_row = 21.6;
    build = 0.0;
  }
  int nv = 0;
  const Variant *vs = m4rm_variants(q, &nv);
  double best = 1e300;
  for (int i = 0; i < nv; ++i) {
    const int64_t rows = int64_t(vs[i].rs) * vs[i].rows_per_slot;
    const int64_t ctas = cdiv(m, rows) * (fq_pitch_words(n) / (vs[i].cols / 64));
    const double scale = double(1 << vs[i].k) / 256.0;
    const double lookups = hand_off + fixed * scale + per_row * double(rows < m ? rows : m);
    const double per_block = lookups > build * scale ? lookups : build * scale;
    const double t = double(cdiv(ctas, sms)) * double(cdiv(l, vs[i].k)) * per_block;
    best = t < best ? t : best;
  }
  return best + 20000.0;
}

// ---- the cache as JSON: {"format": "fq-autotune-1", "entries": [[q, m, l, n, path, kernel], ...]}

constexpr const char *kTuneFormat = "fq-autotune-1";

// A small reader for exactly that document (whitespace anywhere, keys in any
// order, other keys refused): fills `out` or returns false.
struct TuneReader {
  const std::string &t;
  size_t i = 0;
  explicit TuneReader(const std::string &text) : t(text) {}
  void ws() {
    while (i < t.size() && isspace(static_cast<unsigned char>(t[i]))) ++i;
  }
  bool lit(char c) {
    ws();
    if (i < t.size() && t[i] == c) {
      ++i;
      return true;
    }
    return false;
  }
  bool str(std::string *out) {
    if (!lit('"')) return false;
    out->clear();
    while (i < t.size() && t[i] != '"') {
      if (t[i] == '\\' || static_cast<unsigned char>(t[i]) < 0x20) return false;  // no escapes needed
      out->push_back(t[i++]);
    }
    if (i >= t.size()) return false;
    ++i;
    return true;
  }
  bool integer(int64_t *out) {
    ws();
    const size_t b = i;
    if (i < t.size() && t[i] == '-') ++i;
    while (i < t.size() && isdigit(static_cast<unsigned char>(t[i]))) ++i;
    if (i == b || (i == b + 1 && t[b] == '-') || i - b > 19) return false;
    *out = strtoll(t.c_str() + b, nullptr, 10);
    return true;
  }
  bool entries(std::vector<std::array<int64_t, 6>> *out) {
    if (!lit('[')) return false;
    if (lit(']')) return true;
    do {
      std::array<int64_t, 6> e{};
      if (!lit('[')) return false;
      for (int k = 0; k < 6; ++k)
        if ((k > 0 && !lit(',')) || !integer(&e[size_t(k)])) return false;
      if (!lit(']')) return false;
      out->push_back(e);
    } while (lit(','));
    return lit(']');
  }
  bool document(std::vector<std::array<int64_t, 6>> *out) {
    bool have_format = false, have_entries = false;
    if (!lit('{')) return false;
    do {
      std::string key;
      if (!str(&key) || !lit(':')) return false;
      if (key == "format" && !have_format) {
        std::string v;
        if (!str(&v) || v != kTuneFormat) return false;
        have_format = true;
      } else if (key == "entries" && !have_entries) {
        if (!entries(out)) return false;
        have_entries = true;
      } else {
        return false;
      }
    } while (lit(','));
    if (!lit('}')) return false;
    ws();
    return have_format && have_entries && i == t.size();
  }
};

// A remembered choice the library can honour: a field with kernels, sizes >= 0,
// the M4RM path with a compiled kernel (or the planner) or the tensor-core path.
bool valid_entry(const std::array<int64_t, 6> &e) {
  const int64_t q = e[0], path = e[4], kernel = e[5];
  if (!(q == 2 || q == 3 || q == 4 || q == 5 || q == 7) || e[1] < 0 || e[2] < 0 || e[3] < 0) return false;
  if (path == FQ_PATH_MMA) return kernel == 0;
  if (path != FQ_PATH_M4RM) return false;
  int nv = 0;
  m4rm_variants(int(q), &nv);
  return kernel >= 0 && kernel <= nv;
}

}  // namespace fqk

extern "C" {

int fq_autotune_save(const char *path) {
  if (!path) return FQ_EINVAL;
  try {
    std::string text = std::string("{\"format\": \"") + fqk::kTuneFormat + "\", \"entries\": [";
    {
      std::lock_guard<std::mutex> lock(fqk::g_tune_mu);
      bool first = true;
      for (const auto &kv : fqk::g_tuned) {
        char line[160];
        snprintf(line, sizeof(line), "%s\n  [%d, %lld, %lld, %lld, %d, %d]", first ? "" : ",", std::get<0>(kv.first),
                 static_cast<long long>(std::get<1>(kv.first)), static_cast<long long>(std::get<2>(kv.first)),
                 static_cast<long long>(std::get<3>(kv.first)), kv.second.path, kv.second.kernel);
        text += line;
        first = false;
      }
    }
    text += "\n]}\n";
    FILE *f = fopen(path, "wb");
    if (!f) return FQ_EINVAL;
    const bool ok = fwrite(text.data(), 1, text.size(), f) == text.size();
    return (fclose(f) == 0 && ok) ? FQ_OK : FQ_EINVAL;
  } catch (const std::exception &) {
    return FQ_ENOMEM;
  }
}

int fq_autotune_load(const char *path) {
  if (!path) return FQ_EINVAL;
  try {
    FILE *f = fopen(path, "rb");
    if (!f) return FQ_EINVAL;
    std::string text;
    char buf[4096];
    size_t got = 0;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    const bool read_ok = ferror(f) == 0;
    fclose(f);
    if (!read_ok) return FQ_EINVAL;
    std::vector<std::array<int64_t, 6>> entries;
    fqk::TuneReader reader(text);
    if (!reader.document(&entries)) return FQ_EINVAL;
    for (const auto &e : entries)
      if (!fqk::valid_entry(e)) return FQ_EINVAL;
    std::lock_guard<std::mutex> lock(fqk::g_tune_mu);
    for (const auto &e : entries)
      fqk::g_tuned[std::make_tuple(int(e[0]), e[1], e[2], e[3])] = fqk::Choice{int(e[4]), int(e[5])};
    return FQ_OK;
  } catch (const std::exception &) {
    return FQ_ENOMEM;
  }
}

int fq_autotune(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                void *stream, fq_tune_result *out) {
  if (!(q == 2 || q == 3 || q == 4 || q == 5 || q == 7) || m <= 0 || l <= 0 || n <= 0 || !A || !B || !C) return FQ_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nk = 0;
  fqk::m4rm_variants(q, &nk);
  cudaEvent_t e0, e1;
  FQ_CUDA_TRY(cudaEventCreate(&e0));
  if (const cudaError_t e = cudaEventCreate(&e1); e != cudaSuccess) {
    cudaEventDestroy(e0);
    return fqk::record_cuda_error(e);
  }
  fq_tune_result best{};
  best.ms = -1.0f;
  int rc = FQ_OK;
  // candidates: 0 = M4RM planner, 1..nk = compiled M4RM kernels, nk + 1 = MMA
  for (int c = 0; c <= nk + 1 && rc == FQ_OK; ++c) {
    fq_options o{};
    o.path = c == nk + 1 ? FQ_PATH_MMA : FQ_PATH_M4RM;
    o.kernel = (c >= 1 && c <= nk) ? c : 0;
    int r = fq_matmul_ex(q, m, l, n, A, B, C, stream, &o);  // warm-up (and applicability)
    if (r == FQ_ENOTSUP || r == FQ_EINVAL) continue;
    if (r != FQ_OK) {
      rc = r;
      break;
    }
    float ms = 0.0f;
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      if ((r = fq_matmul_ex(q, m, l, n, A, B, C, stream, &o)) != FQ_OK) {
        rc = r;
        break;
      }
      e = cudaEventRecord(e1, s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = fqk::record_cuda_error(e);
      break;
    }
    if (c == 0) best.ms_planner = ms;
    if (c == nk + 1) best.ms_mma = ms;
    if (best.ms < 0 || ms < best.ms) {
      best.ms = ms;
      best.path = o.path;
      best.kernel = o.kernel;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != FQ_OK) return rc;
  if (best.ms < 0) return FQ_ENOTSUP;
  try {
    std::lock_guard<std::mutex> lock(fqk::g_tune_mu);
    fqk::g_tuned[std::make_tuple(q, m, l, n)] = fqk::Choice{best.path, best.kernel};
  } catch (const std::exception &) {
    return FQ_ENOMEM;  // the cache could not grow (or its lock failed); nothing remembered
  }
  if (out) *out = best;
  return FQ_OK;
}

int fq_autotune_lookup(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel) {
  int p = 0, k = 0;
  if (!fqk::tuned_choice(q, m, l, n, &p, &k)) return FQ_ENOTSUP;
  if (path) *path = p;
  if (kernel) *kernel = k;
  return FQ_OK;
}

int fq_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(fqk::g_tune_mu);
  fqk::g_tuned.clear();
  return FQ_OK;
}

}  // extern "C"

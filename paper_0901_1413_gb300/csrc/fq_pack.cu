// Packing residues into bit-planes and back (Section 3, codes of Section 4; the
// extension fields' coefficient planes of Section 4.3), and elementwise
// bitsliced add/sub over the base fields and GF(4).  All three are bandwidth-bound: one thread per
// 64-element word of a row, grid-stride over rows x pitch.
#include "fq_codes.cuh"
#include "fq_fields.cuh"
#include "fq_internal.h"

namespace fqk {

namespace {

template <int Q, int P>
__global__ void pack_kernel(int64_t rows, int64_t cols, const uint8_t *__restrict__ res, int64_t ld,
                            uint64_t *__restrict__ planes, int64_t pitch, unsigned *err, int vec16) {
  const int64_t total = rows * pitch;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / pitch;
    const int64_t w = i - r * pitch;
    const int64_t c0 = w * 64;
    uint64_t out[P];
#pragma unroll
    for (int p = 0; p < P; ++p) out[p] = 0;
    uint32_t bad = 0;
    if (c0 < cols) {
      const uint8_t *src = res + r * ld + c0;
      const int cnt = int(cols - c0 < 64 ? cols - c0 : 64);
      if (vec16 && cnt == 64) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint4 v = __ldg(s4 + j);
          encode4<Q, P>(v.x, out, 16 * j + 0, bad);
          encode4<Q, P>(v.y, out, 16 * j + 4, bad);
          encode4<Q, P>(v.z, out, 16 * j + 8, bad);
          encode4<Q, P>(v.w, out, 16 * j + 12, bad);
        }
      } else {
        for (int e = 0; e < cnt; e += 4) {
          uint32_t v = 0;
          for (int b = 0; b < 4 && e + b < cnt; ++b) v |= uint32_t(src[e + b]) << (8 * b);
          encode4<Q, P>(v, out, e, bad);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) planes[(p * rows + r) * pitch + w] = out[p];
    if (bad) record_error(err, FQ_EVALUE);
  }
}

template <int Q, int P>
__global__ void unpack_kernel(int64_t rows, int64_t cols, const uint64_t *__restrict__ planes, int64_t pitch,
                              uint8_t *__restrict__ res, int64_t ld, int vec16) {
  const int64_t words = (cols + 63) / 64;
  const int64_t total = rows * words;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / words;
    const int64_t w = i - r * words;
    uint64_t in[P];
#pragma unroll
    for (int p = 0; p < P; ++p) in[p] = __ldg(planes + (p * rows + r) * pitch + w);
    const int64_t c0 = w * 64;
    uint8_t *dst = res + r * ld + c0;
    const int cnt = int(cols - c0 < 64 ? cols - c0 : 64);
    if (vec16 && cnt == 64) {
      uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint4 v;
        v.x = decode4<Q, P>(in, 16 * j + 0);
        v.y = decode4<Q, P>(in, 16 * j + 4);
        v.z = decode4<Q, P>(in, 16 * j + 8);
        v.w = decode4<Q, P>(in, 16 * j + 12);
        d4[j] = v;
      }
    } else {
      for (int e = 0; e < cnt; e += 4) {
        const uint32_t v = decode4<Q, P>(in, e);
        for (int b = 0; b < 4 && e + b < cnt; ++b) dst[e + b] = uint8_t(v >> (8 * b));
      }
    }
  }
}

// Extension fields F_{p^n}: code c = sum_j c_j p^j; coefficient j's planes are
// those of a packed F_p matrix (planes j P_p .. (j + 1) P_p - 1).  One element at
// a time: packing is outside the product.
template <int PB>
__host__ __device__ constexpr int base_planes() { return PB == 2 ? 1 : (PB == 3 ? 2 : 3); }

template <int PB, int N>
__global__ void ext_pack_kernel(int64_t rows, int64_t cols, const uint8_t *__restrict__ res, int64_t ld,
                                uint64_t *__restrict__ planes, int64_t pitch, unsigned *err) {
  constexpr int PP = base_planes<PB>();
  constexpr int Q = PB * PB * (N == 3 ? PB : 1);
  const int64_t total = rows * pitch;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / pitch;
    const int64_t w = i - r * pitch;
    const int64_t c0 = w * 64;
    uint64_t out[N][PP];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int p = 0; p < PP; ++p) out[j][p] = 0;
    bool bad = false;
    if (c0 < cols) {
      const uint8_t *src = res + r * ld + c0;
      const int cnt = int(cols - c0 < 64 ? cols - c0 : 64);
      for (int e = 0; e < cnt; ++e) {
        unsigned v = src[e];
        if (v >= unsigned(Q)) {
          bad = true;
          v = 0;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const unsigned d = v % PB;
          v /= PB;
          if constexpr (PB == 3) {             // unit, sign (Section 4.1)
            out[j][0] |= uint64_t(d != 0) << e;
            out[j][1] |= uint64_t(d == 2) << e;
          } else {
#pragma unroll
            for (int p = 0; p < PP; ++p) out[j][p] |= uint64_t((d >> p) & 1u) << e;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int p = 0; p < PP; ++p) planes[((j * PP + p) * rows + r) * pitch + w] = out[j][p];
    if (bad) record_error(err, FQ_EVALUE);
  }
}

template <int PB, int N>
__global__ void ext_unpack_kernel(int64_t rows, int64_t cols, const uint64_t *__restrict__ planes, int64_t pitch,
                                  uint8_t *__restrict__ res, int64_t ld) {
  constexpr int PP = base_planes<PB>();
  const int64_t words = (cols + 63) / 64;
  const int64_t total = rows * words;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / words;
    const int64_t w = i - r * words;
    uint64_t in[N][PP];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int p = 0; p < PP; ++p) in[j][p] = __ldg(planes + ((j * PP + p) * rows + r) * pitch + w);
    const int64_t c0 = w * 64;
    uint8_t *dst = res + r * ld + c0;
    const int cnt = int(cols - c0 < 64 ? cols - c0 : 64);
    for (int e = 0; e < cnt; ++e) {
      unsigned v = 0;
#pragma unroll
      for (int j = N - 1; j >= 0; --j) {
        unsigned d;
        if constexpr (PB == 3) {
          const unsigned unit = unsigned(in[j][0] >> e) & 1u, sign = unsigned(in[j][1] >> e) & 1u;
          d = unit + (unit & sign);
        } else {
          d = 0;
#pragma unroll
          for (int p = 0; p < PP; ++p) d |= (unsigned(in[j][p] >> e) & 1u) << p;
          d = d >= unsigned(PB) ? d - PB : d;    // F_5, F_7 codes read mod p
        }
        v = v * PB + d;
      }
      dst[e] = uint8_t(v);
    }
  }
}

template <class F>
__global__ void add_kernel(int64_t rows, int64_t pitch, const uint64_t *X, const uint64_t *Y, uint64_t *Z,
                           int sub) {
  constexpr int P = F::P;
  const int64_t total = rows * pitch;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    uint32_t lo[P], hi[P], ylo[P], yhi[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t x = X[p * total + i], y = Y[p * total + i];
      lo[p] = uint32_t(x);
      hi[p] = uint32_t(x >> 32);
      ylo[p] = uint32_t(y);
      yhi[p] = uint32_t(y >> 32);
    }
    if (sub) {
      F::sub(lo, ylo);
      F::sub(hi, yhi);
    } else {
      F::add(lo, ylo);
      F::add(hi, yhi);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) Z[p * total + i] = uint64_t(lo[p]) | (uint64_t(hi[p]) << 32);
  }
}

template <class F>
__global__ void canon_kernel(int64_t total, uint64_t *Z) {
  constexpr int P = F::P;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    uint32_t lo[P], hi[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t z = Z[p * total + i];
      lo[p] = uint32_t(z);
      hi[p] = uint32_t(z >> 32);
    }
    F::canon(lo);
    F::canon(hi);
#pragma unroll
    for (int p = 0; p < P; ++p) Z[p * total + i] = uint64_t(lo[p]) | (uint64_t(hi[p]) << 32);
  }
}

inline int grid_for(int64_t total, int threads) {
  const int64_t want = cdiv(total, threads);
  const int64_t cap = 152 * 32;
  return int(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

int launch_pack(int q, int64_t rows, int64_t cols, const uint8_t *res, int64_t ld, uint64_t *planes,
                cudaStream_t s) {
  unsigned *err = nullptr;
  if (int rc = status_word(&err)) return rc;
  const int64_t pitch = fq_pitch_words(cols);
  const int64_t total = rows * pitch;
  if (total == 0) return FQ_OK;
  const int vec16 = (reinterpret_cast<uintptr_t>(res) % 16 == 0) && (ld % 16 == 0);
  const int th = 256, gr = grid_for(total, th);
  switch (q) {
    case 2: pack_kernel<2, 1><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err, vec16); break;
    case 3: pack_kernel<3, 2><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err, vec16); break;
    case 4: pack_kernel<4, 2><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err, vec16); break;
    case 5: pack_kernel<5, 3><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err, vec16); break;
    case 7: pack_kernel<7, 3><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err, vec16); break;
    case 8: ext_pack_kernel<2, 3><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err); break;
    case 9: ext_pack_kernel<3, 2><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err); break;
    case 25: ext_pack_kernel<5, 2><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err); break;
    case 27: ext_pack_kernel<3, 3><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err); break;
    case 49: ext_pack_kernel<7, 2><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err); break;
    case 125: ext_pack_kernel<5, 3><<<gr, th, 0, s>>>(rows, cols, res, ld, planes, pitch, err); break;
    default: return FQ_EINVAL;
  }
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

int launch_unpack(int q, int64_t rows, int64_t cols, const uint64_t *planes, uint8_t *res, int64_t ld,
                  cudaStream_t s) {
  const int64_t pitch = fq_pitch_words(cols);
  const int64_t total = rows * cdiv(cols, 64);
  if (total == 0) return FQ_OK;
  const int vec16 = (reinterpret_cast<uintptr_t>(res) % 16 == 0) && (ld % 16 == 0);
  const int th = 256, gr = grid_for(total, th);
  switch (q) {
    case 2: unpack_kernel<2, 1><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld, vec16); break;
    case 3: unpack_kernel<3, 2><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld, vec16); break;
    case 4: unpack_kernel<4, 2><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld, vec16); break;
    case 5: unpack_kernel<5, 3><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld, vec16); break;
    case 7: unpack_kernel<7, 3><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld, vec16); break;
    case 8: ext_unpack_kernel<2, 3><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld); break;
    case 9: ext_unpack_kernel<3, 2><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld); break;
    case 25: ext_unpack_kernel<5, 2><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld); break;
    case 27: ext_unpack_kernel<3, 3><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld); break;
    case 49: ext_unpack_kernel<7, 2><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld); break;
    case 125: ext_unpack_kernel<5, 3><<<gr, th, 0, s>>>(rows, cols, planes, pitch, res, ld); break;
    default: return FQ_EINVAL;
  }
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

int launch_add(int q, int64_t rows, int64_t cols, const uint64_t *X, const uint64_t *Y, uint64_t *Z, int sub,
               cudaStream_t s) {
  const int64_t pitch = fq_pitch_words(cols);
  const int64_t total = rows * pitch;
  if (total == 0) return FQ_OK;
  const int th = 256, gr = grid_for(total, th);
  switch (q) {
    case 2: add_kernel<F2><<<gr, th, 0, s>>>(rows, pitch, X, Y, Z, sub); break;
    case 3: add_kernel<F3><<<gr, th, 0, s>>>(rows, pitch, X, Y, Z, sub); break;
    case 4: add_kernel<GF4><<<gr, th, 0, s>>>(rows, pitch, X, Y, Z, sub); break;
    case 5: add_kernel<F5><<<gr, th, 0, s>>>(rows, pitch, X, Y, Z, sub); break;
    case 7: add_kernel<F7><<<gr, th, 0, s>>>(rows, pitch, X, Y, Z, sub); break;
    default: return FQ_EINVAL;
  }
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

int launch_canon(int q, int64_t rows, int64_t cols, uint64_t *Z, cudaStream_t s) {
  const int64_t total = rows * fq_pitch_words(cols);
  if (total == 0) return FQ_OK;
  const int th = 256, gr = grid_for(total, th);
  switch (q) {
    case 5: canon_kernel<F5><<<gr, th, 0, s>>>(total, Z); break;
    case 7: canon_kernel<F7><<<gr, th, 0, s>>>(total, Z); break;
    default: return FQ_OK;  // F_2, F_3 and GF(4) codes are unique
  }
  FQ_LAUNCH_CHECK();
  return FQ_OK;
}

}  // namespace fqk

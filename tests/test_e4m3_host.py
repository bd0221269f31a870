"""The plane-word to e4m3 conversion of the tensor-core operands (e4m3x32
and its 16-element form e4m3x16 in csrc/fq_e4m3.cuh), built for the host
with nvcc and checked on the CPU byte for byte against PyTorch's own e4m3
conversion of each element's balanced value.  The element codes are those of the library's planes (Sections 4.1
and 4.2): F_3 unit | sign << 1, F_5 and F_7 a 3-bit code read mod p, and F_2
(each F_2 product of GF(4)) one bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_0901_1413_gb300", "csrc", "fq_e4m3.cuh")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
PLANES = {2: 1, 3: 2, 5: 3, 7: 3}

HARNESS = r"""
#include <cstdio>
#include "%s"
template <int Q, int P>
void run(int words) {
  for (int i = 0; i < words; ++i) {
    uint32_t t[P];
    for (int p = 0; p < P; ++p) if (std::scanf("%%x", &t[p]) != 1) return;
    uint4 lo, hi;
    fqk::e4m3x32<Q, P>(t, lo, hi);
    const uint4 h0 = fqk::e4m3x16<Q, P>(t, 0), h1 = fqk::e4m3x16<Q, P>(t, 1);
    std::printf("%%08x %%08x %%08x %%08x %%08x %%08x %%08x %%08x ", lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w);
    std::printf("%%08x %%08x %%08x %%08x %%08x %%08x %%08x %%08x\n", h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w);
  }
}
int main() {
  int q = 0, words = 0;
  if (std::scanf("%%d %%d", &q, &words) != 2) return 1;
  if (q == 2) run<2, 1>(words);
  if (q == 3) run<3, 2>(words);
  if (q == 5) run<5, 3>(words);
  if (q == 7) run<7, 3>(words);
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if not (os.path.exists(NVCC) or shutil.which("nvcc")):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("e4m3")
    src, exe = d / "h.cu", d / "h"
    src.write_text(HARNESS % HEADER)
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), str(src)], check=True, capture_output=True)
    return str(exe)


def balanced(q, code):
    """An element's balanced value from its code (the plane bits, plane 0 lowest)."""
    if q == 2:
        return code & 1
    if q == 3:
        return {0: 0, 1: 1, 2: 0, 3: -1}[code]
    r = code % q
    return r - q if r > q // 2 else r


@pytest.mark.parametrize("q", (2, 3, 5, 7))
def test_e4m3x32_matches_the_e4m3_format(harness, q):
    """Random words, so that every code sits at every one of the 32 element
    positions many times: each output byte is the e4m3 encoding of the
    element's balanced value (F_3's unused code 2, a sign without a unit,
    gives -0, which adds nothing to a product)."""
    P, words = PLANES[q], 4096
    rng = np.random.default_rng(q)
    t = rng.integers(0, 1 << 32, size=(words, P), dtype=np.uint64)
    t[0] = 0
    t[1] = 0xFFFFFFFF
    text = "%d %d\n" % (q, words) + "\n".join(" ".join("%x" % int(v) for v in row) for row in t)
    out = subprocess.run([harness], input=text, capture_output=True, text=True, check=True).stdout.split()
    got = np.array([int(x, 16) for x in out], dtype=np.uint64).reshape(words, 2, 8)
    got_bytes = got.astype("<u4").view(np.uint8).reshape(words, 2, 32)
    bits = (t[:, :, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)        # words x P x 32
    codes = sum(bits[:, p, :].astype(np.int64) << p for p in range(P))              # words x 32
    table = torch.tensor([float(balanced(q, c)) for c in range(1 << P)])
    want_of_code = table.to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    if q == 3:
        want_of_code[2] = 0x80
    assert np.array_equal(got_bytes[:, 0], want_of_code[codes])      # 32 elements at once
    assert np.array_equal(got_bytes[:, 1], want_of_code[codes])      # the two 16-element halves

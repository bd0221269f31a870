"""Host-side helpers of bench.py: the kernel-source digest that keys recorded
ncu counters (a stale record reads as null traffic), the second roofline
denominator, and the conversion's byte count (no GPU)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_digest_ignores_comments_but_not_code(tmp_path):
    bench = _bench()
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n  return x + 1;  // one\n}\n")
    base = bench.sources_digest([str(a)])
    a.write_text("// a new header\nint f(int x) {\n\n  return x + 1;  /* still one */\n}\n")
    assert bench.sources_digest([str(a)]) == base
    a.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.sources_digest([str(a)]) != base


def test_pipe_peak_denominator():
    bench = _bench()
    rec = bench.pipe_peak(4000.0, {"sm_mhz": 2000.0})
    assert abs(rec["peak"] - 16384 * 152 * 2000e6 / 1e12) < 1e-6
    assert abs(rec["frac"] - 4000.0 / rec["peak"]) < 1e-12
    assert bench.pipe_peak(1.0, None)["sm_mhz"] == 2070.0


def test_prepare_bytes_counts_planes_in_and_e4m3_out():
    bench = _bench()
    # 8192^3 F_3: planes of A and B (2 planes x 8192 rows x 128 words x 8 bytes
    # each) read, A and B^T (8192 x 8192 bytes each) written
    assert bench.prepare_bytes(8192, 8192, 8192) == 2 * (2 * 8192 * 128 * 8) + 2 * 8192 * 8192
    # ragged: l rounded up to 128, n's rows of B^T to the 1024-column pitch
    assert bench.prepare_bytes(100, 200, 300) == 2 * (100 * 16 + 200 * 16) * 8 + (100 + 1024) * 256


def test_prepare_bytes_fp4_form():
    bench = _bench()
    # form 5: packed e2m1, half a byte per element, l rounded up to 256
    assert bench.prepare_bytes(8192, 8192, 8192, 3, 5) == 2 * (2 * 8192 * 128 * 8) + 2 * 8192 * 4096
    assert bench.prepare_bytes(300, 2100, 300, 3, 5) == 2 * (300 * 48 + 2100 * 16) * 8 + (300 + 1024) * 1152
    assert bench.prepare_bytes(8192, 8192, 8192, 4, 5) == 3 * (2 * (2 * 8192 * 128 * 8) + 2 * 8192 * 4096)


def test_tc_roofline_per_form():
    bench = _bench()
    peaks = {"fp8": 3000.0, "fp4": 9000.0, "note_fp8": "x2", "note_fp4": "x6"}
    r4 = bench.tc_roofline(peaks, 5, 4500.0, {"sm_mhz": 2000.0})
    assert r4["frac"] == 0.5 and r4["operands"] == "fp4" and "mxf4" in r4["kernel"]
    assert abs(r4["pipe"]["peak"] - 32768 * 152 * 2000e6 / 1e12) < 1e-6
    r8 = bench.tc_roofline(peaks, 4, 1500.0, {"sm_mhz": 2000.0})
    assert r8["frac"] == 0.5 and r8["operands"] == "fp8"
    assert abs(r8["pipe"]["peak"] - 16384 * 152 * 2000e6 / 1e12) < 1e-6


def test_prepare_bytes_other_fields():
    bench = _bench()
    # F_5 / F_7: three planes read; GF(4): three rounds (one per F_2 product)
    # of both planes read and e4m3 written
    assert bench.prepare_bytes(8192, 8192, 8192, q=5) == 3 * (2 * 8192 * 128 * 8) + 2 * 8192 * 8192
    assert bench.prepare_bytes(8192, 8192, 8192, q=4) == 3 * (2 * (2 * 8192 * 128 * 8) + 2 * 8192 * 8192)
    assert bench.tensor_flops(4, 2, 3, 5) == 3 * 60.0 and bench.tensor_flops(7, 2, 3, 5) == 60.0


def test_algorithmic_lop3_counts():
    bench = _bench()
    # F_3 at k = 8: ceil(l/8) blocks x ceil(n/32) words x (8 LOP3 per row + 4 per table entry)
    assert bench.algorithmic_lop3(64, 16, 64, 8) == 2 * 2 * (64 * 8 + 255 * 4)
    assert bench.algorithmic_lop3(64, 16, 64, 8, q=3) == bench.algorithmic_lop3(64, 16, 64, 8)
    # ragged: l = 17 needs three blocks, n = 33 two words
    assert bench.algorithmic_lop3(1, 17, 33, 8, q=5) == 3 * 2 * (30 + 255 * 11)
    assert bench.algorithmic_lop3(10, 7, 32, 7, q=7) == 1 * 1 * (10 * 22 + 127 * 10)
    assert bench.algorithmic_lop3(10, 7, 32, 7, q=4) == 10 * 3 + 127 * 2


def test_batched_compulsory_bytes():
    bench = _bench()
    # one F_3 product 100 x 200 x 300: la = 256, nr = 512; planes of A over la
    # columns and of B over nr columns read (2 bits per element), C's two
    # planes of 100 rows x 16 words written
    assert bench.batched_compulsory_bytes(3, [(100, 200, 300)]) == 2 * (100 * 256 + 200 * 512) // 8 + 2 * 100 * 16 * 8
    assert bench.batched_compulsory_bytes(5, [(64, 128, 256)] * 2) == 2 * (3 * (64 * 128 + 128 * 256) // 8
                                                                          + 3 * 64 * 16 * 8)

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

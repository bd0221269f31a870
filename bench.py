#!/usr/bin/env python
"""Throughput of exact F_q matrix products on GB300: one JSON line on stdout.

Workload (one step): the F_3 square products n = 4096, 8192 and 16384 with
entries uniform on {0, 1, 2}, and n = 8192 with A 90% zeros (i.i.d.).
Metric: field operations per second, 2 m l n / t (the paper's normalisation
against the classical product's work).

* ``value``: packed inputs resident in HBM, device time (CUDA events on the
  launching stream), L2 flushed before every step; each product runs in the
  form FQ_PATH_AUTO takes for its shape (for these F_3 shapes the tcgen05
  tensor-core form from packed e2m1 operands on SM pairs: operand
  conversion, then the product kernel).
* ``m4rm``: the same products by the plain bitsliced Four-Russians path, with
  ``speedup_vs_m4rm`` the factor between the two.
* ``e2e``: the same products through the public API from pinned host residues:
  host->device copy, fq_pack, fq_matmul, fq_unpack, device->host copy (bound
  by the host link: 1 byte per element up, about 210 GB/s on GB300).
* ``e2e_packed``: the same with the host holding the library's bit-planes
  (the paper's representation): planes up, fq_matmul, C's planes down.
* ``roofline``: the dominant kernel, the tcgen05 product, at 2 m l n flops
  per launch over its own event time, against the dense peak of its operand
  type: the measured cuBLAS bf16 burst times the nominal ratio (fp4 13.5 /
  2.25 = 6, fp8 4.5 / 2.25 = 2), and beside it the instruction kind's own
  pipe rate (fp4 kind::mxf4 32768, fp8 16384 ops/clk/SM, measured by the
  microbenchmark) at the sampled SM clock;
  ``prepare``: the operand conversion's bytes over its time, against the
  measured HBM copy bandwidth;
  ``m4rm.roofline``: the M4RM kernels against the integer-logic (LOP3) issue
  rate (the algorithmic LOP3 of every M4RM launch over the products' time).
* ``batched``: 4096 independent products over F_3 and over F_5 (m, l, n
  uniform over multiples of 64 in [64, 1024]) in one graph-captured launch
  sequence: products/s and 2mln/s for the FQ_PATH_AUTO plan and for the
  Four-Russians-only plan; the AUTO plan's stages timed one by one, with the
  persistent tcgen05 kernel (conversion and tiles in one launch) against the
  fp8 peak and against HBM.
* ``more_workloads``: F_5, F_7 and GF(4) at n = 8192, then F_5 32768^3 and F_3
  65536 x 4096 x 4096, each product on both paths (the tcgen05 form as
  conversion + product kernel, the Four-Russians path), each with its
  roofline (fp8 tensor peak, HBM, LOP3 issue rate) and the two results
  compared bit for bit.
* ``pack_unpack``: fq_pack of the step's operands and fq_unpack of its results,
  timed apart from the product (the metric excludes them).
* ``cpu_baseline``: the CPU oracle on a bounded sample of rows of the same
  products, all host cores (and single-threaded on a smaller sample), with
  the host CPU's model.

``--impl reference`` times the oracle alone (the reference arm).  Under
torchrun with N > 1 ranks every rank runs the whole workload on its own GPU
(independent replicas, weak scaling) and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "F_q matmul 2mln/s: bitsliced M4RM vs INT8-TC path; batched products/s"
UNIT = "field-ops/s (2mln/t)"
Q = 3
# (m, l, n, A law)
PRODUCTS = [(4096, 4096, 4096, "uniform"), (8192, 8192, 8192, "uniform"),
            (16384, 16384, 16384, "uniform"), (8192, 8192, 8192, "sparse90")]
WORKLOAD = "F_3 square products n=4096, 8192, 16384 uniform + n=8192 with A 90% zeros"

# The other workloads, each product timed on both paths: F_5, F_7 and GF(4) at
# n = 8192; the large F_5 32768^3 and F_3 65536 x 4096 x 4096.
MORE_WORKLOADS = [
    ("F_5, F_7 and GF(4) square products n=8192 uniform",
     [(5, 8192, 8192, 8192), (7, 8192, 8192, 8192), (4, 8192, 8192, 8192)]),
    ("large: F_5 square n=32768 and F_3 65536 x 4096 x 4096, uniform",
     [(5, 32768, 32768, 32768), (3, 65536, 4096, 4096)]),
]

# Integer-logic issue rate: 64 LOP3 lane-ops per clock per SM (the ALU pipe;
# measured 63.99 on this GPU), 152 SMs, 2070 MHz maximum SM clock.
ALU_PEAK_TLOPS = 64 * 152 * 2.070e9 / 1e12
# Algorithmic LOP3 lane-ops of the Four-Russians arithmetic per 32-column word:
# LOOKUP_LOP3 for one row and k-row block (its D lookups accumulated: F_3 an
# add and a subtract of four LOP3s each; GF(4) two three-input XORs and one
# XOR; F_7 two carry-save adders mod 7 and one add; F_5 two carry-save adders
# and an end-around add into a four-bit accumulator mod 15, folded once at the
# store), TABLE_LOP3 for one table entry (one bitsliced add: F_3 4, GF(4) 2,
# F_7 10, F_5 11).
LOOKUP_LOP3 = {3: 8, 4: 3, 5: 30, 7: 22}
TABLE_LOP3 = {3: 4, 4: 2, 5: 11, 7: 10}
PLANES = {2: 1, 3: 2, 4: 2, 5: 3, 7: 3}
L2_FLUSH_BYTES = 256 << 20


def cdiv(a, b):
    return -(-a // b)


# Launches of one F_3 tensor-core product: A's planes converted, B's planes
# converted to B^T, the tcgen05 product.
TC_LAUNCHES = 3

# The tcgen05 product forms (fq_tc_form): kernel, operand type, dense
# ops/clk/SM of the instruction kind (the microbenchmark's measured pipe
# rate), nominal peak as a multiple of the bf16 peak.
TC_FORMS = {
    2: ("tc_gemm_kernel (tcgen05.mma.cta_group::1 kind::f8f6f4, e4m3, single SMs, 128x256 tiles)", "fp8", 16384, 2.0),
    3: ("tc_gemm2_kernel (tcgen05.mma.cta_group::2 kind::f8f6f4, e4m3, SM pairs, 256x256 tiles)", "fp8", 16384, 2.0),
    4: ("tc_gemm2_kernel (tcgen05.mma.cta_group::2 kind::f8f6f4, e4m3, SM pairs, 256x512 tiles)", "fp8", 16384, 2.0),
    5: ("tc_gemm4_kernel (tcgen05.mma.cta_group::2 kind::mxf4, packed e2m1, block scales 1.0, SM pairs, "
        "256x448 tiles)", "fp4", 32768, 6.0),
}


def pitch_words(cols):
    return cdiv(max(cols, 1), 1024) * 16


def prepare_bytes(m, l, n, q=3, form=3):
    """Algorithmic DRAM bytes of the operand conversion: every plane of A and
    of B read, A and B^T written, e4m3 (one byte per element, la = l rounded up
    to 128) or, for form 5, packed e2m1 (half a byte, la = l rounded up to
    256) (GF(4): three rounds, one per F_2 product)."""
    if form == 5:
        la = cdiv(l, 256) * 256
        row = la // 2
    else:
        la = cdiv(l, 128) * 128
        row = la
    npad = pitch_words(n) * 64
    rounds = 3 if q == 4 else 1
    return rounds * (PLANES[q] * (m * pitch_words(l) + l * pitch_words(n)) * 8 + (m + npad) * row)


def tensor_flops(q, m, l, n):
    """Tensor-pipe work of one product: 2 m l n (three F_2 products for GF(4))."""
    return (3 if q == 4 else 1) * 2.0 * m * l * n


def algorithmic_lop3(m, l, n, k, q=3):
    """LOP3 lane-ops of one product by M4RM: for every row and k-row block the
    D lookups are accumulated into ceil(n/32) column words (LOOKUP_LOP3 each),
    and every block's table of 2^k - 1 nonzero combinations is built once
    (one bitsliced add per entry and word)."""
    words = cdiv(n, 32)
    blocks = cdiv(l, k)
    return words * blocks * (m * LOOKUP_LOP3[q] + (2 ** k - 1) * TABLE_LOP3[q])


def batched_compulsory_bytes(q, shapes):
    """Compulsory DRAM bytes of the batched tcgen05 kernel for its products:
    A's planes over la = l rounded up to 128 columns and B's over nr = n
    rounded up to 256 columns read once (the e4m3 operands never leave L2),
    C's planes written (its row pitch of 64-bit words)."""
    total = 0
    for (m, l, n) in shapes:
        la, nr = cdiv(l, 128) * 128, cdiv(n, 256) * 256
        total += PLANES[q] * (m * la + l * nr) // 8 + PLANES[q] * m * pitch_words(n) * 8
    return total


def our_launches(levels):
    """Kernels of this library one F_3 product launches: the M4RM kernel, or per
    Strassen level twelve quadrant copies, fifteen bitsliced additions and
    seven sub-products."""
    return 1 if levels == 0 else 27 + 7 * our_launches(levels - 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sizes", type=str, default="",
                    help="comma-separated n list (uniform square products) instead of the workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 4096-product batched workloads")
    ap.add_argument("--no-more", action="store_true",
                    help="skip the F_5/F_7/GF(4) 8192 and the large F_5 / F_3 workloads")
    ap.add_argument("--cpu-rows", type=int, default=1024,
                    help="oracle rows sampled per product (about 11 s of oracle work on 16 cores)")
    return ap.parse_args()


def batched_leg(torch, fq, inputs, dist, dev, reps=10):
    """The batched workloads: 4096 products over F_3 and over F_5 with m, l, n
    uniform over multiples of 64 in [64, 1024], one plan each, its launch
    captured in a CUDA graph and replayed (device time, CUDA events on the
    replaying stream); the FQ_PATH_AUTO plan (per-product choice between the
    two paths) beside the Four-Russians-only plan.  Every rank runs its own
    batch; the slowest rank's time counts."""
    out = {}
    for q in (3, 5):
        shapes = [tuple(int(x) for x in s) for s in inputs.batch_shapes(4096, seed=q)]
        a, b, c = [], [], []
        for p, (m, l, n) in enumerate(shapes):
            a.append(fq.pack(q, inputs.uniform_torch(q, m, l, seed=q, stream=100 + 2 * p, device="cuda")))
            b.append(fq.pack(q, inputs.uniform_torch(q, l, n, seed=q, stream=101 + 2 * p, device="cuda")))
            c.append(fq.empty(q, m, n))
        ptr = lambda xs: torch.tensor([x.data.data_ptr() for x in xs], dtype=torch.int64, device=dev)
        pa, pb, pc = ptr(a), ptr(b), ptr(c)
        ops = sum(2.0 * m * l * n for m, l, n in shapes)
        rec = {"count": len(shapes), "shapes": "m, l, n uniform over multiples of 64 in [64, 1024]"}
        results = {}
        for name, path in (("auto", fq.PATH_AUTO), ("m4rm", fq.PATH_M4RM)):
            plan = fq.BatchPlan(q, shapes, path=path)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                plan.run(pa, pb, pc, stream=stream)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                plan.run(pa, pb, pc, stream=stream)
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            dist.barrier()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                with torch.cuda.stream(stream):
                    g.replay()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = dist.max(statistics.median(ms), dev)
            results[name] = torch.cat([x.data for x in c]).clone()
            entry = {"ms": t, "products_per_s": dist.world * len(shapes) / (t * 1e-3),
                     "field_ops_per_s": dist.world * ops / (t * 1e-3),
                     "tc_products": plan.tc_products, "m4rm_items": plan.items}
            if name == "auto" and plan.tc_products > 0:
                entry.update(batched_stage_rooflines(torch, fq, plan, q, shapes, pa, pb, pc, stream, reps))
            rec[name] = entry
            del g, plan
        if not torch.equal(results["auto"], results["m4rm"]):
            raise SystemExit("batched F_%d: the two plans give different products" % q)
        if fq.status() != fq.OK:
            raise SystemExit("device error in the batched workload")
        rec["speedup_auto_vs_m4rm"] = rec["m4rm"]["ms"] / rec["auto"]["ms"]
        out["F_%d" % q] = rec
        del a, b, c, results
        torch.cuda.empty_cache()
    return out


def batched_stage_rooflines(torch, fq, plan, q, shapes, pa, pb, pc, stream, reps):
    """The AUTO plan's launch stages timed one at a time (fq_matmul_batched_stages,
    CUDA events on the launching stream, median of `reps`): the persistent
    tcgen05 kernel (operand conversion and tiles in one launch) against the
    fp8 tensor peak and against HBM for its compulsory bytes, then the
    Four-Russians kernel (if the plan has items)."""
    peaks = measured_peaks()
    tc = [sh for sh, path in zip(shapes, plan.product_paths()) if path == fq.PATH_MMA]
    ms = {"tcgen05": [], "m4rm": []}
    for r in range(reps + 2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            plan.run_stages(pa, pb, pc, fq.STAGE_TC, stream=stream)
            ev[1].record(stream)
            plan.run_stages(pa, pb, pc, fq.STAGE_M4RM, stream=stream)
            ev[2].record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            ms["tcgen05"].append(ev[0].elapsed_time(ev[1]))
            ms["m4rm"].append(ev[1].elapsed_time(ev[2]))
    if fq.status() != fq.OK:
        raise SystemExit("device error in the batched stages")
    tc_ms = statistics.median(ms["tcgen05"])
    flops = sum(2.0 * m * l * n for (m, l, n) in tc)
    dram = batched_compulsory_bytes(q, tc)
    tflops = flops / (tc_ms * 1e-3) / 1e12
    gbs = dram / (tc_ms * 1e-3) / 1e9
    return {
        "stages_ms": {k: statistics.median(v) for k, v in ms.items()},
        "tile_roofline": {"bound": "tensor", "kernel": "tc_batched_kernel", "achieved": tflops,
                          "peak": peaks["fp8"], "unit": "TFLOP/s", "frac": tflops / peaks["fp8"],
                          "peak_note": peaks["note"], "flops": flops},
        "hbm_roofline": {"bound": "hbm", "kernel": "tc_batched_kernel", "achieved": gbs, "peak": peaks["hbm"],
                         "unit": "GB/s", "frac": gbs / peaks["hbm"], "bytes": dram, "peak_note": peaks["hbm_note"],
                         "note": "compulsory bytes: the planes of A and B read once, C's planes written"},
        "stages_note": "each stage called on its own (fq_matmul_batched_stages), median of %d; the graph "
                       "replay above runs them back to back" % reps,
    }


def product_leg(torch, fq, inputs, dist, dev, flush, workload, prods, clk, reps=3, warmup=1):
    """One product at a time, on both paths, inputs resident in HBM and L2
    flushed before every timed product: the tcgen05 form as its two stages
    (conversion, product kernel) and the plain bitsliced Four-Russians path,
    each against its roofline; the two results must agree bit for bit."""
    peaks = measured_peaks()
    stream = torch.cuda.current_stream()
    out = {"workload": workload, "products": []}
    tot_tc = tot_m4 = 0.0
    ops_all = 0.0
    for (q, m, l, n) in prods:
        A = inputs.uniform_torch(q, m, l, seed=0, stream=inputs.STREAM_A, device=dev)
        B = inputs.uniform_torch(q, l, n, seed=0, stream=inputs.STREAM_B, device=dev)
        a, b = fq.pack(q, A), fq.pack(q, B)
        del A, B
        c_tc, c_m4 = fq.empty(q, m, n), fq.empty(q, m, n)
        ops = fq.TensorOperands(a, b)
        form = fq.tc_form(q, m, l, n)
        t_prep, t_mul, t_m4 = [], [], []
        for r in range(warmup + reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            flush.fill_(r)
            ev[0].record(stream)
            ops.prepare(a, b)
            ev[1].record(stream)
            ops.multiply(out=c_tc)
            ev[2].record(stream)
            flush.fill_(r + 1)
            ev[3].record(stream)
            fq.matmul(a, b, out=c_m4, path=fq.PATH_M4RM)
            ev[4].record(stream)
            torch.cuda.synchronize()
            if r >= warmup:
                t_prep.append(ev[0].elapsed_time(ev[1]))
                t_mul.append(ev[1].elapsed_time(ev[2]))
                t_m4.append(ev[3].elapsed_time(ev[4]))
        if fq.status() != fq.OK:
            raise SystemExit("device error in the F_%d %dx%dx%d product" % (q, m, l, n))
        agree = bool(torch.equal(c_tc.data, c_m4.data))
        if not agree:
            raise SystemExit("F_%d %dx%dx%d: the two paths give different products" % (q, m, l, n))
        prep_ms = dist.max(statistics.median(t_prep), dev)
        mul_ms = dist.max(statistics.median(t_mul), dev)
        m4_ms = dist.max(statistics.median(t_m4), dev)
        field_ops = 2.0 * m * l * n
        tflops = tensor_flops(q, m, l, n) / (mul_ms * 1e-3) / 1e12
        pbytes = prepare_bytes(m, l, n, q, form)
        levels = fq.strassen_levels(q, m, l, n, path=fq.PATH_M4RM)
        leaf = (m >> levels, l >> levels, n >> levels)
        k = fq.planned_kernel(q, *leaf, path=fq.PATH_M4RM)["k"]
        lop3 = 7 ** levels * algorithmic_lop3(*leaf, k, q)
        lop3_t = lop3 / (m4_ms * 1e-3) / 1e12
        out["products"].append({
            "q": q, "m": m, "l": l, "n": n, "paths_agree": agree,
            "tensor": {"ms": prep_ms + mul_ms, "prepare_ms": prep_ms, "multiply_ms": mul_ms,
                       "field_ops_per_s": dist.world * field_ops / ((prep_ms + mul_ms) * 1e-3),
                       "roofline": tc_roofline(peaks, form, tflops, clk),
                       "prepare_roofline": {"bound": "hbm", "achieved": pbytes / (prep_ms * 1e-3) / 1e9,
                                            "peak": peaks["hbm"], "unit": "GB/s",
                                            "frac": pbytes / (prep_ms * 1e-3) / 1e9 / peaks["hbm"],
                                            "bytes": pbytes}},
            "m4rm": {"ms": m4_ms, "field_ops_per_s": dist.world * field_ops / (m4_ms * 1e-3),
                     "strassen_levels": levels, "k": k,
                     "roofline": {"bound": "alu", "achieved": lop3_t, "peak": ALU_PEAK_TLOPS, "unit": "Tlop3/s",
                                  "frac": lop3_t / ALU_PEAK_TLOPS, "lop3": lop3,
                                  "peak_note": "derived: 64 LOP3 lanes/clk/SM x 152 SMs x 2070 MHz"}},
            "speedup_tensor_vs_m4rm": m4_ms / (prep_ms + mul_ms),
        })
        tot_tc += prep_ms + mul_ms
        tot_m4 += m4_ms
        ops_all += field_ops
        del ops, a, b, c_tc, c_m4
        torch.cuda.empty_cache()
    out["tensor_field_ops_per_s"] = dist.world * ops_all / (tot_tc * 1e-3)
    out["m4rm_field_ops_per_s"] = dist.world * ops_all / (tot_m4 * 1e-3)
    out["speedup_tensor_vs_m4rm"] = tot_m4 / tot_tc
    out["timing"] = ("per product: median of %d after %d warm-up, CUDA events on the launching stream, L2 flushed "
                     "(256 MiB write) before each path" % (reps, warmup))
    return out


def products_for(args):
    if args.sizes:
        return [(n, n, n, "uniform") for n in (int(x) for x in args.sizes.split(","))]
    return PRODUCTS


class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float, device) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def done(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; only the
    samples stamped inside the timed window (mark_start .. mark_stop) count."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None
        self.window = [None, None]

    def start(self):
        """Start sampling and wait (up to 5 s) for the first sample."""
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="fq_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def mark_start(self):
        self.window[0] = time.time()

    def mark_stop(self):
        self.window[1] = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        lo, hi = self.window
        inside = [r for r in rows if lo is not None and hi is not None and
                  (self._stamp(r[0]) or 0.0) >= lo - 0.025 and (self._stamp(r[0]) or 0.0) <= hi + 0.025]
        use = inside or rows
        sm = [float(r[1]) for r in use if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use),
                "window": "timed region" if inside else "whole run (no sample stamped inside the timed region)"}


def sources_digest(names):
    """Digest of the code in these sources: comments, blank lines and trailing
    blanks do not count, so that counters stay attached to a kernel whose
    commentary changes."""
    import re
    h = hashlib.sha256()
    for name in names:
        with open(name, encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [line.rstrip() for line in text.splitlines()]
        h.update("\n".join(line for line in lines if line).encode())
    return h.hexdigest()[:16]


def kernel_sources_digest():
    """Digest of the sources the M4RM kernels are compiled from."""
    import glob
    csrc = os.path.join(ROOT, "paper_0901_1413_gb300", "csrc")
    return sources_digest(sorted(glob.glob(os.path.join(csrc, "fq_m4rm*")) +
                                 [os.path.join(csrc, n) for n in ("fq_fields.cuh", "fq_common.cuh")]))


def tc_sources_digest():
    """Digest of the sources the tcgen05 product kernel is compiled from."""
    csrc = os.path.join(ROOT, "paper_0901_1413_gb300", "csrc")
    return sources_digest([os.path.join(csrc, n) for n in ("fq_tc.cu", "fq_common.cuh", "fq_e4m3.cuh")])


def measured_traffic(name, digest):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_sources_sha256_16") != digest:
        return None
    return rec


def measured_peaks():
    """Peaks for the rooflines: the measured dense bf16 burst of
    MEASURED_PEAKS.json (else 1900 TFLOP/s, an earlier GB300 measurement); the
    dense fp8 (e4m3) and fp4 (e2m1) peaks as 2 and 6 times that, the nominal
    ratios (4.5 and 13.5 against 2.25 PFLOP/s); the measured HBM copy
    bandwidth (else 6800 GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            rec = json.load(f)
        bf16, hbm = float(rec["bf16_tflops"]), float(rec["hbm_gbs"])
        src, hbm_note = "of measured: cuBLAS bf16 burst", "of measured: HBM copy (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        bf16, hbm = 1900.0, 6800.0
        src, hbm_note = "of fallback: 1.9 PFLOP/s bf16", "of fallback: 6.8 TB/s"
    return {"bf16": bf16, "fp8": 2.0 * bf16, "fp4": 6.0 * bf16,
            "note": src + " x 2 (nominal fp8/bf16 ratio)",
            "note_fp8": src + " x 2 (nominal fp8/bf16 ratio)",
            "note_fp4": src + " x 6 (nominal fp4/bf16 ratio)",
            "hbm": hbm, "hbm_note": hbm_note}


def tc_roofline(peaks, form, achieved_tflops, clk):
    """Roofline of a tcgen05 product kernel in `form`: against its operand
    type's dense peak, and against its instruction kind's pipe at the sampled
    SM clock."""
    kernel, dtype, opc, _ = TC_FORMS[form]
    return {"bound": "tensor", "achieved": achieved_tflops, "peak": peaks[dtype], "unit": "TFLOP/s",
            "frac": achieved_tflops / peaks[dtype], "peak_note": peaks["note_" + dtype], "kernel": kernel,
            "operands": dtype, "pipe": pipe_peak(achieved_tflops, clk, opc)}


# The f8f6f4 tensor pipe's own peak, as the hardware counters state it
# (sm__ops_path_tensor_op_utcqmma_src_fp8_dst_fp32...peak_sustained) and the
# microbenchmark measures it; kind::mxf4 (packed e2m1) measured at twice that.
FP8_OPS_PER_CLK_PER_SM = 16384
SMS = 152


def pipe_peak(achieved_tflops, clk, ops_per_clk=FP8_OPS_PER_CLK_PER_SM):
    """A second roofline denominator for the tensor-core product: the
    instruction kind's pipe peak at the SM clock sampled in the timed region
    (the measured bf16 figure was taken at a lower, power-capped clock)."""
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = ops_per_clk * SMS * mhz * 1e6 / 1e12
    return {"peak": peak, "unit": "TFLOP/s", "frac": achieved_tflops / peak, "sm_mhz": mhz,
            "note": "%d ops/clk/SM (tcgen05 microbenchmark, operands resident) x 152 SMs x the median SM clock "
                    "of the timed region" % ops_per_clk}


def make_inputs(torch, inputs, prods, seed=0):
    out = []
    for (m, l, n, law) in prods:
        gen = inputs.sparse_torch if law == "sparse90" else inputs.uniform_torch
        A = gen(Q, m, l, seed=seed, stream=inputs.STREAM_A, device="cuda")
        B = inputs.uniform_torch(Q, l, n, seed=seed, stream=inputs.STREAM_B, device="cuda")
        out.append((A, B))
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), best effort."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def cpu_baseline(prods, rows_per_product, seed=0, steps=1, threads=0):
    """The oracle (as it stands) on the first rows_per_product rows of every
    product, on `threads` host threads (0: all)."""
    import numpy as np

    import oracle
    from paper_0901_1413_gb300 import inputs
    work = []
    for (m, l, n, law) in prods:
        r = min(rows_per_product, m)
        A = (inputs.sparse if law == "sparse90" else inputs.uniform)(Q, r, l, seed=seed, stream=inputs.STREAM_A)
        B = inputs.uniform(Q, l, n, seed=seed, stream=inputs.STREAM_B)
        work.append((A, B, r, l, n))
    oracle.matmul(Q, work[0][0][:1], work[0][1])          # load and warm
    times = []
    ops = sum(2.0 * r * l * n for (_, _, r, l, n) in work)
    for _ in range(steps):
        t0 = time.perf_counter()
        for (A, B, _, _, _) in work:
            C = oracle.matmul(Q, A, B, threads)
            assert C.dtype == np.uint8
        times.append(time.perf_counter() - t0)
    return ops, times, oracle.threads_used(threads), sum(r for (_, _, r, _, _) in work)


def run_reference(args, dist):
    if dist.rank != 0:
        return
    prods = products_for(args)
    rows = max(1, min(args.cpu_rows, 16))
    ops, times, cores, nrows = cpu_baseline(prods, rows, steps=args.warmup + args.steps)
    t = times[args.warmup:]
    mean = sum(t) / len(t)
    value = ops / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.sizes else "F_3 square n=" + args.sizes, "q": Q,
                   "sample": "first %d rows of each product" % rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "first %d rows of each of the %d products (%d rows total)"
                                   % (rows, len(prods), nrows)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        dist.init("gloo")
        run_reference(args, dist)
        dist.done()
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")

    import torch

    from paper_0901_1413_gb300 import fq, inputs

    torch.cuda.set_device(dist.local)
    dist.init("nccl")
    dev = torch.device("cuda", dist.local)
    fq.load()
    prods = products_for(args)

    # ---- inputs, packed and resident -------------------------------------
    res = make_inputs(torch, inputs, prods)
    packed = []
    for (A, B), (m, l, n, _) in zip(res, prods):
        a, b = fq.pack(Q, A), fq.pack(Q, B)
        packed.append((a, b, fq.empty(Q, m, n)))
    if fq.status() != fq.OK:
        raise SystemExit("device error while packing")
    # Each product runs in the form FQ_PATH_AUTO takes for its shape (the
    # library's time model, the same with or without a profiler attached).  A
    # tensor-core product runs as its two stages, operand conversion and the
    # tcgen05 product, so that the product kernel can be timed on its own.
    forms = ["tensor" if fq.auto_choice(Q, m, l, n)[0] == fq.PATH_MMA else "m4rm" for (m, l, n, _) in prods]
    tc_forms = [fq.tc_form(Q, m, l, n) if f == "tensor" else None for f, (m, l, n, _) in zip(forms, prods)]
    tops = [fq.TensorOperands(a, b) if f == "tensor" else None for f, (a, b, c) in zip(forms, packed)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(evs=None):
        # evs[j] = (start, operands ready, product done)
        for j, ((a, b, c), t) in enumerate(zip(packed, tops)):
            if evs is not None:
                evs[j][0].record(stream)
            if t is not None:
                t.prepare(a, b)
            if evs is not None:
                evs[j][1].record(stream)
            if t is not None:
                t.multiply(out=c)
            else:
                fq.matmul(a, b, out=c)
            if evs is not None:
                evs[j][2].record(stream)

    def timed(step_fn, steps, warmup, sampler=None):
        for w in range(warmup):
            flush.fill_(w)
            step_fn()
        torch.cuda.synchronize()
        if fq.status() != fq.OK:
            raise SystemExit("device error during warm-up")
        evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in packed] for _ in range(steps)]
        dist.barrier()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.mark_start()
        for s_ in range(steps):
            flush.fill_(s_ + 1)
            step_fn(evs[s_])
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.mark_stop()
        dist.barrier()
        if fq.status() != fq.OK:
            raise SystemExit("device error in the timed region")
        stage = [[[evs[s_][j][0].elapsed_time(evs[s_][j][1]), evs[s_][j][1].elapsed_time(evs[s_][j][2])]
                  for j in range(len(packed))] for s_ in range(steps)]
        step_ms = [evs[s_][0][0].elapsed_time(evs[s_][-1][2]) for s_ in range(steps)]
        return stage, dist.max(sum(step_ms) / len(step_ms), dev)

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "")) or str(dist.local)
    clocks = ClockSampler(uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if len(uuid) > 30 else uuid))
    clocks.start()
    stage, mean_ms = timed(step, args.steps, args.warmup, clocks)
    clk = clocks.stop()
    ops_step = sum(2.0 * m * l * n for (m, l, n, _) in prods)
    value = ops_step * dist.world / (mean_ms * 1e-3)
    per_product = [sum(stage[s_][j][0] + stage[s_][j][1] for s_ in range(args.steps)) / args.steps
                   for j in range(len(prods))]
    product_ms = [sum(stage[s_][j][1] for s_ in range(args.steps)) / args.steps for j in range(len(prods))]

    # Pack and unpack, reported apart from the product: the step's eight
    # operands packed from device-resident residues, its four results unpacked.
    def pack_unpack_ms(reps=10):
        outs = [torch.empty((m, n), dtype=torch.uint8, device=dev) for (m, l, n, _) in prods]
        tp, tu = [], []
        for _ in range(reps + 2):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            for (A, B), (a, b, c) in zip(res, packed):
                fq.pack(Q, A, out=a)
                fq.pack(Q, B, out=b)
            e[1].record(stream)
            for (a, b, c), o in zip(packed, outs):
                fq.unpack(c, out=o)
            e[2].record(stream)
            torch.cuda.synchronize()
            tp.append(e[0].elapsed_time(e[1]))
            tu.append(e[1].elapsed_time(e[2]))
        if fq.status() != fq.OK:
            raise SystemExit("device error in pack / unpack")
        in_bytes = sum(m * l + l * n for (m, l, n, _) in prods)
        out_bytes = sum(m * n for (m, l, n, _) in prods)
        p_ms, u_ms = statistics.median(tp[2:]), statistics.median(tu[2:])
        planes = lambda r, c: 2 * r * pitch_words(c) * 8
        p_bytes = in_bytes + sum(planes(m, l) + planes(l, n) for (m, l, n, _) in prods)
        u_bytes = out_bytes + sum(planes(m, n) for (m, l, n, _) in prods)
        return {"pack_ms": p_ms, "unpack_ms": u_ms, "pack_gbs": p_bytes / (p_ms * 1e-3) / 1e9,
                "unpack_gbs": u_bytes / (u_ms * 1e-3) / 1e9,
                "note": "per step: 8 operands packed (residues in, planes out), 4 results unpacked; "
                        "bytes = residues + planes; median of 10 after 2 warm-ups"}

    pack_unpack = pack_unpack_ms()

    # Roofline of the dominant kernel, the tcgen05 product: 2 m l n flops per
    # launch over the product stage's event time, for the form that takes the
    # most product time (each form against its own operand type's peak).
    peaks = measured_peaks()
    form_ms = {}
    for tf, t in zip(tc_forms, product_ms):
        if tf is not None:
            form_ms[tf] = form_ms.get(tf, 0.0) + t
    main_form = max(form_ms, key=form_ms.get) if form_ms else None
    t_flops = sum(2.0 * m * l * n for tf, (m, l, n, _) in zip(tc_forms, prods) if tf is not None and tf == main_form)
    t_ms = form_ms.get(main_form, 0.0)
    achieved = t_flops / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0
    # The conversion stage: e4m3 bytes written (A: m x la, B^T: 64 pitch(n) x
    # la) plus the planes read (A; B, then B^T's planes written and read).
    prep_ms = sum(sum(stage[s_][j][0] for s_ in range(args.steps)) / args.steps
                  for j, f in enumerate(forms) if f == "tensor")
    prep_bytes = sum(prepare_bytes(m, l, n, Q, tf) for tf, (m, l, n, _) in zip(tc_forms, prods) if tf is not None)
    prep_gbs = prep_bytes / (prep_ms * 1e-3) / 1e9 if prep_ms > 0 else 0.0
    traffic_rec = measured_traffic("tc_fp4_f3_dram_traffic.json" if main_form == 5 else "tc_f3_dram_traffic.json",
                                   tc_sources_digest())
    traffic = traffic_rec.get("bytes_per_launch") if traffic_rec else None

    # ---- the plain bitsliced M4RM path on the same products, for the factor --
    m_levels = [fq.strassen_levels(Q, m, l, n, path=fq.PATH_M4RM) for (m, l, n, _) in prods]
    leaves = [(m >> lv, l >> lv, n >> lv) for lv, (m, l, n, _) in zip(m_levels, prods)]
    leaf_k = [fq.planned_kernel(Q, *leaf, path=fq.PATH_M4RM)["k"] for leaf in leaves]

    def m4rm_step(evs=None):
        for j, (a, b, c) in enumerate(packed):
            if evs is not None:
                evs[j][0].record(stream)
                evs[j][1].record(stream)
            fq.matmul(a, b, out=c, path=fq.PATH_M4RM)
            if evs is not None:
                evs[j][2].record(stream)

    auto_results = [c.data.clone() for (a, b, c) in packed]
    m_steps = max(3, min(args.steps, 5))
    m_stage, m_ms = timed(m4rm_step, m_steps, 3)
    for ref, (a, b, c) in zip(auto_results, packed):
        if not torch.equal(ref, c.data):
            raise SystemExit("the Four-Russians path and the headline path give different products")
    del auto_results
    m_value = ops_step * dist.world / (m_ms * 1e-3)
    m_per_product = [sum(m_stage[s_][j][1] for s_ in range(m_steps)) / m_steps for j in range(len(prods))]
    lop3_step = sum(7 ** lv * algorithmic_lop3(m >> lv, l >> lv, n >> lv, k, Q)
                    for lv, k, (m, l, n, _) in zip(m_levels, leaf_k, prods))
    m_achieved = lop3_step / (sum(m_per_product) * 1e-3) / 1e12
    m_traffic_rec = measured_traffic("m4rm_f3_dram_traffic.json", kernel_sources_digest())
    m4rm = {"value": m_value, "unit": UNIT, "ms_per_step": m_ms, "steps": m_steps, "per_product_ms": m_per_product,
            "strassen_levels": m_levels, "k": leaf_k,
            "gpu_launches": m_steps * sum(our_launches(lv) for lv in m_levels),
            "roofline": {"bound": "alu", "achieved": m_achieved, "peak": ALU_PEAK_TLOPS, "unit": "Tlop3/s",
                         "frac": m_achieved / ALU_PEAK_TLOPS,
                         "traffic": m_traffic_rec.get("bytes_per_m4rm_launch") if m_traffic_rec else None,
                         "peak_note": "derived: 64 LOP3 lanes/clk/SM x 152 SMs x 2070 MHz"}}

    # ---- end to end through the public API, host buffers -------------------
    e2e = e2e_packed = None
    if not args.no_e2e:
        host = []
        for (A, B), (m, l, n, _) in zip(res, prods):
            host.append((A.cpu().pin_memory(), B.cpu().pin_memory(),
                         torch.empty((m, n), dtype=torch.uint8).pin_memory()))
        dbuf = [(torch.empty_like(A), torch.empty_like(B)) for (A, B) in res]
        pk = [(fq.empty(Q, m, l), fq.empty(Q, l, n), fq.empty(Q, m, n), torch.empty((m, n), dtype=torch.uint8,
                                                                                   device=dev))
              for (m, l, n, _) in prods]

        # Copies in and out run on their own streams so that they overlap the
        # products: product j's inputs go up while product j - 1 computes, its
        # result comes down while product j + 1 computes.  Events keep each
        # product's device buffers from being overwritten before they are read.
        h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
        ev = {name: [torch.cuda.Event() for _ in prods] for name in ("in", "packed", "out", "read")}
        started = [False]

        def e2e_step():
            for j, ((hA, hB, hC), (dA, dB), (a, b, c, dC)) in enumerate(zip(host, dbuf, pk)):
                with torch.cuda.stream(h2d_s):
                    if started[0]:
                        h2d_s.wait_event(ev["packed"][j])      # last step's pack has read dA, dB
                    dA.copy_(hA, non_blocking=True)
                    dB.copy_(hB, non_blocking=True)
                    ev["in"][j].record(h2d_s)
                stream.wait_event(ev["in"][j])
                fq.pack(Q, dA, out=a)
                fq.pack(Q, dB, out=b)
                ev["packed"][j].record(stream)
                fq.matmul(a, b, out=c)
                if started[0]:
                    stream.wait_event(ev["read"][j])           # last step's result has left dC
                fq.unpack(c, out=dC)
                ev["out"][j].record(stream)
                with torch.cuda.stream(d2h_s):
                    d2h_s.wait_event(ev["out"][j])
                    hC.copy_(dC, non_blocking=True)
                    ev["read"][j].record(d2h_s)
            started[0] = True

        def join():
            stream.wait_stream(h2d_s)
            stream.wait_stream(d2h_s)

        for _ in range(args.warmup):
            e2e_step()
        join()
        torch.cuda.synchronize()
        e_steps = max(3, min(args.steps, 10))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(e_steps):
            e2e_step()
        join()
        e1.record(stream)
        torch.cuda.synchronize()
        # the results that reached the host equal the device-resident products
        for (hA, hB, hC), (a, b, c) in zip(host, packed):
            if not torch.equal(hC, fq.unpack(c).cpu()):
                raise SystemExit("end-to-end result differs from the device-resident product")
        dist.barrier()
        if fq.status() != fq.OK:
            raise SystemExit("device error in the end-to-end region")
        e_ms = dist.max(e0.elapsed_time(e1) / e_steps, dev)
        e2e = {"value": ops_step * dist.world / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": sum(m * l + l * n for (m, l, n, _) in prods),
               "d2h_bytes_per_step": sum(m * n for (m, l, n, _) in prods),
               "ms_per_step": e_ms, "steps": e_steps,
               "inputs": "uint8 residues in pinned host memory; fq_pack, fq_matmul, fq_unpack on the device"}

        # The same with the host holding matrices in the library's own format
        # (the paper's bit-planes, 2 bits per F_3 element): planes up, fq_matmul,
        # C's planes down, copies overlapped as above.
        del dbuf
        hp = [(a.data.cpu().pin_memory(), b.data.cpu().pin_memory(), torch.empty_like(c.data, device="cpu").pin_memory())
              for (a, b, c) in packed]
        dp = [(fq.empty(Q, m, l), fq.empty(Q, l, n), fq.empty(Q, m, n)) for (m, l, n, _) in prods]
        evp = {name: [torch.cuda.Event() for _ in prods] for name in ("in", "used", "out", "read")}
        startedp = [False]

        def e2e_packed_step():
            for j, ((hA, hB, hC), (a, b, c)) in enumerate(zip(hp, dp)):
                with torch.cuda.stream(h2d_s):
                    if startedp[0]:
                        h2d_s.wait_event(evp["used"][j])       # last step's product has read a, b
                    a.data.copy_(hA, non_blocking=True)
                    b.data.copy_(hB, non_blocking=True)
                    evp["in"][j].record(h2d_s)
                stream.wait_event(evp["in"][j])
                if startedp[0]:
                    stream.wait_event(evp["read"][j])          # last step's C has left the device
                fq.matmul(a, b, out=c)
                evp["used"][j].record(stream)
                evp["out"][j].record(stream)
                with torch.cuda.stream(d2h_s):
                    d2h_s.wait_event(evp["out"][j])
                    hC.copy_(c.data, non_blocking=True)
                    evp["read"][j].record(d2h_s)
            startedp[0] = True

        for _ in range(args.warmup):
            e2e_packed_step()
        join()
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(e_steps):
            e2e_packed_step()
        join()
        e1.record(stream)
        torch.cuda.synchronize()
        for (hA, hB, hC), (a, b, c) in zip(hp, packed):
            if not torch.equal(hC, c.data.cpu()):
                raise SystemExit("end-to-end (packed) result differs from the device-resident product")
        dist.barrier()
        if fq.status() != fq.OK:
            raise SystemExit("device error in the end-to-end (packed) region")
        p_ms = dist.max(e0.elapsed_time(e1) / e_steps, dev)
        e2e_packed = {"value": ops_step * dist.world / (p_ms * 1e-3), "unit": UNIT,
                      "h2d_bytes_per_step": sum(a.data.numel() * 8 + b.data.numel() * 8 for (a, b, c) in packed),
                      "d2h_bytes_per_step": sum(c.data.numel() * 8 for (a, b, c) in packed),
                      "ms_per_step": p_ms, "steps": e_steps,
                      "inputs": "bit-planes (fq_pack's format) in pinned host memory; fq_matmul on the device"}

    batched = None if args.no_batched else batched_leg(torch, fq, inputs, dist, dev)

    more = None
    if not args.sizes and not args.no_more:
        torch.cuda.empty_cache()
        more = [product_leg(torch, fq, inputs, dist, dev, flush, name, ps, clk) for name, ps in MORE_WORKLOADS]

    base = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        ops, times, cores, nrows = cpu_baseline(prods, args.cpu_rows)
        rows1 = max(1, args.cpu_rows // 48)
        ops1, times1, _, nrows1 = cpu_baseline(prods, rows1, threads=1)
        base = {"value": ops / times[0], "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                "sample": "first %d rows of each of the %d products (%d rows), one pass"
                          % (args.cpu_rows, len(prods), nrows),
                "single_thread": {"value": ops1 / times1[0], "unit": UNIT, "cores": 1,
                                  "sample": "first %d rows of each product (%d rows), one pass" % (rows1, nrows1)}}

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("e2m1" if main_form == 5 else "e4m3") + " (exact integers, fp32 sums)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.sizes else "F_3 square n=" + args.sizes,
                       "q": Q, "products": [list(p) for p in prods],
                       "path": forms, "tc_form": tc_forms,
                       "path_choice": "FQ_PATH_AUTO per shape (fq_auto_choice: the library's "
                                      "time model of M4RM and the tensor-core path; fq_tc_form: the tcgen05 form)",
                       "l2": "flushed (256 MiB write) before every step",
                       "parallelism": "replicas" if dist.world > 1 else "single GPU"},
            "roofline": dict(tc_roofline(peaks, main_form, achieved, clk) if main_form else {},
                             traffic=traffic, kernel_ms_per_step=t_ms),
            "prepare": {"bound": "hbm", "ms_per_step": prep_ms, "bytes": prep_bytes, "achieved": prep_gbs,
                        "peak": peaks["hbm"], "unit": "GB/s", "frac": prep_gbs / peaks["hbm"],
                        "peak_note": peaks["hbm_note"]},
            "per_product_ms": per_product,
            "product_stage_ms": product_ms,
            "m4rm": m4rm,
            "speedup_vs_m4rm": value / m_value,
            "pack_unpack": pack_unpack,
            "e2e": e2e,
            "e2e_packed": e2e_packed,
            "batched": batched,
            "more_workloads": more,
            "cpu_baseline": base,
            "clocks": clk,
            "gpu_launches": args.steps * sum(TC_LAUNCHES if f == "tensor" else 1 for f in forms),
        }
        print(json.dumps(line), flush=True)
    dist.done()


if __name__ == "__main__":
    main()

"""Time the product configurations on cuda:0 and print a Markdown table.

    python -m paper_0901_1413_gb300.measure [--quick]

Every row is measured with CUDA events on the current stream, best of a few
runs after one warm-up, inputs resident in device memory (seeded synthetic
residues, uniform unless stated).  Throughput is 2 m l n / t in field
operations per second; batched rows also give products per second.  Both
product paths are timed where the configuration asks for them: the bitsliced
Four-Russians path (M4RM) and the exact tensor-core path (MMA), each with its
direct kernels and, where the time model takes them, with Strassen-Winograd
levels ("+strassen"); for the
extension fields these name the path of the base-field products inside
Section 4.3's matrix-level product, and "karatsuba" is GF(4) by three F_2
products.
"""
from __future__ import annotations

import argparse

import torch

from . import fq, inputs


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _operands(q, m, l, n, sparse=False):
    gen = inputs.sparse_torch if sparse else inputs.uniform_torch
    a = fq.pack(q, gen(q, m, l, seed=0, stream=inputs.STREAM_A))
    b = fq.pack(q, inputs.uniform_torch(q, l, n, seed=0, stream=inputs.STREAM_B))
    return a, b, fq.empty(q, m, n)


def product_rows(q, m, l, n, paths=("m4rm",), sparse=False, reps=3):
    """Each path's direct kernels (no Strassen-Winograd level), then, where the
    time model takes levels, the same path with them ("+strassen")."""
    a, b, c = _operands(q, m, l, n, sparse)
    ops = 2.0 * m * l * n
    out = []
    for p in paths:
        path = {"m4rm": fq.PATH_M4RM, "mma": fq.PATH_MMA, "karatsuba": fq.PATH_KARATSUBA}[p]
        t = _time(lambda: fq.matmul(a, b, out=c, path=path, strassen=-1), reps)
        out.append((p, t, ops / t * 1e3))
        if p != "karatsuba" and q in (2, 3, 4, 5, 7) and fq.strassen_levels(q, m, l, n, path=path) > 0:
            t = _time(lambda: fq.matmul(a, b, out=c, path=path), reps)
            out.append((p + "+strassen", t, ops / t * 1e3))
    if fq.status() != fq.OK:
        raise RuntimeError("device reported an error")
    return out


def batched_row(q, count=4096, reps=5, path=None):
    shapes = [tuple(int(x) for x in s) for s in inputs.batch_shapes(count, seed=q)]
    a, b, c = [], [], []
    for p, (m, l, n) in enumerate(shapes):
        a.append(fq.pack(q, inputs.uniform_torch(q, m, l, seed=q, stream=100 + 2 * p)))
        b.append(fq.pack(q, inputs.uniform_torch(q, l, n, seed=q, stream=101 + 2 * p)))
        c.append(fq.empty(q, m, n))
    ptr = lambda xs: torch.tensor([x.data.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    pa, pb, pc = ptr(a), ptr(b), ptr(c)
    plan = fq.BatchPlan(q, shapes, path=fq.PATH_AUTO if path is None else path)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.run(pa, pb, pc, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.run(pa, pb, pc, stream=stream)
    t = _time(graph.replay, reps)
    if fq.status() != fq.OK:
        raise RuntimeError("device reported an error")
    ops = sum(2.0 * m * l * n for m, l, n in shapes)
    return t, count / t * 1e3, ops / t * 1e3, plan.items


def one_case(spec, reps):
    """--case q,m,l,n[,path[,kernel]]: one product, `reps` timed runs after a warm-up."""
    parts = spec.split(",")
    q, m, l, n = (int(x) for x in parts[:4])
    path = parts[4] if len(parts) > 4 else "auto"
    kernel = int(parts[5]) if len(parts) > 5 else 0
    a, b, c = _operands(q, m, l, n)
    code = {"auto": fq.PATH_AUTO, "m4rm": fq.PATH_M4RM, "mma": fq.PATH_MMA, "karatsuba": fq.PATH_KARATSUBA}[path]
    t = _time(lambda: fq.matmul(a, b, out=c, path=code, kernel=kernel), reps)
    if fq.status() != fq.OK:
        raise RuntimeError("device reported an error")
    print("| q=%d %dx%dx%d | %s | %.3f | %.3e |" % (q, m, l, n, path, t, 2.0 * m * l * n / t * 1e3))


def strassen_table():
    """Direct product against one and two Strassen-Winograd levels, and the
    levels the time model takes (M4RM base products)."""
    print("| field | n | model levels | direct ms | 1 level ms | 2 levels ms |")
    print("|---|---:|---:|---:|---:|---:|")
    for q, n in ((3, 8192), (3, 16384), (3, 32768), (2, 8192), (2, 16384), (2, 32768), (4, 8192), (4, 16384),
                 (5, 8192), (5, 16384), (7, 8192), (7, 16384)):
        a, b, c = _operands(q, n, n, n)
        t = {}
        for lv in (-1, 1, 2):
            if lv == 2 and n < 16384:
                continue
            t[lv] = _time(lambda: fq.matmul(a, b, out=c, path=fq.PATH_M4RM, strassen=lv), 3)
        model = fq.strassen_levels(q, n, n, n, path=fq.PATH_M4RM)
        two = "%.3f" % t[2] if 2 in t else "-"
        print("| %d | %d | %d | %.3f | %.3f | %s |" % (q, n, model, t[-1], t[1], two), flush=True)
        del a, b, c
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="skip the n = 32768 product")
    ap.add_argument("--case", help="time one product only: q,m,l,n[,path[,kernel]]")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--strassen", action="store_true", help="direct vs Strassen-Winograd levels only")
    ap.add_argument("--batched", help="the batch only: q[,auto|m4rm|mma[,count]] (4096 products by default)")
    args = ap.parse_args()
    fq.load()
    if args.case:
        one_case(args.case, args.reps)
        return
    if args.strassen:
        strassen_table()
        return
    if args.batched:
        parts = args.batched.split(",")
        q = int(parts[0])
        path = {"auto": fq.PATH_AUTO, "m4rm": fq.PATH_M4RM, "mma": fq.PATH_MMA}[parts[1] if len(parts) > 1 else "auto"]
        count = int(parts[2]) if len(parts) > 2 else 4096
        t, pps, ops, items = batched_row(q, count=count, reps=args.reps, path=path)
        print("| batched F_%d (%s, %d products) | %.3f ms | %.3e products/s | %.3e field-ops/s | %d items |" % (
            q, parts[1] if len(parts) > 1 else "auto", count, t, pps, ops, items))
        return
    print("| configuration | path | ms | field-ops/s |")
    print("|---|---|---:|---:|")

    def emit(name, rows):
        for p, t, r in rows:
            print("| %s | %s | %.3f | %.3e |" % (name, p, t, r), flush=True)

    for n in (512, 1024, 2048, 4096, 8192, 16384):
        emit("F_3 %d^3" % n, product_rows(3, n, n, n, paths=("m4rm", "mma")))
    emit("F_3 8192^3, A 90% zeros", product_rows(3, 8192, 8192, 8192, sparse=True, paths=("m4rm", "mma")))
    for q, name in ((5, "F_5"), (7, "F_7"), (4, "GF(4)")):
        emit("%s 8192^3" % name, product_rows(q, 8192, 8192, 8192, paths=("m4rm", "mma")))
    emit("F_2 8192^3", product_rows(2, 8192, 8192, 8192, paths=("m4rm", "mma")))
    emit("GF(4) 8192^3, three F_2 products", product_rows(4, 8192, 8192, 8192, paths=("karatsuba",)))
    for q, name in ((8, "F_8"), (9, "F_9"), (25, "F_25"), (27, "F_27"), (49, "F_49"), (125, "F_125")):
        emit("%s 8192^3 (base products on each path)" % name, product_rows(q, 8192, 8192, 8192, paths=("m4rm", "mma")))
    emit("F_3 65536 x 4096 x 4096", product_rows(3, 65536, 4096, 4096, paths=("m4rm", "mma")))
    if not args.quick:
        emit("F_5 32768^3", product_rows(5, 32768, 32768, 32768, paths=("m4rm", "mma"), reps=2))
    print()
    print("| batched (4096 products, m, l, n uniform on 64..1024 step 64, one graph replay) | ms | products/s | field-ops/s | items |")
    print("|---|---:|---:|---:|---:|")
    for q, name in ((3, "F_3"), (5, "F_5")):
        t, pps, ops, items = batched_row(q)
        print("| %s | %.3f | %.3e | %.3e | %d |" % (name, t, pps, ops, items), flush=True)


if __name__ == "__main__":
    main()

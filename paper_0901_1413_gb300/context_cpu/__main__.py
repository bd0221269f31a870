"""Times the CPU bitsliced M4RM at the sizes of the paper's Table 1 (n = 100,
500, 1000, 2500; F_3, F_5, F_7, GF(4)) on one thread and on all host threads,
and, when a GPU is present, the GPU library on the same products.

    python -m paper_0901_1413_gb300.context_cpu [--sizes 100,500,1000,2500]
"""
from __future__ import annotations

import argparse

from . import matmul, threads_used
from .. import inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="100,500,1000,2500")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    sizes = [int(x) for x in args.sizes.split(",")]
    gpu = None
    try:
        import torch
        if torch.cuda.is_available():
            from .. import fq
            from ..measure import _time
            fq.load()
            gpu = (torch, fq, _time)
    except Exception:  # no GPU: CPU columns only
        gpu = None
    allt = threads_used(0)
    print("| field | n | CPU 1 thread ms | CPU %d threads ms | GPU ms |" % allt)
    print("|---|---:|---:|---:|---:|")
    for q, name in ((3, "F_3"), (5, "F_5"), (7, "F_7"), (4, "GF(4)")):
        for n in sizes:
            A = inputs.uniform(q, n, n, seed=n, stream=inputs.STREAM_A)
            B = inputs.uniform(q, n, n, seed=n, stream=inputs.STREAM_B)
            one = min(matmul(q, A, B, threads=1)[1] for _ in range(args.reps))
            many = min(matmul(q, A, B, threads=0)[1] for _ in range(args.reps))
            g = "-"
            if gpu is not None:
                torch, fq, _time = gpu
                a, b = fq.pack(q, torch.from_numpy(A).cuda()), fq.pack(q, torch.from_numpy(B).cuda())
                c = fq.empty(q, n, n)
                g = "%.4f" % _time(lambda: fq.matmul(a, b, out=c), 5)
            print("| %s | %d | %.3f | %.3f | %s |" % (name, n, one, many, g), flush=True)


if __name__ == "__main__":
    main()

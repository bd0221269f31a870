"""fq_matmul_batched_static: the batched product for callers that cannot
allocate device memory (its work list lives in a fixed array inside the
library).  Its results must equal those of fq_matmul_batched on the same
inputs, bit for bit, on consecutive calls with different plans."""
import ctypes

import numpy as np
import pytest
import torch

from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu


def _entry(lib):
    fn = lib.fq_matmul_batched_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 5
    return fn


def _batch(fq, q, shapes, seed):
    a, b = [], []
    for p, (m, l, n) in enumerate(shapes):
        a.append(fq.pack(q, inputs.uniform_torch(q, m, l, seed=seed, stream=2 * p)))
        b.append(fq.pack(q, inputs.uniform_torch(q, l, n, seed=seed, stream=2 * p + 1)))
    return a, b


def _ptrs(xs):
    return torch.tensor([x.data.data_ptr() for x in xs], dtype=torch.int64, device="cuda")


def _outputs(fq, q, shapes):
    outs = []
    for m, l, n in shapes:
        c = fq.empty(q, m, n)
        c.data.fill_(-1)
        outs.append(c)
    return outs


def test_static_workspace_matches_workspace_entry_on_consecutive_calls(fq):
    lib = fq.load()
    run_static = _entry(lib)
    cases = [(3, [(300, 200, 520), (64, 1024, 64), (1, 1, 1), (700, 90, 1100)], 5),
             (5, [(128, 640, 256), (513, 257, 1025), (40, 30, 20)], 6)]
    expected, got = [], []
    for q, shapes, seed in cases:
        a, b = _batch(fq, q, shapes, seed)
        ref = _outputs(fq, q, shapes)
        plan = fq.BatchPlan(q, shapes, path=fq.PATH_M4RM)   # work lists only: fits the fixed array
        ra, rb, rc_ = _ptrs(a), _ptrs(b), _ptrs(ref)
        plan.run(ra, rb, rc_)
        torch.cuda.synchronize()
        expected.append([r.data.clone() for r in ref])
        out = _outputs(fq, q, shapes)
        pa, pb, pc = _ptrs(a), _ptrs(b), _ptrs(out)      # kept alive until the launch is done
        stream = torch.cuda.current_stream()
        rc = run_static(plan._h, ctypes.c_void_p(pa.data_ptr()), ctypes.c_void_p(pb.data_ptr()),
                        ctypes.c_void_p(pc.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == fq.OK
        torch.cuda.synchronize()
        got.append([o.data.clone() for o in out])
    assert fq.status() == fq.OK
    for exp, res in zip(expected, got):
        for e, r in zip(exp, res):
            assert torch.equal(e, r)


def test_static_workspace_refuses_plans_that_do_not_fit(fq):
    lib = fq.load()
    run_static = _entry(lib)
    shapes = np.full((40000, 3), 8, np.int64)           # 40000 products: > 1 MiB of work list
    plan = fq.BatchPlan(3, shapes)
    assert lib.fq_batched_workspace_bytes(plan._h) > (1 << 20)
    rc = run_static(plan._h, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None)
    assert rc == fq.ENOTSUP


def test_static_workspace_refuses_plans_with_tensor_core_products(fq):
    """A plan with tcgen05 products needs its e4m3 arenas, which the fixed
    array cannot hold: refused before anything is enqueued."""
    lib = fq.load()
    run_static = _entry(lib)
    plan = fq.BatchPlan(3, [(256, 512, 512), (64, 64, 64)], path=fq.PATH_MMA)
    assert plan.tc_products == 2
    rc = run_static(plan._h, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None)
    assert rc == fq.ENOTSUP


def test_static_workspace_refuses_capture(fq):
    """The static entry copies its work list from host memory at every call,
    which a graph replay could not repeat: refused while the stream captures,
    with nothing enqueued (the rest of the capture stays valid)."""
    lib = fq.load()
    run_static = _entry(lib)
    q, shapes = 3, [(64, 64, 64)]
    a, b = _batch(fq, q, shapes, 7)
    out = _outputs(fq, q, shapes)
    plan = fq.BatchPlan(q, shapes, path=fq.PATH_M4RM)
    pa, pb, pc = _ptrs(a), _ptrs(b), _ptrs(out)
    x = torch.zeros(1, device="cuda")
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        x.add_(1)
        rc = run_static(plan._h, ctypes.c_void_p(pa.data_ptr()), ctypes.c_void_p(pb.data_ptr()),
                        ctypes.c_void_p(pc.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == fq.ENOTSUP
    g.replay()
    torch.cuda.synchronize()
    assert x.item() == 1.0
    assert fq.status() == fq.OK

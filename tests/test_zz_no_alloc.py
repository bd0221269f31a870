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


def _tiny_f3_batch(count):
    """`count` F_3 products of 8 x 8 by 8 x 8 in three flat device buffers:
    random valid codes (sign bits only where unit bits are set), zero padding;
    the device pointer arrays of A, B and a C buffer filled with ones."""
    words = 2 * 8 * 16                                   # planes x rows x pitch of one 8 x 8 matrix
    g = torch.Generator(device="cuda").manual_seed(count)

    def operand():
        buf = torch.zeros((count, 2, 8, 16), dtype=torch.int64, device="cuda")
        unit = torch.randint(0, 256, (count, 8), device="cuda", generator=g)
        buf[:, 0, :, 0] = unit
        buf[:, 1, :, 0] = unit & torch.randint(0, 256, (count, 8), device="cuda", generator=g)
        return buf

    a, b = operand(), operand()
    c = torch.full((count, words), -1, dtype=torch.int64, device="cuda")
    ptrs = lambda t: t.data_ptr() + torch.arange(count, dtype=torch.int64, device="cuda") * words * 8
    return a, b, c, ptrs(a), ptrs(b), ptrs(c)


def test_static_workspace_limit_is_the_stated_size(fq):
    """The largest plan of 8 x 8 x 8 Four-Russians products whose work list
    fits FQ_BATCH_STATIC_BYTES runs and equals fq_matmul_batched; one product
    more is refused with FQ_ENOTSUP (the size check, not the tensor-core one:
    the plans hold no tcgen05 products)."""
    lib = fq.load()
    run_static = _entry(lib)
    limit = 1 << 20

    def plan_of(count):
        plan = fq.BatchPlan(3, np.full((count, 3), 8, np.int64), path=fq.PATH_M4RM)
        assert plan.tc_products == 0
        return plan, lib.fq_batched_workspace_bytes(plan._h)

    lo, hi = 1, 40000                                   # largest count whose plan fits
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if plan_of(mid)[1] <= limit:
            lo = mid
        else:
            hi = mid - 1
    plan, nbytes = plan_of(lo)
    assert nbytes <= limit < plan_of(lo + 1)[1]
    a, b, c, pa, pb, pc = _tiny_f3_batch(lo)
    ref = torch.full_like(c, -1)
    pr = ref.data_ptr() + torch.arange(lo, dtype=torch.int64, device="cuda") * ref.shape[1] * 8
    plan.run(pa, pb, pr)
    stream = torch.cuda.current_stream()
    assert run_static(plan._h, ctypes.c_void_p(pa.data_ptr()), ctypes.c_void_p(pb.data_ptr()),
                      ctypes.c_void_p(pc.data_ptr()), ctypes.c_void_p(stream.cuda_stream)) == fq.OK
    torch.cuda.synchronize()
    assert fq.status() == fq.OK
    assert torch.equal(ref, c)
    big, _ = plan_of(lo + 1)
    rc = run_static(big._h, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None)
    assert rc == fq.ENOTSUP


def test_static_calls_allocate_no_device_memory(fq):
    """After a first call on the device (which looks up the array's address),
    further calls leave the device's free memory unchanged."""
    lib = fq.load()
    run_static = _entry(lib)
    q, shapes = 3, [(300, 200, 520), (64, 1024, 64), (700, 90, 1100)]
    a, b = _batch(fq, q, shapes, 9)
    out = _outputs(fq, q, shapes)
    plan = fq.BatchPlan(q, shapes, path=fq.PATH_M4RM)
    pa, pb, pc = _ptrs(a), _ptrs(b), _ptrs(out)
    stream = torch.cuda.current_stream()
    args = (plan._h, ctypes.c_void_p(pa.data_ptr()), ctypes.c_void_p(pb.data_ptr()), ctypes.c_void_p(pc.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
    assert run_static(*args) == fq.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert run_static(*args) == fq.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    assert fq.status() == fq.OK


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

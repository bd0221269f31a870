"""The FQ_DEBUG build (libfq_gb300_debug.so): the same library with bounds
checks on every Four-Russians table index (idx < 2^k) and every store of C
(row < m, words within the row pitch), which record FQ_EBOUNDS instead of
reaching memory they must not.  One product per field on each path, and one
batch with both launch kinds, must give the oracle's result with no check
failing."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg(fq):
    return fq.load_debug()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _pack(dbg, fq, q, R):
    res = torch.from_numpy(np.ascontiguousarray(R)).cuda()
    out = fq.empty(q, *R.shape)
    assert dbg.fq_pack(q, R.shape[0], R.shape[1], ctypes.c_void_p(res.data_ptr()), R.shape[1],
                       ctypes.c_void_p(out.data.data_ptr()), _stream()) == fq.OK
    torch.cuda.synchronize()
    return out


def _unpack(dbg, fq, x):
    out = torch.empty((x.rows, x.cols), dtype=torch.uint8, device="cuda")
    assert dbg.fq_unpack(x.q, x.rows, x.cols, ctypes.c_void_p(x.data.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                         x.cols, _stream()) == fq.OK
    return out.cpu().numpy()


@pytest.mark.parametrize("q", (2, 3, 4, 5, 7))
@pytest.mark.parametrize("mln", [(513, 1000, 700), (64, 4100, 1500)])
def test_debug_build_products_pass_their_checks(fq, dbg, q, mln):
    m, l, n = mln
    A = inputs.uniform(q, m, l, seed=q, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=q, stream=inputs.STREAM_B)
    a, b = _pack(dbg, fq, q, A), _pack(dbg, fq, q, B)
    want = oracle.matmul(q, A, B)
    for path in (fq.PATH_M4RM, fq.PATH_MMA):
        c = fq.empty(q, m, n)
        opt = fq.Options(path=path)
        assert dbg.fq_matmul_ex(q, m, l, n, ctypes.c_void_p(a.data.data_ptr()), ctypes.c_void_p(b.data.data_ptr()),
                                ctypes.c_void_p(c.data.data_ptr()), _stream(), ctypes.byref(opt)) == fq.OK
        assert dbg.fq_status(_stream()) == fq.OK, "a bounds check failed (path %d)" % path
        assert np.array_equal(_unpack(dbg, fq, c), want), "path %d" % path


@pytest.mark.parametrize("q", (3, 5))
def test_debug_build_batch_passes_its_checks(fq, dbg, q):
    """An AUTO batch holding tcgen05 products and Four-Russians items."""
    shapes = [(8, 8, 8), (1024, 1024, 1024), (300, 200, 520), (64, 0, 64), (700, 90, 1100)]
    A, B, a, b, c = [], [], [], [], []
    for p, (m, l, n) in enumerate(shapes):
        A.append(inputs.uniform(q, m, l, seed=7, stream=2 * p))
        B.append(inputs.uniform(q, l, n, seed=7, stream=2 * p + 1))
        a.append(_pack(dbg, fq, q, A[-1]) if m and l else fq.empty(q, m, l))
        b.append(_pack(dbg, fq, q, B[-1]) if l and n else fq.empty(q, l, n))
        c.append(fq.empty(q, m, n))
    ptr = lambda xs: torch.tensor([x.data.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    pa, pb, pc = ptr(a), ptr(b), ptr(c)
    sh = np.asarray(shapes, np.int64)
    m, l, n = (np.ascontiguousarray(sh[:, i]) for i in range(3))
    h = ctypes.c_void_p()
    assert dbg.fq_batched_plan_create(q, len(shapes), m.ctypes.data_as(ctypes.c_void_p),
                                      l.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(h)) == fq.OK
    try:
        assert dbg.fq_batched_tc_products(h) > 0 and dbg.fq_batched_items(h) > 0
        ws = torch.empty(dbg.fq_batched_workspace_bytes(h) // 8 + 16, dtype=torch.int64, device="cuda")
        wp = ctypes.c_void_p((ws.data_ptr() + 63) // 64 * 64)
        assert dbg.fq_batched_plan_upload(h, wp, _stream()) == fq.OK
        assert dbg.fq_matmul_batched(h, ctypes.c_void_p(pa.data_ptr()), ctypes.c_void_p(pb.data_ptr()),
                                     ctypes.c_void_p(pc.data_ptr()), wp, _stream()) == fq.OK
        assert dbg.fq_status(_stream()) == fq.OK, "a bounds check failed"
    finally:
        dbg.fq_batched_plan_destroy(h)
    for p, (mm, ll, nn) in enumerate(shapes):
        if mm and nn:
            assert np.array_equal(_unpack(dbg, fq, c[p]), oracle.matmul(q, A[p], B[p])), p

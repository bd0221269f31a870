"""The bounded-wait failure path of the Four-Russians kernels, driven on purpose.

Every hand-over wait between the warps of a CTA is bounded (about two seconds
by default).  fq_debug_wait_limit shortens the bound to a nanosecond, so that
waits which cannot have completed yet give up: the kernel must record
FQ_ETIMEOUT, stop issuing copies, wait for the copies it already issued, skip
lookups whose tables it never received and exit.  Nothing faults or hangs: the
status is read on the host, and the next product on the same device (with the
default bound restored) is exact.

Each compiled kernel runs a product with one row per CTA and many k-row
blocks, so its CTAs spend most of their time waiting for B blocks and tables
that a nanosecond cannot bring."""
import numpy as np
import pytest
import torch

import oracle
from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = (2, 3, 4, 5, 7)


@pytest.fixture
def short_waits(fq):
    lib = fq.load()
    lib.fq_debug_wait_limit(1)
    try:
        yield lib
    finally:
        lib.fq_debug_wait_limit(0)


@pytest.mark.parametrize("q", FIELDS)
def test_every_kernel_times_out_cleanly_and_the_device_stays_usable(fq, short_waits, q):
    m, l, n = 48, 6000, 1100
    A = inputs.uniform(q, m, l, seed=31, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=31, stream=inputs.STREAM_B)
    a, b = fq.pack(q, torch.from_numpy(A).cuda()), fq.pack(q, torch.from_numpy(B).cuda())
    assert fq.status() == fq.OK
    c = fq.empty(q, m, n)
    for info in fq.kernels(q):
        fq.matmul(a, b, out=c, path=fq.PATH_M4RM, kernel=info["index"] + 1, variant=1, strassen=-1)
        torch.cuda.synchronize()                      # the kernel returned: no hang, no fault
        assert fq.status() == fq.ETIMEOUT, info
        assert fq.status() == fq.OK                   # read and cleared
    short_waits.fq_debug_wait_limit(0)
    want = oracle.matmul(q, A, B)
    for info in fq.kernels(q):
        got = fq.unpack(fq.matmul(a, b, path=fq.PATH_M4RM, kernel=info["index"] + 1, variant=1,
                                  strassen=-1)).cpu().numpy()
        assert np.array_equal(got, want), info
    assert fq.status() == fq.OK


def test_default_bound_is_restored(fq, short_waits):
    """fq_debug_wait_limit(0) restores the default bound: a full-size product
    after a timed-out one is exact, on the planner's kernel and with a tile
    of the planner's height."""
    q, m, l, n = 3, 1000, 3000, 1500
    A = inputs.uniform(q, m, l, seed=32, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=32, stream=inputs.STREAM_B)
    a, b = fq.pack(q, torch.from_numpy(A).cuda()), fq.pack(q, torch.from_numpy(B).cuda())
    fq.matmul(a, b, path=fq.PATH_M4RM, variant=1)
    assert fq.status() == fq.ETIMEOUT
    short_waits.fq_debug_wait_limit(0)
    got = fq.unpack(fq.matmul(a, b, path=fq.PATH_M4RM)).cpu().numpy()
    assert fq.status() == fq.OK
    assert np.array_equal(got, oracle.matmul(q, A, B))

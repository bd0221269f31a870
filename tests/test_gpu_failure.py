"""The bounded-wait failure path of the Four-Russians kernels, driven on purpose.

Every hand-over wait between the warps of a CTA is bounded (about two seconds
by default).  fq_debug_stall_block makes one thread of every CTA, on reaching
a chosen k-row block, wait on a barrier that nothing ever completes, and
fq_debug_wait_limit shortens the bound so the test is quick.  The kernel must
record FQ_ETIMEOUT, stop issuing copies, wait for the copies it already issued,
skip lookups whose tables it never received and exit.  Nothing faults or
hangs: the status is read on the host, and the next product on the same
device (with the hooks turned off) is exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = (2, 3, 4, 5, 7)


@pytest.fixture
def hooks(fq):
    lib = fq.load()
    try:
        yield lib
    finally:
        lib.fq_debug_stall_block(-1)
        lib.fq_debug_wait_limit(0)


def _operands(fq, q, m, l, n, seed):
    A = inputs.uniform(q, m, l, seed=seed, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=seed, stream=inputs.STREAM_B)
    return A, B, fq.pack(q, torch.from_numpy(A).cuda()), fq.pack(q, torch.from_numpy(B).cuda())


@pytest.mark.parametrize("q", FIELDS)
def test_every_kernel_times_out_cleanly_and_the_device_stays_usable(fq, hooks, q):
    """Each compiled kernel, stalled at its first block and half way through
    (one row per CTA and full-height tiles), reports FQ_ETIMEOUT and returns;
    afterwards every kernel computes the exact product again."""
    m, l, n = 300, 6000, 1100
    A, B, a, b = _operands(fq, q, m, l, n, seed=31)
    assert fq.status() == fq.OK
    c = fq.empty(q, m, n)
    hooks.fq_debug_wait_limit(50_000)
    for info in fq.kernels(q):
        blocks = -(-l // info["k"])
        for stall in (0, blocks // 2):
            for variant in (1, 0):
                hooks.fq_debug_stall_block(stall)
                fq.matmul(a, b, out=c, path=fq.PATH_M4RM, kernel=info["index"] + 1, variant=variant, strassen=-1)
                torch.cuda.synchronize()                  # the kernel returned: no hang, no fault
                assert fq.status() == fq.ETIMEOUT, (info, stall, variant)
                assert fq.status() == fq.OK               # read and cleared
    hooks.fq_debug_stall_block(-1)
    hooks.fq_debug_wait_limit(0)
    want = oracle.matmul(q, A, B)
    for info in fq.kernels(q):
        got = fq.unpack(fq.matmul(a, b, path=fq.PATH_M4RM, kernel=info["index"] + 1, strassen=-1)).cpu().numpy()
        assert np.array_equal(got, want), info
    assert fq.status() == fq.OK


@pytest.mark.parametrize("q", FIELDS)
def test_tiny_wait_limit_is_harmless(fq, hooks, q):
    """With every wait bounded at one nanosecond of polling, a wait gives up
    whenever its phase has not completed by the time the polling starts to
    count: the kernels may or may not time out, but they always return, and
    the exact product follows."""
    m, l, n = 48, 6000, 1100
    A, B, a, b = _operands(fq, q, m, l, n, seed=33)
    hooks.fq_debug_wait_limit(1)
    for info in fq.kernels(q):
        fq.matmul(a, b, path=fq.PATH_M4RM, kernel=info["index"] + 1, variant=1, strassen=-1)
        torch.cuda.synchronize()
        assert fq.status() in (fq.OK, fq.ETIMEOUT), info
    hooks.fq_debug_wait_limit(0)
    got = fq.unpack(fq.matmul(a, b, path=fq.PATH_M4RM)).cpu().numpy()
    assert fq.status() == fq.OK
    assert np.array_equal(got, oracle.matmul(q, A, B))

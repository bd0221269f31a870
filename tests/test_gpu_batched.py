"""Many products in one persistent launch (fq_matmul_batched), bit-exact
against the oracle, including under CUDA-graph capture and replay."""
import numpy as np
import pytest
import torch

import oracle
from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = (3, 4, 5, 7)


def make_batch(fq, q, shapes, seed):
    A, B, a, b, c = [], [], [], [], []
    for p, (m, l, n) in enumerate(shapes):
        Ap = inputs.uniform(q, m, l, seed=seed, stream=100 + 2 * p)
        Bp = inputs.uniform(q, l, n, seed=seed, stream=101 + 2 * p)
        A.append(Ap)
        B.append(Bp)
        a.append(fq.pack(q, torch.from_numpy(Ap).cuda()) if m and l else fq.empty(q, m, l))
        b.append(fq.pack(q, torch.from_numpy(Bp).cuda()) if l and n else fq.empty(q, l, n))
        out = fq.empty(q, m, n)
        out.data.fill_(-1)
        c.append(out)
    ptr = lambda xs: torch.tensor([x.data.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    return A, B, a, b, c, ptr(a), ptr(b), ptr(c)


PATHS = {"auto": 0, "m4rm": 1, "mma": 2}


def check(fq, q, A, B, c):
    for p in range(len(A)):
        m, n = A[p].shape[0], B[p].shape[1]
        if m == 0 or n == 0:
            continue
        got = fq.unpack(c[p]).cpu().numpy()
        assert np.array_equal(got, oracle.matmul(q, A[p], B[p])), "product %d %s" % (p, (m, A[p].shape[1], n))
        # padding: bits past n and words past them are zero in every plane
        v = c[p].planes_view().cpu().numpy().view(np.uint64)
        w = (n + 63) // 64
        assert not v[:, :, w:].any(), "product %d: padding words" % p
        if n % 64:
            assert not (v[:, :, w - 1] >> np.uint64(n % 64)).any(), "product %d: bits past n" % p


@pytest.mark.parametrize("path", ["auto", "m4rm", "mma"])
@pytest.mark.parametrize("q", FIELDS)
def test_batched_matches_oracle(fq, q, path):
    rng = np.random.default_rng(q)
    shapes = [tuple(int(x) for x in rng.choice(np.arange(64, 577, 64), 3)) for _ in range(20)]
    shapes += [(1, 1, 1), (7, 100, 70), (300, 65, 1100), (1200, 130, 90), (5, 0, 9), (0, 5, 9), (4, 9, 0),
               (129, 1000, 257), (2, 3000, 300)]
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=q)
    plan = fq.BatchPlan(q, shapes, path=PATHS[path])
    if path == "m4rm" or q == 4:
        assert plan.tc_products == 0 and plan.items >= 26
    if path == "mma" and q != 4:
        assert plan.tc_products == len(shapes) - 3      # all but l = 0, m = 0, n = 0
    plan.run(pa, pb, pc)
    assert fq.status() == fq.OK
    check(fq, q, A, B, c)
    # l = 0: C = 0
    assert not c[len(shapes) - 5].data.cpu().numpy()[: 2 * 5 * 16].any()


@pytest.mark.parametrize("q", [3, 5, 7])
def test_batched_mixed_paths_in_one_plan(fq, q):
    """An AUTO plan with products on both paths (an l = 0 product is always a
    Four-Russians zero fill): both launches of one call give the oracle's
    results."""
    shapes = [(8, 8, 8), (16, 40, 24), (1024, 1024, 1024), (512, 896, 768), (64, 0, 64), (960, 320, 1000)]
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=q + 20)
    plan = fq.BatchPlan(q, shapes)
    assert plan.tc_products == 5 and plan.items > 0
    plan.run(pa, pb, pc)
    assert fq.status() == fq.OK
    check(fq, q, A, B, c)


@pytest.mark.parametrize("q", [3, 5, 7])
def test_batched_tensor_core_depth_and_width_edges(fq, q):
    """The tcgen05 batch kernel's operands are padded to 128-deep k-slices and
    256-column tiles, and C is cleared past n: depths from 1 to 257 around
    multiples of 32, widths from 1 to 513 (a last tile holding one to eight
    32-column words, in the first, second and third column block) and row
    counts about one and two 128-row blocks, all in one plan."""
    depths = (1, 31, 32, 33, 64, 65, 96, 97, 127, 128, 129, 200, 255, 257)
    widths = (1, 31, 32, 33, 96, 128, 160, 192, 224, 255, 256, 257, 288, 513)
    rows = (1, 127, 128, 129, 255, 300)
    shapes = [(rows[i % len(rows)], d, widths[(3 * i) % len(widths)]) for i, d in enumerate(depths)]
    shapes += [(rows[(i + 2) % len(rows)], depths[(5 * i) % len(depths)], w) for i, w in enumerate(widths)]
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=q + 60)
    plan = fq.BatchPlan(q, shapes, path=fq.PATH_MMA)
    assert plan.tc_products == len(shapes) and plan.items == 0
    plan.run(pa, pb, pc)
    assert fq.status() == fq.OK
    check(fq, q, A, B, c)


@pytest.mark.parametrize("q", [3, 5])
def test_batched_tensor_core_pairs_with_single_tile_products(fq, q):
    """The tcgen05 batch kernel gives each product to a pair of CTAs that take
    alternate 128 x 256 tiles, so in a one-tile product one CTA of the pair
    has nothing to compute yet takes part in the buffer hand-overs.  Nine
    hundred such products (and a few with several tiles in between) put about
    a dozen on every pair, with runs of one-tile products in the same scratch
    buffer; run twice with new inputs behind the same pointers."""
    rng = np.random.default_rng(70 + q)
    shapes = [(int(rng.choice([1, 37, 64, 100, 128])), int(rng.choice([1, 64, 130, 300])),
               int(rng.choice([1, 64, 200, 256]))) for _ in range(900)]
    shapes[::97] = [(300, 200, 600)] * len(shapes[::97])
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=q + 80)
    plan = fq.BatchPlan(q, shapes, path=fq.PATH_MMA)
    assert plan.tc_products == len(shapes) and plan.items == 0
    plan.run(pa, pb, pc)
    assert fq.status() == fq.OK
    sample = list(range(0, len(shapes), 7)) + list(range(0, len(shapes), 97))
    check(fq, q, [A[i] for i in sample], [B[i] for i in sample], [c[i] for i in sample])
    A2, B2 = [], []
    for p, (m, l, n) in enumerate(shapes):
        A2.append(inputs.uniform(q, m, l, seed=5, stream=2 * p))
        B2.append(inputs.uniform(q, l, n, seed=5, stream=2 * p + 1))
        fq.pack(q, torch.from_numpy(A2[-1]).cuda(), out=a[p])
        fq.pack(q, torch.from_numpy(B2[-1]).cuda(), out=b[p])
    plan.run(pa, pb, pc)
    assert fq.status() == fq.OK
    check(fq, q, [A2[i] for i in sample], [B2[i] for i in sample], [c[i] for i in sample])


@pytest.mark.parametrize("path", ["m4rm", "mma"])
@pytest.mark.parametrize("q", [3, 5])
def test_batched_graph_capture_and_replay(fq, q, path):
    rng = np.random.default_rng(10 + q)
    shapes = [tuple(int(x) for x in rng.choice(np.arange(64, 449, 64), 3)) for _ in range(12)]
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=1)
    plan = fq.BatchPlan(q, shapes, path=PATHS[path])
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        plan.run(pa, pb, pc, stream=stream)          # warm up outside capture
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.run(pa, pb, pc, stream=stream)
    for c_ in c:
        c_.data.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert fq.status() == fq.OK
    check(fq, q, A, B, c)
    # new inputs behind the same pointers, replay again
    A2, B2 = [], []
    for p, (m, l, n) in enumerate(shapes):
        A2.append(inputs.uniform(q, m, l, seed=99, stream=2 * p))
        B2.append(inputs.uniform(q, l, n, seed=99, stream=2 * p + 1))
        fq.pack(q, torch.from_numpy(A2[-1]).cuda(), out=a[p])
        fq.pack(q, torch.from_numpy(B2[-1]).cuda(), out=b[p])
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    check(fq, q, A2, B2, c)


@pytest.mark.slow
@pytest.mark.parametrize("q", [3, 5])
def test_batched_4096_products(fq, q):
    """4096 products with m, l, n uniform over multiples of 64 in [64, 1024]:
    every 97th product against the full oracle, every 7th by a 32-trial
    Freivalds check."""
    shapes = [tuple(int(x) for x in s) for s in inputs.batch_shapes(4096, seed=q)]
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=q)
    plan = fq.BatchPlan(q, shapes)          # AUTO: the time models pick each product's path
    plan.run(pa, pb, pc)
    assert fq.status() == fq.OK
    sample = list(range(0, 4096, 97))
    check(fq, q, [A[i] for i in sample], [B[i] for i in sample], [c[i] for i in sample])
    for p in range(0, 4096, 7):
        got = fq.unpack(c[p]).cpu().numpy()
        assert oracle.freivalds(q, A[p], B[p], got, trials=32, seed=p)


def _tc_max_l(fq, q):
    """Longest l the tcgen05 form takes for q (found through the workspace query)."""
    lib = fq.load()
    lo, hi = 1, 1 << 26
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if lib.fq_tc_workspace_bytes(q, 1, mid, 1) >= 0:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.slow
@pytest.mark.parametrize("q, l, codes", [(7, None, (1, 2, 3)), (3, 1 << 22, (0, 1))])
def test_batched_tensor_core_exact_at_its_range(fq, q, l, codes):
    """The batched tcgen05 kernel at the end of the exact fp32 range.  Deep
    products whose rows of A are all +3 (F_7, at the longest l the form takes:
    partial sums up to 2^24 - 1) or all +1 (F_3, l = 2^22) against random
    positive B, so every step of the tensor-core sum adds a random amount and
    an accumulation that dropped low bits would change the residues; C = A B
    is then a column sum of B.  Short products share the plan, and the deep
    ones are on one and on two 128-row blocks."""
    l = l or _tc_max_l(fq, q)
    a_val = 3 if q == 7 else 1
    n = 70
    rng = np.random.default_rng(q)
    deep = [(3, l, n), (130, l, n)]
    short = [(64, 128, 64), (200, 300, 100)]
    shapes = deep + short
    A, B, a, b, c = [], [], [], [], []
    for p, (m, ll, nn) in enumerate(shapes):
        if p < len(deep):
            Ap = np.full((m, ll), a_val, np.uint8)
            Bp = rng.choice(np.array(codes, np.uint8), size=(ll, nn))
        else:
            Ap = inputs.uniform(q, m, ll, seed=3, stream=2 * p)
            Bp = inputs.uniform(q, ll, nn, seed=3, stream=2 * p + 1)
        A.append(Ap)
        B.append(Bp)
        a.append(fq.pack(q, torch.from_numpy(Ap).cuda()))
        b.append(fq.pack(q, torch.from_numpy(Bp).cuda()))
        out = fq.empty(q, m, nn)
        out.data.fill_(-1)
        c.append(out)
    ptr = lambda xs: torch.tensor([x.data.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    plan = fq.BatchPlan(q, shapes, path=fq.PATH_MMA)
    assert plan.tc_products == len(shapes) and plan.items == 0
    plan.run(ptr(a), ptr(b), ptr(c))
    assert fq.status() == fq.OK
    for p, (m, ll, nn) in enumerate(shapes):
        got = fq.unpack(c[p]).cpu().numpy()
        if p < len(deep):
            want = (a_val * B[p].sum(axis=0, dtype=np.int64)) % q
            assert (got == want[None, :]).all(), "deep product %d" % p
        else:
            assert np.array_equal(got, oracle.matmul(q, A[p], B[p])), "product %d" % p


@pytest.mark.parametrize("q", [3, 5])
def test_batched_stages_one_at_a_time(fq, q):
    """fq_matmul_batched_stages: the tcgen05 kernel and the Four-Russians
    kernel run as separate calls give the oracle's results, like one
    fq_matmul_batched; a plan's product paths are reported."""
    shapes = [(8, 8, 8), (1024, 1024, 1024), (512, 896, 768), (64, 0, 64), (300, 200, 520)]
    A, B, a, b, c, pa, pb, pc = make_batch(fq, q, shapes, seed=q + 40)
    plan = fq.BatchPlan(q, shapes)
    paths = plan.product_paths()
    assert paths.count(fq.PATH_MMA) == plan.tc_products and paths[3] == fq.PATH_M4RM
    for stage in (fq.STAGE_TC, fq.STAGE_M4RM):
        plan.run_stages(pa, pb, pc, stage)
    assert fq.status() == fq.OK
    check(fq, q, A, B, c)

"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/fq.h declares, and the host-only calls behave.  No
kernel is launched (this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fq.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fq_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_0901_1413_gb300 import fq
    return fq.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fq_pack", "fq_unpack", "fq_matmul", "fq_matmul_ex", "fq_add", "fq_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_layout_helpers(lib):
    assert [lib.fq_planes(q) for q in (2, 3, 4, 5, 6, 7, 8)] == [1, 2, 2, 3, 0, 3, 3]
    assert [lib.fq_planes(q) for q in (9, 16, 25, 27, 49, 125, 343)] == [4, 0, 6, 6, 6, 9, 0]
    assert lib.fq_pitch_words(0) == 0
    assert lib.fq_pitch_words(1) == 16
    assert lib.fq_pitch_words(1024) == 16
    assert lib.fq_pitch_words(1025) == 32
    assert lib.fq_pitch_words(-1) == -1
    assert lib.fq_planes_words(5, 3, 65) == 3 * 3 * 16
    assert lib.fq_planes_words(6, 3, 65) == -1


def test_argument_errors_return_before_any_launch(lib):
    from paper_0901_1413_gb300 import fq
    vp = ctypes.c_void_p
    # bad field, negative sizes, null or misaligned pointers: all EINVAL, no CUDA call
    assert lib.fq_matmul(6, 4, 4, 4, vp(16), vp(32), vp(48), None) == fq.EINVAL
    assert lib.fq_matmul(3, -1, 4, 4, vp(16), vp(32), vp(48), None) == fq.EINVAL
    assert lib.fq_matmul(3, 4, 4, 4, None, vp(32), vp(48), None) == fq.EINVAL
    assert lib.fq_matmul(3, 4, 4, 4, vp(16), vp(32), vp(8), None) == fq.EINVAL
    assert lib.fq_matmul(3, 4, 4, 4, vp(16), vp(32), vp(16), None) == fq.EINVAL   # C aliases A
    assert lib.fq_pack(3, 2, 70, vp(16), 69, vp(16), None) == fq.EINVAL           # ld < cols
    assert lib.fq_unpack(5, 2, 3, None, vp(16), 3, None) == fq.EINVAL
    assert lib.fq_add(3, 2, 3, vp(16), vp(16), vp(16), 2, None) == fq.EINVAL      # sub flag
    opt = fq.Options(path=7)
    assert lib.fq_matmul_ex(3, 4, 4, 4, vp(16), vp(32), vp(48), None, ctypes.byref(opt)) == fq.EINVAL
    opt = fq.Options(k=11)
    assert lib.fq_matmul_ex(3, 4, 4, 4, vp(16), vp(32), vp(48), None, ctypes.byref(opt)) == fq.EINVAL
    # the matrix-level (Karatsuba) path exists for GF(4) and the extension fields only
    opt = fq.Options(path=fq.PATH_KARATSUBA)
    for q in (2, 3, 5, 7):
        assert lib.fq_matmul_ex(q, 4, 4, 4, vp(16), vp(32), vp(48), None, ctypes.byref(opt)) == fq.EINVAL
    assert lib.fq_matmul(16, 4, 4, 4, vp(16), vp(32), vp(48), None) == fq.EINVAL  # no F_16
    assert lib.fq_matmul(9, 4, 4, 4, vp(16), vp(32), vp(16), None) == fq.EINVAL   # C aliases A
    # empty products are no-ops
    assert lib.fq_matmul(3, 0, 4, 4, None, None, None, None) == fq.OK
    assert lib.fq_matmul(3, 4, 4, 0, None, None, None, None) == fq.OK


def test_error_strings(lib):
    assert lib.fq_error_string(0) == b"ok"
    assert lib.fq_error_string(4) == b"bounded device wait timed out"
    assert lib.fq_error_string(7) == b"bounds check failed (debug build)"
    assert lib.fq_error_string(99) == b"unknown status"


def test_kernel_table(lib):
    from paper_0901_1413_gb300 import fq
    for q in (2, 3, 4, 5, 7):
        ks = fq.kernels(q)
        assert ks and all(6 <= k["k"] <= 10 and k["max_rows"] > 0 and k["cols"] % 512 == 0 for k in ks)
    assert lib.fq_kernel_count(6) == 0
    assert lib.fq_kernel_count(9) == 0          # extension fields use their base field's kernels
    k = ctypes.c_int()
    assert lib.fq_kernel_info(3, 10_000, ctypes.byref(k), None, None, None) == fq.EINVAL


def _plan_layout_model(q, shapes, path):
    """Workspace bytes, items, tcgen05 products and tiles of a batched plan
    forced onto one path, from the layout include/fq.h describes: header 64,
    shapes 24 each (64-aligned), Four-Russians items 32 each (tiles of C's
    pitch: 512 rows x 512 columns for F_3 and GF(4), 256 x 1024 for F_5 and
    F_7); for tcgen05 products 64-byte records, the 77 group list starts and
    the product list (4 bytes each), the 2 x 76 buffer starts (8 bytes), each
    part 64-aligned; then the groups' scratch buffers, 1024-aligned, of
    128-byte rows.  Products go to 76 groups (pairs of CTAs) longest first,
    each to the least-loaded one by the plan's cost model; a group takes its
    products in the reverse order, and its buffer b holds the largest of its
    products b, b + 2, ...:
    m rounded up to 128 plus n rounded up to 256, times l rounded up to 128
    over 128, rows."""
    from paper_0901_1413_gb300 import fq
    cdiv = lambda a, b: -(-a // b)
    up = lambda x, a: cdiv(x, a) * a
    tc_max_l = ((1 << 24) - 1) // max(1, (q - 1) // 2) ** 2
    # Four-Russians item tiles: rows x 64-bit words (two-plane fields / three-plane fields)
    mt, ctw = (512, 8) if q in (3, 4) else (256, 16)
    items = tiles = 0
    tc = []
    for m, l, n in shapes:
        if m == 0 or n == 0:
            continue
        if path == fq.PATH_MMA and q in (3, 5, 7) and 0 < l <= tc_max_l and n <= (1 << 30):
            la, nr = up(l, 128), up(n, 256)
            tiles += cdiv(m, 128) * (nr // 256)
            cycles = (cdiv(m, 128) * (nr // 256)) * (la // 128) * 760.0 + float((m + n) * la) * (2.07e9 * 152.0 / 3.0e12)
            tc.append((cycles, cdiv(m, 128) * la + nr * (la // 128)))
        else:
            items += cdiv(m, mt) * (fq.pitch_words(n) // ctw)
    off = 64 + up(24 * len(shapes), 64) + 32 * items
    if tc:
        order = sorted(range(len(tc)), key=lambda i: -tc[i][0])
        load, per = [0.0] * 76, [[] for _ in range(76)]
        for i in order:
            c = min(range(76), key=lambda k: (load[k], k))
            per[c].append(i)
            load[c] += tc[i][0]
        rows = 0
        for c in range(76):
            lst = per[c][::-1]
            rows += max([tc[i][1] for i in lst[0::2]] or [0]) + max([tc[i][1] for i in lst[1::2]] or [0])
        for size in (64 * len(tc), 4 * 77, 4 * len(tc), 8 * 152):
            off = up(off, 64) + size
        off = up(off, 1024) + 128 * rows
    return off, items, len(tc), tiles


def test_batch_plan_layout_matches_model(lib):
    """Random shape sets (ragged sizes, empty products, l = 0) on both forced
    paths: the library's plan has the model's workspace bytes and counts."""
    import numpy as np
    from paper_0901_1413_gb300 import fq
    i64p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rng = np.random.default_rng(2024)
    for trial in range(40):
        q = (3, 5, 7, 4)[trial % 4]
        count = int(rng.integers(1, 60))
        sh = rng.integers(0, 1500, size=(count, 3)).astype(np.int64)
        sh[rng.random((count, 3)) < 0.05] = 0
        m, l, n = (np.ascontiguousarray(sh[:, i]) for i in range(3))
        for path in (fq.PATH_M4RM, fq.PATH_MMA):
            h = ctypes.c_void_p()
            assert lib.fq_batched_plan_create_ex(q, count, i64p(m), i64p(l), i64p(n), path, ctypes.byref(h)) == fq.OK
            want = _plan_layout_model(q, sh.tolist(), path)
            got = (lib.fq_batched_workspace_bytes(h), lib.fq_batched_items(h), lib.fq_batched_tc_products(h),
                   lib.fq_batched_tc_tiles(h))
            assert lib.fq_batched_plan_destroy(h) == fq.OK
            assert got == want, (q, path, trial)


def test_batch_plan_32_bit_limits(lib):
    """The batched tcgen05 kernel addresses scratch rows with 32-bit TMA
    coordinates: a plan whose scratch would reach 2^31 rows of 128 bytes is
    refused (and none is made); n above 2^30 keeps a product off the tcgen05
    path."""
    import numpy as np
    from paper_0901_1413_gb300 import fq
    i64p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    la = (1 << 24) - 128            # within F_3's exact fp32 range; 131071 k-slices
    n = np.array([64], np.int64)
    l = np.array([la], np.int64)
    h = ctypes.c_void_p()
    # 16512 rows (129 row blocks) x 131071 k-slices = 2^31 + 16.6e6 scratch rows for A alone
    m = np.array([16512], np.int64)
    assert lib.fq_batched_plan_create_ex(3, 1, i64p(m), i64p(l), i64p(n), fq.PATH_MMA, ctypes.byref(h)) == fq.ENOTSUP
    assert not h.value
    # 128 rows of the same depth: 16.8e6 rows of A and 33.6e6 of B^T, accepted
    m = np.array([128], np.int64)
    assert lib.fq_batched_plan_create_ex(3, 1, i64p(m), i64p(l), i64p(n), fq.PATH_MMA, ctypes.byref(h)) == fq.OK
    assert lib.fq_batched_tc_products(h) == 1
    assert lib.fq_batched_tc_tiles(h) == 1
    assert lib.fq_batched_workspace_bytes(h) > (128 + 256) * la
    assert lib.fq_batched_plan_destroy(h) == fq.OK
    # n = 2^30 + 64: Four Russians even when the tensor path is asked for
    m, l, n = (np.array([v], np.int64) for v in (1, 64, (1 << 30) + 64))
    assert lib.fq_batched_plan_create_ex(3, 1, i64p(m), i64p(l), i64p(n), fq.PATH_MMA, ctypes.byref(h)) == fq.OK
    assert lib.fq_batched_tc_products(h) == 0
    assert lib.fq_batched_items(h) == fq.pitch_words((1 << 30) + 64) // 8
    assert lib.fq_batched_plan_destroy(h) == fq.OK


def test_batch_plan_host_side(lib):
    """Plan creation is host-only: sizes, item count, workspace bytes, errors."""
    import numpy as np
    from paper_0901_1413_gb300 import fq
    i64p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m = np.array([100, 2000, 0, 64], np.int64)
    l = np.array([70, 64, 5, 0], np.int64)
    n = np.array([600, 64, 9, 1100], np.int64)
    h = ctypes.c_void_p()
    assert lib.fq_batched_plan_create_ex(3, 4, i64p(m), i64p(l), i64p(n), fq.PATH_M4RM, ctypes.byref(h)) == fq.OK
    # items: one per row tile x column tile of the pitch (512-row x 512-column
    # tiles; tiles of padding only are zero-fill items): 1 x 2, 4 x 2, 0, 1 x 4
    assert lib.fq_batched_items(h) == 2 + 8 + 0 + 4
    assert lib.fq_batched_tc_products(h) == 0
    assert lib.fq_batched_workspace_bytes(h) == 64 + 128 + 14 * 32
    assert lib.fq_batched_plan_destroy(h) == fq.OK
    # every product the tcgen05 form takes (l > 0; m = 0 needs no work): 100 x 70
    # x 600 (1 x 3 tiles of 128 x 256) and 2000 x 64 x 64 (16 x 1); l = 0 stays
    # a Four-Russians product (4 zero-fill items).  Tables: header 64, shapes 128,
    # items 4 x 32, products 2 x 64, group list starts 77 x 4, group lists 2 x 4,
    # buffer starts 152 x 8, each part 64-byte aligned -> 1440 bytes; scratch
    # (1024-aligned): the larger product (2000 x 64 x 64: 16 row blocks x 128
    # rows of A + 256 rows of B^T) on group 0, the other on group 1, each in its
    # buffer 0: 2304 and 128 + 768 rows of 128 bytes.
    assert lib.fq_batched_plan_create_ex(3, 4, i64p(m), i64p(l), i64p(n), fq.PATH_MMA, ctypes.byref(h)) == fq.OK
    assert lib.fq_batched_items(h) == 4
    assert lib.fq_batched_tc_products(h) == 2
    assert lib.fq_batched_tc_tiles(h) == 3 + 16
    assert lib.fq_batched_workspace_bytes(h) == 2048 + (2304 + 896) * 128
    assert [lib.fq_batched_product_path(h, p) for p in range(4)] == [fq.PATH_MMA, fq.PATH_MMA, fq.PATH_M4RM,
                                                                     fq.PATH_M4RM]
    assert lib.fq_batched_product_path(h, 4) == -fq.EINVAL
    assert lib.fq_batched_product_path(h, -1) == -fq.EINVAL
    assert lib.fq_batched_product_path(None, 0) == -fq.EINVAL
    # stage masks outside 0 .. FQ_BATCH_STAGE_ALL are refused before any launch
    for bad_mask in (-1, 4, 100):
        assert lib.fq_matmul_batched_stages(h, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8),
                                            ctypes.c_void_p(64), None, bad_mask) == fq.EINVAL
    assert lib.fq_batched_plan_destroy(h) == fq.OK
    assert lib.fq_batched_plan_create_ex(3, 4, i64p(m), i64p(l), i64p(n), 9, ctypes.byref(h)) == fq.EINVAL
    assert lib.fq_batched_tc_products(None) == -1
    # GF(4) products stay on Four Russians even when the tensor path is asked for
    assert lib.fq_batched_plan_create_ex(4, 4, i64p(m), i64p(l), i64p(n), fq.PATH_MMA, ctypes.byref(h)) == fq.OK
    assert lib.fq_batched_tc_products(h) == 0
    assert lib.fq_batched_plan_destroy(h) == fq.OK
    # the 4096-product batch workload: the models put (almost) every product on
    # the tcgen05 path (a 128 x 256 tile costs ~760 cycles per 128-deep step;
    # a Four-Russians item pays ~2000 units of set-up alone)
    from paper_0901_1413_gb300 import inputs
    bs = np.asarray(inputs.batch_shapes(4096, seed=3), np.int64).reshape(-1, 3)
    bm, bl, bn = (np.ascontiguousarray(bs[:, i]) for i in range(3))
    assert lib.fq_batched_plan_create(3, 4096, i64p(bm), i64p(bl), i64p(bn), ctypes.byref(h)) == fq.OK
    assert lib.fq_batched_tc_products(h) > 4000
    assert lib.fq_batched_plan_destroy(h) == fq.OK
    assert lib.fq_batched_plan_create(3, 4, i64p(m), i64p(l), i64p(n), ctypes.byref(h)) == fq.OK
    assert lib.fq_batched_plan_upload(h, ctypes.c_void_p(8), None) == fq.EINVAL      # misaligned
    assert lib.fq_matmul_batched(h, None, None, None, ctypes.c_void_p(64), None) == fq.EINVAL
    assert lib.fq_matmul_batched_static(h, None, None, None, None) == fq.EINVAL
    assert lib.fq_matmul_batched_static(None, None, None, None, None) == fq.EINVAL
    assert lib.fq_batched_plan_destroy(h) == fq.OK
    bad = np.array([-1], np.int64)
    assert lib.fq_batched_plan_create(3, 1, i64p(bad), i64p(bad), i64p(bad), ctypes.byref(h)) == fq.EINVAL
    assert lib.fq_batched_plan_create(6, 1, i64p(m), i64p(l), i64p(n), ctypes.byref(h)) == fq.EINVAL
    assert lib.fq_batched_workspace_bytes(None) == -1


def test_autotune_cache_host_side(lib):
    from paper_0901_1413_gb300 import fq
    assert lib.fq_autotune_clear() == fq.OK
    assert lib.fq_autotune_lookup(3, 10, 10, 10, None, None) == fq.ENOTSUP
    assert lib.fq_autotune(6, 10, 10, 10, None, None, None, None, None) == fq.EINVAL
    p, k = ctypes.c_int(-1), ctypes.c_int(-1)
    assert lib.fq_auto_choice(6, 10, 10, 10, ctypes.byref(p), ctypes.byref(k)) == fq.EINVAL
    assert lib.fq_auto_choice(3, -1, 10, 10, ctypes.byref(p), ctypes.byref(k)) == fq.EINVAL
    assert lib.fq_auto_choice(3, 10, 10, 10, None, ctypes.byref(k)) == fq.EINVAL
    # an empty product needs no device and takes the M4RM planner
    assert lib.fq_auto_choice(3, 0, 10, 10, ctypes.byref(p), ctypes.byref(k)) == fq.OK
    assert (p.value, k.value) == (fq.PATH_M4RM, 0)
    # tensor-core workspace sizes (host-only)
    # e4m3 operand bytes (A: m x la, B transposed: 64 pitch(n) x la, la = l up
    # to a multiple of 128); GF(4): three such pairs (A0 B0, A1 B1, (A0+A1)(B0+B1))
    assert lib.fq_tc_workspace_bytes(3, 100, 200, 300) == (100 + 1024) * 256
    assert lib.fq_tc_workspace_bytes(5, 100, 200, 3000) == (100 + 3072) * 256
    assert lib.fq_tc_workspace_bytes(4, 100, 200, 300) == 3 * (100 + 1024) * 256
    assert lib.fq_tc_workspace_bytes(4, 1, 128, 1) == 3 * (1 + 1024) * 128
    assert lib.fq_tc_workspace_bytes(4, 1, 129, 1) == 3 * (1 + 1024) * 256
    assert lib.fq_tc_workspace_bytes(4, 1, (1 << 24) - 1, 1) > 0
    assert lib.fq_tc_workspace_bytes(4, 1, 1 << 24, 1) == -1
    assert lib.fq_tc_workspace_bytes(6, 100, 200, 300) == -1
    assert lib.fq_tc_workspace_bytes(9, 100, 200, 300) == -1
    assert lib.fq_tc_workspace_bytes(7, 10, 2_000_000, 10) == -1                 # beyond exact fp32 sums
    # packed e2m1 operands (form 5: more than 128 rows, l >= 2048): rows of
    # la / 2 bytes, la = l up to a multiple of 256
    assert lib.fq_tc_workspace_bytes(3, 300, 2100, 300) == (300 + 1024) * 2304 // 2
    assert lib.fq_tc_workspace_bytes(4, 129, 2048, 1025) == 3 * (129 + 2048) * 1024
    assert lib.fq_tc_workspace_bytes(3, 300, 2047, 300) == (300 + 1024) * 2048    # e4m3, form 3
    # the form a shape takes (host-only)
    assert lib.fq_tc_form(3, 128, 5000, 300) == 2
    assert lib.fq_tc_form(3, 129, 2047, 300) == 3
    assert lib.fq_tc_form(5, 129, 2048, 300) == 5
    assert lib.fq_tc_form(7, 16384, 16384, 16384) == 5
    assert lib.fq_tc_form(7, 10, 2_000_000, 10) == -fq.ENOTSUP
    assert lib.fq_tc_form(6, 10, 10, 10) == -fq.EINVAL
    assert lib.fq_tc_form(3, -1, 10, 10) == -fq.EINVAL
    vp = ctypes.c_void_p
    assert lib.fq_tc_prepare(7, 10, 2_000_000, 10, vp(16), vp(16), vp(16), None) == fq.ENOTSUP
    assert lib.fq_tc_multiply(6, 10, 10, 10, vp(16), vp(16), None) == fq.EINVAL
    # planned kernel query: argument errors and device-free answers
    assert lib.fq_planned_kernel(6, 10, 10, 10, None) == -fq.EINVAL
    assert lib.fq_planned_kernel(9, 10, 10, 10, None) == -fq.EINVAL      # extension fields: none
    opt = fq.Options(kernel=2)
    assert lib.fq_planned_kernel(3, 10, 10, 10, ctypes.byref(opt)) == 2
    opt = fq.Options(kernel=10_000)
    assert lib.fq_planned_kernel(3, 10, 10, 10, ctypes.byref(opt)) == -fq.EINVAL
    # Strassen level query: argument errors and device-free answers
    opt = fq.Options(strassen=-2)
    assert lib.fq_strassen_levels(3, 4096, 4096, 4096, ctypes.byref(opt)) == -fq.EINVAL
    assert lib.fq_strassen_levels(6, 4096, 4096, 4096, None) == -fq.EINVAL
    assert lib.fq_strassen_levels(3, 0, 4096, 4096, None) == 0
    assert lib.fq_strassen_levels(9, 4096, 4096, 4096, None) == 0
    # extension fields always take the matrix-level products
    for q in (8, 9, 25, 27, 49, 125):
        assert lib.fq_auto_choice(q, 100, 100, 100, ctypes.byref(p), ctypes.byref(k)) == fq.OK
        assert (p.value, k.value) == (fq.PATH_KARATSUBA, 0)


def test_wait_limit_hook_is_host_only(lib):
    """fq_debug_wait_limit and fq_debug_stall_block only store what later
    launches carry: they need no device, accept any value, and 0 (-1) turn
    them off."""
    from paper_0901_1413_gb300 import fq
    assert lib.fq_debug_wait_limit(1) == fq.OK
    assert lib.fq_debug_wait_limit(-5) == fq.OK
    assert lib.fq_debug_wait_limit(0) == fq.OK
    assert lib.fq_debug_stall_block(3) == fq.OK
    assert lib.fq_debug_stall_block(-1) == fq.OK


def test_autotune_cache_save_and_load(lib, tmp_path):
    """The autotune cache round-trips through its JSON file (host only); a
    malformed file or an entry the library cannot honour is refused whole."""
    import json
    from paper_0901_1413_gb300 import fq
    nk3 = lib.fq_kernel_count(3)
    good = {"format": "fq-autotune-1",
            "entries": [[3, 100, 200, 300, fq.PATH_M4RM, nk3], [5, 8192, 8192, 8192, fq.PATH_MMA, 0],
                        [2, 1, 1, 1, fq.PATH_M4RM, 0]]}
    src = tmp_path / "tune.json"
    src.write_text(json.dumps(good, indent=3))
    assert lib.fq_autotune_clear() == fq.OK
    assert lib.fq_autotune_load(str(src).encode()) == fq.OK
    path, kernel = ctypes.c_int(), ctypes.c_int()
    for q, m, l, n, p, k in good["entries"]:
        assert lib.fq_autotune_lookup(q, m, l, n, ctypes.byref(path), ctypes.byref(kernel)) == fq.OK
        assert (path.value, kernel.value) == (p, k)
    dst = tmp_path / "saved.json"
    assert lib.fq_autotune_save(str(dst).encode()) == fq.OK
    saved = json.loads(dst.read_text())
    assert saved["format"] == "fq-autotune-1"
    assert sorted(map(tuple, saved["entries"])) == sorted(map(tuple, good["entries"]))
    # loading merges: a later file replaces the choice of the same shape
    src.write_text(json.dumps({"entries": [[3, 100, 200, 300, fq.PATH_MMA, 0]], "format": "fq-autotune-1"}))
    assert lib.fq_autotune_load(str(src).encode()) == fq.OK
    assert lib.fq_autotune_lookup(3, 100, 200, 300, ctypes.byref(path), ctypes.byref(kernel)) == fq.OK
    assert (path.value, kernel.value) == (fq.PATH_MMA, 0)
    before = dst.read_text()
    bad_docs = [
        "", "{}", "[]", '{"format": "fq-autotune-1"}', '{"entries": []}',
        '{"format": "fq-autotune-2", "entries": []}',
        '{"format": "fq-autotune-1", "entries": [[3, 1, 1, 1, 1]]}',            # five numbers
        '{"format": "fq-autotune-1", "entries": [[3, 1, 1, 1, 1, 0]], "x": 1}',  # unknown key
        '{"format": "fq-autotune-1", "entries": [[3, 1, 1, 1, 1, 0]]} trailing',
        '{"format": "fq-autotune-1", "entries": [[6, 1, 1, 1, 1, 0]]}',          # no F_6
        '{"format": "fq-autotune-1", "entries": [[9, 1, 1, 1, 1, 0]]}',          # F_9: no kernels of its own
        '{"format": "fq-autotune-1", "entries": [[3, -1, 1, 1, 1, 0]]}',         # negative size
        '{"format": "fq-autotune-1", "entries": [[3, 1, 1, 1, 3, 0]]}',          # Karatsuba is no tuned path
        '{"format": "fq-autotune-1", "entries": [[3, 1, 1, 1, 2, 1]]}',          # tensor path with a kernel
        '{"format": "fq-autotune-1", "entries": [[3, 1, 1, 1, 1, %d]]}' % (nk3 + 1),  # no such kernel
        '{"format": "fq-autotune-1", "entries": [[3, 7, 7, 7, 1, 0], [3, 1, 1, 1, 1, -1]]}',  # one bad entry
    ]
    for doc in bad_docs:
        src.write_text(doc)
        assert lib.fq_autotune_load(str(src).encode()) == fq.EINVAL, doc
    assert lib.fq_autotune_lookup(3, 7, 7, 7, None, None) == fq.ENOTSUP       # nothing of a refused file merged
    assert lib.fq_autotune_load(str(tmp_path / "missing.json").encode()) == fq.EINVAL
    assert lib.fq_autotune_load(None) == fq.EINVAL
    assert lib.fq_autotune_save(None) == fq.EINVAL
    assert lib.fq_autotune_save(str(tmp_path / "no" / "dir.json").encode()) == fq.EINVAL
    assert lib.fq_autotune_clear() == fq.OK
    assert lib.fq_autotune_save(str(dst).encode()) == fq.OK
    assert json.loads(dst.read_text())["entries"] == []
    assert before  # the earlier save was a full document


def test_injected_host_allocation_failure(lib):
    """Every host allocation point of plan building, made to fail in turn,
    gives FQ_ENOMEM and no plan; past the last point the plan is made; the
    upload's host image of the tables fails before any device call."""
    import numpy as np
    from paper_0901_1413_gb300 import fq
    i64p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m = np.array([100, 2000, 0, 64], np.int64)
    l = np.array([70, 64, 5, 0], np.int64)
    n = np.array([600, 64, 9, 1100], np.int64)
    h = ctypes.c_void_p()
    failures = 0
    try:
        for after in range(200):
            assert lib.fq_debug_fail_host_alloc(after) == fq.OK
            rc = lib.fq_batched_plan_create_ex(3, 4, i64p(m), i64p(l), i64p(n), fq.PATH_MMA, ctypes.byref(h))
            if rc == fq.OK:
                break
            assert rc == fq.ENOMEM
            assert not h.value
            failures += 1
        else:
            raise AssertionError("plan creation never succeeded")
        assert failures >= 6          # the plan object, four shapes, a tcgen05 product, an item ...
        lib.fq_debug_fail_host_alloc(-1)
        assert lib.fq_batched_tc_products(h) == 2
        lib.fq_debug_fail_host_alloc(0)
        assert lib.fq_batched_plan_upload(h, ctypes.c_void_p(64), None) == fq.ENOMEM
    finally:
        lib.fq_debug_fail_host_alloc(-1)
        if h.value:
            lib.fq_batched_plan_destroy(h)

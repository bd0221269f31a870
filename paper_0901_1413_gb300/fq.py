"""Python binding of the C ABI in ``include/fq.h`` (ctypes; argument marshalling only).

Every computation runs in the CUDA library ``_build/libfq_gb300.so``; PyTorch is
used only for device memory and streams.  There is no CPU path: if the library
cannot be built or loaded, ``load()`` raises.

A packed matrix is a ``Packed``: field size q, shape (rows, cols) and a flat
int64 CUDA tensor holding the plane-major bit-planes (``fq_planes(q) * rows *
fq_pitch_words(cols)`` 64-bit words).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import build as _build

OK, EINVAL, EVALUE, ECUDA, ETIMEOUT, ENOTSUP, ENOMEM, EBOUNDS = range(8)
PATH_AUTO, PATH_M4RM, PATH_MMA, PATH_KARATSUBA = 0, 1, 2, 3
STAGE_TC, STAGE_M4RM, STAGE_ALL = 1, 2, 3

_lib = None


class FqError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = "%s failed: %s" % (what, _lib.fq_error_string(status).decode() if _lib else status)
        if status == ECUDA and _lib is not None:
            msg += " (%s)" % _lib.fq_last_cuda_error().decode()
        super().__init__(msg)


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("k", ctypes.c_int), ("chunk", ctypes.c_int64),
                ("variant", ctypes.c_int), ("kernel", ctypes.c_int), ("strassen", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


_lib_debug = None


def load():
    """Build (if stale) and load the CUDA library; returns the ctypes handle."""
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


def load_debug():
    """Build (if stale) and load the FQ_DEBUG library (same ABI; its kernels
    bounds-check table indices and stores and record FQ_EBOUNDS); returns its
    own ctypes handle, independent of load()'s."""
    global _lib_debug
    if _lib_debug is None:
        _lib_debug = _bind(ctypes.CDLL(_build.build(debug=True)))
    return _lib_debug


def _bind(lib):
    """Argument and result types of every entry point of include/fq.h."""
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    sig = {
        "fq_planes": (i32, [i32]),
        "fq_pitch_words": (i64, [i64]),
        "fq_planes_words": (i64, [i32, i64, i64]),
        "fq_pack": (i32, [i32, i64, i64, vp, i64, vp, vp]),
        "fq_unpack": (i32, [i32, i64, i64, vp, vp, i64, vp]),
        "fq_add": (i32, [i32, i64, i64, vp, vp, vp, i32, vp]),
        "fq_matmul": (i32, [i32, i64, i64, i64, vp, vp, vp, vp]),
        "fq_matmul_ex": (i32, [i32, i64, i64, i64, vp, vp, vp, vp, ctypes.POINTER(Options)]),
        "fq_status": (i32, [vp]),
        "fq_release_scratch": (i32, []),
        "fq_kernel_count": (i32, [i32]),
        "fq_kernel_info": (i32, [i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                 ctypes.POINTER(i32)]),
        "fq_batched_plan_create": (i32, [i32, i32, vp, vp, vp, ctypes.POINTER(vp)]),
        "fq_batched_plan_create_ex": (i32, [i32, i32, vp, vp, vp, i32, ctypes.POINTER(vp)]),
        "fq_batched_workspace_bytes": (i64, [vp]),
        "fq_batched_items": (i64, [vp]),
        "fq_batched_tc_products": (i64, [vp]),
        "fq_batched_tc_tiles": (i64, [vp]),
        "fq_batched_plan_upload": (i32, [vp, vp, vp]),
        "fq_matmul_batched": (i32, [vp, vp, vp, vp, vp, vp]),
        "fq_matmul_batched_static": (i32, [vp, vp, vp, vp, vp]),
        "fq_matmul_batched_stages": (i32, [vp, vp, vp, vp, vp, vp, i32]),
        "fq_batched_product_path": (i32, [vp, i32]),
        "fq_debug_wait_limit": (i32, [i64]),
        "fq_debug_stall_block": (i32, [i64]),
        "fq_debug_fail_host_alloc": (i32, [i64]),
        "fq_batched_plan_destroy": (i32, [vp]),
        "fq_autotune": (i32, [i32, i64, i64, i64, vp, vp, vp, vp, vp]),
        "fq_autotune_lookup": (i32, [i32, i64, i64, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "fq_autotune_clear": (i32, []),
        "fq_autotune_save": (i32, [ctypes.c_char_p]),
        "fq_autotune_load": (i32, [ctypes.c_char_p]),
        "fq_auto_choice": (i32, [i32, i64, i64, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "fq_strassen_levels": (i32, [i32, i64, i64, i64, ctypes.POINTER(Options)]),
        "fq_planned_kernel": (i32, [i32, i64, i64, i64, ctypes.POINTER(Options)]),
        "fq_tc_form": (i32, [i32, i64, i64, i64]),
        "fq_tc_workspace_bytes": (i64, [i32, i64, i64, i64]),
        "fq_tc_prepare": (i32, [i32, i64, i64, i64, vp, vp, vp, vp]),
        "fq_tc_multiply": (i32, [i32, i64, i64, i64, vp, vp, vp]),
        "fq_error_string": (ctypes.c_char_p, [i32]),
        "fq_last_cuda_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _check(rc: int, what: str):
    if rc != OK:
        raise FqError(rc, what)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def planes(q: int) -> int:
    return load().fq_planes(q)


def pitch_words(cols: int) -> int:
    return load().fq_pitch_words(cols)


@dataclass
class Packed:
    q: int
    rows: int
    cols: int
    data: torch.Tensor  # flat int64, device

    @property
    def pitch(self) -> int:
        return pitch_words(self.cols)

    def planes_view(self) -> torch.Tensor:
        """(planes, rows, pitch) view of the words."""
        return self.data.view(planes(self.q), self.rows, self.pitch)


def empty(q: int, rows: int, cols: int, device=None) -> Packed:
    words = load().fq_planes_words(q, rows, cols)
    if words < 0:
        raise FqError(EINVAL, "fq_planes_words")
    dev = torch.device("cuda") if device is None else torch.device(device)
    return Packed(q, rows, cols, torch.empty(max(words, 1), dtype=torch.int64, device=dev))


def pack(q: int, res: torch.Tensor, out: Packed | None = None, stream=None) -> Packed:
    """fq_pack: (rows, cols) uint8 CUDA tensor of residues -> Packed."""
    if res.dtype != torch.uint8 or res.dim() != 2 or not res.is_cuda:
        raise ValueError("expected a 2-D uint8 CUDA tensor")
    if res.stride(1) != 1:
        res = res.contiguous()
    rows, cols = res.shape
    out = empty(q, rows, cols, res.device) if out is None else out
    _check(load().fq_pack(q, rows, cols, ctypes.c_void_p(res.data_ptr()), res.stride(0),
                          ctypes.c_void_p(out.data.data_ptr()), _stream(stream)), "fq_pack")
    return out


def unpack(x: Packed, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """fq_unpack: Packed -> (rows, cols) uint8 residues on the same device."""
    if out is None:
        out = torch.empty((x.rows, x.cols), dtype=torch.uint8, device=x.data.device)
    _check(load().fq_unpack(x.q, x.rows, x.cols, ctypes.c_void_p(x.data.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream(stream)), "fq_unpack")
    return out


def add(x: Packed, y: Packed, sub: bool = False, out: Packed | None = None, stream=None) -> Packed:
    """fq_add: elementwise x + y (or x - y) with the bitsliced formulas."""
    if (x.q, x.rows, x.cols) != (y.q, y.rows, y.cols):
        raise ValueError("shape mismatch")
    out = empty(x.q, x.rows, x.cols, x.data.device) if out is None else out
    _check(load().fq_add(x.q, x.rows, x.cols, ctypes.c_void_p(x.data.data_ptr()),
                         ctypes.c_void_p(y.data.data_ptr()), ctypes.c_void_p(out.data.data_ptr()),
                         int(sub), _stream(stream)), "fq_add")
    return out


def matmul(a: Packed, b: Packed, out: Packed | None = None, path: int = PATH_AUTO, k: int = 0,
           chunk: int = 0, variant: int = 0, kernel: int = 0, strassen: int = 0, stream=None) -> Packed:
    """fq_matmul_ex: C = A B over F_q."""
    if a.q != b.q or a.cols != b.rows:
        raise ValueError("shape mismatch")
    m, l, n = a.rows, a.cols, b.cols
    out = empty(a.q, m, n, a.data.device) if out is None else out
    opt = Options(path=path, k=k, chunk=chunk, variant=variant, kernel=kernel, strassen=strassen)
    _check(load().fq_matmul_ex(a.q, m, l, n, ctypes.c_void_p(a.data.data_ptr()),
                               ctypes.c_void_p(b.data.data_ptr()), ctypes.c_void_p(out.data.data_ptr()),
                               _stream(stream), ctypes.byref(opt)), "fq_matmul")
    return out


def kernels(q: int) -> list[dict]:
    """The compiled M4RM kernels of field q: k, rows and columns per CTA, warps."""
    lib = load()
    out = []
    for i in range(lib.fq_kernel_count(q)):
        k, rows, cols, warps = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.fq_kernel_info(q, i, ctypes.byref(k), ctypes.byref(rows), ctypes.byref(cols), ctypes.byref(warps)),
               "fq_kernel_info")
        out.append({"index": i, "k": k.value, "max_rows": rows.value, "cols": cols.value, "warps": warps.value})
    return out


class TuneResult(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("kernel", ctypes.c_int), ("ms", ctypes.c_float),
                ("ms_planner", ctypes.c_float), ("ms_mma", ctypes.c_float)]


def autotune(a: Packed, b: Packed, out: Packed | None = None, stream=None) -> dict:
    """fq_autotune: time every candidate on these operands; later AUTO products of
    this shape use the fastest.  Returns the measurement."""
    m, l, n = a.rows, a.cols, b.cols
    out = empty(a.q, m, n, a.data.device) if out is None else out
    r = TuneResult()
    _check(load().fq_autotune(a.q, m, l, n, ctypes.c_void_p(a.data.data_ptr()), ctypes.c_void_p(b.data.data_ptr()),
                              ctypes.c_void_p(out.data.data_ptr()), _stream(stream), ctypes.byref(r)), "fq_autotune")
    return {"path": r.path, "kernel": r.kernel, "ms": r.ms, "ms_planner": r.ms_planner, "ms_mma": r.ms_mma}


def strassen_levels(q: int, m: int, l: int, n: int, path: int = PATH_AUTO, k: int = 0, strassen: int = 0) -> int:
    """fq_strassen_levels: Strassen-Winograd levels a product of this shape takes."""
    opt = Options(path=path, k=k, strassen=strassen)
    r = load().fq_strassen_levels(q, m, l, n, ctypes.byref(opt))
    if r < 0:
        raise FqError(-r, "fq_strassen_levels")
    return r


def planned_kernel(q: int, m: int, l: int, n: int, path: int = PATH_AUTO, k: int = 0, kernel: int = 0) -> dict:
    """fq_planned_kernel: the compiled M4RM kernel a direct product runs (its
    kernels() entry)."""
    opt = Options(path=path, k=k, kernel=kernel)
    r = load().fq_planned_kernel(q, m, l, n, ctypes.byref(opt))
    if r <= 0:
        raise FqError(-r, "fq_planned_kernel")
    return kernels(q)[r - 1]


def auto_choice(q: int, m: int, l: int, n: int) -> tuple[int, int]:
    """fq_auto_choice: the (path, kernel) an AUTO product of this shape takes."""
    path, kernel = ctypes.c_int(), ctypes.c_int()
    _check(load().fq_auto_choice(q, m, l, n, ctypes.byref(path), ctypes.byref(kernel)), "fq_auto_choice")
    return path.value, kernel.value


def tc_form(q: int, m: int, l: int, n: int) -> int:
    """fq_tc_form: the tcgen05 product form of this shape (2 single SMs, 3 and 4
    SM pairs from e4m3 operands, 5 SM pairs from packed e2m1 operands)."""
    r = load().fq_tc_form(q, m, l, n)
    if r < 0:
        raise FqError(-r, "fq_tc_form")
    return r


class TensorOperands:
    """fq_tc_prepare / fq_tc_multiply: the tensor-core path's converted operands
    of A and B, kept in a device workspace (a torch buffer) for reuse."""

    def __init__(self, a: Packed, b: Packed, stream=None):
        if a.q != b.q or a.cols != b.rows:
            raise ValueError("shape mismatch")
        self.q, self.m, self.l, self.n = a.q, a.rows, a.cols, b.cols
        nbytes = load().fq_tc_workspace_bytes(self.q, self.m, self.l, self.n)
        if nbytes < 0:
            raise FqError(ENOTSUP, "fq_tc_workspace_bytes")
        self.workspace = torch.empty(max(2, (nbytes + 7) // 8), dtype=torch.int64, device=a.data.device)
        self.prepare(a, b, stream)

    def prepare(self, a: Packed, b: Packed, stream=None):
        _check(load().fq_tc_prepare(self.q, self.m, self.l, self.n, ctypes.c_void_p(a.data.data_ptr()),
                                    ctypes.c_void_p(b.data.data_ptr()), ctypes.c_void_p(self.workspace.data_ptr()),
                                    _stream(stream)), "fq_tc_prepare")

    def multiply(self, out: Packed | None = None, stream=None) -> Packed:
        out = empty(self.q, self.m, self.n, self.workspace.device) if out is None else out
        _check(load().fq_tc_multiply(self.q, self.m, self.l, self.n, ctypes.c_void_p(self.workspace.data_ptr()),
                                     ctypes.c_void_p(out.data.data_ptr()), _stream(stream)), "fq_tc_multiply")
        return out


class BatchPlan:
    """fq_batched_plan_*: a plan for many products over one field, with its
    device workspace (a torch buffer) already uploaded.  path: PATH_AUTO (per
    product by the time models), PATH_M4RM or PATH_MMA."""

    def __init__(self, q: int, shapes, device=None, stream=None, path: int = PATH_AUTO):
        import numpy as np
        lib = load()
        sh = np.ascontiguousarray(np.asarray(shapes, dtype=np.int64).reshape(-1, 3))
        self.q = q
        self.shapes = sh
        m, l, n = (np.ascontiguousarray(sh[:, i]) for i in range(3))
        h = ctypes.c_void_p()
        _check(lib.fq_batched_plan_create_ex(q, len(sh), m.ctypes.data_as(ctypes.c_void_p),
                                             l.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                             path, ctypes.byref(h)), "fq_batched_plan_create_ex")
        self._h = h
        nbytes = lib.fq_batched_workspace_bytes(h)
        self.items = lib.fq_batched_items(h)
        self.tc_products = lib.fq_batched_tc_products(h)
        self.tc_tiles = lib.fq_batched_tc_tiles(h)
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.workspace = torch.empty((nbytes + 63) // 64 * 8 + 8, dtype=torch.int64, device=dev)
        _check(lib.fq_batched_plan_upload(h, ctypes.c_void_p(self._ws_ptr()), _stream(stream)),
               "fq_batched_plan_upload")

    def _ws_ptr(self) -> int:
        p = self.workspace.data_ptr()
        return (p + 63) // 64 * 64

    def run(self, A_ptrs: torch.Tensor, B_ptrs: torch.Tensor, C_ptrs: torch.Tensor, stream=None):
        """fq_matmul_batched; *_ptrs are int64 CUDA tensors of device pointers."""
        _check(load().fq_matmul_batched(self._h, ctypes.c_void_p(A_ptrs.data_ptr()),
                                        ctypes.c_void_p(B_ptrs.data_ptr()), ctypes.c_void_p(C_ptrs.data_ptr()),
                                        ctypes.c_void_p(self._ws_ptr()), _stream(stream)), "fq_matmul_batched")

    def run_stages(self, A_ptrs: torch.Tensor, B_ptrs: torch.Tensor, C_ptrs: torch.Tensor, stages: int,
                   stream=None):
        """fq_matmul_batched_stages: only the launch stages in the mask
        (STAGE_TC, STAGE_M4RM), for timing them apart."""
        _check(load().fq_matmul_batched_stages(self._h, ctypes.c_void_p(A_ptrs.data_ptr()),
                                               ctypes.c_void_p(B_ptrs.data_ptr()),
                                               ctypes.c_void_p(C_ptrs.data_ptr()), ctypes.c_void_p(self._ws_ptr()),
                                               _stream(stream), int(stages)), "fq_matmul_batched_stages")

    def product_paths(self) -> list[int]:
        """fq_batched_product_path of every product: PATH_MMA or PATH_M4RM."""
        lib = load()
        return [lib.fq_batched_product_path(self._h, p) for p in range(len(self.shapes))]

    def run_static(self, A_ptrs: torch.Tensor, B_ptrs: torch.Tensor, C_ptrs: torch.Tensor, stream=None):
        """fq_matmul_batched_static: the same products with the work list in the
        library's fixed device array instead of this plan's workspace (plans of
        Four-Russians items within FQ_BATCH_STATIC_BYTES; not while the stream
        is being captured)."""
        _check(load().fq_matmul_batched_static(self._h, ctypes.c_void_p(A_ptrs.data_ptr()),
                                               ctypes.c_void_p(B_ptrs.data_ptr()),
                                               ctypes.c_void_p(C_ptrs.data_ptr()), _stream(stream)),
               "fq_matmul_batched_static")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fq_batched_plan_destroy(self._h)
            self._h = None


def status(stream=None) -> int:
    """fq_status: synchronize and return (and clear) device-detected errors."""
    return load().fq_status(_stream(stream))

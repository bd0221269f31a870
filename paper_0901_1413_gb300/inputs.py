"""Seeded synthetic inputs: residue matrices drawn from a counter-based splitmix64.

This module holds no arithmetic of the method; both the CUDA path's tests and
the CPU oracle take their inputs from it.

Definition.  splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) advances a 64-bit state by the odd constant
GAMMA = 0x9E3779B97F4A7C15 and outputs mix64(state), where

    mix64(z): z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
              z = (z ^ (z >> 27)) * 0x94D049BB133111EB
              return z ^ (z >> 31)                        (all mod 2^64).

Stream ``stream`` of seed ``seed`` starts from state
s0 = mix64(seed ^ (stream << 40) ^ 0x5851F42D4C957F2D), and its element i is
h_i = mix64(s0 + (i + 1) * GAMMA), i.e. the (i+1)-th splitmix64 output, so any
element can be drawn on its own.  Element (r, c) of a rows x cols matrix is
stream element r * cols + c.

* ``uniform``: entry = floor(h * q / 2^64), uniform on [0, q).
* ``sparse``: entry is 0 when floor(h_mask * 10 / 2^64) < 9 (probability 0.9,
  i.i.d.), else 1 + floor(h_value * (q - 1) / 2^64), uniform on [1, q); the mask
  and the value come from streams ``stream`` and ``stream + 1000``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_SALT = 0x5851F42D4C957F2D
_MASK64 = (1 << 64) - 1

# stream ids used by the tests and the benchmark
STREAM_A = 0
STREAM_B = 1
STREAM_SHAPES = 2


def _mix64_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_start(seed: int, stream: int) -> int:
    return _mix64_int((int(seed) ^ (int(stream) << 40) ^ _SALT) & _MASK64)


def hashes(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """h_i for i in [start, start + count), uint64."""
    s0 = np.uint64(stream_start(seed, stream))
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(s0 + i * GAMMA)


def _scale(h: np.ndarray, q: int) -> np.ndarray:
    """floor(h * q / 2^64) without 128-bit arithmetic (exact for q < 2^31)."""
    hi = h >> np.uint64(32)
    lo = h & np.uint64(0xFFFFFFFF)
    qq = np.uint64(q)
    return (hi * qq + ((lo * qq) >> np.uint64(32))) >> np.uint64(32)


_CHUNK = 1 << 22


def uniform(q: int, rows: int, cols: int, seed: int, stream: int, row0: int = 0,
            total_cols: int | None = None) -> np.ndarray:
    """rows x cols residues uniform on [0, q); rows row0.. of a matrix with
    ``total_cols`` columns (default cols) -- a sub-block of the same matrix."""
    tc = cols if total_cols is None else total_cols
    out = np.empty((rows, cols), dtype=np.uint8)
    if rows == 0 or cols == 0:
        return out
    flat_rows = max(1, _CHUNK // max(cols, 1))
    for r in range(0, rows, flat_rows):
        rr = min(flat_rows, rows - r)
        if tc == cols:
            h = hashes(seed, stream, (row0 + r) * tc, rr * tc).reshape(rr, cols)
        else:
            h = np.stack([hashes(seed, stream, (row0 + r + i) * tc, cols) for i in range(rr)])
        out[r:r + rr] = _scale(h, q).astype(np.uint8)
    return out


def sparse(q: int, rows: int, cols: int, seed: int, stream: int, row0: int = 0) -> np.ndarray:
    """rows x cols residues, zero with probability 0.9 i.i.d., else uniform on [1, q)."""
    out = np.empty((rows, cols), dtype=np.uint8)
    if rows == 0 or cols == 0:
        return out
    flat_rows = max(1, _CHUNK // max(cols, 1))
    for r in range(0, rows, flat_rows):
        rr = min(flat_rows, rows - r)
        hm = hashes(seed, stream, (row0 + r) * cols, rr * cols)
        hv = hashes(seed, stream + 1000, (row0 + r) * cols, rr * cols)
        zero = _scale(hm, 10) < np.uint64(9)
        val = (np.uint64(1) + _scale(hv, q - 1)).astype(np.uint8)
        out[r:r + rr] = np.where(zero, np.uint8(0), val).reshape(rr, cols)
    return out


def batch_shapes(count: int, seed: int, lo: int = 64, hi: int = 1024, step: int = 64) -> np.ndarray:
    """count x 3 array of (m, l, n), each uniform on {lo, lo + step, ..., hi}."""
    choices = (hi - lo) // step + 1
    h = hashes(seed, STREAM_SHAPES, 0, 3 * count)
    return (lo + step * _scale(h, choices).astype(np.int64)).reshape(count, 3)


# ------------------------------------------------------ same draws, on a GPU --
# The definitions above, evaluated with torch int64 arithmetic (wrapping
# multiplication; logical shifts by masking), for large benchmark inputs.

def _t_lsr(x, s: int):
    import torch
    return (x >> s) & torch.tensor((1 << (64 - s)) - 1, dtype=torch.int64, device=x.device)


def _t_mix64(z):
    import torch
    c1 = torch.tensor(0xBF58476D1CE4E5B9 - (1 << 64), dtype=torch.int64, device=z.device)
    c2 = torch.tensor(0x94D049BB133111EB - (1 << 64), dtype=torch.int64, device=z.device)
    z = (z ^ _t_lsr(z, 30)) * c1
    z = (z ^ _t_lsr(z, 27)) * c2
    return z ^ _t_lsr(z, 31)


def _as_i64(v: int) -> int:
    v &= _MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _t_hashes(seed: int, stream: int, start: int, count: int, device):
    import torch
    s0 = stream_start(seed, stream)
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    g = torch.tensor(_as_i64(int(GAMMA)), dtype=torch.int64, device=device)
    return _t_mix64(torch.tensor(_as_i64(s0), dtype=torch.int64, device=device) + i * g)


def _t_scale(h, q: int):
    hi = _t_lsr(h, 32)
    lo = h & 0xFFFFFFFF
    return (hi * q + _t_lsr(lo * q, 32)) >> 32


def uniform_torch(q: int, rows: int, cols: int, seed: int, stream: int, device="cuda"):
    """``uniform`` evaluated on a torch device; identical values."""
    import torch
    out = torch.empty((rows, cols), dtype=torch.uint8, device=device)
    step = max(1, (1 << 24) // max(cols, 1))
    for r in range(0, rows, step):
        rr = min(step, rows - r)
        h = _t_hashes(seed, stream, r * cols, rr * cols, device)
        out[r:r + rr] = _t_scale(h, q).to(torch.uint8).view(rr, cols)
    return out


def sparse_torch(q: int, rows: int, cols: int, seed: int, stream: int, device="cuda"):
    """``sparse`` evaluated on a torch device; identical values."""
    import torch
    out = torch.empty((rows, cols), dtype=torch.uint8, device=device)
    step = max(1, (1 << 24) // max(cols, 1))
    for r in range(0, rows, step):
        rr = min(step, rows - r)
        hm = _t_hashes(seed, stream, r * cols, rr * cols, device)
        hv = _t_hashes(seed, stream + 1000, r * cols, rr * cols, device)
        zero = _t_scale(hm, 10) < 9
        val = (1 + _t_scale(hv, q - 1)).to(torch.uint8)
        out[r:r + rr] = torch.where(zero, torch.zeros_like(val), val).view(rr, cols)
    return out

"""The exact tensor-core form's arithmetic, pinned on the CPU.

The tcgen05 path feeds residues in their balanced form {-B, .., B} (B = (p-1)/2,
B = 1 for the F_2 products of GF(4)) as e4m3 or packed e2m1 values (the latter
with block scale factors 1.0) and accumulates the products in fp32.  That is exact when (a) every balanced residue is an e4m3
value and (b) every partial sum is an integer of magnitude below 2^24, which
holds for any order of additions while l * B^2 < 2^24.  These tests check both
facts with PyTorch's own e4m3 conversion, the e2m1 format's definition and
numpy's float32 arithmetic, and that the library's range for the form ends
exactly there."""
import numpy as np
import pytest
import torch

FIELDS = {2: 1, 3: 1, 4: 1, 5: 2, 7: 3}     # q -> B, the largest balanced magnitude


@pytest.fixture(scope="module")
def lib():
    from paper_0901_1413_gb300 import fq
    return fq.load()


def bound(q):
    """The longest l with l * B^2 < 2^24."""
    return ((1 << 24) - 1) // FIELDS[q] ** 2


@pytest.mark.parametrize("q", (3, 5, 7))
def test_balanced_residues_are_e4m3_values(q):
    b = FIELDS[q]
    r = torch.arange(-b, b + 1, dtype=torch.float32)
    assert torch.equal(r.to(torch.float8_e4m3fn).to(torch.float32), r)


def test_e4m3_bytes_of_the_balanced_residues():
    """The byte constants the conversion kernels write: 1.0 = 0x38, 2.0 = 0x40,
    3.0 = 0x44, a negative value sets bit 7, zero is 0x00."""
    r = torch.tensor([0.0, 1.0, 2.0, 3.0, -1.0, -2.0, -3.0])
    got = r.to(torch.float8_e4m3fn).view(torch.uint8).tolist()
    assert got == [0x00, 0x38, 0x40, 0x44, 0xB8, 0xC0, 0xC4]


def e2m1_value(nib):
    """The OCP MX E2M1 format: sign bit 3, exponent bits 2..1 biased by 1,
    mantissa bit 0; exponent 0 holds the subnormals 0 and 0.5."""
    sign = -1.0 if nib & 8 else 1.0
    e, m = (nib >> 1) & 3, nib & 1
    return sign * (0.5 * m if e == 0 else 2.0 ** (e - 1) * (1.0 + 0.5 * m))


def test_e2m1_nibbles_of_the_balanced_residues():
    """The nibble constants of the fp4 conversion (kind::mxf4 operands): 1 =
    0x2, 2 = 0x4, 3 = 0x5, a negative value sets bit 3, zero is 0x0; and each
    balanced residue has exactly that nibble (besides -0 for zero)."""
    table = {0: 0x0, 1: 0x2, 2: 0x4, 3: 0x5, -1: 0xA, -2: 0xC, -3: 0xD}
    for v, nib in table.items():
        assert e2m1_value(nib) == v
        assert [x for x in range(16) if e2m1_value(x) == v] == ([0x0, 0x8] if v == 0 else [nib])


def test_unit_block_scale():
    """The fp4 form's block scale factors are ue8m0 0x7F, 2^(127 - 127) = 1.0,
    so every scaled block sum is the plain integer sum."""
    assert 2.0 ** (0x7F - 127) == 1.0


@pytest.mark.parametrize("q", (3, 5, 7))
def test_fp32_running_sum_exact_up_to_the_bound(q):
    """At l = bound(q) the worst case (every product B^2, or alternating in
    sign) keeps a sequential float32 sum equal to the integer sum."""
    b2 = FIELDS[q] ** 2
    l = bound(q)
    terms = np.full(l, b2, np.float32)
    assert int(np.cumsum(terms, dtype=np.float32)[-1]) == l * b2
    assert l * b2 < 1 << 24 <= (l + 1) * b2
    rng = np.random.default_rng(q)
    prods = (rng.integers(-FIELDS[q], FIELDS[q] + 1, l) * rng.integers(-FIELDS[q], FIELDS[q] + 1, l))
    assert int(np.cumsum(prods.astype(np.float32), dtype=np.float32)[-1]) == int(prods.sum())


@pytest.mark.parametrize("q", (3, 5, 7))
def test_fp32_running_sum_fails_past_the_bound(q):
    """At most B^2 + 1 terms past the bound an input exists whose float32
    running sum is wrong: the bound is where exactness ends, not a margin."""
    b2 = FIELDS[q] ** 2
    l = bound(q)
    # bound(q) products of B^2 reach 2^24 - 1 - ((2^24 - 1) mod B^2); ones then
    # climb to 2^24 + 1, which float32 cannot hold
    lead = l * b2
    ones = (1 << 24) + 1 - lead
    terms = np.concatenate([np.full(l, b2, np.float32), np.ones(ones, np.float32)])
    assert len(terms) <= l + b2 + 1
    assert int(np.cumsum(terms, dtype=np.float32)[-1]) != lead + ones


@pytest.mark.parametrize("q", (2, 3, 4, 5, 7))
def test_library_range_of_the_tensor_core_form(lib, q):
    """fq_tc_workspace_bytes is -1 exactly from l = bound(q) + 1 on."""
    assert lib.fq_tc_workspace_bytes(q, 1, bound(q), 1) > 0
    assert lib.fq_tc_workspace_bytes(q, 1, bound(q) + 1, 1) == -1

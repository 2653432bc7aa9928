"""C ABI checks that need no GPU: the library loads, exports every entry
point include/paco.h declares, computes the digit reversal of Sect. 3.2
exactly like the oracle's digit-array reversal, and rejects illegal plans
before touching a device."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paco.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(paco_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2609_06449_gb300 as paco
    lib = ctypes.CDLL(paco.library_path)
    names = _declared()
    assert "paco_execute" in names and "paco_plan_create" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in paco.h but not exported"


@pytest.mark.parametrize("b", [2, 4, 8, 16])
def test_digit_reverse_matches_oracle(b):
    import paper_2609_06449_gb300 as paco
    t = b.bit_length() - 1
    for ell in range(1, 31 // t + 1):
        n = b ** ell
        us = np.arange(n) if n <= 4096 else np.random.default_rng(ell).integers(0, n, 4096)
        for u in us:
            assert paco.digit_reverse(int(u), b, ell) == oracle.digit_reverse(int(u), b, ell)


def test_digit_reverse_rejects_bad_arguments():
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError):
        paco.digit_reverse(8, 2, 3)       # 8 has 4 binary digits
    with pytest.raises(paco.PacoError):
        paco.digit_reverse(1, 3, 2)       # b must be a power of two <= 16


@pytest.mark.parametrize("N1,N2,b,p,msg", [
    (256, 256, 3, 0, "radix"),
    (96, 256, 2, 0, "N1"),
    (256, 128, 4, 0, "N2"),            # 128 is not a power of 4
    (256, 256, 2, 3, "p="),
    (256, 256, 4, 2, "p="),            # 2 is not a power of 4
    (16, 16, 2, 32, "p="),             # p does not divide N1
    (2 ** 16, 16, 2, 0, "2^14"),       # factor not built
])
def test_plan_rejects_illegal_sizes(N1, N2, b, p, msg):
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError) as ei:
        paco.Plan(N1, N2, b, 1, paco.C64, p=p)
    assert msg in str(ei.value)
    assert ei.value.status in (1, 2)


def test_plan_rejects_negative_batch_and_bad_dtype():
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError):
        paco.Plan(16, 16, 2, -1, paco.C64)
    with pytest.raises(paco.PacoError):
        paco.Plan(16, 16, 2, 1, 9)


@pytest.mark.parametrize("lengths,msg", [
    ([256, 48], "powers of two"),
    ([8], "powers of two"),            # below 2^4
    ([2 ** 21], "powers of two"),      # above 2^20
])
def test_batched_plan_rejects_unsupported_lengths(lengths, msg):
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError) as ei:
        paco.BatchedPlan(lengths)
    assert msg in str(ei.value) and ei.value.status == 2


def test_batched_plan_rejects_bad_arguments():
    import paper_2609_06449_gb300 as paco
    L = paco.lib
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 2)(256, 1024)
    assert L.paco_plan_create_batched(ctypes.byref(h), arr, 2, paco.C128) == 2   # dtype
    assert L.paco_plan_create_batched(ctypes.byref(h), None, 3, paco.C64) == 1   # NULL list
    assert L.paco_plan_create_batched(ctypes.byref(h), arr, -1, paco.C64) == 1
    o = paco.BatchedOpts(0, 3, 1, 0)                                             # radix 3
    assert L.paco_plan_create_batched_ex(ctypes.byref(h), arr, 2, paco.C64, ctypes.byref(o)) == 1
    assert L.paco_plan_batched_config(None, 256, None, None, None, None) == 1


@pytest.mark.parametrize("dtype_name", ["C64_TC_BF16X3", "C64_TC_FP16"])
def test_tc_forms_reject_small_factors(dtype_name):
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError) as ei:
        paco.Plan(128, 256, 2, 1, getattr(paco, dtype_name))
    assert ei.value.status == 2 and "2^8" in str(ei.value)


@pytest.mark.parametrize("N1,N2,N3,b,dtype_name,msg", [
    (256, 16, 64, 2, "C64", "2^5..2^8"),        # N2 below one pass
    (256, 64, 512, 2, "C64", "2^5..2^8"),       # N3 above one pass
    (256, 128, 256, 2, "C64", "exceeds 2^14"),  # N2 N3 = 2^15
    (256, 32, 64, 4, "C64", "powers of b"),     # 32 is not a power of 4
    (256, 64, 48, 2, "C64", "powers of b"),
    (256, 64, 64, 2, "C128", "complex64"),
    (256, 64, 64, 2, "C64_TC_BF16X3", "complex64"),
])
def test_3d_plan_rejects_unsupported_shapes(N1, N2, N3, b, dtype_name, msg):
    """dims = 3 checks its shape before touching a device."""
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError) as ei:
        paco.Plan(N1, N2, b, 1, getattr(paco, dtype_name), dims=3, N3=N3)
    assert ei.value.status == 2 and msg in str(ei.value)


def test_dims_and_n3_arguments_checked():
    import paper_2609_06449_gb300 as paco
    with pytest.raises(paco.PacoError) as ei:
        paco.Plan(256, 256, 2, 1, paco.C64, N3=64)          # N3 without dims = 3
    assert ei.value.status == 1 and "dims = 3" in str(ei.value)
    with pytest.raises(paco.PacoError) as ei:
        paco.Plan(256, 256, 2, 1, paco.C64, dims=4)
    assert ei.value.status == 1 and "dims" in str(ei.value)
    with pytest.raises(paco.PacoError) as ei:                 # the pipeline's factor N2 N3 checked too
        paco.Plan(2 ** 15, 64, 2, 1, paco.C64, dims=3, N3=64)
    assert "2^14" in str(ei.value)


def test_sharded_plan_rejects_dims_3():
    """The 3-D form is not built for the sharded form: refused before any device work."""
    import paper_2609_06449_gb300 as paco
    from paper_2609_06449_gb300.sharded import ShardedPlan
    with pytest.raises(paco.PacoError) as ei:
        ShardedPlan(256, 1024, 2, 4, 0, dims=3)
    assert ei.value.status == 2 and "sharded" in str(ei.value)

"""paco_execute_noalloc: the allocation-free entry point, checked against
paco_execute.

Some callers cannot allocate device memory -- code running while a CUDA graph
is captured, or inside a framework whose memory pool owns the device -- so the
library offers one entry point that runs the N1 = N2 = 2^14 complex64
transform entirely out of device arrays it reserves when it is loaded.  This
file calls it through the C ABI twice in a row, on different inputs, and
compares each result with the plan-based paco_execute within the tolerance
of the parity tests (relative L2 error <= 5e-7 * log2 N); runs the b = 2
layout with batch = 2 against paco_execute and the FP64 oracle; and checks
that a device-side timeout is reported by paco_noalloc_check().  It sits last
in collection order so that a failure here stops a `-x` run only after every
other test has run."""

import ctypes

import numpy as np
import pytest

from paco_inputs import gaussian, uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402

N1 = N2 = 2 ** 14
N = N1 * N2
TOL = 5e-7 * 28


def _rel(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


def _noalloc(x, out, b, batch, dir=-1):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return paco.lib.paco_execute_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         int(b), int(batch), int(dir), stream)


def test_noalloc_matches_paco_execute_twice():
    plan = paco.Plan(N1, N2, 4, 1, paco.C64, p=64)
    ref = torch.empty(N, dtype=torch.complex64, device="cuda")
    got = torch.empty_like(ref)
    for call, (gen, seed, d) in enumerate([(uniform, 11, -1), (gaussian, 12, +1)]):
        x = torch.from_numpy(gen(N, seed, np.complex64)).cuda()
        got.fill_(float("nan"))
        rc = _noalloc(x, got, 4, 1, d)
        assert rc == 0, paco.lib.paco_last_error().decode()
        plan.execute(x, ref, d)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(got)).all(), f"call {call}: non-finite output"
        err = _rel(got, ref)
        assert err <= TOL, f"call {call}: rel L2 vs paco_execute {err:.3e} > {TOL:.3e}"
        del x
    torch.cuda.empty_cache()


def test_noalloc_b2_batch2_matches_plan_and_oracle():
    """The b = 2 layout (a different run structure of the digit-reversed rows
    that stage 2 reads) with batch = 2 (the batch folded into the last tensor
    dimension, twice the counters): element-wise against paco_execute on a
    b = 2, batch = 2 plan and, per transform, against the FP64 oracle."""
    import oracle
    batch = 2
    xh = np.stack([uniform(N, 31, np.complex64), gaussian(N, 32, np.complex64)])
    x = torch.from_numpy(xh).cuda()
    got = torch.full_like(x, float("nan"))
    plan = paco.Plan(N1, N2, 2, batch, paco.C64, p=128)
    ref = torch.empty_like(x)
    for d in (-1, +1):
        rc = _noalloc(x, got, 2, batch, d)
        assert rc == 0, paco.lib.paco_last_error().decode()
        plan.execute(x, ref, d)
        torch.cuda.synchronize()
        assert paco.lib.paco_noalloc_check() == 0
        for t in range(batch):
            err = _rel(got[t], ref[t])
            assert err <= TOL, f"dir {d} transform {t}: rel L2 vs paco_execute {err:.3e}"
        gh = got.cpu().numpy()
        for t in range(batch):
            want = oracle.fft(xh[t].astype(np.complex128).reshape(1, -1), dir=d).ravel()
            err = np.linalg.norm(gh[t].astype(np.complex128) - want) / np.linalg.norm(want)
            assert err <= TOL, f"dir {d} transform {t}: rel L2 vs oracle {err:.3e} > {TOL:.3e}"
            del want
    del x, got, ref
    torch.cuda.empty_cache()


def test_noalloc_reports_a_forced_timeout():
    """A bounded wait that gives up inside paco_execute_noalloc is reported by
    the next paco_noalloc_check() (PACO_ERR_TIMEOUT); the check clears it, the
    context stays usable and the next normal call is correct.  The timeout is
    forced with the test hook: a short poll limit and a dependency target no
    counter reaches, so every wait ends by itself."""
    x = torch.from_numpy(uniform(N, 41, np.complex64)).cuda()
    got = torch.empty_like(x)
    assert paco.lib.paco_noalloc_check() == 0                 # nothing pending
    paco.lib.paco_debug_noalloc_set_waits(2000, 1 << 20)
    try:
        assert _noalloc(x, got, 4, 1) == 0                    # enqueued fine
        torch.cuda.synchronize()
        assert paco.lib.paco_noalloc_check() == 5             # PACO_ERR_TIMEOUT
        assert b"bounded" in paco.lib.paco_last_error()
    finally:
        paco.lib.paco_debug_noalloc_set_waits(0, 0)
    assert paco.lib.paco_noalloc_check() == 0                 # cleared by the check
    assert _noalloc(x, got, 4, 1) == 0
    plan = paco.Plan(N1, N2, 4, 1, paco.C64, p=64)
    ref = torch.empty_like(x)
    plan.execute(x, ref, -1)
    torch.cuda.synchronize()
    assert paco.lib.paco_noalloc_check() == 0
    assert _rel(got, ref) <= TOL
    del x, got, ref
    torch.cuda.empty_cache()


def test_noalloc_rejects_out_of_range_arguments():
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(x, y, 4, 17) == 1                  # batch above PACO_NOALLOC_MAX_BATCH
    assert b"batch" in paco.lib.paco_last_error()
    assert _noalloc(x, y, 8, 1) == 1                   # only b = 2 or 4 at N1 = N2 = 2^14
    assert _noalloc(x, y, 4, 1, 0) == 1                # bad direction
    assert _noalloc(x, y, 4, 0) == 0                   # empty batch: nothing to do

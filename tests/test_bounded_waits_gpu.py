"""The kernels' bounded waits (failure detection without a GPU fault): a
dependency target that nothing can meet makes every wait give up after its
poll limit; the launch ends, paco_plan_check reports PACO_ERR_TIMEOUT, and the
next normal execution on the same context is correct (checked against the
FP64 oracle)."""

import math

import numpy as np
import pytest

import oracle
from paco_inputs import gaussian, uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402

TIMEOUT = 5


def _rel(y, x):
    ref = oracle.fft(x.astype(np.complex128))
    return float(np.max(np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


def _expect_timeout_then_recover(plan, x, run):
    plan.debug_set_waits(spin_limit=20000, wait_bias=1)
    run()
    torch.cuda.synchronize()
    with pytest.raises(paco.PacoError) as ei:
        plan.check()
    assert ei.value.status == TIMEOUT
    plan.debug_set_waits(0, 0)
    y = run()
    torch.cuda.synchronize()
    plan.check()
    return y


def test_panel_pipeline_wait_gives_up_and_context_survives():
    # stage 1 with N1 = 2^14 over 128 columns runs on the panel pipeline,
    # whose Phase-B tiles wait on the Phase-A completion counter
    N1, N2 = 2 ** 14, 128
    x = gaussian(N1 * N2, 41, np.complex64)
    plan = paco.Plan(N1, N2, 2, 1, paco.C64)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)

    def run():
        plan.execute(xt, out, -1)
        return out
    y = _expect_timeout_then_recover(plan, x, run)
    assert _rel(y.cpu().numpy().reshape(1, -1), x.reshape(1, -1)) <= 5e-7 * math.log2(N1 * N2)


def test_batched_phase3_wait_gives_up_and_context_survives():
    lengths = [2 ** 14] * 4 + [256] * 8
    x = gaussian(sum(lengths), 42, np.complex64)
    plan = paco.BatchedPlan(lengths, autotune=False)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)

    def run():
        plan.execute(xt, out, -1)
        return out
    y = _expect_timeout_then_recover(plan, x, run).cpu().numpy()
    off = 0
    for n in lengths:
        assert _rel(y[off:off + n].reshape(1, -1), x[off:off + n].reshape(1, -1)) <= 5e-7 * math.log2(n)
        off += n


def test_one_launch_cluster_wait_gives_up_and_context_survives():
    """The one-launch form's transaction barrier made to expect bytes that no
    CTA sends: every CTA's 2 s wait gives up, the status word reads
    PACO_ERR_TIMEOUT, and the next transform is correct."""
    N = 65536
    plan = paco.Plan(256, 256, 2, 1, paco.C64, p=4)
    assert plan.info.fused_cluster == 1
    x = np.asarray(uniform(N, 95, np.complex64)).reshape(1, N)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)

    def run():
        plan.execute(xt, out, -1)
        return out.cpu().numpy()

    y = _expect_timeout_then_recover(plan, x, run)
    assert _rel(y, x) <= 5e-7 * 16

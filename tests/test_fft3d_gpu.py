"""dims = 3: the 3-D DFT of the N1 x N2 x N3 array (the PACO pipeline on the
N1 x (N2 N3) view without its top-level twiddle, Phase III as the split
stage over the N2 x N3 planes with ones for its twiddle), returned with its
axes reversed.  Each path the plan can take (generic or split Phase I,
Phase III planes of 2^10..2^14, the middle axis shorter or longer than the
last, radices 2, 4, 8) against the 3-D reference built from the oracle,
element by element."""

import math

import numpy as np
import pytest

import oracle2d
from paco_inputs import uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402


def _rel(got, want):
    got = np.asarray(got, np.complex128).reshape(want.shape)
    return float(np.max(np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)))


@pytest.mark.parametrize("N1,N2,N3,b,batch,dirs", [
    (256, 64, 64, 2, 2, (-1, 1)),      # Phase III plane 2^12
    (128, 32, 256, 2, 1, (-1, 1)),     # middle axis shorter than the last, 2^13
    (4096, 32, 32, 2, 1, (-1,)),       # Phase I split too (real twiddles), plane 2^10
    (256, 128, 128, 2, 1, (-1,)),      # plane 2^14 (the 1-D plan would take the L2 panel)
    (512, 64, 64, 8, 1, (-1, 1)),      # radix 8
    (64, 256, 64, 4, 1, (1,)),         # radix 4, middle axis longer than the last
])
def test_3d_dft_against_oracle(N1, N2, N3, b, batch, dirs):
    N = N1 * N2 * N3
    plan = paco.Plan(N1, N2, b, batch, paco.C64, dims=3, N3=N3)
    inf = plan.info
    assert (inf.dims, inf.N1, inf.N2, inf.N3, inf.N) == (3, N1, N2, N3, N)
    assert inf.stage_split[1] == 1
    x = uniform(batch * N, N1 + N2 + 3 * N3 + b, np.complex64).reshape(batch, N)
    xt = torch.from_numpy(x).cuda()
    for d in dirs:
        out = torch.empty_like(xt)
        plan.execute(xt, out, d)
        torch.cuda.synchronize()
        plan.check()
        want = oracle2d.fft3_reversed(x, N1, N2, N3, d)
        assert _rel(out.cpu().numpy(), want) <= 5e-7 * math.log2(N)


def test_fft3_helper_and_2d_plan_differ():
    """paco.fft3 matches the reference; the 2-D plan of the N1 x (N2 N3)
    view does not (its Phase III is the 1-D DFT of length N2 N3), so the
    ones really replace the split's twiddle."""
    N1, N2, N3 = 64, 32, 64
    N = N1 * N2 * N3
    x = uniform(N, 13, np.complex64).reshape(1, -1)
    xt = torch.from_numpy(x).cuda()
    y3 = paco.fft3(xt, N1, N2, N3, 2)
    want = oracle2d.fft3_reversed(x, N1, N2, N3)
    assert _rel(y3.cpu().numpy(), want) <= 5e-7 * math.log2(N)
    y2 = paco.fft2(xt, N1, N2 * N3, 2)
    assert _rel(y2.cpu().numpy(), want) > 0.1


def test_3d_plan_rejects_the_weighted_entry_points():
    N1, N2, N3 = 64, 32, 32
    plan = paco.Plan(N1, N2, 2, 1, paco.C64, dims=3, N3=N3)
    x = torch.zeros(N1 * N2 * N3, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(x)
    w = torch.ones(x.numel(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(paco.PacoError) as ei:
        plan.execute_weighted_power(x, out, w, loss)
    assert ei.value.status == 2 and "dims = 3" in str(ei.value)

"""dims = 2: the 2-D DFT of the N1 x N2 view (the PACO pipeline without its
top-level twiddle, returned transposed) -- a slab decomposition of the 2-D
FFT with one redistribution.  Every path the plan can take (one-launch
cluster, split stage, L2 panel, generic stages, complex128, the sharded
form) against the 2-D reference built from the oracle, element by element."""

import math

import numpy as np
import pytest

import oracle2d
import shard_np
from paco_inputs import uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402


def _rel(got, want):
    got = np.asarray(got, np.complex128).reshape(want.shape)
    return float(np.max(np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)))


@pytest.mark.parametrize("N1,N2,b,batch,dtype", [
    (256, 256, 2, 3, paco.C64), (4096, 256, 4, 1, paco.C64), (16384, 128, 2, 1, paco.C64),
    (64, 1024, 4, 2, paco.C64), (256, 512, 2, 2, paco.C128)])
@pytest.mark.parametrize("d", [-1, 1])
def test_2d_dft_against_oracle(N1, N2, b, batch, dtype, d):
    N = N1 * N2
    npdt = np.complex64 if dtype == paco.C64 else np.complex128
    plan = paco.Plan(N1, N2, b, batch, dtype, dims=2)
    assert plan.info.dims == 2
    x = uniform(batch * N, N1 + N2 + b, npdt).reshape(batch, N)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    plan.execute(xt, out, d)
    torch.cuda.synchronize()
    plan.check()
    want = oracle2d.fft2_transposed(x, N1, N2, d)
    tol = (5e-7 if dtype == paco.C64 else 1e-14) * math.log2(N)
    assert _rel(out.cpu().numpy(), want) <= tol


def test_fft2_helper_and_1d_plan_differ():
    """paco.fft2 matches the reference; the 1-D plan of the same shape does
    not (it applies the top-level twiddle), so the option is really taken."""
    N1, N2 = 128, 256
    x = uniform(N1 * N2, 9, np.complex64).reshape(1, -1)
    xt = torch.from_numpy(x).cuda()
    y2 = paco.fft2(xt, N1, N2, 2)
    want = oracle2d.fft2_transposed(x, N1, N2)
    assert _rel(y2.cpu().numpy(), want) <= 5e-7 * 15
    y1 = paco.fft(xt, N1, N2, 2)
    assert _rel(y1.cpu().numpy(), want) > 0.1


def test_sharded_2d_slab_decomposition():
    """The sharded form with dims = 2 (G = 4 rank programs on one GPU,
    device copies for the all-to-all): the assembled output is the
    transposed 2-D DFT."""
    from paper_2609_06449_gb300.sharded import ShardedPlan
    N1, N2, b, G, batch = 256, 1024, 4, 4, 2
    N = N1 * N2
    x = uniform(batch * N, 11, np.complex64).reshape(batch, N)
    plans = [ShardedPlan(N1, N2, b, G, g, batch, dims=2) for g in range(G)]
    sends = []
    for g in range(G):
        s = torch.empty(G * batch * plans[g].block, dtype=torch.complex64, device="cuda")
        plans[g].stage1(torch.from_numpy(shard_np.slab(x, g, G, N1, N2)).cuda(), s, -1)
        sends.append(s)
    ys = []
    for q in range(G):
        recv = torch.empty_like(sends[q])
        for g in range(G):
            recv.view(G, -1)[g].copy_(sends[g].view(G, -1)[q])
        yl = torch.empty(batch * N2 * (N1 // G), dtype=torch.complex64, device="cuda")
        plans[q].stage2(recv, yl, -1)
        ys.append(yl.cpu().numpy())
    got = shard_np.assemble(ys, G, N1, N2)
    assert _rel(got, oracle2d.fft2_transposed(x, N1, N2)) <= 5e-7 * math.log2(N)

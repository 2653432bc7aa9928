"""The sharded form on one GPU: the G rank programs (paco_shard_stage1,
exchange, paco_shard_stage2) run one after another, device copies standing
in for the all-to-all (block q of rank g -> slot g of rank q).  Checked
against the oracle: every rank's send blocks against the NumPy statement of
the layout (tests/shard_np.py), and the assembled output of every transform
element by element against the oracle's DFT.  Measured on hardware only as
this emulation: the GPU pool has one GPU per box."""

import math

import numpy as np
import pytest

import oracle
import shard_np
from paco_inputs import gaussian

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402
from paper_2609_06449_gb300.sharded import ShardedPlan  # noqa: E402


def _rel(a, b):
    a = np.asarray(a, np.complex128).reshape(np.asarray(b).shape[0], -1)
    b = np.asarray(b, np.complex128).reshape(a.shape)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("N1,N2,b,G,batch", [(256, 256, 2, 4, 1), (256, 256, 4, 4, 3), (1024, 1024, 4, 16, 2),
                                             (4096, 256, 4, 4, 1), (16384, 1024, 4, 4, 1), (64, 4096, 2, 8, 2)])
@pytest.mark.parametrize("dir", [-1, 1])
def test_sharded_form_against_oracle(N1, N2, b, G, batch, dir):
    N = N1 * N2
    tol = 5e-7 * math.log2(N)
    x = gaussian(batch * N, N1 + N2 + G, np.complex64).reshape(batch, N)
    plans = [ShardedPlan(N1, N2, b, G, g, batch) for g in range(G)]
    assert plans[0].block == N // (G * G)
    info = paco.PlanInfo()
    paco._check(paco.lib.paco_plan_info(plans[1]._h, paco.ctypes.byref(info)))
    assert (info.shard_G, info.shard_rank) == (G, 1)
    sends = []
    for g in range(G):
        xl = torch.from_numpy(shard_np.slab(x, g, G, N1, N2)).cuda()
        s = torch.empty(G * batch * plans[g].block, dtype=torch.complex64, device="cuda")
        plans[g].stage1(xl, s, dir)
        sends.append(s)
    torch.cuda.synchronize()
    # rank 0's blocks against the NumPy statement of the layout
    want0 = shard_np.stage1(shard_np.slab(x.astype(np.complex128), 0, G, N1, N2), 0, G, N1, N2, b, dir)
    got0 = sends[0].cpu().numpy().reshape(want0.shape)
    assert _rel(got0.reshape(G * batch, -1), want0.reshape(G * batch, -1)) <= tol
    ys = []
    for q in range(G):
        recv = torch.empty_like(sends[q])
        rv = recv.view(G, -1)
        for g in range(G):
            rv[g].copy_(sends[g].view(G, -1)[q])
        yl = torch.empty(batch * N2 * (N1 // G), dtype=torch.complex64, device="cuda")
        plans[q].stage2(recv, yl, dir)
        ys.append(yl.cpu().numpy())
    y = shard_np.assemble(ys, G, N1, N2)
    ref = oracle.fft(x.astype(np.complex128), dir, threads=0)
    assert _rel(y, ref) <= tol


def test_sharded_plan_refuses_other_calls():
    """A sharded plan runs only through the two shard calls; bad G or rank is
    an argument error; nothing is launched."""
    pl = ShardedPlan(256, 256, 2, 4, 0, 1)
    x = torch.zeros(65536, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(paco.PacoError) as e:
        paco._check(paco.lib.paco_execute(pl._h, paco._ptr(x), paco._ptr(y), -1, paco._stream(None)))
    assert e.value.status == 2
    for G, r in ((3, 0), (4, 4), (1, 0), (512, 0)):
        with pytest.raises(paco.PacoError):
            ShardedPlan(256, 256, 2, G, r, 1)


@pytest.mark.parametrize("N1,N2,b,G,batch", [(256, 256, 4, 4, 2), (1024, 256, 4, 4, 1), (256, 4096, 2, 8, 2)])
def test_restore_input_ownership_against_oracle(N1, N2, b, G, batch):
    """The sharded transform, then the second redistribution on the GPU
    (paco_shard_restore_pack / _unpack, the uneven all-to-all emulated by
    device copies): rank r ends with y viewed N1 x N2, columns
    [r Cl, (r+1) Cl), element by element against the oracle's y."""
    N = N1 * N2
    tol = 5e-7 * math.log2(N)
    Cl, K1 = N2 // G, N1 // G
    x = gaussian(batch * N, N1 + 5 * G, np.complex64).reshape(batch, N)
    plans = [ShardedPlan(N1, N2, b, G, g, batch, restore=True) for g in range(G)]
    sends = []
    for g in range(G):
        s = torch.empty(G * batch * plans[g].block, dtype=torch.complex64, device="cuda")
        plans[g].stage1(torch.from_numpy(shard_np.slab(x, g, G, N1, N2)).cuda(), s, -1)
        sends.append(s)
    ylocals = []
    for q in range(G):
        recv = torch.empty_like(sends[q])
        for g in range(G):
            recv.view(G, -1)[g].copy_(sends[g].view(G, -1)[q])
        yl = torch.empty(batch * N2 * K1, dtype=torch.complex64, device="cuda")
        plans[q].stage2(recv, yl, -1)
        ylocals.append(yl)
    # second redistribution
    counts = [p.restore_counts() for p in plans]
    packs = []
    for q in range(G):
        sb = torch.empty_like(ylocals[q])
        plans[q].restore_pack(ylocals[q], sb)
        packs.append(sb)
    ref = oracle.fft(x.astype(np.complex128), -1, threads=0).reshape(batch, N1, N2)
    for r in range(G):
        parts = []
        for q in range(G):
            sc = counts[q][0]
            start = batch * sum(sc[:r])
            parts.append(packs[q][start:start + batch * sc[r]])
            assert sc[r] == counts[r][1][q]
        recv = torch.cat(parts)
        out = torch.empty(batch * N1 * Cl, dtype=torch.complex64, device="cuda")
        plans[r].restore_unpack(recv, out)
        got = out.cpu().numpy().reshape(batch, N1 * Cl)
        want = ref[:, :, r * Cl:(r + 1) * Cl].reshape(batch, N1 * Cl)
        err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
        assert float(err.max()) <= tol, (r, err)

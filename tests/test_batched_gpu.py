"""GPU parity of the uneven batch (paco_plan_create_batched): every
transform of a mixed-length batch against the FP64 oracle, per length, at the
complex64 tolerance 5e-7*log2(N_i); fixed and autotuned configurations; CUDA
graph capture; the full-size mix on sampled transforms plus Parseval on all."""

import math

import numpy as np
import pytest

import oracle
from paco_inputs import gaussian, uneven_lengths

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402


def offsets(lengths):
    return np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)


def check_all(lengths, x, y, d, idx=None):
    off = offsets(lengths)
    by_len = {}
    for i in (range(len(lengths)) if idx is None else idx):
        by_len.setdefault(int(lengths[i]), []).append(i)
    worst = 0.0
    for n, ids in by_len.items():
        xs = np.stack([x[off[i]:off[i] + n] for i in ids]).astype(np.complex128)
        ys = np.stack([y[off[i]:off[i] + n] for i in ids]).astype(np.complex128)
        ref = oracle.fft(xs, dir=d)
        err = np.linalg.norm(ys - ref, axis=1) / np.linalg.norm(ref, axis=1)
        tol = 5e-7 * math.log2(n)
        assert err.max() <= tol, f"N={n} rel_l2={err.max():.3e} tol={tol:.3e}"
        worst = max(worst, float(err.max() / tol))
    return worst


def run(plan, x, d=-1):
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    plan.execute(xt, out, d)
    torch.cuda.synchronize()
    plan.check()
    return out.cpu().numpy()


MIX = (2 ** uneven_lengths(count=160, seed=5, lo=4, hi=20, total_log2=23)).astype(np.int64)


@pytest.mark.parametrize("d", [-1, 1])
def test_uneven_mix_autotuned(d):
    plan = paco.BatchedPlan(MIX)
    x = gaussian(int(MIX.sum()), 31, np.complex64)
    y = run(plan, x, d)
    check_all(MIX, x, y, d)


@pytest.mark.parametrize("b,ctas,lag", [(2, 1, 1), (4, 1, 2), (8, 2, 4), (16, 2, 1)])
def test_uneven_mix_fixed_configs(b, ctas, lag):
    plan = paco.BatchedPlan(MIX, autotune=False, b=b, ctas_per_sm=ctas, lag=lag)
    x = gaussian(int(MIX.sum()), 32, np.complex64)
    y = run(plan, x, -1)
    check_all(MIX, x, y, -1)
    for n in set(MIX.tolist()):
        bb, n1, c, lg = plan.config(n)
        assert n % n1 == 0 and bb in (2, 4, 8, 16) and c == ctas and lg == lag


def test_every_length_and_partial_groups():
    # every supported length, with counts that leave the last small group partial
    lengths = []
    for e in range(4, 21):
        lengths += [2 ** e] * (3 if e < 14 else 1)
    lengths = np.array(lengths[::-1] + lengths, dtype=np.int64)
    plan = paco.BatchedPlan(lengths, autotune=False)
    x = gaussian(int(lengths.sum()), 33, np.complex64)
    for d in (-1, 1):
        check_all(lengths, x, run(plan, x, d), d)


def test_single_length_matches_plan():
    n1 = n2 = 128
    lengths = np.full(24, n1 * n2, dtype=np.int64)
    x = gaussian(int(lengths.sum()), 34, np.complex64)
    yb = run(paco.BatchedPlan(lengths), x)
    plan = paco.Plan(n1, n2, 2, 24, paco.C64)
    ys = run(plan, x.reshape(24, -1)).reshape(-1)
    assert np.linalg.norm(yb - ys) / np.linalg.norm(ys) <= 5e-7 * 14


def test_graph_capture_replay():
    lengths = MIX
    plan = paco.BatchedPlan(lengths)
    x = torch.from_numpy(gaussian(int(lengths.sum()), 35, np.complex64)).cuda()
    out = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.execute(x, out, -1, stream=s)          # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = out.clone()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g):
        plan.execute(x, out, -1)
    for _ in range(3):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, eager)
    check_all(lengths, x.cpu().numpy(), out.cpu().numpy(), -1)


def test_empty_and_errors():
    plan = paco.BatchedPlan([])
    plan.execute(0, 0, -1)
    with pytest.raises(paco.PacoError):
        paco.BatchedPlan([48])
    with pytest.raises(paco.PacoError):
        paco.BatchedPlan([2 ** 21])
    pl = paco.BatchedPlan([256, 4096])
    xt = torch.zeros(256 + 4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(paco.PacoError):
        pl.execute_stage1(xt, torch.empty_like(xt))
    with pytest.raises(paco.PacoError):
        pl.execute(xt, xt)                           # aliasing


def test_full_size_uneven_batch():
    """The uneven benchmark workload: 4096 lengths (exponents uniform over
    8..20, reduced to a 2^28 total) plus 2^14 transforms of 2^12, N(0,1).
    Every one of the 20 480 transforms, element by element, against the
    oracle's FP64 FFT (grouped by length, the oracle's batch spread over the
    host cores): relative L2 error <= 5e-7 * log2 N_i per transform."""
    e = uneven_lengths()
    lengths = np.concatenate([2 ** e, np.full(2 ** 14, 2 ** 12)]).astype(np.int64)
    total = int(lengths.sum())
    plan = paco.BatchedPlan(lengths)
    g = torch.Generator(device="cuda").manual_seed(0)
    xr = torch.randn(total, 2, generator=g, device="cuda", dtype=torch.float32)
    x = torch.view_as_complex(xr)
    out = torch.empty_like(x)
    plan.execute(x, out, -1)
    torch.cuda.synchronize()
    plan.check()
    xh = x.cpu().numpy()
    yh = out.cpu().numpy()
    del x, xr, out
    torch.cuda.empty_cache()
    offs = offsets(lengths)
    worst = {}
    for v in np.unique(lengths):
        ids = np.flatnonzero(lengths == v)
        n = int(v)
        xs = np.stack([xh[offs[i]:offs[i] + n] for i in ids]).astype(np.complex128)
        ys = np.stack([yh[offs[i]:offs[i] + n] for i in ids]).astype(np.complex128)
        ref = oracle.fft(xs, -1, threads=0)
        errs = np.linalg.norm(ys - ref, axis=1) / np.linalg.norm(ref, axis=1)
        worst[n] = float(errs.max())
        assert worst[n] <= 5e-7 * math.log2(n), (n, worst[n], int(ids[int(np.argmax(errs))]))
    assert sum(int(np.count_nonzero(lengths == n)) for n in worst) == len(lengths)

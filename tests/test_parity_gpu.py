"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Floating-point tolerance (relative L2 error per transform against the FP64
oracle on the same rounded inputs): 5e-7*log2(N) for complex64 and
1e-14*log2(N) for complex128.  Index work (where each value lands) is checked
through the intermediates of Eq. (17) and Lemma 1 against the step-by-step
simulator."""

import math

import numpy as np
import pytest

import oracle
from oracle import paco_sim as ps
from paco_inputs import gaussian, uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402

TOL = {paco.C64: 5e-7, paco.C128: 1e-14}
NP = {paco.C64: np.complex64, paco.C128: np.complex128}
TT = {paco.C64: torch.complex64, paco.C128: torch.complex128}


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128).reshape(ref.shape)
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return float(np.max(num / den))


def run(plan, x_np, dir=-1):
    x = torch.from_numpy(x_np).cuda()
    out = torch.empty_like(x)
    plan.execute(x, out, dir)
    torch.cuda.synchronize()
    plan.check()
    return out.cpu().numpy()


CASES = [  # (N1, N2, b, p)
    (2, 2, 2, 2), (2, 8, 2, 2), (8, 2, 2, 2), (4, 4, 2, 2), (4, 4, 4, 4),
    (16, 16, 2, 2), (16, 16, 4, 4), (16, 16, 16, 16), (32, 32, 2, 2),
    (64, 16, 4, 4), (16, 64, 4, 4), (8, 64, 8, 8), (256, 256, 2, 4),
    (128, 512, 2, 4), (512, 128, 2, 8), (1024, 1024, 4, 4), (4096, 64, 4, 16),
    (64, 4096, 4, 4), (2048, 2048, 2, 16), (8192, 16, 2, 2), (16, 8192, 2, 2),
    (4096, 4096, 16, 16), (16384, 16, 4, 4), (16, 16384, 4, 16),
    (16384, 128, 2, 2), (128, 16384, 2, 4), (16384, 256, 4, 16), (256, 16384, 4, 4),
]


@pytest.mark.parametrize("dtype", [paco.C64, paco.C128])
@pytest.mark.parametrize("N1,N2,b,p", CASES)
def test_end_to_end_vs_oracle(N1, N2, b, p, dtype):
    N = N1 * N2
    batch = 3 if N <= 2 ** 16 else 1
    x = uniform(batch * N, N1 + 7 * N2, NP[dtype]).reshape(batch, N)
    plan = paco.Plan(N1, N2, b, batch, dtype, p=p)
    tol = TOL[dtype] * max(1.0, math.log2(N))
    for d in (-1, 1):
        got = run(plan, x, d)
        ref = oracle.fft(x.astype(np.complex128), dir=d)
        err = rel_l2(got, ref)
        assert err <= tol, f"dir={d} rel_l2={err:.3e} tol={tol:.3e}"


@pytest.mark.parametrize("dtype", [paco.C64, paco.C128])
@pytest.mark.parametrize("N1,N2,b,p", [(16, 16, 2, 2), (64, 16, 4, 4), (16, 64, 4, 4),
                                       (64, 64, 8, 8), (256, 16, 16, 16), (256, 256, 2, 4),
                                       (64, 256, 4, 16), (16384, 256, 4, 4), (256, 16384, 4, 4)])
def test_intermediates_vs_simulator(N1, N2, b, p, dtype):
    """Stage-1 output is W = Z-hat (Eq. (17)) and Phase I alone is A-tilde
    (Lemma 1) -- both compared with the step-by-step simulator, so every
    value must sit at the position the paper's permutation assigns."""
    N = N1 * N2
    x = gaussian(N, 3, NP[dtype])
    plan = paco.Plan(N1, N2, b, 1, dtype, p=p)
    ref = ps.simulate(x.astype(np.complex128), N1, N2, b, p, phase1="lemma")
    xt = torch.from_numpy(x).cuda()
    W = torch.empty_like(xt)
    plan.execute_stage1(xt, W)
    At = torch.empty_like(xt)
    plan.execute_phase1(xt, At)
    torch.cuda.synchronize()
    tol = TOL[dtype] * math.log2(N)
    Wg = W.cpu().numpy().reshape(N2, N1)
    assert np.linalg.norm(Wg - ref["W"]) / np.linalg.norm(ref["W"]) <= tol
    Ag = At.cpu().numpy().reshape(N1, N2)
    assert np.linalg.norm(Ag - ref["A_tilde"]) / np.linalg.norm(ref["A_tilde"]) <= tol
    # stage 2 in place on W gives the transform
    plan.execute_stage2(W, W)
    torch.cuda.synchronize()
    assert rel_l2(W.cpu().numpy(), ref["Y"].reshape(1, N)) <= tol


def test_config_a_and_direct_dft_subcase():
    """N = 2^16 as 256 x 256, b = 2, p = 4, U[-1,1) from seed 0, forward; and
    the 2^10 sub-case against the long-double direct DFT."""
    x = uniform(2 ** 16, 0, np.complex64)
    plan = paco.Plan(256, 256, 2, 1, paco.C64, p=4)
    got = run(plan, x.reshape(1, -1))
    ref = oracle.fft(x.astype(np.complex128))
    assert rel_l2(got, ref.reshape(1, -1)) <= 5e-7 * 16
    x10 = uniform(2 ** 10, 0, np.complex64)
    plan10 = paco.Plan(32, 32, 2, 1, paco.C64, p=2)
    got10 = run(plan10, x10.reshape(1, -1))
    ref10 = oracle.dft_direct(x10.astype(np.complex128))
    assert rel_l2(got10, ref10.reshape(1, -1)) <= 5e-7 * 10


@pytest.mark.parametrize("b,p", [(2, 4), (2, 8), (4, 4)])
def test_one_launch_cluster_form(b, p):
    """N1 = N2 = 256 with p = 4 or 8 runs as one cluster launch (CTA q =
    processor q): against the oracle in both directions with a ragged batch
    of 3, against the two-launch path (stage 1 + stage 2 through W in global
    memory), and the all-to-all's item counts per ordered pair, measured in
    the kernel, equal to batch * N/p^2 (Theorem 4)."""
    N1 = N2 = 256
    N, batch = N1 * N2, 3
    plan = paco.Plan(N1, N2, b, batch, paco.C64, p=p)
    assert plan.info.fused_cluster == 1
    x = uniform(batch * N, 70 + p + b, np.complex64).reshape(batch, N)
    xt = torch.from_numpy(x).cuda()
    for d in (-1, 1):
        got = run(plan, x, d)
        ref = oracle.fft(x.astype(np.complex128), dir=d)
        assert rel_l2(got, ref) <= 5e-7 * 16, d
        two = torch.empty_like(xt)
        plan.execute_stage1(xt, two, d)
        plan.execute_stage2(two, two, d)
        torch.cuda.synchronize()
        assert rel_l2(got, two.cpu().numpy().astype(np.complex128)) <= 5e-7 * 16
    out = torch.empty_like(xt)
    counts = plan.debug_exchange_counts(xt, out)
    assert counts == [[batch * N // (p * p)] * p for _ in range(p)]
    assert rel_l2(out.cpu().numpy(), oracle.fft(x.astype(np.complex128))) <= 5e-7 * 16


def test_one_launch_form_batch_limit():
    """The one-launch form takes up to 16 transforms; 17 run as two stage
    launches.  Both against the oracle."""
    N = 65536
    for batch, fused in ((16, 1), (17, 0)):
        plan = paco.Plan(256, 256, 2, batch, paco.C64, p=4)
        assert plan.info.fused_cluster == fused
        x = uniform(batch * N, 90 + batch, np.complex64).reshape(batch, N)
        assert rel_l2(run(plan, x), oracle.fft(x.astype(np.complex128))) <= 5e-7 * 16


@pytest.mark.parametrize("N1,N2,b,batch,split", [
    (4096, 4096, 4, 2, (1, 1)), (4096, 4096, 2, 1, (1, 1)), (4096, 4096, 8, 1, (1, 1)),
    (4096, 4096, 16, 1, (0, 0)), (8192, 4096, 2, 1, (1, 1)), (4096, 8192, 2, 1, (1, 1)),
    (8192, 256, 2, 3, (1, 0)), (256, 8192, 2, 3, (0, 1)), (4096, 64, 4, 5, (1, 0))])
@pytest.mark.parametrize("d", [-1, 1])
def test_split_stages_against_oracle(N1, N2, b, batch, split, d):
    """Stages of 2^12 and 2^13 (complex64) run as two passes through the
    plan's scratch (pass A of length 2^ceil(l/2) with the twiddle
    w_L^{-k_a j_b}, pass B with the stage's epilogue); radix 16 at 2^12 keeps
    the single pass (its half-lengths are not powers of 16).  Every transform
    element by element against the oracle, both directions."""
    N = N1 * N2
    plan = paco.Plan(N1, N2, b, batch, paco.C64)
    assert tuple(plan.info.stage_split) == split
    x = uniform(batch * N, N1 + 3 * N2 + b, np.complex64).reshape(batch, N)
    got = run(plan, x, d)
    ref = oracle.fft(x.astype(np.complex128), dir=d, threads=0)
    assert rel_l2(got, ref) <= 5e-7 * math.log2(N), (N1, N2, b)


@pytest.mark.parametrize("N1,N2,b,batch", [(16384, 2048, 2, 2), (16384, 4096, 4, 1), (4096, 16384, 4, 2),
                                            (16384, 512, 2, 1), (16384, 16384, 4, 1)])
@pytest.mark.parametrize("d", [-1, 1])
def test_split_2p14_option(N1, N2, b, batch, d):
    """split=1: the 2^14 stages as two passes too (2^8 x 2^6 for b = 4, 2^7 x
    2^7 for b = 2) -- every transform element by element against the oracle,
    both directions, three times with identical results."""
    N = N1 * N2
    plan = paco.Plan(N1, N2, b, batch, paco.C64, split=1)
    want = tuple(int(L >= 4096) for L in (N1, N2))
    assert tuple(plan.info.stage_split) == want
    x = uniform(batch * N, N1 + N2 + 7 * b, np.complex64).reshape(batch, N)
    ref = oracle.fft(x.astype(np.complex128), dir=d, threads=0)
    first = None
    for _ in range(3):
        got = run(plan, x, d)
        assert rel_l2(got, ref) <= 5e-7 * math.log2(N), (N1, N2, b)
        if first is None:
            first = got
        assert np.array_equal(got, first)


def test_closed_forms_on_gpu():
    """delta -> constant; single tone -> N delta; Parseval."""
    N1 = N2 = 256
    N = N1 * N2
    plan = paco.Plan(N1, N2, 4, 1, paco.C64, p=4)
    d = np.zeros((1, N), np.complex64); d[0, 0] = 1
    assert np.allclose(run(plan, d), 1.0, atol=1e-6)
    f = 12345
    tone = np.exp(2j * np.pi * f * np.arange(N) / N).astype(np.complex64).reshape(1, N)
    y = run(plan, tone)
    want = np.zeros(N); want[f] = N
    assert np.max(np.abs(y[0] - want)) <= 5e-7 * 16 * N
    x = gaussian(N, 1, np.complex64).reshape(1, N)
    y = run(plan, x)
    e_y = np.sum(np.abs(y.astype(np.complex128)) ** 2)
    e_x = np.sum(np.abs(x.astype(np.complex128)) ** 2)
    assert abs(e_y - N * e_x) / (N * e_x) < 1e-5


def test_edge_cases():
    # batch 0 is a no-op
    plan0 = paco.Plan(64, 64, 4, 0, paco.C64)
    plan0.execute(0, 0, -1)
    # aliasing and bad direction are errors
    plan = paco.Plan(64, 64, 4, 1, paco.C64)
    x = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(paco.PacoError) as ei:
        plan.execute(x, x, -1)
    assert ei.value.status == 3
    y = torch.empty_like(x)
    with pytest.raises(paco.PacoError):
        plan.execute(x, y, 0)
    with pytest.raises(paco.PacoError):
        plan.execute(x[1:], y, -1)   # misaligned (8-byte offset)
    # the largest stage length built (2^14) in both factors: c64, b = 2
    xs = uniform(2 ** 14 * 16, 2, np.complex64).reshape(1, -1)
    planb = paco.Plan(2 ** 14, 16, 2, 1, paco.C64)
    assert rel_l2(run(planb, xs), oracle.fft(xs.astype(np.complex128))) <= 5e-7 * 18


def test_host_buffer_entry_point():
    N1, N2 = 1024, 256
    N = N1 * N2
    x = uniform(2 * N, 4, np.complex64).reshape(2, N)
    plan = paco.Plan(N1, N2, 4, 2, paco.C64)
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty(h_in.shape, dtype=h_in.dtype, device="cuda")
    d_out = torch.empty_like(d_in)
    plan.execute_host(h_in, h_out, d_in, d_out, -1)
    torch.cuda.synchronize()
    assert rel_l2(h_out.numpy(), oracle.fft(x.astype(np.complex128))) <= 5e-7 * 18


def test_torch_wrapper_and_stream():
    N1, N2 = 256, 64
    x = torch.from_numpy(gaussian(4 * N1 * N2, 8, np.complex64)).reshape(4, N1 * N2).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y = paco.fft(x, N1, N2, 4)
    s.synchronize()
    ref = oracle.fft(x.cpu().numpy().astype(np.complex128))
    assert rel_l2(y.cpu().numpy(), ref) <= 5e-7 * 14


def test_full_size_bench_configuration():
    """N = 2^28 c64 as 2^14 x 2^14, b = 4, p = 64 -- the configuration and
    launch bench.py times (the 2^14 panel pipeline in both stages) --
    element by element against the oracle's full FP64 FFT, forward and
    conjugate; tolerance 5e-7 * log2 N on the relative L2 error."""
    N1 = N2 = 2 ** 14
    N = N1 * N2
    x = uniform(N, 0, np.complex64)
    plan = paco.Plan(N1, N2, 4, 1, paco.C64, p=64)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    x128 = x.astype(np.complex128).reshape(1, N)
    del x
    for d in (-1, 1):
        yd.fill_(float("nan"))
        plan.execute(xd, yd, d)
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.fft(x128, dir=d, threads=0).reshape(N)
        got = yd.cpu().numpy()
        err = np.linalg.norm(got.astype(np.complex128) - ref) / np.linalg.norm(ref)
        assert err <= 5e-7 * 28, f"dir={d} rel_l2={err:.3e}"
        del ref, got
    del xd, yd
    torch.cuda.empty_cache()


@pytest.mark.parametrize("N1,N2,b", [(16384, 2048, 2), (2048, 16384, 2),
                                     (16384, 4096, 4), (4096, 16384, 4)])
def test_panel_ring_wraps(N1, N2, b):
    """The 2^14 panel pipeline over 16 or 32 panels of 128 columns per
    transform, batch 2: its ring of three L2 panel buffers is reused many
    times, so the A tiles that wait for a released buffer and the B tiles of
    late panels all run.  Element-wise against the oracle, both directions."""
    batch = 2
    N = N1 * N2
    x = uniform(batch * N, N1 + 3 * N2 + b, np.complex64).reshape(batch, N)
    plan = paco.Plan(N1, N2, b, batch, paco.C64)
    tol = 5e-7 * math.log2(N)
    x128 = x.astype(np.complex128)
    for d in (-1, 1):
        got = run(plan, x, d)
        ref = oracle.fft(x128, dir=d)
        err = rel_l2(got, ref)
        assert err <= tol, f"dir={d} rel_l2={err:.3e} tol={tol:.3e}"


def test_full_size_complex128():
    """complex128 N = 2^27 as 2^13 x 2^14, b = 2, p = 128 (the FP64
    configuration of the large-scale workload), forward and conjugate, against
    the oracle's full FP64 FFT; tolerance 1e-14 * log2 N."""
    N1, N2 = 2 ** 13, 2 ** 14
    N = N1 * N2
    x = uniform(N, 0, np.complex128)
    plan = paco.Plan(N1, N2, 2, 1, paco.C128, p=128)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    for d in (-1, 1):
        plan.execute(xd, yd, d)
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.fft(x, dir=d, threads=0)
        err = np.linalg.norm(yd.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-14 * 27, f"dir={d} rel_l2={err:.3e}"
    del xd, yd
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [paco.C64, paco.C128])
@pytest.mark.parametrize("N1,N2,b,p", [(2, 8, 2, 2), (16, 16, 4, 4), (64, 16, 2, 2), (16, 64, 4, 4),
                                       (256, 256, 2, 4), (512, 64, 8, 8), (128, 512, 2, 8),
                                       (4096, 64, 4, 16), (16384, 256, 4, 4), (256, 16384, 4, 4)])
def test_unfused_pipeline(N1, N2, b, p, dtype):
    """Phase I alone -> paco_permute (PARA-CO-DRP as its own pass) -> Phase
    III equals the transform; the permuted array equals Z-hat of Eq. (17)
    from the simulator and the fused stage-1 output."""
    N = N1 * N2
    batch = 2 if N <= 2 ** 16 else 1
    x = gaussian(batch * N, 5, NP[dtype]).reshape(batch, N)
    plan = paco.Plan(N1, N2, b, batch, dtype, p=p)
    tol = TOL[dtype] * max(1.0, math.log2(N))
    xt = torch.from_numpy(x).cuda()
    for d in (-1, 1):
        At = torch.empty_like(xt)
        W = torch.empty_like(xt)
        Wf = torch.empty_like(xt)
        y = torch.empty_like(xt)
        plan.execute_phase1(xt, At, d)
        plan.permute(At, W, d)
        plan.execute_stage1(xt, Wf, d)
        plan.execute_stage2(W, y, d)
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.fft(x.astype(np.complex128), dir=d)
        assert rel_l2(y.cpu().numpy(), ref) <= tol
        Wn, Wfn = W.cpu().numpy(), Wf.cpu().numpy()
        assert rel_l2(Wn, Wfn.astype(np.complex128)) <= tol
        if d == -1:
            sim = ps.simulate(x[0].astype(np.complex128), N1, N2, b, p, phase1="lemma")
            assert rel_l2(Wn[0].reshape(1, -1), sim["W"].reshape(1, -1)) <= tol


def test_permute_rejects_aliasing():
    plan = paco.Plan(64, 64, 2, 1, paco.C64)
    xt = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(paco.PacoError):
        plan.permute(xt, xt)


def test_fp64_peak_probe_is_plausible():
    """paco_probe_fp64_peak (the complex128 roofline's denominator): a DFMA
    rate between a tenth and twice GB300's nominal 1.25 TFLOP/s, over a
    launch long enough to time."""
    gflops, ms = paco.probe_fp64_peak(iters=1024)
    assert ms > 0.05
    assert 125.0 <= gflops <= 2500.0, gflops

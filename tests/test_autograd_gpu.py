"""Differentiation (the backward form): PacoFFT's hand-written backward is the
unnormalised conjugate transform (dir = +1).  The paper defines only the
forward transform; for y = F x with F symmetric, the vector-Jacobian product
PyTorch asks for is F^H g = conj(F) g, i.e. the dir = +1 transform of g.

For L = sum(w * |F x|^2), PyTorch's complex convention gives
grad_x = 2 F^H (w * F x)."""

import math

import numpy as np
import pytest

import oracle
from paco_inputs import gaussian, weights

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402


def loss_np(x, w, N1, N2):
    """The loss evaluated by the oracle (FP64 recursive FFT)."""
    y = oracle.fft(x.reshape(-1, N1 * N2))
    return float(np.sum(w * np.abs(y) ** 2))


def test_gradcheck_complex128():
    """torch.autograd.gradcheck on a c128 plan, N = 2^10, batch 4."""
    N1 = N2 = 32
    x = torch.from_numpy(gaussian(4 * N1 * N2, 3, np.complex128)).reshape(4, N1 * N2).cuda()
    x.requires_grad_(True)
    f = lambda t: paco.PacoFFT.apply(t, N1, N2, 2, 2)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=False)


def test_finite_differences_complex64():
    """FP64 central finite differences of the oracle loss versus the c64 GPU
    gradient of L = sum(w |F x|^2), N = 2^10, batch 4."""
    N1 = N2 = 32
    N = N1 * N2
    xc = gaussian(4 * N, 5, np.complex64).reshape(4, N)
    w = weights(4 * N, 6).reshape(4, N).astype(np.float64)
    x = torch.from_numpy(xc).cuda().requires_grad_(True)
    y = paco.PacoFFT.apply(x, N1, N2, 2, 2)
    loss = (torch.from_numpy(w.astype(np.float32)).cuda() * y.abs() ** 2).sum()
    loss.backward()
    g = x.grad.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(7)
    x64 = xc.astype(np.complex128)
    h = 1e-4
    for _ in range(12):
        t, j = int(rng.integers(4)), int(rng.integers(N))
        fd = []
        for dv in (1.0, 1j):
            xp = x64.copy(); xp[t, j] += h * dv
            xm = x64.copy(); xm[t, j] -= h * dv
            fd.append((loss_np(xp, w, N1, N2) - loss_np(xm, w, N1, N2)) / (2 * h))
        want = fd[0] + 1j * fd[1]                     # dL/dRe + i dL/dIm
        scale = np.sqrt(np.mean(np.abs(g) ** 2))
        assert abs(g[t, j] - want) <= 1e-4 * scale + 1e-6 * abs(want), (t, j, g[t, j], want)


def test_analytic_adjoint_full_size():
    """256 x N = 2^20 (the differentiation workload): the GPU gradient of
    L = sum(w |F x|^2) against 2 F^H (w * F x) computed by the oracle, for
    every transform, element by element: relative L2 error per transform
    <= 5e-7 * log2 N."""
    N1 = N2 = 1024
    N = N1 * N2
    batch = 256
    xh = gaussian(batch * N, 0, np.complex64).reshape(batch, N)
    wh = weights(batch * N, 1).reshape(batch, N)
    x = torch.from_numpy(xh).cuda()
    wt = torch.from_numpy(wh).cuda()
    x.requires_grad_(True)
    y = paco.PacoFFT.apply(x, N1, N2, 4, 4)
    (wt * y.abs() ** 2).sum().backward()
    g = x.grad.cpu().numpy()
    del x, wt, y
    torch.cuda.empty_cache()
    yo = oracle.fft(xh.astype(np.complex128), -1, threads=0)
    yo *= wh.astype(np.float64)
    want = oracle.fft(yo, +1, threads=0)
    want *= 2.0
    del yo
    errs = np.linalg.norm(g.astype(np.complex128) - want, axis=1) / np.linalg.norm(want, axis=1)
    tol = 5e-7 * math.log2(N)
    assert float(errs.max()) <= tol, f"max rel_l2 {errs.max():.3e} over {batch} gradients"


@pytest.mark.parametrize("N1,N2,b,batch", [(32, 32, 2, 3), (64, 256, 4, 2), (1024, 1024, 4, 4)])
def test_fused_weighted_power_loss(N1, N2, b, batch):
    """weighted_power_loss (the loss summed by the Phase III kernel, the
    backward's w-product applied by the conjugate transform's loads): the
    loss against sum(w |F x|^2) from the oracle (relative error <= 1e-6, the
    FP32 rounding of y), the output y against the oracle's F x, and the
    gradient with an upstream factor of 3 against 6 F^H (w * F x), every
    transform element by element within 5e-7 * log2 N."""
    N = N1 * N2
    xh = gaussian(batch * N, 11 + b, np.complex64).reshape(batch, N)
    wh = weights(batch * N, 12 + b).reshape(batch, N)
    x = torch.from_numpy(xh).cuda().requires_grad_(True)
    wt = torch.from_numpy(wh).cuda()
    loss = paco.weighted_power_loss(x, wt, N1, N2, b)
    assert loss.dtype == torch.float64 and loss.dim() == 0
    (3.0 * loss).backward()
    yo = oracle.fft(xh.astype(np.complex128), -1, threads=0)
    want_loss = float(np.sum(wh.astype(np.float64) * np.abs(yo) ** 2))
    assert abs(loss.item() - want_loss) <= 1e-6 * want_loss
    want = 6.0 * oracle.fft(yo * wh.astype(np.float64), +1, threads=0)
    g = x.grad.cpu().numpy().astype(np.complex128)
    errs = np.linalg.norm(g - want, axis=1) / np.linalg.norm(want, axis=1)
    assert float(errs.max()) <= 5e-7 * math.log2(N), errs.max()


def test_fused_loss_matches_unfused_path():
    """The fused loss and gradient equal the unfused composition
    (PacoFFT + PyTorch's w |y|^2) to FP32 rounding."""
    N1 = N2 = 64
    N, batch = N1 * N2, 5
    xh = gaussian(batch * N, 21, np.complex64).reshape(batch, N)
    wt = torch.from_numpy(weights(batch * N, 22).reshape(batch, N)).cuda()
    xa = torch.from_numpy(xh).cuda().requires_grad_(True)
    xb = torch.from_numpy(xh).cuda().requires_grad_(True)
    la = paco.weighted_power_loss(xa, wt, N1, N2, 2)
    la.backward()
    yb = paco.PacoFFT.apply(xb, N1, N2, 2)
    lb = (wt * torch.view_as_real(yb).pow(2).sum(-1)).sum()
    lb.backward()
    assert abs(la.item() - lb.item()) <= 1e-5 * abs(lb.item())
    d = (xa.grad - xb.grad).abs().max().item()
    assert d <= 1e-5 * xb.grad.abs().max().item()


def test_fused_loss_rejects_panel_plans():
    """Plans with a 2^14 complex64 factor (panel stages) do not take the
    weighted terms: PACO_ERR_UNSUPPORTED, nothing launched."""
    N1, N2 = 1 << 14, 128
    x = torch.zeros(N1 * N2, dtype=torch.complex64, device="cuda")
    w = torch.ones(N1 * N2, dtype=torch.float32, device="cuda")
    with pytest.raises(paco.PacoError) as e:
        paco.weighted_power_loss(x, w, N1, N2, 2)
    assert e.value.status == 2                               # PACO_ERR_UNSUPPORTED


def test_weighted_entry_points_directly():
    """The two C-ABI calls behind weighted_power_loss, each form:
    out_weighted = 0 / 1 (y or w * y stored, the loss the same) and the
    weighted input with a weight array, with a scalar only, and with both."""
    N1 = N2 = 64
    N, batch = N1 * N2, 3
    plan = paco.Plan(N1, N2, 2, batch, paco.C64)
    xh = gaussian(batch * N, 31, np.complex64).reshape(batch, N)
    wh = weights(batch * N, 32).reshape(batch, N)
    x = torch.from_numpy(xh).cuda()
    w = torch.from_numpy(wh).cuda()
    y = torch.empty_like(x)
    u = torch.empty_like(x)
    l0 = torch.empty((), dtype=torch.float64, device="cuda")
    l1 = torch.empty((), dtype=torch.float64, device="cuda")
    plan.execute_weighted_power(x, y, w, l0, -1)
    plan.execute_weighted_power(x, u, w, l1, -1, out_weighted=True)
    yo = oracle.fft(xh.astype(np.complex128))
    want = float(np.sum(wh * np.abs(yo) ** 2))
    assert abs(l0.item() - want) <= 1e-6 * want and abs(l1.item() - want) <= 1e-6 * want
    assert np.allclose(u.cpu().numpy(), wh * y.cpu().numpy(), rtol=1e-6, atol=1e-6 * np.abs(yo).max())
    g = torch.full((), 0.75, dtype=torch.float64, device="cuda")
    for wt, sc, mult, factor in ((w, None, 3.0, 3.0 * wh), (None, g, 2.0, 1.5), (w, g, 2.0, 1.5 * wh)):
        out = torch.empty_like(x)
        plan.execute_weighted_input(x, out, wt, sc, mult, +1)
        ref = oracle.fft(factor * xh.astype(np.complex128), +1)
        err = np.linalg.norm(out.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert float(err.max()) <= 5e-7 * math.log2(N)

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

"""GPU parity of the tensor-core precision forms: radix-16 sub-DFTs as
BF16 3-term split or FP16 per-block-scaled contractions with FP32
accumulation, against the FP64 oracle.  Bounds: the BF16x3 form must meet
the complex64 bound 5e-7*log2(N); the FP16 form the FP16 bound 1e-3
(relative L2 per transform)."""

import math

import numpy as np
import pytest

import oracle
from paco_inputs import loguniform, uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402

FORMS = {"bf16x3": paco.C64_TC_BF16X3, "fp16": paco.C64_TC_FP16}


def bound(form, N):
    return 5e-7 * math.log2(N) if form == "bf16x3" else 1e-3


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128).reshape(ref.shape)
    return float(np.max(np.linalg.norm(got - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("N1,N2,b,batch", [(256, 256, 4, 3), (256, 256, 2, 1), (1024, 256, 4, 2),
                                           (256, 4096, 16, 1), (4096, 4096, 4, 2)])
@pytest.mark.parametrize("gen", ["uniform", "loguniform"])
def test_tc_form_vs_oracle(form, N1, N2, b, batch, gen):
    N = N1 * N2
    mk = uniform if gen == "uniform" else loguniform
    x = mk(batch * N, N1 + N2 + batch, np.complex64).reshape(batch, N)
    plan = paco.Plan(N1, N2, b, batch, FORMS[form])
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    for d in (-1, 1):
        plan.execute(xt, out, d)
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.fft(x.astype(np.complex128), dir=d)
        err = rel_l2(out.cpu().numpy(), ref)
        assert err <= bound(form, N), f"{form} dir={d} rel_l2={err:.3e}"


@pytest.mark.parametrize("form", list(FORMS))
def test_tc_form_full_size(form):
    """N = 2^28 (2^14 x 2^14, b = 4, p = 64), the size the precision forms
    are benchmarked at: the whole output against the oracle's full FP64 FFT,
    both directions, at the form's bound (relative L2)."""
    N1 = N2 = 2 ** 14
    N = N1 * N2
    plan = paco.Plan(N1, N2, 4, 1, FORMS[form], p=64)
    xh = uniform(N, 0, np.complex64)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    x128 = xh.astype(np.complex128).reshape(1, N)
    del xh
    for d in (-1, 1):
        plan.execute(x, y, d)
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.fft(x128, dir=d, threads=0).reshape(N)
        got = y.cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= bound(form, N), f"{form} dir={d} rel_l2={err:.3e}"
        del ref, got
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", ["plain", "bf16x3", "fp16"])
def test_precision_workload_full_size(form):
    """The precision benchmark's configuration: 16 transforms of 2^24
    (4096 x 4096, b = 4) with log-uniform magnitudes 1e-4..1e4 and uniform
    phases.  Every transform, element by element, against the oracle's FP64
    FFT at the form's bound (5e-7 * log2 N, or 1e-3 for FP16)."""
    from paco_inputs import loguniform
    N1 = N2 = 4096
    N, B = N1 * N2, 16
    dt = {"plain": paco.C64, "bf16x3": paco.C64_TC_BF16X3, "fp16": paco.C64_TC_FP16}[form]
    x = np.concatenate([loguniform(N, 100 + i, np.complex64) for i in range(B)])
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    plan = paco.Plan(N1, N2, 4, B, dt)
    plan.execute(xt, y, -1)
    torch.cuda.synchronize()
    plan.check()
    bound_ = 5e-7 * 24 if form != "fp16" else 1e-3
    yh = y.cpu().numpy().reshape(B, N)
    ref = oracle.fft(x.astype(np.complex128).reshape(B, N), dir=-1, threads=0)
    errs = np.linalg.norm(yh.astype(np.complex128) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert float(errs.max()) <= bound_, (form, errs)

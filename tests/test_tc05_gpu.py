"""The tcgen05 probe (paco_probe_tc05_dft128): the 128-point DFT sub-pass as
a BF16x3 complex GEMM on the tensor cores, against the FP64 DFT of the same
input, per sequence.  The operands are kept to about 2^-17 relative (two bf16
terms each, the cross term of the two low parts dropped), so the stated
bound is 2e-5 relative L2 per sequence."""

import numpy as np
import pytest

from paco_inputs import gaussian

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_06449_gb300 as paco  # noqa: E402


def _dft128_columns(x):
    """y[b][k][c] = sum_j exp(-2 pi i jk / 128) x[b][j][c], FP64."""
    j = np.arange(128)
    F = np.exp(-2j * np.pi * np.outer(j, j) / 128)
    return np.einsum("kj,bjc->bkc", F, x.astype(np.complex128))


@pytest.mark.parametrize("batch,C", [(1, 64), (2, 128), (8, 4096), (3, 1216)])
def test_tc05_dft128_against_fp64(batch, C):
    x = gaussian(batch * 128 * C, 7 + C, np.complex64).reshape(batch, 128, C)
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)
    paco.probe_tc05_dft128(xt, yt, batch, C, timed=True)
    y = yt.cpu().numpy().astype(np.complex128)
    ref = _dft128_columns(x)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)    # per (b, c) sequence
    assert float(err.max()) <= 2e-5, float(err.max())


def test_tc05_rejects_bad_shapes():
    x = torch.zeros(128 * 96, dtype=torch.complex64, device="cuda")
    with pytest.raises(paco.PacoError):
        paco.probe_tc05_dft128(x, torch.empty_like(x), 1, 96)

"""Pins of the CPU oracle's DFT against facts the mathematics fixes.

The oracle evaluates the canonical DFT of Sect. 2 (y = Omega_N x,
(Omega_N)_{k,j} = w_N^{-kj}, w_N = e^{2 pi i/N}).  Each test below checks it
against something other than itself: closed forms of the definition, the
brute-force direct sum on small inputs, and an independent library FFT."""

import numpy as np
import pytest

import oracle
from paco_inputs import gaussian, uniform

SIZES_SMALL = [1, 2, 4, 8, 16, 32, 64, 256, 1024]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("f", ["direct", "fft"])
@pytest.mark.parametrize("n", [8, 64, 512])
def test_delta_and_constant(f, n):
    fn = oracle.dft_direct if f == "direct" else oracle.fft
    # delta at 0 -> all ones
    d = np.zeros(n, complex); d[0] = 1
    assert np.allclose(fn(d), np.ones(n), atol=1e-13)
    # delta at j0 -> w^{-k j0} = exp(-2 pi i k j0 / n)
    j0 = n // 3 if n > 2 else 1
    d = np.zeros(n, complex); d[j0] = 1
    k = np.arange(n)
    assert np.allclose(fn(d), np.exp(-2j * np.pi * k * j0 / n), atol=1e-13)
    # constant -> n * delta_{k,0}
    e = np.zeros(n, complex); e[0] = n
    assert np.allclose(fn(np.ones(n, complex)), e, atol=1e-12 * n)


@pytest.mark.parametrize("f", ["direct", "fft"])
@pytest.mark.parametrize("n", [16, 256])
def test_single_tone(f, n):
    """x_j = w^{+f j} -> y_k = n * delta_{k,f}: fixes the sign convention."""
    fn = oracle.dft_direct if f == "direct" else oracle.fft
    for fr in [1, 3, n - 1]:
        x = np.exp(2j * np.pi * fr * np.arange(n) / n)
        y = fn(x)
        want = np.zeros(n, complex); want[fr] = n
        assert np.allclose(y, want, atol=1e-11 * n)


@pytest.mark.parametrize("n", [64, 1024, 4096])
def test_parseval_linearity_real_symmetry(n):
    x = gaussian(n, 11, np.complex128)
    z = gaussian(n, 12, np.complex128)
    y = oracle.fft(x)
    assert abs(np.vdot(y, y).real - n * np.vdot(x, x).real) <= 1e-12 * n * np.vdot(x, x).real
    a, b = 0.75 - 0.5j, -1.25 + 2j
    assert _rel(oracle.fft(a * x + b * z), a * y + b * oracle.fft(z)) < 1e-14
    r = x.real.astype(complex)
    yr = oracle.fft(r)
    k = np.arange(1, n)
    assert np.allclose(yr[n - k], np.conj(yr[k]), atol=1e-12 * np.sqrt(n))


@pytest.mark.parametrize("n", [2, 16, 1024])
def test_round_trip(n):
    """dir=+1 after dir=-1 gives n*x (unnormalised conjugate transform)."""
    x = uniform(n, 5, np.complex128)
    back = oracle.fft(oracle.fft(x, dir=-1), dir=+1)
    assert _rel(back, n * x) < 1e-14
    back_d = oracle.dft_direct(oracle.dft_direct(x, -1), +1)
    assert _rel(back_d, n * x) < 1e-15


@pytest.mark.parametrize("n", SIZES_SMALL + [4096])
def test_fft_equals_direct_sum(n):
    """Brute force on small inputs: recursive FFT vs the O(n^2) sum."""
    x = gaussian(n, n, np.complex128)
    for d in (-1, 1):
        assert _rel(oracle.fft(x, d), oracle.dft_direct(x, d)) < 1e-14


@pytest.mark.parametrize("n", [2 ** 12, 2 ** 16, 2 ** 20])
def test_fft_matches_independent_library(n):
    """numpy's pocketfft shares no code with the oracle."""
    x = uniform(n, 3, np.complex128)
    assert _rel(oracle.fft(x), np.fft.fft(x)) < 1e-14
    assert _rel(oracle.fft(x, +1), np.fft.ifft(x) * n) < 1e-14


def test_batched_fft_is_per_row():
    x = gaussian(8 * 256, 2, np.complex128).reshape(8, 256)
    y = oracle.fft(x, threads=4)
    for t in range(8):
        assert _rel(y[t], oracle.dft_direct(x[t])) < 1e-14


@pytest.mark.parametrize("n", [4096, 2 ** 16])
def test_dft_at_matches(n):
    x = uniform(n, 9, np.complex128)
    ks = np.array([0, 1, 7, n // 2, n - 1, 12345 % n])
    ref = np.fft.fft(x)[ks]
    for d, r in ((-1, ref), (1, np.fft.ifft(x)[ks] * n)):
        got = oracle.dft_at(x, ks, d)
        assert np.max(np.abs(got - r)) / np.max(np.abs(r)) < 1e-13
    if n <= 4096:
        assert np.allclose(oracle.dft_at(x, ks), oracle.dft_direct(x)[ks], atol=1e-10)


def test_bad_arguments_are_rejected():
    with pytest.raises(ValueError):
        oracle.fft(np.zeros(12, complex))          # not a power of two
    with pytest.raises(ValueError):
        oracle.dft_at(np.zeros(8, complex), [8])   # k out of range


@pytest.mark.parametrize("lg,batch", [(15, 1), (18, 1), (17, 3), (16, 16)])
@pytest.mark.parametrize("d", [-1, 1])
def test_threaded_fft_is_bit_identical(lg, batch, d):
    """The OpenMP forms (top recursion levels as tasks for a few large
    transforms, whole transforms per thread for many) run the same butterflies
    on the same operands as the one-thread recursion: the outputs must be
    equal bit for bit, whatever the thread count."""
    x = uniform(batch << lg, 5, np.complex128).reshape(batch, 1 << lg)
    one = oracle.fft(x, dir=d, threads=1)
    for t in (2, 3, 8):
        assert np.array_equal(oracle.fft(x, dir=d, threads=t), one)


def test_oracle_2d_dft_against_numpy_fft2():
    """The 2-D reference of the dims = 2 tests (the oracle's 1-D DFT down the
    columns, then along the rows, returned transposed) against numpy's fft2,
    an independent library routine, both directions."""
    import oracle2d
    rng = np.random.default_rng(17)
    for N1, N2 in ((8, 16), (32, 32), (64, 8)):
        x = rng.standard_normal((3, N1 * N2)) + 1j * rng.standard_normal((3, N1 * N2))
        got = oracle2d.fft2_transposed(x, N1, N2, -1)
        want = np.stack([np.fft.fft2(xi.reshape(N1, N2)).T.reshape(-1) for xi in x])
        assert np.allclose(got, want, atol=1e-10 * np.abs(want).max())
        got = oracle2d.fft2_transposed(x, N1, N2, +1)
        want = np.stack([(N1 * N2 * np.fft.ifft2(xi.reshape(N1, N2))).T.reshape(-1) for xi in x])
        assert np.allclose(got, want, atol=1e-10 * np.abs(want).max())


def test_oracle_3d_dft_against_numpy_fftn():
    """The 3-D reference of the dims = 3 tests (the oracle's 1-D DFT along
    each axis in turn, returned with the axes reversed) against numpy's fftn,
    an independent library routine, both directions; unequal axes, so that a
    swapped pair of axes or a missed transpose fails."""
    import oracle2d
    rng = np.random.default_rng(23)
    for N1, N2, N3 in ((4, 8, 16), (16, 4, 8), (8, 32, 2)):
        N = N1 * N2 * N3
        x = rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))
        got = oracle2d.fft3_reversed(x, N1, N2, N3, -1)
        want = np.stack([np.fft.fftn(xi.reshape(N1, N2, N3)).transpose(2, 1, 0).reshape(-1) for xi in x])
        assert np.allclose(got, want, atol=1e-10 * np.abs(want).max())
        got = oracle2d.fft3_reversed(x, N1, N2, N3, +1)
        want = np.stack([(N * np.fft.ifftn(xi.reshape(N1, N2, N3))).transpose(2, 1, 0).reshape(-1) for xi in x])
        assert np.allclose(got, want, atol=1e-10 * np.abs(want).max())

"""Seeded synthetic inputs for the PACO hot path.

This module holds random-number recipes only: no transform arithmetic, no
index maps, nothing of the method.  The CPU oracle, the tests and the
benchmark all draw their inputs here, so that both sides of a parity check see
the same bytes.  Every generator takes an explicit integer seed and uses
numpy's PCG64 ``default_rng``.

Workload recipes (the method itself fixes none of them; the paper has no
experiments, so these stand in for its workloads):

* ``uniform``      -- real and imaginary parts i.i.d. U[-1, 1)
* ``gaussian``     -- real and imaginary parts i.i.d. N(0, 1)
* ``loguniform``   -- magnitude 10**U[-4, 4), phase U[0, 2*pi)
* ``weights``      -- real weights U[0, 1)
* ``uneven_lengths`` -- log2-lengths of the uneven batch (see its docstring)
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "complex_input",
    "uniform",
    "gaussian",
    "loguniform",
    "weights",
    "uneven_lengths",
]


def _real_dtype(dtype) -> type:
    dtype = np.dtype(dtype)
    if dtype == np.complex64:
        return np.float32
    if dtype == np.complex128:
        return np.float64
    raise ValueError(f"unsupported complex dtype {dtype}")


def uniform(n: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """``n`` complex values with Re, Im i.i.d. U[-1, 1), drawn in the real
    dtype of ``dtype`` (so a complex64 draw is exactly representable)."""
    rt = _real_dtype(dtype)
    rng = np.random.default_rng(seed)
    v = rng.random(size=2 * int(n), dtype=rt)
    v *= rt(2.0)
    v -= rt(1.0)
    return v.view(np.dtype(dtype))


def gaussian(n: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """``n`` complex values with Re, Im i.i.d. N(0, 1)."""
    rt = _real_dtype(dtype)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(size=2 * int(n), dtype=rt)
    return v.view(np.dtype(dtype))


def loguniform(n: int, seed: int, dtype=np.complex64,
               lo_exp: float = -4.0, hi_exp: float = 4.0) -> np.ndarray:
    """``n`` complex values with magnitude 10**U[lo_exp, hi_exp) and phase
    U[0, 2*pi): a wide dynamic range for the precision study."""
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(lo_exp, hi_exp, size=int(n))
    ph = rng.uniform(0.0, 2.0 * np.pi, size=int(n))
    return (mag * np.exp(1j * ph)).astype(dtype)


def weights(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    """``n`` real weights i.i.d. U[0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.random(size=int(n), dtype=np.dtype(dtype).type)


def complex_input(kind: str, n: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """Dispatch by recipe name: 'uniform', 'gaussian' or 'loguniform'."""
    if kind == "uniform":
        return uniform(n, seed, dtype)
    if kind == "gaussian":
        return gaussian(n, seed, dtype)
    if kind == "loguniform":
        return loguniform(n, seed, dtype)
    raise ValueError(f"unknown input recipe {kind!r}")


def uneven_lengths(count: int = 4096, seed: int = 0, lo: int = 8, hi: int = 20,
                   total_log2: int = 28) -> np.ndarray:
    """log2-lengths for the uneven batch: ``count`` exponents drawn i.i.d.
    uniform over {lo..hi}; then, while the total length exceeds
    2**total_log2, the largest exponent (first on ties) is decremented, never
    below ``lo``.  Returns an int64 array of exponents."""
    rng = np.random.default_rng(seed)
    e = rng.integers(lo, hi + 1, size=int(count)).astype(np.int64)
    limit = 1 << int(total_log2)
    total = int(np.sum(np.left_shift(np.int64(1), e)))
    while total > limit:
        i = int(np.argmax(e))
        if e[i] <= lo:
            break
        total -= 1 << int(e[i] - 1)
        e[i] -= 1
    return e

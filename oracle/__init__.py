"""CPU oracle for the PACO hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product library: the two share no code.

Contents
--------
* ``dft_direct``, ``fft``, ``dft_at``: the canonical DFT of Sect. 2,
  ``y = Omega_N x`` with ``(Omega_N)_{k,j} = w_N^{-kj}``, ``w_N = e^{2 pi i/N}``,
  evaluated by the C reference in ``oracle.c`` (long-double direct sum, FP64
  recursive radix-2 Cooley-Tukey, FP64 exact-residue sum at chosen outputs).
* ``digit_reverse`` / ``digit_reverse_table``: base-b digit reversal
  ``pi_ell`` (Sect. 3.2, App. A.1) from explicit digit arrays.
* ``paco_sim``: the paper's procedures written step by step -- the
  cache-oblivious batched local FFT over digit-field views (Fig. "cofft",
  App. B; views and splits of App. A.3-A.4), Macro-Digit-Reversal and
  Fused-Macro-Digit-Reversal (App. C.1-C.2), and PARA-CO-DRP_b (App. C.5) with
  p simulated processors and an explicit all-to-all.  It produces the
  intermediates the CUDA path exposes (the Phase-I output slab, the
  redistributed array ``W = Z-hat`` of Eq. (17)) and the end-to-end result.

``dir = -1`` is the paper's forward transform; ``dir = +1`` is the
unnormalised conjugate transform, which the paper does not define (reading:
every root ``w^{-r}`` becomes ``w^{+r}``).
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

__all__ = [
    "load",
    "num_threads",
    "dft_direct",
    "fft",
    "dft_at",
    "digit_reverse",
    "digit_reverse_table",
]

_lib = None


def _declare(lib):
    i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_dft_direct.argtypes = [i64, dp, dp, i32]
    lib.oracle_dft_direct.restype = i32
    lib.oracle_fft.argtypes = [i64, i64, dp, dp, i32, i32]
    lib.oracle_fft.restype = i32
    lib.oracle_dft_at.argtypes = [i64, dp, i64, dp, dp, i32, i32]
    lib.oracle_dft_at.restype = i32
    lib.oracle_digit_reverse.argtypes = [i64, i64, i32]
    lib.oracle_digit_reverse.restype = i64
    lib.oracle_digit_reverse_table.argtypes = [i64, i32, dp]
    lib.oracle_digit_reverse_table.restype = i32
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = i32
    return lib


def load():
    """Build (if stale) and load liboracle.so."""
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(_build.build()))
    return _lib


class Bound:
    """The oracle's entry points bound to a given build of oracle.c (the
    tests bind planted-mistake builds this way)."""

    def __init__(self, path: str):
        self.lib = _declare(ctypes.CDLL(path))

    def dft_direct(self, x, dir=-1):
        return dft_direct(x, dir, lib=self.lib)

    def fft(self, x, dir=-1, threads=0):
        return fft(x, dir, threads, lib=self.lib)

    def dft_at(self, x, ks, dir=-1, threads=0):
        return dft_at(x, ks, dir, threads, lib=self.lib)

    def digit_reverse(self, u, b, ell):
        return digit_reverse(u, b, ell, lib=self.lib)

    def digit_reverse_table(self, b, ell):
        return digit_reverse_table(b, ell, lib=self.lib)


def num_threads() -> int:
    return int(load().oracle_num_threads())


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def dft_direct(x, dir: int = -1, lib=None) -> np.ndarray:
    """Direct O(n^2) DFT of a 1-D vector, long-double accumulation."""
    x = _c128(x).ravel()
    y = np.empty_like(x)
    rc = (lib or load()).oracle_dft_direct(x.size, _ptr(x), _ptr(y), int(dir))
    if rc != 0:
        raise ValueError(f"oracle_dft_direct failed ({rc})")
    return y


def fft(x, dir: int = -1, threads: int = 0, lib=None) -> np.ndarray:
    """FP64 recursive radix-2 FFT along the last axis (length a power of 2)."""
    x = _c128(x)
    n = x.shape[-1] if x.ndim else 1
    batch = x.size // n if n else 0
    y = np.empty_like(x)
    rc = (lib or load()).oracle_fft(n, batch, _ptr(x), _ptr(y), int(dir), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_fft failed ({rc})")
    return y


def dft_at(x, ks, dir: int = -1, threads: int = 0, lib=None) -> np.ndarray:
    """The DFT definition evaluated only at output indices ``ks`` (FP64,
    exact residues, pairwise summation): O(n) work per output."""
    x = _c128(x).ravel()
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64).ravel())
    out = np.empty(ks.size, dtype=np.complex128)
    rc = (lib or load()).oracle_dft_at(x.size, _ptr(x), ks.size, _ptr(ks), _ptr(out),
                              int(dir), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_dft_at failed ({rc})")
    return out


def digit_reverse(u: int, b: int, ell: int, lib=None) -> int:
    """pi_ell(u) in base b, from an explicit digit array."""
    r = int((lib or load()).oracle_digit_reverse(int(u), int(b), int(ell)))
    if r < 0:
        raise ValueError("digit_reverse: bad argument")
    return r


def digit_reverse_table(b: int, ell: int, lib=None) -> np.ndarray:
    """[pi_ell(u) for u in range(b**ell)]."""
    n = int(b) ** int(ell)
    out = np.empty(n, dtype=np.int64)
    rc = (lib or load()).oracle_digit_reverse_table(int(b), int(ell), _ptr(out))
    if rc != 0:
        raise ValueError("digit_reverse_table: bad argument")
    return out

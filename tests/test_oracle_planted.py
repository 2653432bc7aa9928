"""The pins catch plausible mistakes: each build of oracle.c with one planted
error (ORACLE_PLANT, see oracle.c) must fail at least one pin check."""

import numpy as np
import pytest

import oracle
from oracle import build as obuild
from paco_inputs import gaussian


def _pins(o):
    """Run the core pins against a bound oracle; return the names that fail."""
    bad = []
    n = 64
    k = np.arange(n)
    d = np.zeros(n, complex); d[5] = 1
    want = np.exp(-2j * np.pi * k * 5 / n)
    if not np.allclose(o.dft_direct(d), want, atol=1e-12):
        bad.append("delta-direct")
    if not np.allclose(o.fft(d), want, atol=1e-12):
        bad.append("delta-fft")
    tone = np.exp(2j * np.pi * 3 * k / n)
    t = np.zeros(n, complex); t[3] = n
    if not np.allclose(o.fft(tone), t, atol=1e-9):
        bad.append("tone-fft")
    x = gaussian(n, 1, np.complex128)
    if not np.allclose(o.dft_direct(x), np.fft.fft(x), atol=1e-10):
        bad.append("direct-vs-library")
    if not np.allclose(o.dft_at(x, [0, 3, 17]), np.fft.fft(x)[[0, 3, 17]], atol=1e-10):
        bad.append("dft_at-vs-library")
    if list(o.digit_reverse_table(2, 3)) != [0, 4, 2, 6, 1, 5, 3, 7] or \
            o.digit_reverse(0b011011, 4, 3) != 0b111001:
        bad.append("digit-reversal")
    return bad


def test_clean_build_passes_pins():
    assert _pins(oracle.Bound(obuild.build())) == []


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5, 6])
def test_planted_mistake_is_caught(plant, tmp_path):
    path = obuild.build(plant=plant, out=str(tmp_path / f"liboracle_plant{plant}.so"))
    assert _pins(oracle.Bound(path)) != []

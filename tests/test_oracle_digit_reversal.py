"""Pins of the oracle's base-b digit reversal pi_ell (Sect. 3.2, App. A.1)."""

import itertools

import numpy as np
import pytest

import oracle


def test_hand_computed_examples():
    # b = 2 on 3 bits: the classic bit-reversal order
    assert list(oracle.digit_reverse_table(2, 3)) == [0, 4, 2, 6, 1, 5, 3, 7]
    # b = 4, ell = 3: digits (1,2,3) -> (3,2,1): 0b01_10_11 -> 0b11_10_01
    assert oracle.digit_reverse(0b011011, 4, 3) == 0b111001
    # b = 8, ell = 2: 8*d1 + d0 -> 8*d0 + d1
    assert oracle.digit_reverse(8 * 5 + 3, 8, 2) == 8 * 3 + 5
    # b = 16, ell = 3: 0x1A7 -> 0x7A1
    assert oracle.digit_reverse(0x1A7, 16, 3) == 0x7A1
    # base 4 keeps the bit order inside a digit: not bit reversal
    assert oracle.digit_reverse(0b0001, 4, 2) == 0b0100
    assert oracle.digit_reverse(0b0001, 2, 4) == 0b1000
    # the paper's Fig. 1 caption: on 2 bits, 1 <-> 2, 0 and 3 fixed
    assert list(oracle.digit_reverse_table(2, 2)) == [0, 2, 1, 3]


@pytest.mark.parametrize("b", [2, 4, 8, 16])
def test_involution_and_bijection(b):
    for ell in range(0, 5 if b <= 4 else 4):
        t = oracle.digit_reverse_table(b, ell)
        n = b ** ell
        assert sorted(t.tolist()) == list(range(n))
        assert np.array_equal(t[t], np.arange(n))


@pytest.mark.parametrize("b", [2, 4, 8, 16])
def test_composition_identity(b):
    """pi_l(a*n2 + c) = pi_l1(a) + pi_l2(c)*n1 (App. A.6, the step from
    Eq. (finalfreq) to the parent coordinate), and its global form
    pi_m(a ++ c) = pi_m2(c) ++ pi_m1(a) (Eq. full-middle-digit-reversal)."""
    for l1, l2 in itertools.product(range(0, 3), range(0, 3)):
        n1, n2 = b ** l1, b ** l2
        t = oracle.digit_reverse_table(b, l1 + l2)
        t1 = oracle.digit_reverse_table(b, l1)
        t2 = oracle.digit_reverse_table(b, l2)
        a = np.repeat(np.arange(n1), n2)
        c = np.tile(np.arange(n2), n1)
        assert np.array_equal(t[a * n2 + c], t1[a] + t2[c] * n1)


def test_rejects_too_many_digits():
    with pytest.raises(ValueError):
        oracle.digit_reverse(16, 2, 4)   # 16 needs 5 binary digits

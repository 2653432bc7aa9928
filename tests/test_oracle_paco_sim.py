"""Pins of the step-by-step PACO simulator (oracle/paco_sim.py).

Each check compares the procedures against an independent statement of what
they must produce: the paper's worked example (Fig. 1), closed forms of the
intermediates (Lemma 1; Eq. (17)), the DFT itself (Theorem 3, via numpy's
independent FFT), and the balance counts of Theorem 4."""

import os

import numpy as np
import pytest

from oracle import paco_sim as ps
from paco_inputs import gaussian, uniform

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_para_co_drp.txt")

CONFIGS = [  # (N1, N2, b, p)
    (4, 4, 2, 2), (16, 16, 2, 2), (16, 64, 4, 4), (64, 16, 4, 4),
    (64, 64, 8, 8), (256, 16, 16, 16), (256, 256, 2, 4), (64, 256, 4, 16),
]


def _read_golden():
    panels, cur = {}, None
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("panel"):
                cur = line.split()[1]
                panels[cur] = []
                continue
            panels[cur].append([tuple(int(v) for v in cell.split(",")) for cell in line.split()])
    return {k: np.array(v) for k, v in panels.items()}   # (rows, cols, 3)


def test_fig1_worked_example():
    """Fig. 1: N1 = N2 = 4, p = 2, b = 2; every panel, every cell and owner."""
    g = _read_golden()
    N1 = N2 = 4
    p, b = 2, 2
    w1, w2 = N1 // p, N2 // p
    labels = np.arange(N1 * N2).reshape(N1, N2)         # label = a*N2 + c
    slabs = [labels[:, q * w2:(q + 1) * w2] for q in range(p)]
    tr = {}
    out = ps.para_co_drp(slabs, N1, N2, b, p, twiddle=False, trace=tr)

    def cells(arr, owner):
        r, c = np.indices(arr.shape)
        return np.stack([arr // N2, arr % N2, owner(r, c)], axis=-1)

    init = np.concatenate(slabs, axis=1)
    assert np.array_equal(cells(init, lambda r, c: c // w2), g["initial"])
    packed = np.concatenate(tr["packed"], axis=1)
    assert np.array_equal(cells(packed, lambda r, c: c // w2), g["packed"])
    # received: processor q' holds the packed rows of its row slab, assembled
    # from the raw regions R_{q',q} in source order.
    recv = np.concatenate([np.concatenate([tr["raw"][(qd, q)] for q in range(p)], axis=1)
                           for qd in range(p)], axis=0)
    assert np.array_equal(cells(recv, lambda r, c: r // w1), g["received"])
    transposed = np.concatenate(tr["transposed"], axis=1)
    assert np.array_equal(cells(transposed, lambda r, c: c // w1), g["transposed"])
    output = np.concatenate(out, axis=1)
    assert np.array_equal(cells(output, lambda r, c: c // w1), g["output"])


@pytest.mark.parametrize("N1,N2,b,p", CONFIGS)
def test_coordinate_trace(N1, N2, b, p):
    """The procedure realises (a, c) -> (pi_m2(c), pi_m1(a)) (Eq. (18))."""
    import oracle
    labels = np.arange(N1 * N2).reshape(N1, N2)
    w2 = N2 // p
    out = ps.para_co_drp([labels[:, q * w2:(q + 1) * w2] for q in range(p)],
                         N1, N2, b, p, twiddle=False)
    W = np.concatenate(out, axis=1)
    m1, m2 = ps.log_b(N1, b), ps.log_b(N2, b)
    pi1 = oracle.digit_reverse_table(b, m1)
    pi2 = oracle.digit_reverse_table(b, m2)
    a, c = labels // N2, labels % N2
    expect = np.empty_like(W)
    expect[pi2[c], pi1[a]] = labels
    assert np.array_equal(W, expect)


@pytest.mark.parametrize("N1,N2,b,p", CONFIGS)
def test_balance_counts(N1, N2, b, p):
    """Theorem 4: exactly N/p^2 items per ordered pair, N/p staying on the
    diagonal (self pairs), h = (N/p)(1 - 1/p) sent by each processor and
    mu = N(1 - 1/p) in all -- counting only the items whose own coordinates
    (source = owner of input column c, destination = owner of output column
    pi_m1(a)) match the route the procedure sent them on."""
    N = N1 * N2
    counts = ps.balance_counts(N1, N2, b, p)
    assert np.all(counts == N // (p * p))
    assert np.all(np.diag(counts) == N // (p * p))
    assert counts.sum() == N                          # every item routed where it belongs
    assert np.all(counts.sum(axis=1) == N // p)       # each processor's slab leaves once
    remote = counts.sum() - np.trace(counts)
    assert remote == N - N // p                       # mu
    assert np.all(counts.sum(axis=1) - np.diag(counts) == N // p - N // (p * p))   # h


@pytest.mark.parametrize("N1,N2,b,p", CONFIGS)
def test_balance_pin_catches_misrouting(N1, N2, b, p):
    """A planted mistake in the simulator -- row blocks chosen by the physical
    row a instead of the frequency pi_m1(a) it holds (no local pack
    reversal) -- must break the balance pin: some items then travel to a
    processor that does not own their output column."""
    N = N1 * N2
    counts = ps.balance_counts(N1, N2, b, p, plant="route_by_a")
    assert not np.all(counts == N // (p * p))


@pytest.mark.parametrize("N1,N2,b,p", [(16, 16, 2, 2), (64, 16, 4, 4), (16, 64, 4, 4),
                                       (64, 64, 8, 8), (256, 16, 16, 16)])
def test_lemma1_output_layout(N1, N2, b, p):
    """CO-Batched-FFT in output layout realises P_pi Omega (Lemma 1;
    Thm A.9): physical row a holds frequency pi_m1(a).  Omega from numpy."""
    import oracle
    x = uniform(N1 * N2, 1, np.complex128).reshape(N1, N2)
    for d in (-1, 1):
        got = ps.co_batched_fft(x, b, d)
        A = np.fft.fft(x, axis=0) if d == -1 else np.fft.ifft(x, axis=0) * N1
        pi = oracle.digit_reverse_table(b, ps.log_b(N1, b))
        assert np.max(np.abs(got - A[pi, :])) < 1e-12 * N1


@pytest.mark.parametrize("N1,N2,b,p", CONFIGS)
def test_redistributed_layout_eq17(N1, N2, b, p):
    """W = Z-hat with Z-hat[u, v] = Z[v, pi_m2(u)], Z[v, c] = A[v, c] w_N^{-vc},
    A the column DFTs (Eq. (17); local pack of Sect. 4.2)."""
    import oracle
    N = N1 * N2
    x = gaussian(N, 4, np.complex128)
    r = ps.simulate(x, N1, N2, b, p, phase1="lemma" if N > 4096 else "cofft")
    A = np.fft.fft(x.reshape(N1, N2), axis=0)
    v = np.arange(N1)[:, None]
    c = np.arange(N2)[None, :]
    Z = A * np.exp(-2j * np.pi * ((v * c) % N) / N)
    pi2 = oracle.digit_reverse_table(b, ps.log_b(N2, b))
    Zhat = Z[:, pi2].T
    assert np.max(np.abs(r["W"] - Zhat)) < 1e-12 * np.sqrt(N) * 8


@pytest.mark.parametrize("N1,N2,b,p", CONFIGS)
@pytest.mark.parametrize("d", [-1, 1])
def test_end_to_end_theorem3(N1, N2, b, p, d):
    """Y[k2, k1] = y[k1 + k2 N1] (Theorem 3), and slab q' holds exactly the
    columns k1 in [q' N1/p, (q'+1) N1/p) (target ownership, Eq. (3))."""
    N = N1 * N2
    x = uniform(N, 7, np.complex128)
    r = ps.simulate(x, N1, N2, b, p, dir=d, phase1="lemma" if N > 4096 else "cofft")
    y = np.fft.fft(x) if d == -1 else np.fft.ifft(x) * N
    assert np.linalg.norm(r["Y"].ravel() - y) / np.linalg.norm(y) < 1e-14
    w1 = N1 // p
    Yfull = r["Y"]
    for q in range(p):
        k1 = np.arange(q * w1, (q + 1) * w1)
        assert np.allclose(ps.phase_three(r["slabs"][q], b, d), Yfull[:, k1], atol=1e-9)


def test_rejects_illegal_sizes():
    x = np.zeros(64, complex)
    with pytest.raises(ValueError):
        ps.simulate(x, 8, 8, 4, 2)      # 8 is not a power of 4
    with pytest.raises(ValueError):
        ps.simulate(x, 8, 8, 2, 16)     # p does not divide N1

"""The PACO procedures, step by step, on the CPU -- TEST INFRASTRUCTURE ONLY.

Written from the paper's definitions, in its notation, with no blocking,
fusion or reordering beyond what the procedures state.  Slow on purpose; sizes
are meant to stay small (N up to ~2^16).  Used by the tests to produce the
intermediates the CUDA path exposes and to check the paper's invariants.

Notation (Sect. 2): N = N1*N2, N1 = b^m1, N2 = b^m2, p processors with
p | N1 and p | N2.  Input view X[j1, j2] = x[j1*N2 + j2] (row-major N1 x N2),
owner0(j1, j2) = floor(j2*p/N2).  Output view Y[k2, k1] = y[k1 + k2*N1]
(row-major N2 x N1), owner1(k2, k1) = floor(k1*p/N1).

Procedures
----------
co_batched_fft          Fig. "cofft" (App. B): batch split when s >= n (outer
                        digit first, then the MSD of C), else a balanced
                        digit-aligned transform split with the layout-aware
                        twiddle w_n^{-pi_l1(a) j2} (Eq. twop, App. A.2) applied
                        before the second child group; natural-order DFT leaves.
                        Output-layout mode: realises P_pi Omega (Lemma 1).
macro_digit_reversal    App. C.1 (two-cycle swaps of contiguous rows).
fused_macro_digit_reversal  App. C.2 (same, times a destination-indexed g).
para_co_drp             App. C.5: pack (fused reversal with g = w_N^{-vc}),
                        one all-to-all of (N1/p) x (N2/p) blocks, per-block
                        transpose, unpack (reversal of the N2 row field).
phase_three             B_m2 = Omega P_pi (Lemma 1, input-layout form).
simulate                the three phases composed (Eq. (10), Theorem 3).
"""

from __future__ import annotations

import numpy as np

from . import digit_reverse_table, fft as _oracle_fft

# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------


def log_b(n: int, b: int) -> int:
    """ell with b**ell == n; raises if n is not a power of b."""
    ell, v = 0, 1
    while v < n:
        v *= b
        ell += 1
    if v != n:
        raise ValueError(f"{n} is not a power of {b}")
    return ell


def root(r, n: int, dir: int = -1):
    """w_n^{dir * r} for exact integer residues r (reduced mod n here)."""
    r = np.mod(np.asarray(r, dtype=np.int64), n)
    ang = 2.0 * np.pi * (r.astype(np.float64) / float(n))
    return np.cos(ang) + 1j * dir * np.sin(ang)


def _small_dft(v: np.ndarray, dir: int) -> np.ndarray:
    """Natural-order DFT along axis 0 of a (n, s) block: the constant-size
    leaf kernel of Fig. "cofft" (its n is at most b)."""
    n = v.shape[0]
    k = np.arange(n)
    mat = root(np.outer(k, k), n, dir)
    return mat @ v


# ---------------------------------------------------------------------------
# CO-Batched-FFT over digit-field views (App. A.3-A.4, App. B)
# ---------------------------------------------------------------------------


class View:
    """V = (T, O, C, F, mode) of App. A.3 for a root array whose physical
    address is sum(digit[slot] * b**slot).  T, O, C are lists of physical slot
    numbers, most significant first; F maps fixed slots to values.  P (label to
    slot) is the identity here: labels are slot numbers, and relabelling T1 as
    the output field A keeps its slots (Eq. relabel)."""

    def __init__(self, T, O, C, F):
        self.T, self.O, self.C, self.F = list(T), list(O), list(C), dict(F)


def _field_values(slots, b):
    """All assignments of a digit field as (count, len(slots)) digit arrays,
    enumerated with the first (most significant) slot varying slowest."""
    k = len(slots)
    n = b ** k
    idx = np.arange(n)
    digs = np.empty((n, k), dtype=np.int64)
    for i in range(k):
        digs[:, i] = (idx // b ** (k - 1 - i)) % b
    return digs


def _addresses(view: View, b: int) -> np.ndarray:
    """addr_V(tau, (eta, chi)) of Eq. (addr) as an (n, s) integer array:
    rows index the transform coordinate tau, columns the batch (eta, chi)."""
    base = sum(v * b ** slot for slot, v in view.F.items())
    tdig = _field_values(view.T, b)
    bdig = _field_values(view.O + view.C, b)
    tw = np.array([b ** s for s in view.T], dtype=np.int64)
    bw = np.array([b ** s for s in view.O + view.C], dtype=np.int64)
    ta = tdig @ tw if view.T else np.zeros(1, dtype=np.int64)
    ba = bdig @ bw if (view.O + view.C) else np.zeros(1, dtype=np.int64)
    return base + ta[:, None] + ba[None, :]


def _co_batched_fft(data: np.ndarray, view: View, b: int, dir: int) -> None:
    n = b ** len(view.T)
    s = b ** (len(view.O) + len(view.C))
    if n <= b and s <= b:                                   # base case
        addr = _addresses(view, b)
        data[addr] = _small_dft(data[addr], dir)
        return
    if s >= n:                                              # batch split
        if view.O:
            d = view.O[0]
            for r in range(b):
                F = dict(view.F)
                F[d] = r
                _co_batched_fft(data, View(view.T, view.O[1:], view.C, F), b, dir)
        else:
            d = view.C[0]                                   # MSD of C
            for r in range(b):
                F = dict(view.F)
                F[d] = r
                _co_batched_fft(data, View(view.T, view.O, view.C[1:], F), b, dir)
        return
    # balanced digit-aligned transform split: |T1| = ceil(l/2), |T2| = floor(l/2)
    ell = len(view.T)
    l1 = (ell + 1) // 2
    T1, T2 = view.T[:l1], view.T[l1:]
    _co_batched_fft(data, View(T1, T2 + view.O, view.C, view.F), b, dir)
    # relabel T1 -> A (same slots); layout-aware twiddle w_n^{-pi_l1(a) j2}
    # on every item of the parent view before the second child group.
    A = T1
    addr = _addresses(View(A + T2, view.O, view.C, view.F), b)   # rows: a*n2 + j2
    n1, n2 = b ** l1, b ** (ell - l1)
    a = np.arange(n1 * n2) // n2
    j2 = np.arange(n1 * n2) % n2
    pi_a = digit_reverse_table(b, l1)[a]
    data[addr] *= root(pi_a * j2, n, dir)[:, None]
    _co_batched_fft(data, View(T2, A + view.O, view.C, view.F), b, dir)


def co_batched_fft(slab: np.ndarray, b: int, dir: int = -1) -> np.ndarray:
    """Output-layout local FFT of every column of an (n, s) row-major slab
    (n and s powers of b): returns the slab whose physical row a holds the
    frequency pi_l(a) of its column's DFT, i.e. (P_pi Omega_n) per column."""
    n, s = slab.shape
    ln, ls = log_b(n, b), log_b(s, b)
    data = np.array(slab, dtype=np.complex128).ravel()
    # physical slots: column digits are slots 0..ls-1 (least significant,
    # contiguous), row digits are slots ls..ls+ln-1.
    T = [ls + i for i in range(ln - 1, -1, -1)]
    C = [i for i in range(ls - 1, -1, -1)]
    _co_batched_fft(data, View(T, [], C, {}), b, dir)
    return data.reshape(n, s)


# ---------------------------------------------------------------------------
# Macro-element digit reversals (App. C.1, C.2)
# ---------------------------------------------------------------------------


def macro_digit_reversal(X: np.ndarray, b: int) -> None:
    """In place: X'[i, :] = X[pi_l(i), :] over the n rows of X, by swapping
    the two macro-elements of each two-cycle i < pi_l(i)."""
    n = X.shape[0]
    pi = digit_reverse_table(b, log_b(n, b))
    for i in range(n):
        k = int(pi[i])
        if i < k:
            tmp = X[i].copy()
            X[i] = X[k]
            X[k] = tmp


def fused_macro_digit_reversal(X: np.ndarray, b: int, g) -> None:
    """In place: X'[i, j] = g(i, j) * X[pi_l(i), j]; g(i) returns the row of
    destination-indexed coefficients for destination row i."""
    n = X.shape[0]
    pi = digit_reverse_table(b, log_b(n, b))
    for i in range(n):
        k = int(pi[i])
        if i < k:
            x = X[i].copy()
            y = X[k].copy()
            X[i] = g(i) * y
            X[k] = g(k) * x
        elif i == k:
            X[i] = g(i) * X[i]


# ---------------------------------------------------------------------------
# PARA-CO-DRP_b (App. C.5) with p simulated processors
# ---------------------------------------------------------------------------


def para_co_drp(slabs, N1: int, N2: int, b: int, p: int, dir: int = -1,
                twiddle: bool = True, trace=None, plant: str | None = None):
    """Run the middle stage on p simulated processors.

    ``slabs[q]`` is processor q's Phase-I slab X_q (N1 x N2/p).  Returns the
    list of target slabs Y_q (N2 x N1/p).  With ``twiddle=False`` the data are
    moved only (for label-tracing).  ``trace``, if a dict, receives the packed
    slabs, the blocks sent per (q, q'), and the raw received regions.
    ``plant`` exists only so that the tests can show their pins catching a
    plausible mistake: ``"route_by_a"`` skips the local pack's digit reversal,
    so the row block sent to q' is chosen by the physical row a instead of
    the frequency pi_m1(a) it holds."""
    N = N1 * N2
    w1, w2 = N1 // p, N2 // p                  # N1/p and N2/p
    packed = []
    sent = {}
    for q in range(p):
        Xq = np.array(slabs[q], copy=True)
        if plant == "route_by_a":
            pass
        elif twiddle:
            c = q * w2 + np.arange(w2)         # global column of each c_loc
            Xq = Xq.astype(np.complex128)
            fused_macro_digit_reversal(Xq, b, lambda v: root(v * c, N, dir))
        else:
            macro_digit_reversal(Xq, b)
        packed.append(Xq)
        for qd in range(p):                    # blocks S_{q,q'}
            sent[(q, qd)] = Xq[qd * w1:(qd + 1) * w1, :].copy()
    # one all-to-all: raw region R_{q',q} on q' receives S_{q,q'}
    raw = {(qd, q): sent[(q, qd)] for q in range(p) for qd in range(p)}
    out = []
    transposed = []
    for qd in range(p):
        Yq = np.empty((N2, w1), dtype=packed[0].dtype)
        for r in range(p):                     # CO-Transpose, then copy to Y_{q,r}
            T = raw[(qd, r)].T.copy()          # (N2/p) x (N1/p)
            Yq[r * w2:(r + 1) * w2, :] = T
        transposed.append(Yq.copy())
        macro_digit_reversal(Yq, b)            # N2-field reversal
        out.append(Yq)
    if trace is not None:
        trace["packed"] = packed
        trace["sent"] = sent
        trace["raw"] = raw
        trace["transposed"] = transposed
    return out


def phase_three(W: np.ndarray, b: int, dir: int = -1) -> np.ndarray:
    """B_m2 = Omega_N2 P_pi applied down every column of W (N2 x N1): the
    logical input j of column v is the physical row pi_m2(j)."""
    N2 = W.shape[0]
    pi = digit_reverse_table(b, log_b(N2, b))
    logical = W[pi, :]                          # (P_pi w)[j] = w[pi(j)]
    return _oracle_fft(logical.T, dir=dir).T


def phase_one(x: np.ndarray, N1: int, N2: int, b: int, dir: int = -1) -> np.ndarray:
    """Phase I on the whole input: the output-layout local FFT (P_pi Omega_N1)
    of every column of X = x.reshape(N1, N2), via co_batched_fft per slab of
    one column block -- returned as the full N1 x N2 array A-tilde."""
    X = np.asarray(x, dtype=np.complex128).reshape(N1, N2)
    return co_batched_fft(X, b, dir) if N2 >= 1 else X


def simulate(x, N1: int, N2: int, b: int, p: int, dir: int = -1,
             phase1: str = "cofft"):
    """End-to-end PACO on p simulated processors.

    Returns a dict with
      'A_tilde'  Phase-I output, N1 x N2 (physical row a holds k1 = pi_m1(a));
      'W'        the redistributed array Z-hat, N2 x N1 (Eq. (17));
      'slabs'    the p target slabs Y_q (N2 x N1/p) of PARA-CO-DRP;
      'Y'        the output view, N2 x N1 (natural-order y when flattened).
    ``phase1='cofft'`` runs the digit-field recursion per input slab;
    ``phase1='lemma'`` forms P_pi Omega from the oracle FFT instead (the
    right-hand side of Lemma 1)."""
    m1, m2 = log_b(N1, b), log_b(N2, b)
    if p < 2 or N1 % p or N2 % p:
        raise ValueError("need p >= 2 with p | N1 and p | N2")
    log_b(p, b)
    X = np.asarray(x, dtype=np.complex128).reshape(N1, N2)
    w2 = N2 // p
    if phase1 == "cofft":
        A_t = np.empty_like(X)
        for q in range(p):
            A_t[:, q * w2:(q + 1) * w2] = co_batched_fft(X[:, q * w2:(q + 1) * w2], b, dir)
    else:
        A = _oracle_fft(X.T, dir=dir).T
        A_t = A[digit_reverse_table(b, m1), :]
    slabs = [A_t[:, q * w2:(q + 1) * w2] for q in range(p)]
    out = para_co_drp(slabs, N1, N2, b, p, dir)
    W = np.concatenate(out, axis=1)
    Y = phase_three(W, b, dir)
    return {"A_tilde": A_t, "W": W, "slabs": out, "Y": Y, "m1": m1, "m2": m2}


def balance_counts(N1: int, N2: int, b: int, p: int, plant: str | None = None) -> np.ndarray:
    """counts[q, q'] = number of items that PARA-CO-DRP sends from processor q
    to processor q' AND that belong on that route by their own coordinates.

    Every item is labelled with its Phase-I position (a, c).  Its source is
    the input owner of column c, q = floor(c / (N2/p)) (Sect. 2, input
    ownership), and its destination is the owner of the output column it
    feeds, k1 = pi_m1(a) (the frequency that physical row a holds after
    Phase I, Lemma 1), q' = floor(pi_m1(a) / (N1/p)) (Eq. (3)).  The
    procedure runs on the labels and every label found in a block it sends
    from q to q' is counted only if its coordinates give that same (q, q').
    Theorem 4 then fixes counts == N/p^2 everywhere; a misrouted item lowers
    some count.  Raises if a label is sent twice or never."""
    import oracle
    N = N1 * N2
    labels = np.arange(N, dtype=np.int64).reshape(N1, N2)   # label = a*N2 + c
    trace = {}
    w1, w2 = N1 // p, N2 // p
    slabs = [labels[:, q * w2:(q + 1) * w2] for q in range(p)]
    para_co_drp(slabs, N1, N2, b, p, twiddle=False, trace=trace, plant=plant)
    pi1 = oracle.digit_reverse_table(b, log_b(N1, b))
    counts = np.zeros((p, p), dtype=np.int64)
    seen = np.zeros(N, dtype=np.int64)
    for (q, qd), blk in trace["sent"].items():
        lab = np.asarray(blk, dtype=np.int64).ravel()
        np.add.at(seen, lab, 1)
        a, c = lab // N2, lab % N2
        ok = (c // w2 == q) & (pi1[a] // w1 == qd)
        counts[q, qd] += int(np.count_nonzero(ok))
    if not np.all(seen == 1):
        raise AssertionError("an item was sent more than once or never")
    return counts

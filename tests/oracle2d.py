"""The 2-D and 3-D DFTs from the oracle's 1-D DFT (test infrastructure).
For every N1 x N2 array X (row-major rows of x), out[k2][k1] = sum_{j1, j2}
X[j1][j2] w_N1^{dir k1 j1} w_N2^{dir k2 j2} -- the layout a dims = 2 plan
returns (transposed); for every N1 x N2 x N3 array, out[k3][k2][k1] -- the
layout a dims = 3 plan returns (axes reversed).  The 1-D oracle applied
along one axis at a time; pinned against numpy's fft2 / fftn in
tests/test_oracle_dft.py."""

import numpy as np

import oracle


def fft2_transposed(x, N1, N2, dir=-1):
    X = np.asarray(x, dtype=np.complex128).reshape(-1, N1, N2)
    out = []
    for Xi in X:
        At = oracle.fft(np.ascontiguousarray(Xi.T), dir)     # [j2][k1]: DFTs over j1
        Y2 = oracle.fft(np.ascontiguousarray(At.T), dir)     # [k1][k2]: DFTs over j2
        out.append(np.ascontiguousarray(Y2.T).reshape(-1))   # [k2][k1]
    return np.stack(out)


def _along_last(A, dir):
    """The oracle's 1-D DFT of every row (last axis) of A."""
    n = A.shape[-1]
    flat = np.ascontiguousarray(A).reshape(-1, n)
    return oracle.fft(flat, dir).reshape(A.shape)


def fft3_reversed(x, N1, N2, N3, dir=-1):
    X = np.asarray(x, dtype=np.complex128).reshape(-1, N1, N2, N3)
    out = []
    for Xi in X:
        A = _along_last(Xi, dir)                                          # [j1][j2][k3]
        A = _along_last(np.ascontiguousarray(A.transpose(0, 2, 1)), dir)  # [j1][k3][k2]
        A = _along_last(np.ascontiguousarray(A.transpose(1, 2, 0)), dir)  # [k3][k2][k1]
        out.append(A.reshape(-1))
    return np.stack(out)

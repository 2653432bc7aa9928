"""The 2-D DFT from the oracle's 1-D DFT (test infrastructure): for every
N1 x N2 array X (row-major rows of x), out[k2][k1] = sum_{j1, j2}
X[j1][j2] w_N1^{dir k1 j1} w_N2^{dir k2 j2} -- the layout a dims = 2 plan
returns (transposed).  The 1-D oracle applied down the columns, then along
the rows; pinned against numpy's fft2 in tests/test_oracle_dft.py."""

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

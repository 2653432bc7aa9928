"""Plain NumPy statement of the sharded form's per-rank stages, in the
buffer layouts that include/paco.h fixes for paco_shard_stage1 / stage2
(test infrastructure: it shares no code with the CUDA path).

x_local [batch][N1][Cl]; send, recv [G][batch][Cl][K1]; y_local [batch][N2][K1]
(Cl = N2/G, K1 = N1/G).  Local DFTs are the oracle's FFT; the top-level
twiddle is w_N^{-k1 c} at the global column c (Eq. two-factor-ct); block
rows are in the order of the digit reversal of the local column (Eq. (17)
with c = g Cl + c_l)."""

import numpy as np

import oracle


def _rev(b, n):
    """Digit reversal table over the base-b digits of [n]."""
    t = {2: 1, 4: 2, 8: 3, 16: 4}[b]
    m = int(round(np.log2(n))) // t
    return np.asarray(oracle.digit_reverse_table(b, m)) if m > 0 else np.zeros(1, dtype=np.int64)


def stage1(x_local, rank, G, N1, N2, b, dir=-1):
    """Phase I of rank `rank`'s input slab, packed into its G send blocks."""
    Cl, K1, N = N2 // G, N1 // G, N1 * N2
    x = np.asarray(x_local, dtype=np.complex128).reshape(-1, N1, Cl)
    batch = x.shape[0]
    # column DFTs of length N1 (over j1), one per local column
    cols = np.transpose(x, (0, 2, 1)).reshape(-1, N1)
    A = oracle.fft(np.ascontiguousarray(cols), dir).reshape(batch, Cl, N1)      # A[b][c_l][k1]
    c = rank * Cl + np.arange(Cl)
    k1 = np.arange(N1)
    Z = A * np.exp(dir * 2j * np.pi * ((np.outer(c, k1) % N) / N))[None]        # w_N^{-k1 c} for dir = -1
    pi = _rev(b, Cl)
    send = np.zeros((G, batch, Cl, K1), complex)
    for q in range(G):
        send[q][:, pi, :] = Z[:, :, q * K1:(q + 1) * K1]                        # row pi(c_l) <- column c_l
    return send


def stage2(recv, rank, G, N1, N2, b, dir=-1):
    """Phase III of rank `rank`'s output columns from its received blocks."""
    Cl, K1 = N2 // G, N1 // G
    r = np.asarray(recv, dtype=np.complex128).reshape(G, -1, Cl, K1)
    batch = r.shape[1]
    pi = _rev(b, Cl)
    # u[b][j][v] = W row pi_m2(j) = row pi(j_l) of the block from rank j_h
    u = np.concatenate([r[jh][:, pi, :] for jh in range(G)], axis=1)          # [batch][N2][K1]
    cols = np.transpose(u, (0, 2, 1)).reshape(-1, N2)
    y = oracle.fft(np.ascontiguousarray(cols), dir).reshape(batch, K1, N2)
    return np.transpose(y, (0, 2, 1))                                           # [batch][N2][K1]


def assemble(y_locals, G, N1, N2):
    """y (batch x N) from the G ranks' output slabs: Y[k2][g K1 + v]."""
    K1 = N1 // G
    batch = np.asarray(y_locals[0]).reshape(-1, N2, K1).shape[0]
    Y = np.zeros((batch, N2, N1), complex)
    for g, yl in enumerate(y_locals):
        Y[:, :, g * K1:(g + 1) * K1] = np.asarray(yl).reshape(batch, N2, K1)
    return Y.reshape(batch, N1 * N2)                                            # y[k1 + k2 N1] = Y[k2][k1]


def slab(x, rank, G, N1, N2):
    """Rank `rank`'s input slab [batch][N1][Cl] of x (batch x N)."""
    Cl = N2 // G
    return np.ascontiguousarray(np.asarray(x).reshape(-1, N1, N2)[:, :, rank * Cl:(rank + 1) * Cl])

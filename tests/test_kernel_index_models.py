"""CPU models of two kernels' index arithmetic, checked before any GPU run
and kept as regression tests (no GPU, no CUDA code):

* the uneven-batch kernel's shared-memory path for whole transforms
  (N <= 2^13): every shared-memory position written and read by the Phase I
  passes, the fused digit-reversal store W[pi_m2(c)][k1] with its XOR column
  swizzle, and the Phase III passes is in bounds, each pass's writes are a
  bijection, and the result is the DFT (numpy FFT as the reference);
* the tensor-core radix-16 contraction's fragment mapping (PTX m16n8k16
  register layouts for A, B and the accumulator): assembling the 32 x 32 real
  DFT matrix from the per-lane fragments and contracting gives the
  16-point DFT of every lane's sequence."""

import numpy as np
import pytest


def drev(u, bits, t):
    """base-2^t digit reversal of a bits-bit integer (plain digit arrays)."""
    digits = [(u >> (t * i)) & ((1 << t) - 1) for i in range(bits // t)]
    out = 0
    for d in digits:
        out = (out << t) | d
    return out


def small_group_model(LG1, LG2, t, xs):
    N1, N2 = 1 << LG1, 1 << LG2
    N = N1 * N2
    G = 8192 // N
    R1 = min(N1, 16); R2 = N1 // R1; Q1 = min(N2, 16); Q2 = N2 // Q1
    LR1, LR2, LQ1, LQ2 = (int(np.log2(v)) for v in (R1, R2, Q1, Q2))
    HM = min(N1, 32) - 1
    NT = 512
    tw = np.exp(-2j * np.pi * np.arange(N) / N)
    gcount = len(xs)
    S = np.full(8192, np.nan, dtype=complex)
    for g in range(gcount):
        S[g * N:(g + 1) * N] = xs[g]
    out = [np.full(N, np.nan, dtype=complex) for _ in range(gcount)]
    regs = {}
    written = np.zeros(8192, int)
    # Phase I pass a
    for tid in range(NT):
        vs = []
        for q in range(16 // R1):
            u = tid + NT * q
            c = u & (N2 - 1); jl = (u >> LG2) & (R2 - 1); g = u >> (LG2 + LR2)
            base = g * N + jl * N2 + c
            idx = [base + r * R2 * N2 for r in range(R1)]
            assert all(0 <= i < 8192 for i in idx)
            y = np.fft.fft(S[idx])
            if R2 > 1:
                y = y * tw[(np.arange(R1) * jl * N2) % N]
                for s_ in range(R1):
                    S[base + s_ * R2 * N2] = y[s_]
                    written[base + s_ * R2 * N2] += 1
            vs.append(y)
        regs[tid] = vs
    if R2 > 1:
        assert (written == 1).all()
        for tid in range(NT):
            vs = []
            for q in range(16 // R2):
                u = tid + NT * q
                c = u & (N2 - 1); kl = (u >> LG2) & (R1 - 1); g = u >> (LG2 + LR1)
                base = g * N + kl * R2 * N2 + c
                vs.append(np.fft.fft(S[[base + r * N2 for r in range(R2)]]))
            regs[tid] = vs
    # top-level twiddle + fused digit reversal into the swizzled W
    W = np.full(8192, np.nan, dtype=complex)
    cnt = np.zeros(8192, int)
    NUf = 16 // R2 if R2 > 1 else 16 // R1
    RF = R2 if R2 > 1 else R1
    for tid in range(NT):
        for q in range(NUf):
            u = tid + NT * q
            c = u & (N2 - 1)
            kl = ((u >> LG2) & (R1 - 1)) if R2 > 1 else 0
            g = (u >> (LG2 + LR1)) if R2 > 1 else (u >> LG2)
            urow = drev(c, LG2, t)
            assert drev(urow, LG2, t) == c
            for k in range(RF):
                k1 = (kl + R1 * k) if R2 > 1 else k
                pos = g * N + urow * N1 + (k1 ^ (c & HM))
                W[pos] = regs[tid][q][k] * tw[k1 * c]
                cnt[pos] += 1
    assert (cnt == 1).all()
    # Phase III
    written[:] = 0
    for tid in range(NT):
        for q in range(16 // Q1):
            u = tid + NT * q
            col = u & (N1 - 1); jl = (u >> LG1) & (Q2 - 1); g = u >> (LG1 + LQ2)
            pos = [g * N + drev(r * Q2 + jl, LG2, t) * N1 + (col ^ ((r * Q2 + jl) & HM)) for r in range(Q1)]
            y = np.fft.fft(W[pos])
            if Q2 > 1:
                y = y * tw[(np.arange(Q1) * jl * N1) % N]
                for s_ in range(Q1):
                    W[pos[s_]] = y[s_]
                    written[pos[s_]] += 1
            elif g < gcount:
                for s_ in range(Q1):
                    out[g][s_ * N1 + col] = y[s_]
    if Q2 > 1:
        assert (written == 1).all()
        for tid in range(NT):
            for q in range(16 // Q2):
                u = tid + NT * q
                col = u & (N1 - 1); kl = (u >> LG1) & (Q1 - 1); g = u >> (LG1 + LQ1)
                pos = [g * N + drev(kl * Q2 + r, LG2, t) * N1 + (col ^ ((kl * Q2 + r) & HM)) for r in range(Q2)]
                y = np.fft.fft(W[pos])
                if g < gcount:
                    for k in range(Q2):
                        out[g][(kl + Q1 * k) * N1 + col] = y[k]
    return out


@pytest.mark.parametrize("lg,t", [(4, 2), (5, 1), (8, 4), (9, 1), (12, 2), (12, 3), (13, 1)])
def test_small_group_index_maps_compute_the_dft(lg, t):
    LG1, LG2 = (lg + 1) // 2, lg // 2
    rng = np.random.default_rng(lg)
    G = 8192 >> lg
    xs = [rng.standard_normal(1 << lg) + 1j * rng.standard_normal(1 << lg) for _ in range(max(1, G - 1))]
    for x, y in zip(xs, small_group_model(LG1, LG2, t, xs)):
        assert np.allclose(y, np.fft.fft(x))


def _dft_matrix_entry(m, kk):
    k, j = m & 15, kk & 15
    c, s = np.cos(2 * np.pi * ((k * j) & 15) / 16), np.sin(2 * np.pi * ((k * j) & 15) / 16)
    if m < 16 and kk < 16:
        return c
    if m < 16:
        return s
    if kk < 16:
        return -s
    return c


def test_tensor_core_fragment_mapping():
    # A fragment: reg r holds rows g + 8 (r & 1), columns 2 q + 8 (r >> 1) + h;
    # B fragment: reg r holds k = 2 q + 8 r + h, column n = g;
    # accumulator: c0, c1 at (g, 2q + {0,1}), c2, c3 at (g + 8, 2q + {0,1}).
    rng = np.random.default_rng(0)
    V = rng.standard_normal((32, 16)) + 1j * rng.standard_normal((32, 16))
    X = np.concatenate([V.real.T, V.imag.T])                 # 32 (k) x 32 (n)
    acc = np.zeros((4, 2, 32, 4))
    for nt in range(4):
        for mt in range(2):
            for ks in range(2):
                A = np.zeros((16, 16)); B = np.zeros((16, 8))
                for lane in range(32):
                    g, q = lane >> 2, lane & 3
                    for r in range(4):
                        for h in range(2):
                            m = 16 * mt + g + 8 * (r & 1)
                            kk = 16 * ks + 2 * q + 8 * (r >> 1) + h
                            A[g + 8 * (r & 1), 2 * q + 8 * (r >> 1) + h] = _dft_matrix_entry(m, kk)
                    for r in range(2):
                        for h in range(2):
                            B[2 * q + 8 * r + h, g] = X[16 * ks + 2 * q + 8 * r + h, 8 * nt + g]
                D = A @ B
                for lane in range(32):
                    g, q = lane >> 2, lane & 3
                    acc[nt, mt, lane] += [D[g, 2 * q], D[g, 2 * q + 1], D[g + 8, 2 * q], D[g + 8, 2 * q + 1]]
    # each lane's outputs: frequencies s = g + 8 si of sequences n = 8 nt + 2 q + h
    Y = np.full((32, 16), np.nan, dtype=complex)
    for lane in range(32):
        g, q = lane >> 2, lane & 3
        for nt in range(4):
            for h in range(2):
                for si in range(2):
                    n = 8 * nt + 2 * q + h
                    Y[n, g + 8 * si] = acc[nt, 0, lane, h + 2 * si] + 1j * acc[nt, 1, lane, h + 2 * si]
    assert np.allclose(Y, np.fft.fft(V, axis=1))

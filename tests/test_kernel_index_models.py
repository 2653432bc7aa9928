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


# ---------------------------------------------------------------------------
# The 2^14 panel pipeline (paco_panel.cuh): one tile of each kind
# ---------------------------------------------------------------------------

def _swz(addr):
    """TMA 128-byte swizzle of a byte offset inside a 1024-aligned buffer:
    the 16-byte chunk index (bits 4-6) is XORed with the row index mod 8
    (bits 7-9)."""
    return addr ^ (((addr >> 7) & 7) << 4)


def _tma_box(box_dims, coord_to_global):
    """Yield (smem byte offset, global index) of every element of a box, the
    first dimension fastest (8-byte elements, 128-byte swizzle)."""
    idx = np.indices(box_dims[::-1]).reshape(len(box_dims), -1)[::-1]   # idx[0] fastest
    lin = np.zeros(idx.shape[1], dtype=np.int64)
    mul = 1
    for k, d in enumerate(box_dims):
        lin += idx[k] * mul
        mul *= d
    return _swz(lin * 8), coord_to_global(*idx)


def land_lo(b, t8):
    return (((t8 & 1) << 2) | (t8 & 2) | ((t8 >> 2) & 1)) if b == 2 else t8


def land_hi(b, s):
    if b == 2:
        return ((s & 1) << 3) | ((s & 2) << 1) | ((s >> 1) & 2) | ((s >> 3) & 1)
    if b == 4:
        return ((s & 3) << 2) | ((s >> 2) & 3)
    return s


NBOX = 2            # TMA boxes (16 sequences x 128 points) per tile
WPG = 8             # consumer warps per tile (one group)


def _lane(warp, lane):
    """(q, column, chunk, half, box byte offset) of lane `lane` of consumer
    warp `warp` (0..7 within its group)."""
    q = lane & 7
    col = 4 * (warp & 3) + (lane >> 3)
    cc, half = col >> 1, col & 1
    return q, col, cc, half, (warp >> 2) * 16384 + half * 8


def _consume(smem, kind, b, conj, TW=None, E1=None, E2=None):
    """The consumer warps of paco_panel_kernel on one landed tile, with the
    kernel's address formulas.  `smem` is the 32 KiB stage buffer as 4096
    complex slots (byte offset / 8).  Returns the per-lane outputs for the
    stage-1 A 16-byte stores as {(warp, lane, k8): (y_h0, y_h1)} and writes the
    in-place store image into smem for the other kinds."""
    w128 = np.exp(-2j * np.pi * np.arange(128) / 128)
    paired = (kind == "1A")
    stores = {}
    reads, writes = set(), set()
    new = {}
    for warp in range(WPG):
        for lane in range(32):
            q, col, cc, half, box = _lane(warp, lane)
            stage2A = (kind == "2A")
            lo = land_lo(b, q) if stage2A else q
            base = box + (lo << 7) + ((cc ^ lo) << 4)
            v = np.array([smem[(base + (land_hi(b, s) if stage2A else s) * 1024) // 8] for s in range(16)])
            for s in range(16):
                reads.add(base + (land_hi(b, s) if stage2A else s) * 1024)
            if kind in ("1A", "2A") and conj:
                v = np.conj(v)
            v = np.fft.fft(v)
            v = v * w128[(np.arange(16) * q) % 128]
            e0 = box + (q << 7) + ((cc ^ q) << 4)
            for k in range(16):
                m = (k >> 1) if paired else (k & 7)
                a = (e0 ^ (m * 0x90)) + k * 1024
                writes.add(a)
                new.setdefault(("x", a), v[k])
            stores[(warp, lane)] = e0
    # exchange: every lane of a warp writes before any lane reads (__syncwarp)
    assert len(writes) == WPG * 32 * 16 and writes == reads    # in place, bijective
    for (_, a), val in new.items():
        smem[a // 8] = val
    out = {}
    images = {}
    kb0 = lambda q: 2 * q if paired else q
    kbs = 1 if paired else 8
    for warp in range(WPG):
        for lane in range(32):
            e0 = stores[(warp, lane)]
            q, col, cc, half, box = _lane(warp, lane)
            rb = e0 + (q * 2048 if paired else q * 1024)
            hs = 1024 if paired else 8192
            res = np.zeros(16, complex)
            for h in range(2):
                xs = np.array([smem[((rb ^ (t * 0x90)) + h * hs) // 8] for t in range(8)])
                res[8 * h:8 * h + 8] = np.fft.fft(xs)
            k = np.array([kb0(q) + kbs * h + 16 * k8 for h in range(2) for k8 in range(8)])
            if kind in ("1A", "2A"):
                res = res * TW[k]
            elif kind == "1B":
                res = res * E1[16 * (warp >> 2) + col] * E2[k]
            if kind in ("1B", "2B") and conj:
                res = np.conj(res)
            if paired:
                for k8 in range(8):
                    out[(warp, lane, k8)] = (res[k8], res[8 + k8])
            else:
                ob = box + (q << 7) + ((cc ^ q) << 4)
                for h in range(2):
                    for k8 in range(8):
                        a = ob + h * 1024 + k8 * 2048
                        assert (a % 16384) // 128 == k[8 * h + k8]   # image row = output index
                        images[a] = res[8 * h + k8]
    if not paired:
        assert len(images) == 4096
        for a, val in images.items():
            smem[a // 8] = val
    return out


@pytest.mark.parametrize("conj", [False, True])
def test_panel_stage1_tiles_model(conj):
    """Stage 1 (N1 = 2^14 rows, C = 256 columns, P = 128): an A tile (TMA
    box (16 c, 1 j_lo, 128 j_hi)) through the consumers to the panel buffer
    [c][j_lo][k_lo] (16-byte stores), then a B tile of that panel buffer
    (box (16 k_lo, 128 j_lo, 1 c)) to W's row pi(c) (box (16 k_lo, 128 k_hi)):
    every value lands where the two-factor DFT, the twiddle w_L^{-k_lo j_lo}
    and the epilogue w_N^{-k1 c} put it."""
    rng = np.random.default_rng(1)
    L, C, P = 16384, 256, 128
    N = L * C
    X = rng.standard_normal((L, C)) + 1j * rng.standard_normal((L, C))
    wL = np.exp(-2j * np.pi * np.arange(L) / L)
    q_panel, slot = 1, 1
    colbase = q_panel * P
    # --- A tile t: j_lo = t >> 2, columns c0 = 32 (t & 3)
    t = 77
    jlo, c0 = t >> 2, 32 * (t & 3)
    smem = np.full(4096, np.nan, complex)
    for x in range(NBOX):
        offs, (cg, jl, jh) = _tma_box((16, 1, 128), lambda a, bb, c: (colbase + c0 + 16 * x + a, jlo + bb, c))
        smem[(x * 16384 + offs) // 8] = X[jl + 128 * jh, cg]
    TW = wL[(np.arange(128) * jlo) % L]
    out = _consume(smem, "1A", 2, conj, TW=TW)
    scratch = {}
    for (warp, lane, k8), (y0, y1) in out.items():
        q, col, _, _, _ = _lane(warp, lane)
        cl = c0 + 16 * (warp >> 2) + col
        base = ((slot * P + cl) * 128 + jlo) * 128 + 2 * q + 16 * k8
        scratch[base] = y0
        scratch[base + 1] = y1
    # dir = +1 conjugates on the A tile's load and on the B tile's store:
    # between the two the panel buffer holds the forward transform of conj(x)
    xc = np.conj(X) if conj else X
    for cl in range(c0, c0 + 32):
        seq = xc[jlo + 128 * np.arange(128), colbase + cl]
        want = np.fft.fft(seq) * TW
        got = np.array([scratch[((slot * P + cl) * 128 + jlo) * 128 + k] for k in range(128)])
        assert np.allclose(got, want)
    # --- B tile: column cl, k0 = 32 (t & 3); its panel buffer filled with the true A results
    cl, k0 = 93, 64
    cglob = colbase + cl
    Acol = np.array([np.fft.fft(xc[jl + 128 * np.arange(128), cglob]) * wL[(np.arange(128) * jl) % L]
                     for jl in range(128)])                    # [j_lo][k_lo]
    smem = np.full(4096, np.nan, complex)
    for x in range(NBOX):
        offs, (kl, jl, c) = _tma_box((16, 128, 1), lambda a, bb, c: (k0 + 16 * x + a, bb, c))
        smem[(x * 16384 + offs) // 8] = Acol[jl, kl]
    E1 = np.exp(-2j * np.pi * (((k0 + np.arange(32)) * cglob) % N) / N)
    E2 = np.exp(-2j * np.pi * ((128 * np.arange(128) * cglob) % N) / N)
    _consume(smem, "1B", 2, conj, E1=E1, E2=E2)
    Wrow = {}
    for x in range(NBOX):
        offs, (kl, kh, _) = _tma_box((16, 128, 1), lambda a, bb, c: (k0 + 16 * x + a, bb, c))
        for o, a_, b_ in zip(offs, kl, kh):
            Wrow[a_ + 128 * b_] = smem[(x * 16384 + o) // 8]
    # Z[k1, c] = A[k1, c] w_N^{-k1 c} for the 32 k_lo of the tile, all k_hi
    # (for dir = +1: the conjugate of that product formed on conj(x))
    full = np.fft.fft(xc[:, cglob])
    assert len(Wrow) == 32 * 128
    for k1, got in Wrow.items():
        want = full[k1] * np.exp(-2j * np.pi * ((k1 * cglob) % N) / N)
        if conj:
            want = np.conj(want)
        assert abs(got - want) < 1e-9 * np.sqrt(L) * 10, (k1, got, want)


@pytest.mark.parametrize("b", [2, 4])
@pytest.mark.parametrize("conj", [False, True])
def test_panel_stage2_tiles_model(b, conj):
    """Stage 2 (W with N2 = 2^14 rows, C = 128 columns, P = 128): an A tile
    loads rows pi(j_lo + 128 j_hi) through the tensor map whose row dimensions
    are ordered as in panel_prepare (b = 2: rank 4; b = 4: rank 5 plus the
    second map for row bit 6) -- the landing order the consumers assume
    (land_lo, land_hi) must give logical j_hi = t8 + 8 s in v[s] -- and is
    stored to the panel buffer [k_lo][j_lo][v]; a B tile of that buffer is
    stored to Y (box (16 v, 1 k_lo, 128 k_hi)).  Values must land where the
    length-2^14 DFT over the digit-reversed rows puts them."""
    import oracle
    rng = np.random.default_rng(2)
    L, C, P = 16384, 128, 128
    t = 2 if b == 4 else 1
    pi = oracle.digit_reverse_table(b, 14 // t)
    W = rng.standard_normal((L, C)) + 1j * rng.standard_normal((L, C))
    wL = np.exp(-2j * np.pi * np.arange(L) / L)
    # --- A tile: j_lo, 64 columns v0
    for jlo in (0, 37, 64 + 5):
        v0 = 96
        u = int(pi[jlo])
        smem = np.full(4096, np.nan, complex)
        for x in range(NBOX):
            if b == 2:
                f = lambda vv, d1, d2, d3: (v0 + 16 * x + vv, d1 * 16 + d2 + 128 * (d3 + (u >> 7)))
                offs, (vg, row) = _tma_box((16, 8, 16, 1), f)
            else:
                base_row = 64 if (u >> 6) & 1 else 0
                f = lambda vv, d1, d2, d3, d4: (v0 + 16 * x + vv,
                                                base_row + 128 * d1 + 16 * d2 + d3 + 256 * (d4 + (u >> 8)))
                offs, (vg, row) = _tma_box((16, 2, 4, 16, 1), f)
            smem[(x * 16384 + offs) // 8] = W[row, vg]
        TW = wL[(np.arange(128) * jlo) % L]
        _consume(smem, "2A", b, conj, TW=TW)
        for x in range(NBOX):
            offs, (vv, jl, kl) = _tma_box((16, 1, 128), lambda a, bb, c: (v0 + 16 * x + a, jlo + bb, c))
            for o, vg, k in zip(offs, vv, kl):
                seq = W[pi[jlo + 128 * np.arange(128)], vg]
                want = np.fft.fft(np.conj(seq) if conj else seq)[k] * TW[k]
                assert abs(smem[(x * 16384 + o) // 8] - want) < 1e-9, (jlo, vg, k)
    # --- B tile: k_lo, 64 columns v0 over a panel buffer [k_lo][j_lo][v]
    klo, v0 = 21, 32
    logical = W[pi, :]                                     # logical rows j
    lc = np.conj(logical) if conj else logical             # dir = +1: conjugated on the A load
    Aall = np.empty((128, 128, C), complex)                # [k_lo][j_lo][v]
    for jl in range(128):
        seqs = lc[jl + 128 * np.arange(128), :]            # (j_hi, v)
        Aall[:, jl, :] = np.fft.fft(seqs, axis=0) * wL[(np.arange(128) * jl) % L][:, None]
    smem = np.full(4096, np.nan, complex)
    for x in range(NBOX):
        offs, (vv, jl, kl) = _tma_box((16, 128, 1), lambda a, bb, c: (v0 + 16 * x + a, bb, klo + c))
        smem[(x * 16384 + offs) // 8] = Aall[kl, jl, vv]
    _consume(smem, "2B", b, conj)
    Yfull = np.fft.fft(lc, axis=0)
    if conj:
        Yfull = np.conj(Yfull)
    for x in range(NBOX):
        offs, (vv, kl, kh) = _tma_box((16, 1, 128), lambda a, bb, c: (v0 + 16 * x + a, klo + bb, c))
        for o, vg, k_lo, k_hi in zip(offs, vv, kl, kh):
            want = Yfull[k_lo + 128 * k_hi, vg]
            assert abs(smem[(x * 16384 + o) // 8] - want) < 1e-9 * 128, (vg, k_lo, k_hi)


def test_panel_shared_accesses_are_conflict_free():
    """Every shared-memory access instruction of a consumer warp (landing
    reads for each tile kind and b, both sides of the exchange in its paired
    and staged forms, the store image) is served without bank conflicts: an
    8-byte access is served per half-warp, and each half-warp's 16 lanes must
    touch each of the 32 four-byte banks exactly once."""
    def conflict_free(addrs):
        for hw in (addrs[:16], addrs[16:]):
            cnt = np.zeros(32, int)
            for a in hw:
                for w in range(2):
                    cnt[((a + 4 * w) // 4) % 32] += 1
            if cnt.max() != 1:
                return False
        return True

    def lanes(f):
        return [f(*_lane(warp, lane)) for lane in range(32)]

    for warp in range(WPG):
        for kind, b in (("A1", 2), ("A2", 2), ("A2", 4), ("B", 2)):
            for s in range(16):
                def f(q, col, cc, half, box, s=s):
                    lo = land_lo(b, q) if kind == "A2" else q
                    hs = land_hi(b, s) if kind == "A2" else s
                    return box + (lo << 7) + ((cc ^ lo) << 4) + hs * 1024
                assert conflict_free(lanes(f)), (kind, b, s)
        for paired in (True, False):
            for k in range(16):
                m = (k >> 1) if paired else (k & 7)
                assert conflict_free(lanes(lambda q, col, cc, half, box:
                                           ((box + (q << 7) + ((cc ^ q) << 4)) ^ (m * 0x90)) + k * 1024))
            for h in range(2):
                for tt in range(8):
                    def f(q, col, cc, half, box):
                        e0 = box + (q << 7) + ((cc ^ q) << 4)
                        rb = e0 + (q * 2048 if paired else q * 1024)
                        return (rb ^ (tt * 0x90)) + h * (1024 if paired else 8192)
                    assert conflict_free(lanes(f)), (paired, h, tt)
        for h in range(2):
            for k8 in range(8):
                assert conflict_free(lanes(lambda q, col, cc, half, box:
                                           box + (q << 7) + ((cc ^ q) << 4) + h * 1024 + k8 * 2048))


# ---------------------------------------------------------------------------
# The one-launch cluster form (paco_cluster.cu): N1 = N2 = 256, p = 4 or 8
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("K,p,b", [(16, 4, 2), (16, 8, 2), (16, 4, 4), (8, 4, 2), (8, 8, 2)])
@pytest.mark.parametrize("conj", [False, True])
def test_cluster_kernel_model(K, p, b, conj):
    """Every CTA of a K-CTA cluster with the kernel's index formulas (CTA r
    owns 256/K input and output columns; processor q is CTAs q K/p ..):
    Phase I through the radix 16 x 16 exchange (pass 2 in the t16-fast role),
    the all-to-all into the destination CTAs' swizzled W parts (each slot
    written exactly once, in bounds -- the bytes each CTA's transaction
    barrier expects; N/K^2 items per ordered pair of CTAs and N/p^2 per
    ordered pair of processors), Phase III over the digit-reversed rows, and
    the output positions -- equal to the DFT.  Every shared-memory access
    pattern is checked for half-warp bank conflicts."""
    import oracle
    L, N = 256, 65536
    t = {2: 1, 4: 2, 16: 4}[b]
    pi = oracle.digit_reverse_table(b, 8 // t)
    W1 = W2 = L // K
    nt = N // K // 16
    rng = np.random.default_rng(K + p + b)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    w256 = np.exp(-2j * np.pi * np.arange(256) / 256)
    wN = lambda r: np.exp(-2j * np.pi * (r % N) / N)
    sw = lambda row: row >> 4

    def banks_ok(addrs):
        """16 lanes of a half-warp, 8-byte words: 16 different banks."""
        return len({a_ % 16 for a_ in addrs}) == 16

    def dft256_cols(vals, W, t16_fast):
        """vals[tid] = the 16 pass-1 inputs of thread tid (col = tid % W,
        t16 = tid // W); returns (outs, roles): outs[tid] = outputs u + 16 k
        of column col2, roles[tid] = (col2, u)."""
        buf = np.full(256 * W, np.nan, complex)
        for tid in range(nt):
            col, t16 = tid % W, tid // W
            v = np.fft.fft(vals[tid]) * w256[(np.arange(16) * t16) % 256]
            for s in range(16):
                i = (s * 16 + t16) * W + (col ^ s)
                assert np.isnan(buf[i])
                buf[i] = v[s]
        role = (lambda tid: (tid // 16, tid % 16)) if t16_fast else (lambda tid: (tid % W, tid // W))
        for hw in range(0, nt, 16):
            for s in range(16):
                assert banks_ok([(s * 16 + tid // W) * W + ((tid % W) ^ s) for tid in range(hw, hw + 16)])
            for tt in range(16):
                assert banks_ok([(role(tid)[1] * 16 + tt) * W + (role(tid)[0] ^ role(tid)[1])
                                 for tid in range(hw, hw + 16)])
        outs = []
        for tid in range(nt):
            col2, u = role(tid)
            outs.append(np.fft.fft(np.array([buf[(u * 16 + tt) * W + (col2 ^ u)] for tt in range(16)])))
        return outs, [role(tid) for tid in range(nt)]

    xin = np.conj(x) if conj else x
    X = xin.reshape(L, L)
    parts = [np.full(N // K, np.nan, complex) for _ in range(K)]
    sent = np.zeros((K, K), int)
    for r in range(K):
        vals = [np.array([X[(tid // W1) + 16 * s, r * W1 + tid % W1] for s in range(16)]) for tid in range(nt)]
        outs, roles = dft256_cols(vals, W1, True)
        for k in range(16):                                   # exchange stores, per half-warp
            for hw in range(0, nt, 16):
                addrs = []
                for tid in range(hw, hw + 16):
                    colB, tB = roles[tid]
                    row = int(pi[r * W1 + colB])
                    vf = tB + 16 * k
                    addrs.append(row * W2 + ((vf % W2) ^ sw(row)))
                assert banks_ok(addrs)
        for tid in range(nt):
            colB, tB = roles[tid]
            c = r * W1 + colB
            row = int(pi[c])
            for k in range(16):
                vf = tB + 16 * k
                z = outs[tid][k] * wN(vf * c)
                rd, vl = vf // W2, vf % W2
                idx = row * W2 + (vl ^ sw(row))
                assert 0 <= idx < N // K and np.isnan(parts[rd][idx])
                parts[rd][idx] = z
                sent[r, rd] += 1
    assert np.all(sent == N // (K * K))
    g = K // p
    per_proc = sent.reshape(p, g, p, g).sum(axis=(1, 3))
    assert np.all(per_proc == N // (p * p))
    y = np.full(N, np.nan, complex)
    for r in range(K):
        assert not np.isnan(parts[r]).any()                   # every byte the barrier expects landed
        for hw in range(0, nt, 16):
            for s_ in range(16):
                assert banks_ok([int(pi[tid // W2 + 16 * s_]) * W2 + ((tid % W2) ^ sw(int(pi[tid // W2 + 16 * s_])))
                                 for tid in range(hw, hw + 16)])
        vals = []
        for tid in range(nt):
            vl, u16 = tid % W2, tid // W2
            rows = [int(pi[u16 + 16 * s]) for s in range(16)]
            vals.append(np.array([parts[r][rr * W2 + (vl ^ sw(rr))] for rr in rows]))
        outs, roles = dft256_cols(vals, W2, False)
        for tid in range(nt):
            vl, u16 = roles[tid]
            for k in range(16):
                k2 = u16 + 16 * k
                y[k2 * L + r * W2 + vl] = np.conj(outs[tid][k]) if conj else outs[tid][k]
    want = np.fft.fft(x) if not conj else np.fft.ifft(x) * N
    assert np.allclose(y, want, atol=1e-8 * np.sqrt(N))


# ---- the tcgen05 probe: operand layout vs the MMA descriptor's addressing ---

def _sw128_off(r, k, R):
    """The kernel's byte offset of element (row r, k) of a K-major bf16
    operand with K = 128 in the 128-byte swizzle layout."""
    return (k >> 6) * (R * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + ((k & 7) << 1)


def _descriptor_address(start, r, kp):
    """Address the MMA reads for element (r, kp) of one K = 16 step from a
    descriptor with this start, stride byte offset 1024 and the 128-byte
    swizzle: 8-row groups 1024 B apart, rows 128 B apart, then address bits
    [4:6] XOR bits [7:9]."""
    a = start + (r >> 3) * 1024 + (r & 7) * 128 + (kp >> 3) * 16 + (kp & 7) * 2
    return a ^ (((a >> 7) & 7) << 4)


@pytest.mark.parametrize("R", [128, 64, 32])
def test_tc05_operand_layout_matches_descriptors(R):
    """The layout the tcgen05 kernel writes (and the table kernel builds) is
    what its descriptors address: for every K = 16 step kk (start = atom
    (kk / 4) + 32 B (kk mod 4)) and every element, and it is a bijection onto
    the operand's R * 256 bytes."""
    seen = set()
    for r in range(R):
        for k in range(128):
            o = _sw128_off(r, k, R)
            assert 0 <= o < R * 256
            seen.add(o)
    assert len(seen) == R * 128
    for kk in range(8):
        start = (kk >> 2) * (R * 128) + (kk & 3) * 32
        for r in range(R):
            for kp in range(16):
                assert _descriptor_address(start, r, kp) == _sw128_off(r, 16 * kk + kp, R)


# ---- the split stages: the four passes' address maps compose to the DFT ------

def _split_pipeline_model(xin, N1, N2, b, lgLa3=0):
    """Both stages as their two passes with the kernels' formulas: Phase I
    pass A (x viewed [La][Lb C], twiddle w_L^{-k_a j_b}, S[j_b][c][k_a]),
    pass B (S rows j_b, w_N^{-k1 c}, W[pi_m2(c)][k_a + La k_b]), Phase III
    pass A (W row pi(j_a) of block pi(j_b), S[j_b][k_a][v]) and pass B
    (y[k_a + La k_b][v]); every slot written once.  lgLa3 > 0: the 3-D
    form -- Phase III's first pass length La = 2^lgLa3 as given, ones for
    the top-level twiddle and for Phase III's split twiddle."""
    import oracle
    t = {2: 1, 4: 2, 8: 3, 16: 4}[b]
    N = N1 * N2

    def split(L, lgLa=0):
        lgL = L.bit_length() - 1
        if not lgLa:
            lgLa = (lgL + 1) // 2
            while lgLa % t:
                lgLa += 1
        return 1 << lgLa, L >> lgLa

    def rev(u, bits):
        return int(oracle.digit_reverse_table(b, bits // t)[u]) if bits else 0

    def twL(L, r):
        return np.exp(-2j * np.pi * (r % L) / L)

    # Phase I (L = N1 over C = N2 columns)
    L, C = N1, N2
    La, Lb = split(L)
    lgC = C.bit_length() - 1
    S = np.full(N, np.nan, complex)
    X = xin.reshape(L, C)
    for cc in range(Lb * C):                             # view column j_b C + c
        jb, c = cc >> lgC, cc & (C - 1)
        col = np.array([X[ja * Lb + jb, c] for ja in range(La)])   # row j_a of [La][Lb C]
        A = np.fft.fft(col)
        for ka in range(La):
            idx = cc * La + ka
            assert np.isnan(S[idx])
            S[idx] = A[ka] * twL(L, ka * jb)
    W = np.full(N, np.nan, complex)
    lgN2 = lgC
    for cc in range(C * La):                             # view column c La + k_a
        c, ka = cc // La, cc % La
        col = np.array([S[jb * (C * La) + cc] for jb in range(Lb)])
        B = np.fft.fft(col)
        for kb in range(Lb):
            k1 = ka + La * kb
            idx = rev(c, lgN2) * L + k1
            assert np.isnan(W[idx])
            top = 1.0 if lgLa3 else np.exp(-2j * np.pi * ((k1 * c) % N) / N)
            W[idx] = B[kb] * top
    # Phase III (L = N2 over C = N1 columns), W as [N2][N1]
    L, C = N2, N1
    La, Lb = split(L, lgLa3)
    lgC = C.bit_length() - 1
    lgLa, lgLb = La.bit_length() - 1, Lb.bit_length() - 1
    S = np.full(N, np.nan, complex)
    for cc in range(Lb * C):                             # view column j_b C + v
        jb, v = cc >> lgC, cc & (C - 1)
        base = rev(jb, lgLb) * La * C + v
        col = np.array([W[rev(ja, lgLa) * C + base] for ja in range(La)])
        A = np.fft.fft(col)
        for ka in range(La):
            idx = ((jb * La + ka) * C) + v
            assert np.isnan(S[idx])
            S[idx] = A[ka] * (1.0 if lgLa3 else twL(L, ka * jb))
    y = np.full(N, np.nan, complex)
    for cc in range(La * C):                             # view column k_a C + v
        ka, v = cc >> lgC, cc & (C - 1)
        col = np.array([S[jb * (La * C) + cc] for jb in range(Lb)])
        B = np.fft.fft(col)
        for kb in range(Lb):
            idx = (ka + La * kb) * N1 + v
            assert np.isnan(y[idx])
            y[idx] = B[kb]
    return y


@pytest.mark.parametrize("N1,N2,b", [(64, 32, 2), (64, 64, 4), (128, 64, 2), (256, 16, 4)])
@pytest.mark.parametrize("conj", [False, True])
def test_split_stage_address_maps(N1, N2, b, conj):
    """The four passes of the split stages compose to the DFT."""
    N = N1 * N2
    rng = np.random.default_rng(N1 + N2 + b)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = _split_pipeline_model(np.conj(x) if conj else x, N1, N2, b)
    if conj:
        y = np.conj(y)
    want = np.fft.fft(x) if not conj else np.fft.ifft(x) * N
    assert np.allclose(y, want, atol=1e-9 * np.sqrt(N) * np.abs(want).max())


@pytest.mark.parametrize("N1,Na,Nb,b", [(16, 8, 4, 2), (8, 4, 16, 2), (16, 16, 4, 4), (32, 4, 4, 4)])
def test_split_stage_address_maps_3d(N1, Na, Nb, b):
    """The same four passes with the 3-D plan's settings (ones for the
    top-level twiddle and for Phase III's split twiddle, Phase III's first
    pass length the middle axis Na, smaller or larger than Nb) compose to
    the 3-D DFT of the N1 x Na x Nb array with its axes reversed; with the
    default split or with the twiddles left in they do not."""
    N2 = Na * Nb
    N = N1 * N2
    rng = np.random.default_rng(N1 + 3 * Na + 7 * Nb + b)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = _split_pipeline_model(x, N1, N2, b, lgLa3=Na.bit_length() - 1)
    want = np.fft.fftn(x.reshape(N1, Na, Nb)).transpose(2, 1, 0).reshape(-1)
    assert np.allclose(y, want, atol=1e-9 * np.sqrt(N) * np.abs(want).max())
    y1 = _split_pipeline_model(x, N1, N2, b)                 # the 1-D DFT instead
    assert not np.allclose(y1, want, atol=1e-3 * np.abs(want).max())

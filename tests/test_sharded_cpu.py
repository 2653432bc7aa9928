"""The sharded form's host side on the CPU (no GPU).

1. The per-rank stages as plain NumPy statements of the layouts include/paco.h
   fixes (tests/shard_np.py), run for G ranks in one process with the
   exchange done by hand: the assembled output equals the oracle's DFT, and
   every block holds N/G^2 items per transform (Theorem 4).
2. paco.sharded.sharded_fft -- the orchestration the GPU ranks run -- over
   gloo with 2 and 4 real processes, its stage callables replaced by the
   NumPy stages: the all-to-all of equal blocks (torch.distributed
   all_to_all_single) delivers block q of every rank to rank q in sender
   order, and the assembled output equals the oracle's DFT."""

import os
import socket

import numpy as np
import pytest

import oracle
import shard_np
from paco_inputs import gaussian

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("N1,N2,b,G", [(16, 16, 2, 2), (64, 16, 4, 4), (32, 64, 2, 8), (256, 64, 4, 16)])
@pytest.mark.parametrize("dir", [-1, 1])
def test_numpy_stages_give_the_dft(N1, N2, b, G, dir):
    N, batch = N1 * N2, 2
    x = gaussian(batch * N, N1 + G, np.complex128).reshape(batch, N)
    sends = [shard_np.stage1(shard_np.slab(x, g, G, N1, N2), g, G, N1, N2, b, dir) for g in range(G)]
    for s in sends:
        assert s.shape == (G, batch, N2 // G, N1 // G) and s[0, 0].size == N // (G * G)
    recvs = [np.stack([sends[g][q] for g in range(G)]) for q in range(G)]   # block q of rank g -> rank q, slot g
    ys = [shard_np.stage2(recvs[q], q, G, N1, N2, b, dir) for q in range(G)]
    y = shard_np.assemble(ys, G, N1, N2)
    ref = oracle.fft(x, dir)
    assert np.max(np.abs(y - ref)) <= 1e-9 * np.sqrt(N) * np.max(np.abs(ref))


def test_numpy_stages_catch_a_misrouted_block():
    """Swapping two ranks' blocks in the exchange breaks the result: the
    check above can fail."""
    N1, N2, b, G = 16, 16, 2, 2
    x = gaussian(N1 * N2, 3, np.complex128).reshape(1, -1)
    sends = [shard_np.stage1(shard_np.slab(x, g, G, N1, N2), g, G, N1, N2, b) for g in range(G)]
    recvs = [np.stack([sends[G - 1 - g][q] for g in range(G)]) for q in range(G)]
    y = shard_np.assemble([shard_np.stage2(recvs[q], q, G, N1, N2, b) for q in range(G)], G, N1, N2)
    assert np.max(np.abs(y - oracle.fft(x))) > 1e-3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, G, port, N1, N2, b, dir, q):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(G))
    import shard_np as snp
    from paco_inputs import gaussian as gen
    import paper_2609_06449_gb300.sharded as sharded
    dist.init_process_group("gloo")
    try:
        batch = 2
        x = gen(batch * N1 * N2, 50 + G, np.complex128).reshape(batch, -1)
        xl = torch.from_numpy(snp.slab(x, rank, G, N1, N2))
        sizes = []

        def stage1(xs, send, d):
            sizes.append(send.numel())
            send.copy_(torch.from_numpy(snp.stage1(xs.numpy(), rank, G, N1, N2, b, d).reshape(-1)))

        def stage2(recv, yl, d):
            yl.copy_(torch.from_numpy(snp.stage2(recv.numpy(), rank, G, N1, N2, b, d).reshape(-1)))

        y = sharded.sharded_fft(xl, N1, N2, b, dir, stage1=stage1, stage2=stage2)
        q.put((rank, y.numpy().copy(), sizes[0]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("G,N1,N2,b", [(2, 32, 64, 2), (4, 64, 64, 4)])
@pytest.mark.parametrize("dir", [-1, 1])
def test_sharded_fft_orchestration_over_gloo(G, N1, N2, b, dir):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, G, port, N1, N2, b, dir, q)) for r in range(G)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(G):
        r, y, n = q.get(timeout=120)
        got[r] = (y, n)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    N, batch = N1 * N2, 2
    for r in range(G):
        assert got[r][1] == G * batch * N // (G * G)          # G blocks of N/G^2 items per transform
    y = shard_np.assemble([got[r][0] for r in range(G)], G, N1, N2)
    x = gaussian(batch * N, 50 + G, np.complex128).reshape(batch, -1)
    ref = oracle.fft(x, dir)
    assert np.max(np.abs(y - ref)) <= 1e-9 * np.sqrt(N) * np.max(np.abs(ref))


# ---- restoring the input's ownership (the second redistribution) ----------

def _restore_by_maps(y, N1, N2, G, batch):
    """Every rank's pack, the uneven exchange by hand, every rank's unpack,
    with the host maps of paco_shard_restore_maps (numpy data movement)."""
    from paper_2609_06449_gb300.sharded import restore_maps
    K1, Cl = N1 // G, N2 // G
    Y = y.reshape(batch, N2, N1)
    maps = [restore_maps(N1, N2, G, q) for q in range(G)]
    sends = []
    for q in range(G):
        yl = np.ascontiguousarray(Y[:, :, q * K1:(q + 1) * K1]).reshape(batch, -1)
        pack, sc, _, _ = maps[q]
        off = np.concatenate([[0], np.cumsum(sc)])
        sends.append([yl[:, pack[off[r]:off[r + 1]]] for r in range(G)])   # block r: [batch][count]
    outs = []
    for r in range(G):
        _, _, unpack, rc = maps[r]
        off = np.concatenate([[0], np.cumsum(rc)])
        out = np.zeros((batch, N1 * Cl), complex)
        for q in range(G):
            blk = sends[q][r]
            assert blk.shape[1] == rc[q]                     # the sizes agree on both sides
            out[:, unpack[off[q]:off[q + 1]]] = blk
        outs.append(out.reshape(batch, N1, Cl))
    return outs


@pytest.mark.parametrize("N1,N2,G", [(16, 16, 4), (64, 16, 4), (16, 64, 4), (32, 8, 2), (8, 32, 8),
                                     (256, 64, 16), (128, 512, 4)])
def test_restore_maps_move_every_item_to_the_input_owner(N1, N2, G):
    """The maps of the second redistribution, by full simulation: rank r ends
    with y viewed N1 x N2, columns [r Cl, (r+1) Cl); every item moves once;
    with N1 = N2 nothing leaves its rank."""
    batch = 2
    rng = np.random.default_rng(N1 + N2 + G)
    y = rng.standard_normal((batch, N1 * N2)) + 1j * rng.standard_normal((batch, N1 * N2))
    outs = _restore_by_maps(y, N1, N2, G, batch)
    Cl = N2 // G
    for r in range(G):
        assert np.array_equal(outs[r], y.reshape(batch, N1, N2)[:, :, r * Cl:(r + 1) * Cl])
    if N1 == N2:
        from paper_2609_06449_gb300.sharded import restore_maps
        for q in range(G):
            sc = restore_maps(N1, N2, G, q)[1]
            assert sc[q] == N1 * N2 // G and sc.sum() == sc[q]


def _restore_worker(rank, G, port, N1, N2, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(G))
    import paper_2609_06449_gb300.sharded as sharded
    dist.init_process_group("gloo")
    try:
        batch, K1 = 2, N1 // G
        rng = np.random.default_rng(5)
        y = rng.standard_normal((batch, N1 * N2)) + 1j * rng.standard_normal((batch, N1 * N2))
        yl = torch.from_numpy(np.ascontiguousarray(y.reshape(batch, N2, N1)[:, :, rank * K1:(rank + 1) * K1]))
        pack, sc, unpack, rc = sharded.restore_maps(N1, N2, G, rank)
        offs = np.concatenate([[0], np.cumsum(sc)])
        offr = np.concatenate([[0], np.cumsum(rc)])

        def do_pack(src, send):                      # [G][batch][count]
            v = src.reshape(batch, -1).numpy()
            send.copy_(torch.from_numpy(np.concatenate(
                [v[:, pack[offs[r]:offs[r + 1]]].reshape(-1) for r in range(G)])))

        def do_unpack(recv, out):
            rv = recv.numpy()
            o = np.zeros((batch, N1 * N2 // G), complex)
            start = 0
            for qq in range(G):
                n = batch * rc[qq]
                o[:, unpack[offr[qq]:offr[qq + 1]]] = rv[start:start + n].reshape(batch, rc[qq])
                start += n
            out.copy_(torch.from_numpy(o.reshape(-1)))

        got = sharded.sharded_restore(yl, N1, N2, pack=do_pack, unpack=do_unpack,
                                      counts=lambda: (list(sc), list(rc)))
        q.put((rank, got.numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("G,N1,N2", [(2, 32, 8), (4, 16, 64)])
def test_sharded_restore_orchestration_over_gloo(G, N1, N2):
    """sharded_restore over gloo: the uneven all-to-all delivers every block,
    and each rank ends with the input's slab of y."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_restore_worker, args=(r, G, port, N1, N2, q)) for r in range(G)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(G))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    batch, Cl = 2, N2 // G
    rng = np.random.default_rng(5)
    y = rng.standard_normal((batch, N1 * N2)) + 1j * rng.standard_normal((batch, N1 * N2))
    for r in range(G):
        assert np.array_equal(got[r], y.reshape(batch, N1, N2)[:, :, r * Cl:(r + 1) * Cl])

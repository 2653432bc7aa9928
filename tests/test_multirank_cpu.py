"""Multi-process paths on the CPU (gloo), no GPU.

1. The benchmark's rank handling (bench.Ranks): barrier, the max over ranks
   of the step time, and the whole-job value = units of all ranks / slowest
   rank -- the N > 1 path of bench.py, whose ranks run independent replicas.
2. PARA-CO-DRP_b (App. C.5) with p real processes: each rank packs its
   Phase-I slab with the fused macro digit reversal (oracle procedures),
   sends every destination its (N1/p) x (N2/p) block over gloo point-to-point
   (one balanced exchange: N/p^2 items per ordered pair, the self block stays
   local), transposes the received blocks and unpacks.  The result must equal
   the single-process procedure and the closed form Z-hat of Eq. (17); the
   items' labels travel the same exchange, and each receiving rank counts, per
   source, the items whose own coordinates route them to it (N/p^2 each)."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))


def _ranks_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    _env(rank, world, port)
    import bench
    r = bench.Ranks("gloo", device="cpu")
    r.barrier()
    step = 1.0 + rank                                  # rank r takes 1 + r seconds
    v = r.job_value(100.0, step)                       # 100 units per rank per step
    m = r.max_over_ranks(step)
    r.close()
    q.put((rank, v, m))


@pytest.mark.parametrize("world", [2, 3])
def test_bench_rank_aggregation_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ranks_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = float(world)
    for rank, v, m in out:
        assert m == slowest
        assert abs(v - 100.0 * world / slowest) < 1e-9


def _drp_worker(rank, p, port, N1, N2, b, q):
    import sys
    sys.path.insert(0, ROOT)
    _env(rank, p, port)
    from oracle import paco_sim as ps
    from paco_inputs import gaussian
    dist.init_process_group("gloo")
    N = N1 * N2
    x = gaussian(N, 21, np.complex128)
    A_t = ps.simulate(x, N1, N2, b, p, phase1="lemma")["A_tilde"]   # Phase-I output, all slabs
    w1, w2 = N1 // p, N2 // p
    Xq = np.array(A_t[:, rank * w2:(rank + 1) * w2])                 # this processor's slab
    c = rank * w2 + np.arange(w2)
    ps.fused_macro_digit_reversal(Xq, b, lambda v: ps.root(v * c, N, -1))   # local pack
    # the labels a*N2 + c of this slab's items, packed by the same reversal
    # (the pack moves whole rows; the fused twiddle does not move anything)
    lab = (np.arange(N1)[:, None] * N2 + rank * w2 + np.arange(w2)[None, :]).astype(np.int64)
    ps.macro_digit_reversal(lab, b)

    def exchange(arr, np_dtype, view):
        recv, reqs, bufs = {}, [], {}
        for qd in range(p):                                           # one balanced exchange
            blk = np.ascontiguousarray(arr[qd * w1:(qd + 1) * w1, :])
            if qd == rank:
                recv[rank] = blk                                      # self block stays local
                continue
            t = torch.from_numpy(blk.view(view).copy())
            reqs.append(dist.isend(t, dst=qd))
            r = torch.empty_like(t)
            bufs[qd] = r
            reqs.append(dist.irecv(r, src=qd))
        for rq in reqs:
            rq.wait()
        for qd, r in bufs.items():
            recv[qd] = r.numpy().view(np_dtype).reshape(w1, w2)
        return recv

    recv = exchange(Xq, np.complex128, np.float64)
    rlab = exchange(lab, np.int64, np.int64)
    # items received from each source whose own coordinates route them here:
    # source = owner of input column c, destination = owner of k1 = pi_m1(a)
    import oracle
    pi1 = oracle.digit_reverse_table(b, ps.log_b(N1, b))
    sizes = {}
    for src, L in rlab.items():
        a, c = L // N2, L % N2
        sizes[src] = int(np.count_nonzero((c // w2 == src) & (pi1[a] // w1 == rank)))
    Yq = np.empty((N2, w1), dtype=np.complex128)
    for src in range(p):                                              # per-block transpose
        Yq[src * w2:(src + 1) * w2, :] = recv[src].T
    ps.macro_digit_reversal(Yq, b)                                    # local unpack
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, Yq, sizes))


@pytest.mark.parametrize("N1,N2,b,p", [(16, 16, 2, 2), (64, 16, 4, 4), (16, 64, 2, 2)])
def test_para_co_drp_over_gloo(N1, N2, b, p):
    import oracle
    from oracle import paco_sim as ps
    from paco_inputs import gaussian
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_drp_worker, args=(r, p, port, N1, N2, b, q)) for r in range(p)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(p):
        rank, Yq, sizes = q.get(timeout=120)
        res[rank] = (Yq, sizes)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    N = N1 * N2
    x = gaussian(N, 21, np.complex128)
    single = ps.simulate(x, N1, N2, b, p, phase1="lemma")
    # exactly N/p^2 correctly routed items per ordered pair (Theorem 4),
    # counted on the receiving rank by the items' own coordinates
    for rank in range(p):
        assert sorted(res[rank][1]) == list(range(p))
        assert all(v == N // (p * p) for v in res[rank][1].values())
    W = np.concatenate([res[r][0] for r in range(p)], axis=1)
    assert np.allclose(W, single["W"], atol=1e-12)
    # closed form of Eq. (17): W[u, v] = Z[v, pi_m2(u)], Z[v, c] = A[v, c] w_N^{-vc}
    A = np.fft.fft(x.reshape(N1, N2), axis=0)
    v = np.arange(N1)[:, None]
    c = np.arange(N2)[None, :]
    Z = A * np.exp(-2j * np.pi * ((v * c) % N) / N)
    pi2 = oracle.digit_reverse_table(b, ps.log_b(N2, b))
    assert np.allclose(W, Z[:, pi2].T, atol=1e-9)

"""The sharded form of PACO across G ranks (one GPU per rank): PARA-CO-DRP
(Sect. 4.2, App. C.5) with the processors of the paper's machine model as
ranks.  Rank g holds input slab g (columns [g Cl, (g+1) Cl) of X = x viewed
N1 x N2, Cl = N2/G) and gets output slab g (columns [g K1, (g+1) K1) of
Y = y viewed N2 x N1, K1 = N1/G); the layouts are those of
``paco_plan_create_sharded`` in include/paco.h:

    x_local [batch][N1][Cl]   send, recv [G][batch][Cl][K1]   y_local [batch][N2][K1]

``sharded_fft`` is the host orchestration: Phase I on the slab into G send
blocks of N/G^2 items per transform (``paco_shard_stage1``), one all-to-all
of equal blocks (``torch.distributed.all_to_all_single``, NCCL grouped
send/recv for CUDA tensors: every rank receives into its own buffer, no peer
loads), Phase III on the received blocks (``paco_shard_stage2``).
``sharded_restore`` is the optional second redistribution that gives every
rank the input's slab of y ([batch][N1][Cl]): pack, an all-to-all with
uneven splits, unpack (``paco_shard_restore_*``).  The stage, pack and
exchange callables can be replaced, which is how the orchestration is tested
without GPUs."""

from __future__ import annotations

import ctypes

from . import C64, ShardOpts, _check, _ptr, _stream, lib


def restore_maps(N1: int, N2: int, G: int, rank: int):
    """``paco_shard_restore_maps`` (host): (pack_map, send_counts, unpack_map,
    recv_counts) of one rank as numpy arrays."""
    import numpy as np
    n = int(N1) * int(N2) // int(G)
    pack = np.empty(n, np.int32)
    unpack = np.empty(n, np.int32)
    sc = np.empty(int(G), np.int64)
    rc = np.empty(int(G), np.int64)
    p32, p64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    _check(lib.paco_shard_restore_maps(int(N1), int(N2), int(G), int(rank), pack.ctypes.data_as(p32),
                                       sc.ctypes.data_as(p64), unpack.ctypes.data_as(p32), rc.ctypes.data_as(p64)))
    return pack, sc, unpack, rc


class ShardedPlan:
    """``paco_plan_create_sharded``: the plan of rank ``rank`` of ``G``
    (``restore``: also the maps of the second redistribution; ``dims=2``:
    the slab-decomposed 2-D DFT of the N1 x N2 view)."""

    def __init__(self, N1: int, N2: int, b: int, G: int, rank: int, batch: int = 1, restore: bool = False,
                 dims: int = 1):
        o = ShardOpts(int(N1), int(N2), int(b), int(G), int(rank), int(batch), C64, 1 if restore else 0, int(dims))
        h = ctypes.c_void_p()
        _check(lib.paco_plan_create_sharded(ctypes.byref(h), ctypes.byref(o)))
        self._h = h
        self.N1, self.N2, self.b, self.G, self.rank, self.batch = int(N1), int(N2), int(b), int(G), int(rank), int(batch)
        self.Cl, self.K1 = self.N2 // self.G, self.N1 // self.G
        self.block = self.Cl * self.K1            # N/G^2 items per transform and ordered pair of ranks

    def stage1(self, x_local, send, dir: int = -1, stream=None) -> None:
        _check(lib.paco_shard_stage1(self._h, _ptr(x_local), _ptr(send), int(dir), _stream(stream)))

    def stage2(self, recv, y_local, dir: int = -1, stream=None) -> None:
        _check(lib.paco_shard_stage2(self._h, _ptr(recv), _ptr(y_local), int(dir), _stream(stream)))

    def restore_counts(self):
        """(send_counts, recv_counts) per transform, G entries each."""
        sc = (ctypes.c_int64 * self.G)()
        rc = (ctypes.c_int64 * self.G)()
        _check(lib.paco_shard_restore_counts(self._h, sc, rc))
        return list(sc), list(rc)

    def restore_pack(self, y_local, send, stream=None) -> None:
        _check(lib.paco_shard_restore_pack(self._h, _ptr(y_local), _ptr(send), _stream(stream)))

    def restore_unpack(self, recv, out, stream=None) -> None:
        _check(lib.paco_shard_restore_unpack(self._h, _ptr(recv), _ptr(out), _stream(stream)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.paco_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exchange_blocks(send, recv, group=None) -> None:
    """The all-to-all of PARA-CO-DRP: block q of ``send`` ([G][...], equal
    blocks) goes to rank q, into block g (the sender's rank) of ``recv``.
    Complex buffers travel as their real view."""
    import torch
    import torch.distributed as dist
    s = torch.view_as_real(send) if send.is_complex() else send
    r = torch.view_as_real(recv) if recv.is_complex() else recv
    dist.all_to_all_single(r, s, group=group)


def sharded_fft(x_local, N1: int, N2: int, b: int, dir: int = -1, group=None, stage1=None, stage2=None,
                exchange=exchange_blocks):
    """This rank's output slab y_local ([batch][N2][K1]) of the N = N1*N2
    transform whose input slabs the G ranks of ``group`` hold (x_local:
    [batch][N1][Cl]).  stage1(x_local, send, dir) and stage2(recv, y_local,
    dir) default to the rank's ``ShardedPlan``; exchange(send, recv, group)
    to ``exchange_blocks``."""
    import torch
    import torch.distributed as dist
    G = dist.get_world_size(group)
    rank = dist.get_rank(group)
    N1, N2 = int(N1), int(N2)
    Cl, K1 = N2 // G, N1 // G
    if x_local.numel() % (N1 * Cl):
        raise ValueError(f"x_local must hold [batch][{N1}][{Cl}] elements")
    batch = x_local.numel() // (N1 * Cl)
    if stage1 is None or stage2 is None:
        plan = ShardedPlan(N1, N2, b, G, rank, batch)
        stage1, stage2 = stage1 or plan.stage1, stage2 or plan.stage2
    x_local = x_local.contiguous()
    send = torch.empty(G * batch * Cl * K1, dtype=x_local.dtype, device=x_local.device)
    stage1(x_local, send, dir)
    recv = torch.empty_like(send)
    exchange(send, recv, group)
    y_local = torch.empty(batch * N2 * K1, dtype=x_local.dtype, device=x_local.device)
    stage2(recv, y_local, dir)
    return y_local.reshape(batch, N2, K1)


def exchange_uneven(send, recv, send_splits, recv_splits, group=None) -> None:
    """All-to-all with uneven blocks: send_splits[r] items of ``send`` to rank
    r, recv_splits[q] items from rank q into ``recv`` (complex buffers travel
    as their real view)."""
    import torch
    import torch.distributed as dist
    f = 2 if send.is_complex() else 1
    s = torch.view_as_real(send).reshape(-1) if send.is_complex() else send
    r = torch.view_as_real(recv).reshape(-1) if recv.is_complex() else recv
    dist.all_to_all_single(r, s, output_split_sizes=[f * int(c) for c in recv_splits],
                           input_split_sizes=[f * int(c) for c in send_splits], group=group)


def sharded_restore(y_local, N1: int, N2: int, group=None, plan=None, pack=None, unpack=None, counts=None,
                    exchange=exchange_uneven):
    """The second redistribution: from this rank's output slab y_local
    ([batch][N2][K1], the result of ``sharded_fft``) to the input's
    ownership of y ([batch][N1][Cl]: y viewed N1 x N2, columns [rank Cl,
    (rank+1) Cl)).  pack(y_local, send), unpack(recv, out) and counts() ->
    (send_counts, recv_counts) per transform default to ``plan`` (a
    ShardedPlan created with restore=True)."""
    import torch
    import torch.distributed as dist
    G = dist.get_world_size(group)
    N1, N2 = int(N1), int(N2)
    n = N1 * N2 // G
    batch = y_local.numel() // n
    if plan is not None:
        pack, unpack, counts = pack or plan.restore_pack, unpack or plan.restore_unpack, counts or plan.restore_counts
    sc, rc = counts()
    y_local = y_local.contiguous()
    send = torch.empty(batch * n, dtype=y_local.dtype, device=y_local.device)
    pack(y_local, send)
    recv = torch.empty_like(send)
    exchange(send, recv, [batch * c for c in sc], [batch * c for c in rc], group)
    out = torch.empty(batch * n, dtype=y_local.dtype, device=y_local.device)
    unpack(recv, out)
    return out.reshape(batch, N1, N2 // G)

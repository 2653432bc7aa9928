"""The uneven-batch work queue (host logic, no GPU): the invariants the
persistent launch relies on, for random length mixes and lags.

* every transform is scheduled exactly once: small ones (N <= 2^13) in
  one group of same-length transforms of at most 8192 / N, large ones as
  N / 8192 Phase I tiles and N / 8192 Phase III tiles;
* every Phase III tile comes after all Phase I tiles of its transform (a
  Phase III item only waits on lower-indexed items, which never wait: the
  deadlock-freedom argument);
* a transform's Phase III tiles come at least `lag` items after its last
  Phase I tile unless the queue ran out of other work."""

import ctypes

import numpy as np
import pytest

from paco_inputs import uneven_lengths


def schedule(lengths, lag):
    import paper_2609_06449_gb300 as paco
    L = paco.lib
    f = L.paco_debug_batched_schedule
    i32p = ctypes.POINTER(ctypes.c_int32)
    f.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.c_int64, i32p, i32p, i32p,
                  ctypes.c_int64, i32p, ctypes.c_int64]
    f.restype = ctypes.c_int64
    n = len(lengths)
    cap = int(sum(max(1, 2 * (int(v) // 8192)) for v in lengths)) + n
    arr = (ctypes.c_int64 * max(1, n))(*[int(v) for v in lengths])
    kind = np.zeros(cap, np.int32); idx = np.zeros(cap, np.int32); tile = np.zeros(cap, np.int32)
    grp = np.zeros(max(1, n), np.int32)
    m = f(arr, n, lag, kind.ctypes.data_as(i32p), idx.ctypes.data_as(i32p), tile.ctypes.data_as(i32p), cap,
          grp.ctypes.data_as(i32p), max(1, n))
    assert m >= 0
    return kind[:m], idx[:m], tile[:m], grp


def check(lengths, lag):
    lengths = np.asarray(lengths, dtype=np.int64)
    kind, idx, tile, grp = schedule(lengths, lag)
    seen_small = np.zeros(len(lengths), int)
    p1 = {}
    p3 = {}
    for pos, (k, i, t) in enumerate(zip(kind, idx, tile)):
        if k == 0:
            members = grp[i:i + t]
            assert t >= 1
            n = lengths[members[0]]
            assert n <= 2 ** 13 and t <= 8192 // n and np.all(lengths[members] == n)
            seen_small[members] += 1
        elif k == 1:
            p1.setdefault(int(i), []).append((pos, int(t)))
        else:
            p3.setdefault(int(i), []).append((pos, int(t)))
    small = lengths <= 2 ** 13
    assert np.all(seen_small[small] == 1) and np.all(seen_small[~small] == 0)
    big = set(np.flatnonzero(~small).tolist())
    assert set(p1) == big and set(p3) == big
    for tr in big:
        nt = int(lengths[tr]) // 8192
        assert sorted(t for _, t in p1[tr]) == list(range(nt))
        assert sorted(t for _, t in p3[tr]) == list(range(nt))
        last1 = max(pos for pos, _ in p1[tr])
        first3 = min(pos for pos, _ in p3[tr])
        assert first3 > last1
        # the lag is kept unless nothing else was left to queue: then only
        # Phase III tiles follow
        if first3 - last1 - 1 < lag:
            assert np.all(kind[first3:] == 2)
    return kind


@pytest.mark.parametrize("lag", [0, 1, 152, 608])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_schedule_invariants_random_mix(seed, lag):
    e = uneven_lengths(count=300, seed=seed, lo=4, hi=20, total_log2=24)
    check(2 ** e, lag)


def test_schedule_benchmark_mix():
    e = uneven_lengths()
    lengths = np.concatenate([2 ** e, np.full(2 ** 14, 2 ** 12)])
    kind = check(lengths, 608)
    # 20 480 transforms: small groups plus two tiles per 8192 elements of the large ones
    assert len(kind) > 0


def test_schedule_rejects_bad_lengths():
    import paper_2609_06449_gb300 as paco
    f = paco.lib.paco_debug_batched_schedule
    arr = (ctypes.c_int64 * 2)(256, 48)
    i32p = ctypes.POINTER(ctypes.c_int32)
    buf = (ctypes.c_int32 * 16)()
    f.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.c_int64, i32p, i32p, i32p,
                  ctypes.c_int64, i32p, ctypes.c_int64]
    f.restype = ctypes.c_int64
    assert f(arr, 2, 0, buf, buf, buf, 16, buf, 16) == -1

"""PACO FFT on one GB300 -- thin Python binding over the C ABI (include/paco.h).

Every step of the transform runs in the CUDA kernels of ``libpaco.so``; this
module only marshals arguments.  PyTorch supplies device memory and streams.
There is no CPU fallback: importing the package raises if the library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``).

Entry points (same names as the C ABI):

* ``Plan(N1, N2, b, batch, dtype, p=0, tile_w=0, cluster=0, ctas_per_sm=0,
  split=0, dims=1, N3=0)`` -- ``paco_plan_create_ex``;
  ``.execute(in_ptr, out_ptr, dir, stream)`` etc.
* ``fft(x, N1, N2, b, p=0, dir=-1)`` -- torch tensors on the GPU;
  ``fft2`` -- the 2-D DFT of the N1 x N2 view (transposed result);
  ``fft3`` -- the 3-D DFT of N1 x N2 x N3 arrays (axes reversed).
* ``PacoFFT`` -- ``torch.autograd.Function`` whose backward is the conjugate
  transform (``dir=+1``).
* ``sharded`` -- the sharded form across G ranks (``ShardedPlan``,
  ``sharded_fft``: Phase I per rank, one all-to-all of N/G^2-item blocks,
  Phase III per rank).
* ``weighted_power_loss(x, w, N1, N2, b)`` -- sum(w |F x|^2) with the loss
  summed in the Phase III kernel and its backward fused into the conjugate
  transform's loads (``paco_execute_weighted_power`` / ``_input``).
"""

from __future__ import annotations

import ctypes
import os

__all__ = [
    "PacoError",
    "Plan",
    "BatchedPlan",
    "lib",
    "library_path",
    "fft",
    "fft2",
    "fft3",
    "PacoFFT",
    "PacoWeightedPowerLoss",
    "weighted_power_loss",
    "digit_reverse",
    "C64",
    "C128",
    "C64_TC_BF16X3",
    "C64_TC_FP16",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libpaco.so")

C64, C128, C64_TC_BF16X3, C64_TC_FP16 = 0, 1, 2, 3

_STATUS = {
    0: "PACO_OK",
    1: "PACO_ERR_INVALID_ARG",
    2: "PACO_ERR_UNSUPPORTED",
    3: "PACO_ERR_ALIASING",
    4: "PACO_ERR_CUDA",
    5: "PACO_ERR_TIMEOUT",
    6: "PACO_ERR_NOMEM",
    7: "PACO_ERR_DEVICE",
}


class PacoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanOpts(ctypes.Structure):
    _fields_ = [
        ("N1", ctypes.c_int64), ("N2", ctypes.c_int64), ("b", ctypes.c_int),
        ("p", ctypes.c_int), ("batch", ctypes.c_int64), ("dtype", ctypes.c_int),
        ("tile_w", ctypes.c_int), ("cluster", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
        ("split", ctypes.c_int), ("dims", ctypes.c_int), ("N3", ctypes.c_int64),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("N1", ctypes.c_int64), ("N2", ctypes.c_int64), ("N", ctypes.c_int64),
        ("batch", ctypes.c_int64), ("b", ctypes.c_int), ("p", ctypes.c_int),
        ("m1", ctypes.c_int), ("m2", ctypes.c_int), ("dtype", ctypes.c_int),
        ("slab_width_ok", ctypes.c_int), ("items_per_pair", ctypes.c_int64),
        ("h", ctypes.c_int64), ("mu", ctypes.c_int64),
        ("stage_tile_w", ctypes.c_int * 2), ("stage_cluster", ctypes.c_int * 2),
        ("stage_threads", ctypes.c_int * 2), ("stage_smem", ctypes.c_int * 2),
        ("fused_cluster", ctypes.c_int),
        ("shard_G", ctypes.c_int),
        ("shard_rank", ctypes.c_int),
        ("stage_split", ctypes.c_int * 2),
        ("dims", ctypes.c_int),
        ("N3", ctypes.c_int64),
    ]


class ShardOpts(ctypes.Structure):
    _fields_ = [
        ("N1", ctypes.c_int64), ("N2", ctypes.c_int64), ("b", ctypes.c_int), ("G", ctypes.c_int),
        ("rank", ctypes.c_int), ("batch", ctypes.c_int64), ("dtype", ctypes.c_int),
        ("restore", ctypes.c_int), ("dims", ctypes.c_int),
    ]


class BatchedOpts(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int), ("b", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("lag", ctypes.c_int)]


def _load():
    if not os.path.exists(library_path):
        raise ImportError(
            f"{library_path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(library_path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    L.paco_plan_create.argtypes = [i64, i64, i32, i64, i32]
    L.paco_plan_create.restype = vp
    L.paco_plan_create_ex.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PlanOpts)]
    L.paco_plan_create_ex.restype = i32
    L.paco_plan_destroy.argtypes = [vp]
    L.paco_plan_destroy.restype = None
    L.paco_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    L.paco_plan_info.restype = i32
    for name in ("paco_execute", "paco_execute_stage1", "paco_execute_stage2",
                 "paco_execute_phase1", "paco_permute"):
        f = getattr(L, name)
        f.argtypes = [vp, vp, vp, i32, vp]
        f.restype = i32
    L.paco_execute_host.argtypes = [vp, vp, vp, vp, vp, i32, vp]
    L.paco_execute_host.restype = i32
    L.paco_plan_check.argtypes = [vp]
    L.paco_plan_check.restype = i32
    L.paco_last_error.argtypes = []
    L.paco_last_error.restype = ctypes.c_char_p
    L.paco_digit_reverse.argtypes = [i64, i32, i32]
    L.paco_digit_reverse.restype = i64
    L.paco_version.argtypes = []
    L.paco_version.restype = ctypes.c_char_p
    L.paco_plan_create_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i32]
    L.paco_plan_create_batched.restype = i32
    L.paco_plan_create_batched_ex.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i32,
                                              ctypes.POINTER(BatchedOpts)]
    L.paco_plan_create_batched_ex.restype = i32
    pi = ctypes.POINTER(i32)
    L.paco_plan_batched_config.argtypes = [vp, i64, pi, pi, pi, pi]
    L.paco_plan_batched_config.restype = i32
    L.paco_debug_exchange_counts.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i64), vp]
    L.paco_debug_exchange_counts.restype = i32
    L.paco_debug_set_waits.argtypes = [vp, ctypes.c_uint, ctypes.c_uint]
    L.paco_debug_set_waits.restype = i32
    L.paco_execute_noalloc.argtypes = [vp, vp, i32, i64, i32, vp]
    L.paco_execute_noalloc.restype = i32
    L.paco_probe_fp64_peak.argtypes = [i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), vp]
    L.paco_probe_fp64_peak.restype = i32
    L.paco_execute_weighted_power.argtypes = [vp, vp, vp, vp, vp, i32, i32, vp]
    L.paco_execute_weighted_power.restype = i32
    L.paco_execute_weighted_input.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, i32, vp]
    L.paco_execute_weighted_input.restype = i32
    L.paco_plan_create_sharded.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ShardOpts)]
    L.paco_plan_create_sharded.restype = i32
    for name in ("paco_shard_stage1", "paco_shard_stage2"):
        f = getattr(L, name)
        f.argtypes = [vp, vp, vp, i32, vp]
        f.restype = i32
    p64, p32 = ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32)
    L.paco_shard_restore_counts.argtypes = [vp, p64, p64]
    L.paco_shard_restore_counts.restype = i32
    for name in ("paco_shard_restore_pack", "paco_shard_restore_unpack"):
        f = getattr(L, name)
        f.argtypes = [vp, vp, vp, vp]
        f.restype = i32
    L.paco_shard_restore_maps.argtypes = [i64, i64, i32, i32, p32, p64, p32, p64]
    L.paco_shard_restore_maps.restype = i32
    L.paco_probe_tc05_dft128.argtypes = [vp, vp, i64, i64, ctypes.POINTER(ctypes.c_float), vp]
    L.paco_probe_tc05_dft128.restype = i32
    L.paco_noalloc_check.argtypes = []
    L.paco_noalloc_check.restype = i32
    L.paco_debug_noalloc_set_waits.argtypes = [ctypes.c_uint, ctypes.c_uint]
    L.paco_debug_noalloc_set_waits.restype = None
    return L


lib = _load()


def _check(status: int) -> None:
    if status != 0:
        raise PacoError(status, lib.paco_last_error().decode())


def execute_noalloc(x, out, b: int, batch: int, dir: int = -1, stream=None) -> None:
    """paco_execute_noalloc: the N1 = N2 = 2^14 complex64 transform without
    any allocation (the library's reserved device arrays); see paco.h."""
    _check(lib.paco_execute_noalloc(_ptr(x), _ptr(out), int(b), int(batch), int(dir), _stream(stream)))


def probe_fp64_peak(iters: int = 4096, stream=None):
    """paco_probe_fp64_peak: (GFLOP/s, ms) of the FP64 FMA rate on the current
    device (FMA = two flops), at the clock the GPU ran."""
    g, t = ctypes.c_double(), ctypes.c_float()
    _check(lib.paco_probe_fp64_peak(int(iters), ctypes.byref(g), ctypes.byref(t), _stream(stream)))
    return g.value, t.value


def noalloc_check() -> None:
    """paco_noalloc_check: raise if a kernel of paco_execute_noalloc on the
    current device recorded an error (e.g. a bounded wait that gave up)."""
    _check(lib.paco_noalloc_check())


def digit_reverse(u: int, b: int, ell: int) -> int:
    """pi_ell(u) in base b, as computed by the library (host function)."""
    r = lib.paco_digit_reverse(int(u), int(b), int(ell))
    if r < 0:
        raise PacoError(1, "digit_reverse: bad argument")
    return int(r)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Plan:
    """A PACO plan (``paco_plan_create_ex``).  Buffers are torch tensors or
    raw device pointers; ``stream`` is a torch stream, a raw handle, or None
    for torch's current stream.  ``dims=2``: the 2-D DFT of the N1 x N2 view;
    ``dims=3`` with ``N3``: the 3-D DFT of N1 x N2 x N3 arrays (then
    ``self.N2`` is the middle axis and ``self.N`` = N1 N2 N3)."""

    def __init__(self, N1: int, N2: int, b: int, batch: int = 1, dtype: int = C64,
                 p: int = 0, tile_w: int = 0, cluster: int = 0, ctas_per_sm: int = 0, split: int = 0,
                 dims: int = 1, N3: int = 0):
        o = PlanOpts(int(N1), int(N2), int(b), int(p), int(batch), int(dtype),
                     int(tile_w), int(cluster), int(ctas_per_sm), int(split), int(dims), int(N3))
        h = ctypes.c_void_p()
        _check(lib.paco_plan_create_ex(ctypes.byref(h), ctypes.byref(o)))
        self._h = h
        inf = PlanInfo()
        _check(lib.paco_plan_info(self._h, ctypes.byref(inf)))
        self.info = inf
        self.N1, self.N2, self.N3, self.N = inf.N1, inf.N2, inf.N3, inf.N
        self.b, self.p, self.batch, self.dtype = inf.b, inf.p, inf.batch, inf.dtype
        self.m1, self.m2 = inf.m1, inf.m2

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.paco_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def execute(self, x, out, dir: int = -1, stream=None) -> None:
        _check(lib.paco_execute(self._h, _ptr(x), _ptr(out), int(dir), _stream(stream)))

    def execute_weighted_power(self, x, out, w, loss, dir: int = -1, stream=None, out_weighted: bool = False) -> None:
        """y = F^dir x, loss[0] = sum(w |y|^2) (float32 w, float64 loss, device);
        out = y, or w * y with ``out_weighted``."""
        _check(lib.paco_execute_weighted_power(self._h, _ptr(x), _ptr(out), _ptr(w), _ptr(loss),
                                               1 if out_weighted else 0, int(dir), _stream(stream)))

    def execute_weighted_input(self, x, out, w, scale=None, mult: float = 1.0, dir: int = -1,
                               stream=None) -> None:
        """out = F^dir (mult * scale[0] * w * x); scale a float64 device scalar or
        None, w a float32 device tensor or None (the scalar alone)."""
        _check(lib.paco_execute_weighted_input(self._h, _ptr(x), _ptr(out), _ptr(w), _ptr(scale),
                                               float(mult), int(dir), _stream(stream)))

    def execute_stage1(self, x, W, dir: int = -1, stream=None) -> None:
        _check(lib.paco_execute_stage1(self._h, _ptr(x), _ptr(W), int(dir), _stream(stream)))

    def execute_stage2(self, W, out, dir: int = -1, stream=None) -> None:
        _check(lib.paco_execute_stage2(self._h, _ptr(W), _ptr(out), int(dir), _stream(stream)))

    def execute_phase1(self, x, out, dir: int = -1, stream=None) -> None:
        _check(lib.paco_execute_phase1(self._h, _ptr(x), _ptr(out), int(dir), _stream(stream)))

    def permute(self, a_tilde, W, dir: int = -1, stream=None) -> None:
        _check(lib.paco_permute(self._h, _ptr(a_tilde), _ptr(W), int(dir), _stream(stream)))

    def execute_host(self, h_in, h_out, d_in, d_out, dir: int = -1, stream=None) -> None:
        _check(lib.paco_execute_host(self._h, _ptr(h_in), _ptr(h_out), _ptr(d_in),
                                     _ptr(d_out), int(dir), _stream(stream)))

    def check(self) -> None:
        _check(lib.paco_plan_check(self._h))

    def debug_exchange_counts(self, x, out, dir: int = -1, stream=None):
        """Test hook: run a one-launch cluster plan once and return the p x p
        counts of items each CTA (processor) wrote to each other CTA."""
        p = int(self.p)
        arr = (ctypes.c_int64 * (p * p))()
        _check(lib.paco_debug_exchange_counts(self._h, _ptr(x), _ptr(out), int(dir), arr, _stream(stream)))
        return [[int(arr[q * p + r]) for r in range(p)] for q in range(p)]

    def debug_set_waits(self, spin_limit: int = 0, wait_bias: int = 0) -> None:
        """Test hook of the bounded waits (``paco_debug_set_waits``)."""
        _check(lib.paco_debug_set_waits(self._h, int(spin_limit), int(wait_bias)))


class BatchedPlan(Plan):
    """An uneven batch (``paco_plan_create_batched``): ``lengths`` complex64
    transforms stored back to back in the given order.  ``autotune=True`` is
    the default constructor; otherwise ``b``, ``ctas_per_sm`` and ``lag`` fix
    the configuration.  ``execute``/``execute_host`` as for ``Plan``."""

    def __init__(self, lengths, autotune: bool = True, b: int = 0, ctas_per_sm: int = 1,
                 lag: int = 0):
        n = len(lengths)
        arr = (ctypes.c_int64 * max(1, n))(*[int(v) for v in lengths])
        h = ctypes.c_void_p()
        if autotune and not b:
            _check(lib.paco_plan_create_batched(ctypes.byref(h), arr, n, C64))
        else:
            o = BatchedOpts(1 if autotune else 0, int(b), int(ctas_per_sm), int(lag))
            _check(lib.paco_plan_create_batched_ex(ctypes.byref(h), arr, n, C64, ctypes.byref(o)))
        self._h = h
        inf = PlanInfo()
        _check(lib.paco_plan_info(self._h, ctypes.byref(inf)))
        self.info = inf
        self.lengths = [int(v) for v in lengths]
        self.N, self.count, self.dtype = inf.N, inf.batch, C64

    def config(self, length: int):
        """(b, N1, ctas_per_sm, lag) the plan uses for `length`."""
        b, n1, c, lag = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.paco_plan_batched_config(self._h, int(length), ctypes.byref(b), ctypes.byref(n1),
                                            ctypes.byref(c), ctypes.byref(lag)))
        return b.value, n1.value, c.value, lag.value


_PLANS: dict = {}


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"PACO takes complex64 or complex128 tensors, got {t.dtype}")


def get_plan(N1: int, N2: int, b: int, batch: int, dtype: int, p: int = 0,
             device: int | None = None, stream: int | None = None, dims: int = 1, N3: int = 0) -> Plan:
    """The cached plan for this shape on ``device`` and ``stream``.

    A plan's executions must not overlap in time (the 2^14 complex64 panel
    pipeline keeps its ring buffers and counters in the plan), so plans are
    cached per stream: calls on one stream are ordered by that stream, and
    calls on different streams get different plans."""
    import torch
    dev = torch.cuda.current_device() if device is None else device
    if stream is None:
        stream = int(torch.cuda.current_stream(dev).cuda_stream)
    key = (N1, N2, b, batch, dtype, p, dev, int(stream), int(dims), int(N3))
    pl = _PLANS.get(key)
    if pl is None:
        with torch.cuda.device(dev):
            pl = Plan(N1, N2, b, batch, dtype, p, dims=dims, N3=N3)
        _PLANS[key] = pl
    return pl


def probe_tc05_dft128(x, y, batch: int, C: int, stream=None, timed: bool = False):
    """``paco_probe_tc05_dft128``: y[b][k][c] = sum_j w_128^{-jk} x[b][j][c] on
    the tcgen05 tensor cores (BF16x3).  Returns the kernel time in ms when
    ``timed`` (the call then waits), else None."""
    ms = ctypes.c_float(0.0)
    _check(lib.paco_probe_tc05_dft128(_ptr(x), _ptr(y), int(batch), int(C),
                                      ctypes.byref(ms) if timed else None, _stream(stream)))
    return ms.value if timed else None


def fft2(x, N1: int, N2: int, b: int, p: int = 0, dir: int = -1, out=None):
    """2-D DFT of every N1 x N2 array in ``x`` (last dimension N1*N2, row
    major), returned transposed: out[..., k2 * N1 + k1] = sum_{j1, j2}
    x[..., j1 * N2 + j2] w_N1^{dir k1 j1} w_N2^{dir k2 j2} (a plan with
    dims = 2: the PACO pipeline without its top-level twiddle)."""
    import torch
    if not x.is_cuda:
        raise ValueError("PACO runs on the GPU: x must be a CUDA tensor")
    N = int(N1) * int(N2)
    if x.shape[-1] != N:
        raise ValueError(f"last dimension {x.shape[-1]} != N1*N2 = {N}")
    x = x.contiguous()
    batch = x.numel() // N
    if out is None:
        out = torch.empty_like(x)
    dev = x.device.index
    stream = int(torch.cuda.current_stream(x.device).cuda_stream)
    with torch.cuda.device(dev):
        pl = get_plan(int(N1), int(N2), int(b), batch, _dtype_code(x), int(p), dev, stream, dims=2)
        pl.execute(x, out, dir, stream)
    return out


def fft3(x, N1: int, N2: int, N3: int, b: int, p: int = 0, dir: int = -1, out=None):
    """3-D DFT of every N1 x N2 x N3 array in ``x`` (last dimension
    N1*N2*N3, row major), returned with its axes reversed:
    out[..., (k3 * N2 + k2) * N1 + k1] = sum x[..., (j1 * N2 + j2) * N3 + j3]
    w_N1^{dir k1 j1} w_N2^{dir k2 j2} w_N3^{dir k3 j3} (a plan with dims = 3:
    the pipeline on the N1 x (N2 N3) view without its top-level twiddle,
    Phase III split over the N2 x N3 planes)."""
    import torch
    if not x.is_cuda:
        raise ValueError("PACO runs on the GPU: x must be a CUDA tensor")
    N = int(N1) * int(N2) * int(N3)
    if x.shape[-1] != N:
        raise ValueError(f"last dimension {x.shape[-1]} != N1*N2*N3 = {N}")
    x = x.contiguous()
    batch = x.numel() // N
    if out is None:
        out = torch.empty_like(x)
    dev = x.device.index
    stream = int(torch.cuda.current_stream(x.device).cuda_stream)
    with torch.cuda.device(dev):
        pl = get_plan(int(N1), int(N2), int(b), batch, _dtype_code(x), int(p), dev, stream, dims=3, N3=int(N3))
        pl.execute(x, out, dir, stream)
    return out


def fft(x, N1: int, N2: int, b: int, p: int = 0, dir: int = -1, out=None):
    """PACO transform of the last dimension of ``x`` (length N1*N2) for every
    leading index: dir=-1 the paper's forward DFT, dir=+1 the unnormalised
    conjugate transform.  ``x`` must be a contiguous complex64/complex128 CUDA
    tensor; returns a new tensor (or fills ``out``).  The work is enqueued on
    the current stream of ``x``'s device, with a plan cached for that stream."""
    import torch
    if not x.is_cuda:
        raise ValueError("PACO runs on the GPU: x must be a CUDA tensor")
    N = int(N1) * int(N2)
    if x.shape[-1] != N:
        raise ValueError(f"last dimension {x.shape[-1]} != N1*N2 = {N}")
    x = x.contiguous()
    batch = x.numel() // N
    if out is None:
        out = torch.empty_like(x)
    elif out.device != x.device:
        raise ValueError("out must be on the device of x")
    dev = x.device.index
    stream = int(torch.cuda.current_stream(x.device).cuda_stream)
    with torch.cuda.device(dev):
        pl = get_plan(int(N1), int(N2), int(b), batch, _dtype_code(x), int(p), dev, stream)
        pl.execute(x, out, dir, stream)
    return out


try:
    import torch as _torch

    class PacoFFT(_torch.autograd.Function):
        """y = PACO(x) with the hand-written backward grad_x = F^H grad_y,
        F^H being the unnormalised conjugate transform (F is symmetric, so
        F^H = conj(F)); it runs the same kernels with dir = +1."""

        @staticmethod
        def forward(ctx, x, N1, N2, b, p=0):
            ctx.cfg = (N1, N2, b, p)
            return fft(x, N1, N2, b, p, dir=-1)

        @staticmethod
        def backward(ctx, g):
            N1, N2, b, p = ctx.cfg
            return fft(g.contiguous(), N1, N2, b, p, dir=+1), None, None, None, None
    class PacoWeightedPowerLoss(_torch.autograd.Function):
        """loss = sum(w |F x|^2) over the whole batch (float64 scalar), F the
        paper's forward transform.  Forward: the two stage kernels, the loss
        summed by the Phase III kernel, which stores u = w ⊙ F x (y itself is
        not returned).  Backward: grad_x = F^H (2 g u), the scalar 2 g applied
        as the conjugate transform's Phase I loads its input.  w (float32, the
        shape of x) is treated as a constant."""

        @staticmethod
        def forward(ctx, x, w, N1, N2, b, p=0):
            if w.requires_grad:
                raise ValueError("weighted_power_loss: w is a constant (requires_grad must be False)")
            xc, wc = x.contiguous(), w.contiguous()
            N = int(N1) * int(N2)
            if xc.dtype != _torch.complex64 or wc.dtype != _torch.float32 or wc.shape != xc.shape:
                raise ValueError("weighted_power_loss: x complex64 and w float32 of the same shape")
            y = _torch.empty_like(xc)
            loss = _torch.empty((), dtype=_torch.float64, device=xc.device)
            stream = int(_torch.cuda.current_stream(xc.device).cuda_stream)
            with _torch.cuda.device(xc.device.index):
                pl = get_plan(int(N1), int(N2), int(b), xc.numel() // N, C64, int(p), xc.device.index, stream)
                pl.execute_weighted_power(xc, y, wc, loss, -1, stream, out_weighted=True)
            ctx.save_for_backward(y)
            ctx.cfg = (int(N1), int(N2), int(b), int(p), stream)
            return loss

        @staticmethod
        def backward(ctx, g):
            (y,) = ctx.saved_tensors
            N1, N2, b, p, _ = ctx.cfg
            g = g.to(_torch.float64).contiguous()
            gx = _torch.empty_like(y)
            stream = int(_torch.cuda.current_stream(y.device).cuda_stream)
            with _torch.cuda.device(y.device.index):
                pl = get_plan(N1, N2, b, y.numel() // (N1 * N2), C64, p, y.device.index, stream)
                pl.execute_weighted_input(y, gx, None, g, 2.0, +1, stream)
            return gx, None, None, None, None, None

    def weighted_power_loss(x, w, N1: int, N2: int, b: int, p: int = 0):
        """sum(w |F x|^2) (float64 scalar) with the fused forward and backward
        of ``PacoWeightedPowerLoss``."""
        return PacoWeightedPowerLoss.apply(x, w, N1, N2, b, p)
except ImportError:  # pragma: no cover - torch is a hard requirement on the GPU machine
    PacoFFT = PacoWeightedPowerLoss = weighted_power_loss = None

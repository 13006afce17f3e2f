"""Python binding of librecon.so, the GB300 grayscale morphological
reconstruction library (C ABI in include/recon.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels behind the C ABI. Functions keep the C names; image arguments are
device addresses (ints, e.g. ``tensor.data_ptr()`` of contiguous uint8 CUDA
tensors), except in the ``*_host`` entry points, which take host addresses.
``run(I, J, conn)`` and ``batch(pairs, conn)`` take the tensors themselves,
check that they are contiguous 2-D uint8 CUDA tensors, and call the same
entry points.
There is no fallback: if librecon.so is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librecon.so")

RECON_OK, RECON_EINVAL, RECON_EMARKER, RECON_ENOMEM, RECON_ECUDA, RECON_ETIMEOUT = range(6)
RECON_FLAG_SYNC, RECON_FLAG_NO_CHECK, RECON_FLAG_LEARNED, RECON_FLAG_NO_GRAPH = 1, 2, 4, 8
(RECON_P_BLOCK_H, RECON_P_SWEEPS, RECON_P_GRID, RECON_P_BANDS, RECON_P_WAIT_NS, RECON_P_ORDER,
 RECON_P_TEST_STALL, RECON_P_TMA, RECON_P_TRACE, RECON_P_LAST_ABORT, RECON_P_REVISIT_SCANS,
 RECON_P_SCAN_GAIN, RECON_P_TUNE_FROM_CACHE) = range(1, 14)
RECON_OP_DILATE, RECON_OP_ERODE, RECON_OP_FILL_HOLES = 0, 1, 2

# every symbol the header declares; tests check the library exports them all
SYMBOLS = ("recon_init", "recon_run", "recon_run_op", "recon_batch", "recon_batch_ex", "recon_run_host",
           "recon_batch_host", "recon_sync", "recon_last_error_tile", "recon_free",
           "recon_strerror", "recon_set_param", "recon_get_param", "recon_get_work",
           "recon_last_kernel_ms", "recon_features", "recon_mlp_forward", "recon_mlp_grad",
           "recon_mlp_adam", "recon_mlp_train", "recon_sched_set_model", "recon_sched_plan_batch",
           "recon_autotune", "recon_sync_for", "recon_trace", "recon_run_noalloc",
           "recon_mb_threads", "recon_mb_random", "recon_mb_atomic", "recon_dt", "recon_dt_levels",
           "recon_mlp_train_resume", "recon_autotune_cache", "recon_autotune_cache_load", "recon_checks")
RECON_NFEAT, RECON_MLP_NPARAMS = 20, 5634


class recon_tile(ctypes.Structure):
    _fields_ = [("I", ctypes.c_void_p), ("J", ctypes.c_void_p), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("pitch", ctypes.c_int), ("conn", ctypes.c_int),
                ("op", ctypes.c_int)]


class recon_work(ctypes.Structure):
    _fields_ = [("visits", ctypes.c_uint64), ("scan_rows", ctypes.c_uint64),
                ("pops", ctypes.c_uint64), ("seeds", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("busy_ns", ctypes.c_uint64), ("phase_ns", ctypes.c_uint64 * 6)]


class ReconError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what or "recon", recon_strerror(status), status))


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Loads librecon.so (built by __graft_entry__.build() or
    paper_1311_0378_gb300.build). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("librecon.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i, u, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_int64
    tp = ctypes.POINTER(recon_tile)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "recon_init": ([ctypes.POINTER(vp), i, vp, u], i),
        "recon_run": ([vp, vp, vp, i, i, i], i),
        "recon_run_op": ([vp, vp, vp, i, i, i, i], i),
        "recon_batch": ([vp, tp, i], i),
        "recon_batch_ex": ([vp, tp, i, ip, ip], i),
        "recon_run_host": ([vp, vp, vp, i, i, i], i),
        "recon_batch_host": ([vp, tp, i], i),
        "recon_sync": ([vp], i),
        "recon_last_error_tile": ([vp], i),
        "recon_free": ([vp], i),
        "recon_strerror": ([i], ctypes.c_char_p),
        "recon_set_param": ([vp, i, i64], i),
        "recon_get_param": ([vp, i], i64),
        "recon_get_work": ([vp, ctypes.POINTER(recon_work), i], i),
        "recon_last_kernel_ms": ([vp, ctypes.POINTER(ctypes.c_float)], i),
        "recon_features": ([vp, tp, i, vp], i),
        "recon_mlp_forward": ([vp, vp, vp, i, vp], i),
        "recon_mlp_grad": ([vp, vp, vp, vp, vp, i, vp, vp], i),
        "recon_mlp_adam": ([vp, vp, vp, vp, vp, i, ctypes.c_float], i),
        "recon_mlp_train": ([vp, vp, vp, vp, i, i, i, ctypes.c_float, ctypes.c_uint64, vp], i),
        "recon_sched_set_model": ([vp, vp, vp, i, i], i),
        "recon_sched_plan_batch": ([vp, tp, i, vp, vp, vp], i),
        "recon_autotune": ([vp, tp, i, i, vp], i),
        "recon_sync_for": ([vp, i], i),
        "recon_trace": ([vp, vp, i], i),
        "recon_run_noalloc": ([vp, vp, i, i, i, vp], i),
        "recon_mb_threads": ([i], i),
        "recon_dt": ([vp, vp, vp, vp, i, i], i),
        "recon_dt_levels": ([vp], i),
        "recon_autotune_cache": ([vp, vp, i], i),
        "recon_checks": ([vp, vp, vp, i], i),
        "recon_autotune_cache_load": ([vp, vp, i], i),
        "recon_mlp_train_resume": ([vp, vp, vp, ip, i, vp, vp, i, i, i, ctypes.c_float, ctypes.c_uint64, vp], i),
        "recon_mb_random": ([vp, i, ctypes.c_uint64, i, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_float)], i),
        "recon_mb_atomic": ([vp, i, i, ctypes.POINTER(ctypes.c_float)], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _tiles(tiles: Sequence[Tuple[int, ...]]):
    """(I, J, H, W, pitch, conn) or (I, J, H, W, pitch, conn, op) per tile."""
    arr = (recon_tile * max(len(tiles), 1))()
    for k, t in enumerate(tiles):
        arr[k] = recon_tile(*t) if len(t) == 7 else recon_tile(*t, RECON_OP_DILATE)
    return arr


def _ints(v):
    if v is None:
        return None
    return (ctypes.c_int * max(len(v), 1))(*[int(x) for x in v])


def recon_init(device: int = 0, stream: int = 0, flags: int = 0) -> ctypes.c_void_p:
    """Creates a context; raises ReconError on failure. `stream` is a
    cudaStream_t address (0: the context makes its own)."""
    ctx = ctypes.c_void_p()
    rc = lib().recon_init(ctypes.byref(ctx), device, ctypes.c_void_p(stream or None), flags)
    if rc != RECON_OK:
        raise ReconError(rc, "recon_init")
    return ctx


def recon_run(ctx, I: int, J: int, H: int, W: int, conn: int) -> int:
    return lib().recon_run(ctx, I, J, H, W, conn)


def recon_run_op(ctx, I: int, J: int, H: int, W: int, conn: int, op: int) -> int:
    return lib().recon_run_op(ctx, I, J, H, W, conn, op)


def recon_batch(ctx, tiles) -> int:
    """tiles: sequence of (I, J, H, W, pitch, conn[, op]) with device addresses."""
    return lib().recon_batch(ctx, _tiles(tiles), len(tiles))


def recon_batch_ex(ctx, tiles, variant=None, order=None) -> int:
    return lib().recon_batch_ex(ctx, _tiles(tiles), len(tiles), _ints(variant), _ints(order))


def recon_run_host(ctx, I: int, J: int, H: int, W: int, conn: int) -> int:
    return lib().recon_run_host(ctx, I, J, H, W, conn)


def recon_batch_host(ctx, tiles) -> int:
    """tiles: sequence of (I, J, H, W, pitch, conn[, op]) with HOST addresses."""
    return lib().recon_batch_host(ctx, _tiles(tiles), len(tiles))


def recon_sync(ctx) -> int:
    return lib().recon_sync(ctx)


def recon_last_error_tile(ctx) -> int:
    return lib().recon_last_error_tile(ctx)


def recon_free(ctx) -> int:
    return lib().recon_free(ctx)


def recon_strerror(status: int) -> str:
    return lib().recon_strerror(status).decode()


def recon_set_param(ctx, key: int, value: int) -> int:
    return lib().recon_set_param(ctx, key, value)


def recon_get_param(ctx, key: int) -> int:
    return lib().recon_get_param(ctx, key)


def recon_get_work(ctx, n: int):
    out = (recon_work * max(n, 1))()
    rc = lib().recon_get_work(ctx, out, n)
    if rc != RECON_OK:
        raise ReconError(rc, "recon_get_work")
    names = ("load", "scan", "seed", "queue", "write", "fetch")
    return [dict(visits=w.visits, scan_rows=w.scan_rows, pops=w.pops, seeds=w.seeds, levels=w.levels,
                 busy_ns=w.busy_ns, phase_ns=dict(zip(names, list(w.phase_ns)))) for w in out[:n]]


def recon_last_kernel_ms(ctx) -> float:
    ms = ctypes.c_float()
    rc = lib().recon_last_kernel_ms(ctx, ctypes.byref(ms))
    if rc != RECON_OK:
        raise ReconError(rc, "recon_last_kernel_ms")
    return ms.value


def check(rc: int, what: str = "") -> None:
    """Raises ReconError unless rc == RECON_OK."""
    if rc != RECON_OK:
        raise ReconError(rc, what)


# ---- learned cost model (device float pointers as ints) ----

def recon_features(ctx, tiles, feat: int) -> int:
    return lib().recon_features(ctx, _tiles(tiles), len(tiles), feat)


def recon_mlp_forward(ctx, theta: int, X: int, n: int, Y: int) -> int:
    return lib().recon_mlp_forward(ctx, theta, X, n, Y)


def recon_mlp_grad(ctx, theta: int, X: int, T: int, idx: int, n: int, grad: int, loss: int) -> int:
    return lib().recon_mlp_grad(ctx, theta, X, T, idx or None, n, grad, loss or None)


def recon_mlp_adam(ctx, theta: int, grad: int, m: int, v: int, t: int, lr: float) -> int:
    return lib().recon_mlp_adam(ctx, theta, grad, m, v, t, lr)


def recon_mlp_train(ctx, theta: int, X: int, T: int, n: int, epochs: int, batch: int, lr: float,
                    seed: int = 0):
    """Returns (status, [mean batch loss per epoch])."""
    losses = (ctypes.c_float * epochs)()
    rc = lib().recon_mlp_train(ctx, theta, X, T, n, epochs, batch, lr, seed, losses)
    return rc, list(losses)


def recon_mlp_train_resume(ctx, theta: int, adam_mv: int, step: int, epoch0: int, X: int, T: int, n: int,
                           epochs: int, batch: int, lr: float, seed: int = 0):
    """Returns (status, step after training, [mean batch loss per epoch])."""
    losses = (ctypes.c_float * epochs)()
    st = ctypes.c_int(step)
    rc = lib().recon_mlp_train_resume(ctx, theta, adam_mv, ctypes.byref(st), epoch0, X, T, n, epochs, batch, lr,
                                      seed, losses)
    return rc, st.value, list(losses)


def recon_sched_set_model(ctx, theta_host: Sequence[float], norm: Sequence[float], variant_a: int,
                          variant_b: int) -> int:
    th = (ctypes.c_float * RECON_MLP_NPARAMS)(*[float(x) for x in theta_host])
    nm = (ctypes.c_float * 4)(*[float(x) for x in norm])
    return lib().recon_sched_set_model(ctx, th, nm, variant_a, variant_b)


def recon_sched_plan_batch(ctx, tiles):
    """Returns (status, variant[n], order[n], pred[2n])."""
    n = len(tiles)
    v = (ctypes.c_int * n)()
    o = (ctypes.c_int * n)()
    p = (ctypes.c_float * (2 * n))()
    rc = lib().recon_sched_plan_batch(ctx, _tiles(tiles), n, v, o, p)
    return rc, list(v), list(o), list(p)


def recon_autotune(ctx, tiles, reps: int = 2):
    """Returns (status, (block_h, bands, scan_pairs, scan_gain)) and installs the best."""
    best = (ctypes.c_int * 4)()
    rc = lib().recon_autotune(ctx, _tiles(tiles), len(tiles), reps, best)
    return rc, tuple(best)


def recon_autotune_cache(ctx):
    """The autotuner's cache: (status, [(bucket, conns, marker_class, bh, bands, k, gain), ...])."""
    n = lib().recon_autotune_cache(ctx, None, 0)
    if n < 0:
        return -n, []
    buf = (ctypes.c_int * max(7 * n, 1))()
    m = lib().recon_autotune_cache(ctx, buf, n)
    return RECON_OK, [tuple(buf[7 * i:7 * i + 7]) for i in range(min(n, m))]


def recon_autotune_cache_load(ctx, entries) -> int:
    flat = [int(x) for e in entries for x in e]
    buf = (ctypes.c_int * max(len(flat), 1))(*flat)
    return lib().recon_autotune_cache_load(ctx, buf, len(entries))


def recon_checks(reset: bool = False):
    """(enabled, failed checks, where-code of the first) of the bounds-checked build."""
    en, viol, first = ctypes.c_int(0), ctypes.c_uint(0), ctypes.c_uint(0)
    st = lib().recon_checks(ctypes.byref(en), ctypes.byref(viol), ctypes.byref(first), 1 if reset else 0)
    if st != 0:
        raise ReconError(RECON_ECUDA, "recon_checks")
    return en.value, viol.value, first.value


def recon_sync_for(ctx, timeout_ms: int) -> int:
    return lib().recon_sync_for(ctx, timeout_ms)


def recon_trace(ctx, n: int):
    out = (ctypes.c_uint * max(n, 1))()
    m = lib().recon_trace(ctx, out, n)
    return list(out[:max(m, 0)])


def recon_run_noalloc(I: int, J: int, H: int, W: int, conn: int, stream: int = 0) -> int:
    """Allocation-free single-tile reconstruction (device pointers; waits)."""
    return lib().recon_run_noalloc(I, J, H, W, conn, ctypes.c_void_p(stream or None))


# ---- tensor-level calls: argument checks, then the C calls above ----

_contexts = {}


def _check_pair(I, J):
    """I and J must be contiguous 2-D uint8 CUDA tensors of one shape on one
    device (the C ABI takes their device addresses, row stride = W)."""
    import torch
    for name, t in (("I", I), ("J", J)):
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch.Tensor" % name)
        if t.dtype != torch.uint8:
            raise TypeError("%s must be uint8, got %s" % (name, t.dtype))
        if t.device.type != "cuda":
            raise ValueError("%s must be a CUDA tensor, got device %s" % (name, t.device))
        if t.dim() != 2:
            raise ValueError("%s must be 2-D (H, W), got shape %s" % (name, tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if I.shape != J.shape or I.device != J.device:
        raise ValueError("I %s on %s and J %s on %s differ in shape or device"
                         % (tuple(I.shape), I.device, tuple(J.shape), J.device))


def context_for(device, stream=None, flags: int = RECON_FLAG_SYNC):
    """A context kept per (device index, stream, flags) for the tensor calls;
    `stream` is a torch.cuda.Stream (None: torch's current stream on that
    device). RECON_FLAG_SYNC makes each call raise on a device error."""
    import torch
    dev = torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    st = stream if stream is not None else torch.cuda.current_stream(idx)
    key = (idx, st.cuda_stream, flags)
    if key not in _contexts:
        _contexts[key] = recon_init(idx, st.cuda_stream, flags)
    return _contexts[key]


def run(I, J, conn: int = 8, op: int = RECON_OP_DILATE, ctx=None):
    """Reconstructs J in place under I (Table II; Algorithm 1 with the hybrid
    scan + queue schedule of Sec. V-C) and returns J. I, J: contiguous uint8
    CUDA tensors of shape (H, W); op: RECON_OP_DILATE (J <= I), RECON_OP_ERODE
    (J >= I) or RECON_OP_FILL_HOLES (J receives FillHoles(I)). Runs on torch's
    current stream unless `ctx` is given; raises ReconError on failure."""
    _check_pair(I, J)
    c = ctx if ctx is not None else context_for(J.device)
    check(recon_run_op(c, I.data_ptr(), J.data_ptr(), int(I.shape[0]), int(I.shape[1]), conn, op), "run")
    return J


def batch(pairs, conn: int = 8, op: int = RECON_OP_DILATE, ctx=None):
    """Reconstructs every (I, J) pair in one persistent launch, each J in place,
    and returns the list of J. Tensors as for run(); tiles may differ in size
    and must not share memory. Raises ReconError (with the failing tile from
    recon_last_error_tile in the message) on failure."""
    pairs = list(pairs)
    if not pairs:
        raise ValueError("batch needs at least one (I, J) pair")
    for I, J in pairs:
        _check_pair(I, J)
    dev = pairs[0][1].device
    if any(J.device != dev for _, J in pairs):
        raise ValueError("all tiles of a batch must be on one device")
    c = ctx if ctx is not None else context_for(dev)
    tiles = [(I.data_ptr(), J.data_ptr(), int(I.shape[0]), int(I.shape[1]), int(I.shape[1]), conn, op)
             for I, J in pairs]
    st = recon_batch(c, tiles)
    if st != RECON_OK:
        raise ReconError(st, "batch (first failing tile %d)" % recon_last_error_tile(c))
    return [J for _, J in pairs]


# ---- device micro-benchmarks (current device, default stream; they wait) ----

def recon_mb_threads(device: int = 0) -> int:
    return lib().recon_mb_threads(device)


def recon_mb_random(matrix: int, log2n: int, ops: int, write: bool, seed: int):
    """Returns (status, checksum or None, ms)."""
    cs = ctypes.c_uint64(0)
    ms = ctypes.c_float(0)
    rc = lib().recon_mb_random(matrix, log2n, ops, 1 if write else 0, seed, ctypes.byref(cs), ctypes.byref(ms))
    return rc, (None if write else cs.value), ms.value


def recon_mb_atomic(counters: int, mode: int, iters: int):
    """Returns (status, ms)."""
    ms = ctypes.c_float(0)
    rc = lib().recon_mb_atomic(counters, mode, iters, ctypes.byref(ms))
    return rc, ms.value


def recon_dt(ctx, B: int, d2: int, site: int, H: int, W: int) -> int:
    """Distance transform (device addresses; site may be 0); waits."""
    return lib().recon_dt(ctx, B, d2, ctypes.c_void_p(site or None), H, W)


def recon_dt_levels(ctx) -> int:
    return lib().recon_dt_levels(ctx)

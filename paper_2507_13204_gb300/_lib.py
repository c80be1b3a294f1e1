"""ctypes binding of libkg.so.

Functions carry the C ABI's names and only marshal arguments: tensors become
device pointers, streams become cudaStream_t handles, statuses become
exceptions.  Every computation happens in the library's CUDA kernels; if the
library is missing this module raises, it never falls back to another path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkg.so")

KG_OK, KG_ERR_INVALID_ARG, KG_ERR_OOM, KG_ERR_CUDA, KG_ERR_BOUNDS, KG_ERR_TIMEOUT, \
    KG_ERR_UNSUPPORTED, KG_ERR_STATE, KG_ERR_RANGE = range(9)
STATUS_NAMES = ["KG_OK", "KG_ERR_INVALID_ARG", "KG_ERR_OOM", "KG_ERR_CUDA", "KG_ERR_BOUNDS",
                "KG_ERR_TIMEOUT", "KG_ERR_UNSUPPORTED", "KG_ERR_STATE", "KG_ERR_RANGE"]
KG_QUADFORM, KG_TETENERGY, KG_LAPLACE1D, KG_SPQUADFORM = 1, 2, 3, 4
KG_F64, KG_F32 = 0, 1
KG_STRATEGY_AUTO, KG_STRATEGY_ATOMIC, KG_STRATEGY_CSR, KG_STRATEGY_TRANSPOSE, KG_STRATEGY_FUSED, \
    KG_STRATEGY_SHARED, KG_STRATEGY_WARP, KG_STRATEGY_TILE = range(8)
KG_MODE_AUTO, KG_MODE_RECOMPUTE, KG_MODE_TAPE = range(3)
KG_ARITH_AUTO, KG_ARITH_NATIVE, KG_ARITH_PAIR = range(3)

# Every symbol include/kg.h declares (checked by the test suite).
EXPORTS = ["kg_options_default", "kg_options_apply_env", "kg_tape_generation", "kg_create", "kg_eval", "kg_grad", "kg_eval_tape",
           "kg_grad_from_tape", "kg_grad_host", "kg_batch_create", "kg_grad_batched",
           "kg_grad_batched_loop", "kg_batch_get_config", "kg_sync", "kg_batch_sync", "kg_last_error",
           "kg_get_config", "kg_workspace_bytes", "kg_last_launch_count", "kg_profile_enable", "kg_profile_read",
           "kg_quadform_grad_noalloc", "kg_hvp", "kg_check_bounded_wait", "kg_measure_box", "kg_destroy", "kg_batch_destroy"]


class kg_options(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("strategy", ctypes.c_int), ("mode", ctypes.c_int),
                ("arith", ctypes.c_int), ("check", ctypes.c_int), ("block", ctypes.c_int),
                ("team", ctypes.c_int), ("tile", ctypes.c_int),
                ("tape_budget_bytes", ctypes.c_size_t)]


class kg_box_rates(ctypes.Structure):
    _fields_ = [("fp64_fma_tflops", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("fp64_red_gops", ctypes.c_double), ("fp32_red_gops", ctypes.c_double),
                ("fp64_log1p_gops", ctypes.c_double), ("fp64_div_gops", ctypes.c_double),
                ("sms", ctypes.c_int), ("l2_bytes", ctypes.c_int),
                ("fp64_gather_gops", ctypes.c_double), ("fp32_gather_gops", ctypes.c_double)]


class KGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


_lock = threading.Lock()
_lib = None


def lib():
    """Opens libkg.so (built by build.build() / __graft_entry__.build())."""
    global _lib
    if _lib is not None:  # opened once; the lock only guards the first open
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "paper_2507_13204_gb300.build.build() (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
            i, st = ctypes.c_int, ctypes.c_int
            optp = ctypes.POINTER(kg_options)
            vpp = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "kg_options_default": (None, [optp]),
                "kg_options_apply_env": (st, [optp]),
                "kg_tape_generation": (st, [vp, ctypes.POINTER(ctypes.c_uint64)]),
                "kg_create": (st, [ctypes.POINTER(vp), i, i64p, i, vpp, i, optp, vp]),
                "kg_eval": (st, [vp, vp, vp, vp]),
                "kg_grad": (st, [vp, vp, vp, vp, vp, vp, i, vp]),
                "kg_eval_tape": (st, [vp, vp, vp, vp]),
                "kg_grad_from_tape": (st, [vp, vp, vp, i, vp]),
                "kg_hvp": (st, [vp, vp, vp, vp, vp, i, vp]),
                "kg_grad_host": (st, [vp, vp, vp, vp, vp]),
                "kg_batch_create": (st, [ctypes.POINTER(vp), vpp, i, optp, vp]),
                "kg_grad_batched": (st, [vp, vpp, vpp, vpp, vp]),
                "kg_grad_batched_loop": (st, [vp, vpp, vpp, vpp, vp]),
                "kg_batch_get_config": (st, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
                "kg_sync": (st, [vp]),
                "kg_batch_sync": (st, [vp]),
                "kg_last_error": (ctypes.c_char_p, []),
                "kg_get_config": (st, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
                "kg_workspace_bytes": (ctypes.c_size_t, [vp]),
                "kg_last_launch_count": (i, []),
                "kg_profile_enable": (st, [i]),
                "kg_profile_read": (st, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_char_p)]),
                "kg_quadform_grad_noalloc": (st, [vp, ctypes.c_int64, ctypes.c_int64, vp, vp, vp, vp]),
                "kg_check_bounded_wait": (st, [vp, ctypes.c_uint64, vp]),
                "kg_measure_box": (st, [ctypes.POINTER(kg_box_rates), vp]),
                "kg_destroy": (None, [vp]),
                "kg_batch_destroy": (None, [vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def ptr(t) -> int | None:
    """Device (or host) address of a tensor / numpy array / int; None stays NULL."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


_current_stream = None  # () -> raw cudaStream_t of torch's current stream, or None


def _current_stream_fn():
    import torch
    if not torch.cuda.is_available():
        return lambda: None
    raw, dev = getattr(torch._C, "_cuda_getCurrentRawStream", None), getattr(torch._C, "_cuda_getDevice", None)
    if raw is not None and dev is not None:  # a few microseconds less a call than current_stream()
        return lambda: raw(dev())
    return lambda: torch.cuda.current_stream().cuda_stream


def stream_handle(stream) -> int | None:
    """None: torch's current stream on the current device."""
    global _current_stream
    if stream is None:
        if _current_stream is None:
            _current_stream = _current_stream_fn()
        return _current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def check(status: int, where: str):
    if status != KG_OK:
        raise KGError(status, where, lib().kg_last_error().decode())


def options(dtype=KG_F64, strategy=KG_STRATEGY_AUTO, mode=KG_MODE_AUTO, arith=KG_ARITH_AUTO,
            check=0, block=0, team=0, tile=0, tape_budget_bytes=0) -> kg_options:
    o = kg_options()
    lib().kg_options_default(ctypes.byref(o))
    o.dtype, o.strategy, o.mode, o.arith = dtype, strategy, mode, arith
    o.check, o.block, o.team, o.tile = check, block, team, tile
    o.tape_budget_bytes = tape_budget_bytes
    return o


# ---------------------------------------------------------------- C names
def kg_create(kind: int, sizes, data, opt: kg_options | None = None, stream=None) -> int:
    h = ctypes.c_void_p()
    sz = (ctypes.c_int64 * len(sizes))(*[int(s) for s in sizes])
    dp = (ctypes.c_void_p * len(data))(*[ptr(d) for d in data])
    check(lib().kg_create(ctypes.byref(h), kind, sz, len(sizes), dp, len(data),
                          ctypes.byref(opt) if opt is not None else None, stream_handle(stream)),
          "kg_create")
    return h.value


def kg_eval(h, x, f, stream=None):
    check(lib().kg_eval(h, ptr(x), ptr(f), stream_handle(stream)), "kg_eval")


def kg_grad(h, x, f, gx, gdata=None, seed=None, accumulate=0, stream=None):
    check(lib().kg_grad(h, ptr(x), ptr(f), ptr(gx), ptr(gdata), ptr(seed), int(accumulate),
                        stream_handle(stream)), "kg_grad")


def kg_hvp(h, x, v, hv, seed=None, accumulate=0, stream=None):
    check(lib().kg_hvp(h, ptr(x), ptr(v), ptr(hv), ptr(seed), int(accumulate), stream_handle(stream)),
          "kg_hvp")


def kg_eval_tape(h, x, f=None, stream=None):
    check(lib().kg_eval_tape(h, ptr(x), ptr(f), stream_handle(stream)), "kg_eval_tape")


def kg_options_apply_env(opt: kg_options) -> kg_options:
    check(lib().kg_options_apply_env(ctypes.byref(opt)), "kg_options_apply_env")
    return opt


def kg_tape_generation(h) -> int:
    g = ctypes.c_uint64()
    check(lib().kg_tape_generation(h, ctypes.byref(g)), "kg_tape_generation")
    return g.value


def kg_measure_box(stream=None) -> dict:
    """FP64/FP32 FMA and red rates, SM count and L2 size of the current GPU."""
    r = kg_box_rates()
    check(lib().kg_measure_box(ctypes.byref(r), stream_handle(stream)), "kg_measure_box")
    return {k: getattr(r, k) for k, _ in kg_box_rates._fields_}


def kg_check_bounded_wait(h, limit_ns: int, stream=None):
    check(lib().kg_check_bounded_wait(h, int(limit_ns), stream_handle(stream)), "kg_check_bounded_wait")


def kg_grad_from_tape(h, gx, seed=None, accumulate=0, stream=None):
    check(lib().kg_grad_from_tape(h, ptr(gx), ptr(seed), int(accumulate), stream_handle(stream)),
          "kg_grad_from_tape")


def kg_grad_host(h, x_host, f_host, gx_host, stream=None):
    check(lib().kg_grad_host(h, ptr(x_host), ptr(f_host), ptr(gx_host), stream_handle(stream)),
          "kg_grad_host")


def _table(items):
    """ctypes array of the items' addresses (an array passes through as is)."""
    if isinstance(items, ctypes.Array):
        return items
    return (ctypes.c_void_p * len(items))(*[ptr(t) for t in items])


def kg_batch_create(problems, opt: kg_options | None = None, stream=None) -> int:
    h = ctypes.c_void_p()
    tab = (ctypes.c_void_p * len(problems))(*problems)
    check(lib().kg_batch_create(ctypes.byref(h), tab, len(problems),
                                ctypes.byref(opt) if opt is not None else None,
                                stream_handle(stream)), "kg_batch_create")
    return h.value


def kg_grad_batched(b, xs, fs, gxs, stream=None):
    check(lib().kg_grad_batched(b, _table(xs), _table(fs), _table(gxs), stream_handle(stream)),
          "kg_grad_batched")


def kg_grad_batched_loop(b, xs, fs, gxs, stream=None):
    check(lib().kg_grad_batched_loop(b, _table(xs), _table(fs), _table(gxs), stream_handle(stream)),
          "kg_grad_batched_loop")


def kg_batch_get_config(b):
    """(arith name, work items, persistent grid) of a batch."""
    a, n, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().kg_batch_get_config(b, ctypes.byref(a), ctypes.byref(n), ctypes.byref(g)),
          "kg_batch_get_config")
    return ["auto", "native", "pair"][a.value], n.value, g.value


def kg_sync(h):
    check(lib().kg_sync(h), "kg_sync")


def kg_batch_sync(b):
    check(lib().kg_batch_sync(b), "kg_batch_sync")


def kg_last_error() -> str:
    return lib().kg_last_error().decode()


def kg_get_config(h):
    """Resolved (strategy, mode, arith) names of a problem."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().kg_get_config(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "kg_get_config")
    strat = ["auto", "atomic", "csr", "transpose", "fused", "shared", "warp", "tile"][a.value]
    return strat, ["auto", "recompute", "tape"][b.value], ["auto", "native", "pair"][c.value]


def kg_workspace_bytes(h) -> int:
    return int(lib().kg_workspace_bytes(h))


def kg_last_launch_count() -> int:
    return int(lib().kg_last_launch_count())


def kg_profile_enable(on: bool):
    check(lib().kg_profile_enable(int(bool(on))), "kg_profile_enable")


def kg_profile_read():
    """Returns (summed main-kernel milliseconds, bracketed launches, kernel name)."""
    ms, n, name = ctypes.c_double(), ctypes.c_int(), ctypes.c_char_p()
    check(lib().kg_profile_read(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(name)),
          "kg_profile_read")
    return ms.value, n.value, (name.value or b"").decode()


def kg_destroy(h):
    if h:
        lib().kg_destroy(h)


def kg_batch_destroy(b):
    if b:
        lib().kg_batch_destroy(b)

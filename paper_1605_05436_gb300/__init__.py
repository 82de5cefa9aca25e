"""GB300 exact floating-point summation.

Goodrich & Eldawy, "Parallel Algorithms for Summing Floating-Point Numbers"
(arXiv:1605.05436): reduce n IEEE values to their exact sum in a carry-free
superaccumulator, then round once.

This module is the thin Python binding of ``libexactsum.so`` (the C ABI in
``include/exactsum.h``).  The functions named ``exactsum_*`` mirror the C
entry points one to one and only marshal arguments; every step of the
summation runs in the library's CUDA kernels.  The torch helpers at the end
(``exact_sum`` and friends) take tensors, pass their device pointers and the
current CUDA stream, and allocate result tensors -- PyTorch supplies memory
and streams only.

There is no CPU fallback: if the library is not built, or no sm_103 GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libexactsum.so")

F64, F32, BF16 = 0, 1, 2
RNE, RTZ, RUP, RDOWN = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, 1, 2, 3, 4, 5
ACC_WORDS = 80
ACC_BYTES = 8 * ACC_WORDS
ITEMSIZE = {F64: 8, F32: 4, BF16: 2}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int

# name -> (argtypes); every entry point returns an int status except
# exactsum_last_error.
_SIGNATURES = {
    "exactsum_create": [ctypes.POINTER(_vp), _int, _i64],
    "exactsum_destroy": [_vp],
    "exactsum_sum": [_vp, _vp, _i64, _int, _int, _int, _vp, _vp],
    "exactsum_sum_host": [_vp, _vp, _i64, _int, _int, _int, _vp, _vp],
    "exactsum_sum_adaptive": [_vp, _vp, _i64, _int, _int, _int, _vp, ctypes.POINTER(_int),
                              ctypes.POINTER(_int), _vp],
    "exactsum_acc_zero": [_vp, _vp, _vp],
    "exactsum_acc_add": [_vp, _vp, _i64, _int, _vp, _vp],
    "exactsum_acc_round": [_vp, _vp, _int, _int, _int, _vp, _vp],
    "exactsum_segmented_sum": [_vp, _vp, _vp, _i64, _int, _int, _int, _vp, _vp],
    "exactsum_sum_each": [_vp, _vp, _vp, _i64, _int, _int, _int, _vp, _vp],
    "exactsum_segmented_autotune": [_vp, _vp, _vp, _i64, _int, _vp, _vp, ctypes.POINTER(_int),
                                    ctypes.POINTER(_int), ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_float)],
    "exactsum_tuning_save": [_vp, ctypes.c_char_p],
    "exactsum_tuning_load": [_vp, ctypes.c_char_p],
    "exactsum_device_status": [_vp, ctypes.POINTER(_i64)],
    "exactsum_server_create": [ctypes.POINTER(_vp), _int, _int, _i64, _i64, _i64, _int],
    "exactsum_server_submit": [_vp, _vp, _i64, _int, _int, _int, _int, ctypes.POINTER(ctypes.c_uint64)],
    "exactsum_server_poll": [_vp, _vp, _int, ctypes.POINTER(_int)],
    "exactsum_server_drain": [_vp, _i64],
    "exactsum_server_set_lanes": [_vp, _i64, _int, _int],
    "exactsum_server_stats": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "exactsum_server_destroy": [_vp],
    "exactsum_segmented_sum_noalloc": [_vp, _vp, _i64, _int, _int, _int, _vp, _vp],
    "exactsum_check_timeout": [_vp, ctypes.c_uint32, _vp, _vp],
}
OPTIONAL_SIGNATURES: dict = {}

_lock = threading.Lock()
_lib = None


class ExactSumError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"exactsum status {status}: {message}")
        self.status = status


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


def library() -> ctypes.CDLL:
    """Load ``libexactsum.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                                   "(paper_1605_05436_gb300.build())")
            # load the CUDA runtime through torch first when available, so that
            # the library and torch share one runtime instance
            try:
                import torch  # noqa: F401
            except ImportError:
                pass
            lib = ctypes.CDLL(LIB_PATH)
            for name, argtypes in {**_SIGNATURES, **OPTIONAL_SIGNATURES}.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    if name in _SIGNATURES:
                        raise RuntimeError(f"{LIB_PATH} does not export {name}")
                    continue
                fn.argtypes = argtypes
                fn.restype = _int
            lib.exactsum_last_error.argtypes = [_vp]
            lib.exactsum_last_error.restype = ctypes.c_char_p
            lib.exactsum_server_last_error.argtypes = [_vp]
            lib.exactsum_server_last_error.restype = ctypes.c_char_p
            lib.exactsum_server_clock_ns.argtypes = []
            lib.exactsum_server_clock_ns.restype = _i64
            _lib = lib
    return _lib


def _check(status: int, handle) -> None:
    if status != OK:
        msg = library().exactsum_last_error(handle)
        raise ExactSumError(status, msg.decode(errors="replace") if msg else "")


# ---------------------------------------------------------------------------
# C entry points (same names and argument order as include/exactsum.h)
# ---------------------------------------------------------------------------

def exactsum_create(device: int = 0, max_segments_hint: int = 0) -> int:
    h = _vp()
    _check(library().exactsum_create(ctypes.byref(h), device, max_segments_hint), None)
    return h.value


def exactsum_destroy(handle: int) -> None:
    _check(library().exactsum_destroy(handle), handle)


def exactsum_last_error(handle) -> str:
    return library().exactsum_last_error(handle).decode(errors="replace")


def exactsum_sum(handle, d_x, n, in_dtype, out_dtype, mode, d_result, stream) -> None:
    _check(library().exactsum_sum(handle, d_x, n, in_dtype, out_dtype, mode, d_result, stream), handle)


def exactsum_sum_host(handle, h_x, n, in_dtype, out_dtype, mode, h_result, stream) -> None:
    _check(library().exactsum_sum_host(handle, h_x, n, in_dtype, out_dtype, mode, h_result, stream),
           handle)


def exactsum_sum_adaptive(handle, d_x, n, in_dtype, out_dtype, mode, d_result, stream) -> tuple:
    """Returns (passes, last_r) (last_r 0 when the exact kernel ran)."""
    passes, last_r = _int(0), _int(0)
    _check(library().exactsum_sum_adaptive(handle, d_x, n, in_dtype, out_dtype, mode, d_result,
                                           ctypes.byref(passes), ctypes.byref(last_r), stream), handle)
    return passes.value, last_r.value


def exactsum_acc_zero(handle, d_acc, stream) -> None:
    _check(library().exactsum_acc_zero(handle, d_acc, stream), handle)


def exactsum_acc_add(handle, d_x, n, in_dtype, d_acc, stream) -> None:
    _check(library().exactsum_acc_add(handle, d_x, n, in_dtype, d_acc, stream), handle)


def exactsum_acc_round(handle, d_acc, in_dtype, out_dtype, mode, d_result, stream) -> None:
    _check(library().exactsum_acc_round(handle, d_acc, in_dtype, out_dtype, mode, d_result, stream),
           handle)


def exactsum_segmented_sum(handle, d_x, d_offsets, num_segments, in_dtype, out_dtype, mode, d_results,
                           stream) -> None:
    _check(library().exactsum_segmented_sum(handle, d_x, d_offsets, num_segments, in_dtype, out_dtype,
                                            mode, d_results, stream), handle)


def exactsum_sum_each(handle, d_x, h_offsets, num_segments, in_dtype, out_dtype, mode, d_results,
                      stream) -> None:
    _check(library().exactsum_sum_each(handle, d_x, h_offsets, num_segments, in_dtype, out_dtype, mode,
                                       d_results, stream), handle)


def exactsum_segmented_autotune(handle, d_x, d_offsets, num_segments, in_dtype, d_results_scratch,
                                stream):
    """Returns (warps, kind, tile, ms) of the fastest reducer configuration
    (kind 0: register streaming, 1: TMA ring, 2: windowed)."""
    w, k, t, ms = _int(0), _int(0), _i64(0), ctypes.c_float(0)
    _check(library().exactsum_segmented_autotune(handle, d_x, d_offsets, num_segments, in_dtype,
                                                 d_results_scratch, stream, ctypes.byref(w), ctypes.byref(k),
                                                 ctypes.byref(t), ctypes.byref(ms)), handle)
    return w.value, k.value, t.value, ms.value


def exactsum_tuning_save(handle, path: str) -> None:
    _check(library().exactsum_tuning_save(handle, path.encode()), handle)


def exactsum_tuning_load(handle, path: str) -> None:
    _check(library().exactsum_tuning_load(handle, path.encode()), handle)


def exactsum_device_status(handle) -> int:
    v = _i64(0)
    _check(library().exactsum_device_status(handle, ctypes.byref(v)), handle)
    return v.value


STATUS_BAD_OFFSETS, STATUS_MAP_OVERFLOW, STATUS_TIMEOUT = 1, 2, 4


def exactsum_check_timeout(handle, polls, d_elapsed_ns, stream) -> None:
    """Run one bounded wait that is never satisfied (the kernels' timeout
    path); afterwards exactsum_device_status reports STATUS_TIMEOUT."""
    _check(library().exactsum_check_timeout(handle, polls, d_elapsed_ns, stream), handle)
NOALLOC_MAX_SEGMENTS = 2048


def exactsum_segmented_sum_noalloc(d_x, d_offsets, num_segments, in_dtype, out_dtype, mode, d_results,
                                   stream) -> None:
    """Segmented sum that allocates nothing (fixed scratch inside the
    library; at most NOALLOC_MAX_SEGMENTS segments; overlapping calls race)."""
    _check(library().exactsum_segmented_sum_noalloc(d_x, d_offsets, num_segments, in_dtype, out_dtype, mode,
                                                    d_results, stream), None)


class exactsum_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
                ("result_bits", ctypes.c_uint64), ("n", ctypes.c_int64), ("submit_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


def _check_server(status: int, server) -> None:
    if status != OK:
        msg = library().exactsum_server_last_error(server) if server else b"invalid argument"
        raise ExactSumError(status, msg.decode(errors="replace") if msg else "")


def exactsum_server_create(device: int, max_slots: int, mem_budget_bytes: int, chunk_elems: int,
                           tile_elems: int, max_steps_per_request: int = 0) -> int:
    h = _vp()
    _check_server(library().exactsum_server_create(ctypes.byref(h), device, max_slots, mem_budget_bytes,
                                                   chunk_elems, tile_elems, max_steps_per_request), None)
    return h.value


def exactsum_server_submit(server, x, n, in_dtype, out_dtype, mode, x_on_host) -> int:
    rid = ctypes.c_uint64(0)
    _check_server(library().exactsum_server_submit(server, x, n, in_dtype, out_dtype, mode, x_on_host,
                                                   ctypes.byref(rid)), server)
    return rid.value


def exactsum_server_poll(server, max_out: int = 4096) -> list:
    buf = (exactsum_completion * max_out)()
    cnt = _int(0)
    _check_server(library().exactsum_server_poll(server, buf, max_out, ctypes.byref(cnt)), server)
    return [buf[i] for i in range(cnt.value)]


def exactsum_server_set_lanes(server, express_max_bytes: int, express_sms: int, resident: int = 1) -> None:
    """Bulk/express lane split (before the first submission); express_max_bytes
    < 0 sends every request to the express lane; resident 1: the express lane
    is a resident kernel fed from a host ring, 0: continuous-batching steps."""
    _check_server(library().exactsum_server_set_lanes(server, express_max_bytes, express_sms, resident), server)


def exactsum_server_drain(server, timeout_ms: int) -> None:
    _check_server(library().exactsum_server_drain(server, timeout_ms), server)


def exactsum_server_stats(server):
    a, b, c = _i64(0), _i64(0), _i64(0)
    _check_server(library().exactsum_server_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                  server)
    return {"steps": a.value, "peak_active": b.value, "outstanding": c.value}


def exactsum_server_clock_ns() -> int:
    return library().exactsum_server_clock_ns()


def exactsum_server_last_error(server) -> str:
    return library().exactsum_server_last_error(server).decode(errors="replace")


def exactsum_server_destroy(server) -> None:
    _check_server(library().exactsum_server_destroy(server), server)


# ---------------------------------------------------------------------------
# torch helpers (memory and streams only)
# ---------------------------------------------------------------------------
_handles: dict = {}


def handle_for(device: int):
    """A cached library handle for a CUDA device index."""
    with _lock:
        h = _handles.get(device)
    if h is None:
        h = exactsum_create(device, 0)
        with _lock:
            _handles[device] = h
    return h


def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    """Input format of a tensor: float64/float32/bfloat16, or raw IEEE bits
    held in int64/uint64 (FP64), int32/uint32 (FP32), int16/uint16 (BF16)."""
    torch = _torch()
    m = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16,
         torch.int64: F64, torch.int32: F32, torch.int16: BF16}
    for name, code in (("uint64", F64), ("uint32", F32), ("uint16", BF16)):
        if hasattr(torch, name):
            m[getattr(torch, name)] = code
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def result_tensor(out_dtype: int, device, count: int = 1):
    torch = _torch()
    td = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[out_dtype]
    return torch.empty(count, dtype=td, device=device)


def _stream_ptr(stream, device):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def exact_sum(x, out_dtype: int | None = None, mode: int = RNE, stream=None, out=None):
    """Exact sum of a contiguous CUDA tensor, rounded once; returns a
    one-element tensor of the output format (float64/float32/bfloat16)."""
    if not x.is_cuda:
        raise ValueError("exact_sum takes a CUDA tensor (use exact_sum_host for host memory)")
    if not x.is_contiguous():
        raise ValueError("input must be contiguous")
    in_dtype = dtype_code(x)
    out_dtype = in_dtype if out_dtype is None else out_dtype
    dev = x.device.index
    if out is None:
        out = result_tensor(out_dtype, x.device)
    exactsum_sum(handle_for(dev), x.data_ptr() if x.numel() else None, x.numel(), in_dtype,
                 out_dtype, mode, out.data_ptr(), _stream_ptr(stream, dev))
    return out


def adaptive_sum(x, out_dtype: int | None = None, mode: int = RNE, stream=None, out=None):
    """The condition-number-sensitive sum of a contiguous CUDA tensor (the
    same correctly rounded result as exact_sum); returns (result tensor,
    passes, last_r)."""
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("adaptive_sum takes a contiguous CUDA tensor")
    in_dtype = dtype_code(x)
    out_dtype = in_dtype if out_dtype is None else out_dtype
    dev = x.device.index
    if out is None:
        out = result_tensor(out_dtype, x.device)
    passes, last_r = exactsum_sum_adaptive(handle_for(dev), x.data_ptr() if x.numel() else None, x.numel(),
                                           in_dtype, out_dtype, mode, out.data_ptr(), _stream_ptr(stream, dev))
    return out, passes, last_r


def exact_sum_host(x, out_dtype: int | None = None, mode: int = RNE, device: int = 0, stream=None):
    """End to end from host memory (a CPU tensor, ideally pinned): returns the
    result's raw bits as a Python int after the stream has finished."""
    if x.is_cuda or not x.is_contiguous():
        raise ValueError("exact_sum_host takes a contiguous CPU tensor")
    in_dtype = dtype_code(x)
    out_dtype = in_dtype if out_dtype is None else out_dtype
    res = ctypes.c_uint64(0)
    exactsum_sum_host(handle_for(device), x.data_ptr() if x.numel() else None, x.numel(), in_dtype,
                      out_dtype, mode, ctypes.addressof(res), _stream_ptr(stream, device))
    return res.value & ((1 << (8 * ITEMSIZE[out_dtype])) - 1)


def new_accumulator(device):
    """A zeroed device accumulator (EXACTSUM_ACC_WORDS int64 words)."""
    torch = _torch()
    return torch.zeros(ACC_WORDS, dtype=torch.int64, device=device)


def acc_add(acc, x, stream=None):
    in_dtype = dtype_code(x)
    dev = x.device.index
    exactsum_acc_add(handle_for(dev), x.data_ptr() if x.numel() else None, x.numel(), in_dtype,
                     acc.data_ptr(), _stream_ptr(stream, dev))
    return acc


def acc_round(acc, in_dtype: int, out_dtype: int | None = None, mode: int = RNE, stream=None):
    out_dtype = in_dtype if out_dtype is None else out_dtype
    dev = acc.device.index
    out = result_tensor(out_dtype, acc.device)
    exactsum_acc_round(handle_for(dev), acc.data_ptr(), in_dtype, out_dtype, mode, out.data_ptr(),
                       _stream_ptr(stream, dev))
    return out


def segmented_sum(x, offsets, out_dtype: int | None = None, mode: int = RNE, stream=None, out=None):
    """Exact sums of CSR segments: ``offsets`` is an int64 CUDA tensor of
    S + 1 entries; returns S results of the output format."""
    if not (x.is_cuda and offsets.is_cuda):
        raise ValueError("segmented_sum takes CUDA tensors")
    torch = _torch()
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous int64 tensor")
    in_dtype = dtype_code(x)
    out_dtype = in_dtype if out_dtype is None else out_dtype
    S = offsets.numel() - 1
    dev = x.device.index
    if out is None:
        out = result_tensor(out_dtype, x.device, max(S, 0))
    exactsum_segmented_sum(handle_for(dev), x.data_ptr() if x.numel() else None, offsets.data_ptr(), S,
                           in_dtype, out_dtype, mode, out.data_ptr() if S > 0 else None,
                           _stream_ptr(stream, dev))
    return out


def sum_each(x, offsets_host, out_dtype: int | None = None, mode: int = RNE, stream=None, out=None):
    """One exactsum_sum launch per segment (host int64 offsets): the baseline."""
    torch = _torch()
    off = offsets_host.to(torch.int64).contiguous()
    in_dtype = dtype_code(x)
    out_dtype = in_dtype if out_dtype is None else out_dtype
    S = off.numel() - 1
    dev = x.device.index
    if out is None:
        out = result_tensor(out_dtype, x.device, max(S, 0))
    exactsum_sum_each(handle_for(dev), x.data_ptr() if x.numel() else None, off.data_ptr(), S, in_dtype,
                      out_dtype, mode, out.data_ptr() if S > 0 else None, _stream_ptr(stream, dev))
    return out

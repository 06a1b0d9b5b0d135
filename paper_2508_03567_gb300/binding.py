"""Python binding of the C ABI in include/nbldpc.h (argument marshalling only).

Functions carry the C names.  Device buffers are torch CUDA tensors (PyTorch
supplies memory and streams); every decode step runs in the library's CUDA
kernels.  There is no CPU fallback: if libnbldpc.so is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbldpc.so")

NBLDPC_OK = 0
NBLDPC_ERR_ARG = -1
NBLDPC_ERR_POLY = -2
NBLDPC_ERR_H = -3
NBLDPC_ERR_CUDA = -4
NBLDPC_ERR_NOMEM = -5
NBLDPC_ERR_TIMEOUT = -6
NBLDPC_ERR_UNSUPPORTED = -7

EXPORTED = ("nbldpc_code_create", "nbldpc_code_destroy", "nbldpc_code_info",
            "nbldpc_decode_workspace_size", "nbldpc_decode", "nbldpc_decode_host_workspace_size",
            "nbldpc_decode_host", "nbldpc_decode_batch_workspace_size", "nbldpc_decode_batch",
            "nbldpc_code_get_tuning", "nbldpc_code_set_tuning", "nbldpc_code_autotune_workspace_size",
            "nbldpc_code_autotune", "nbldpc_code_set_message_bits", "nbldpc_code_get_message_bits",
            "nbldpc_code_set_cnp_schedule", "nbldpc_code_get_cnp_schedule", "nbldpc_code_set_work_counter",
            "nbldpc_fftspa_workspace_size", "nbldpc_fftspa_decode",
            "nbldpc_fftspa_decode_host_workspace_size", "nbldpc_fftspa_decode_host",
            "nbldpc_server_create", "nbldpc_server_create_custom", "nbldpc_server_submit", "nbldpc_server_poll",
            "nbldpc_server_stats_get", "nbldpc_server_destroy",
            "nbldpc_decode_noalloc", "nbldpc_kernel_launch_count", "nbldpc_probe_minmax",
            "nbldpc_status_string")

NBLDPC_MAX_BATCH_JOBS = 32
NBLDPC_CNP_MINIMAL = 0
NBLDPC_CNP_TABLE1 = 1


class nbldpc_job(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("gamma_dev", ctypes.c_void_p), ("frames", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("early_stop", ctypes.c_int), ("out_sym_dev", ctypes.c_void_p),
                ("out_iters_dev", ctypes.c_void_p), ("out_ok_dev", ctypes.c_void_p)]


class nbldpc_tune_result(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("frames_per_block", ctypes.c_int), ("ms", ctypes.c_float)]

_lib = None
_lock = threading.Lock()


class nbldpc_request(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("gamma_host", ctypes.c_void_p), ("frames", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("early_stop", ctypes.c_int), ("out_sym_host", ctypes.c_void_p),
                ("out_iters_host", ctypes.c_void_p), ("out_ok_host", ctypes.c_void_p), ("user", ctypes.c_void_p),
                ("id", ctypes.c_uint64)]


_REQP = ctypes.POINTER(nbldpc_request)
REQUEST_BYTES_FN = ctypes.CFUNCTYPE(ctypes.c_size_t, ctypes.c_void_p, _REQP)
LAUNCH_BYTES_FN = ctypes.CFUNCTYPE(ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(_REQP), ctypes.c_int, ctypes.c_int)
START_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(_REQP), ctypes.c_int, ctypes.c_int,
                            ctypes.c_int, ctypes.POINTER(ctypes.c_uint64))
TOKEN_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64)


class nbldpc_server_executor(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("request_bytes", REQUEST_BYTES_FN), ("launch_bytes", LAUNCH_BYTES_FN),
                ("start", START_FN), ("done", TOKEN_FN), ("finish", TOKEN_FN)]


class nbldpc_server_stats(ctypes.Structure):
    _fields_ = [("used_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t), ("launches", ctypes.c_uint64),
                ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("waiting", ctypes.c_int),
                ("admitted", ctypes.c_int), ("in_flight", ctypes.c_int)]


class NbldpcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {nbldpc_status_string(status)} ({status})")


def lib() -> ctypes.CDLL:
    """Load libnbldpc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA decoder library not built: {LIB_PATH} is missing "
                                   "(run paper_2508_03567_gb300.build.build_library())")
            L = ctypes.CDLL(LIB_PATH)
            vp, sz = ctypes.c_void_p, ctypes.c_size_t
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.nbldpc_code_create.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                             i32p, i32p, ctypes.POINTER(ctypes.c_uint8),
                                             ctypes.POINTER(vp)]
            L.nbldpc_code_destroy.argtypes = [vp]
            L.nbldpc_code_destroy.restype = None
            L.nbldpc_code_info.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 4
            L.nbldpc_decode_workspace_size.argtypes = [vp, ctypes.c_int, ctypes.POINTER(sz)]
            L.nbldpc_decode.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                        vp, sz, vp]
            L.nbldpc_decode_host_workspace_size.argtypes = [vp, ctypes.c_int, ctypes.POINTER(sz)]
            L.nbldpc_decode_host.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                             vp, ctypes.c_int, vp, sz, vp]
            L.nbldpc_decode_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                                vp, vp]
            jp = ctypes.POINTER(nbldpc_job)
            ip = ctypes.POINTER(ctypes.c_int)
            L.nbldpc_decode_batch_workspace_size.argtypes = [jp, ctypes.c_int, ctypes.POINTER(sz)]
            L.nbldpc_decode_batch.argtypes = [jp, ctypes.c_int, vp, sz, vp]
            L.nbldpc_code_get_tuning.argtypes = [vp, ip, ip]
            L.nbldpc_code_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.nbldpc_code_set_message_bits.argtypes = [vp, ctypes.c_int]
            L.nbldpc_code_get_message_bits.argtypes = [vp, ip]
            L.nbldpc_code_set_cnp_schedule.argtypes = [vp, ctypes.c_int]
            L.nbldpc_code_get_cnp_schedule.argtypes = [vp, ip]
            L.nbldpc_code_set_work_counter.argtypes = [vp, vp]
            L.nbldpc_fftspa_workspace_size.argtypes = [vp, ctypes.c_int, ctypes.POINTER(sz)]
            L.nbldpc_fftspa_decode.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                               vp, sz, vp]
            L.nbldpc_fftspa_decode_host_workspace_size.argtypes = [vp, ctypes.c_int, ctypes.POINTER(sz)]
            L.nbldpc_fftspa_decode_host.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                                    ctypes.c_int, vp, sz, vp]
            srvp = ctypes.POINTER(ctypes.c_void_p)
            L.nbldpc_server_create.argtypes = [sz, ctypes.c_int, ctypes.c_int, ctypes.c_int, srvp]
            L.nbldpc_server_create_custom.argtypes = [ctypes.POINTER(nbldpc_server_executor), sz, ctypes.c_int,
                                                      ctypes.c_int, ctypes.c_int, srvp]
            L.nbldpc_server_submit.argtypes = [vp, ctypes.POINTER(nbldpc_request), ctypes.POINTER(ctypes.c_uint64)]
            L.nbldpc_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ip]
            L.nbldpc_server_stats_get.argtypes = [vp, ctypes.POINTER(nbldpc_server_stats)]
            L.nbldpc_server_destroy.argtypes = [vp]
            L.nbldpc_server_destroy.restype = None
            L.nbldpc_code_autotune_workspace_size.argtypes = [vp, ctypes.c_int, ctypes.POINTER(sz)]
            L.nbldpc_code_autotune.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, sz, vp,
                                               ctypes.POINTER(nbldpc_tune_result), ctypes.c_int, ip]
            L.nbldpc_probe_minmax.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double),
                                              ip, vp]
            L.nbldpc_kernel_launch_count.argtypes = []
            L.nbldpc_kernel_launch_count.restype = ctypes.c_uint64
            L.nbldpc_status_string.argtypes = [ctypes.c_int]
            L.nbldpc_status_string.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(st: int, what: str) -> None:
    if st != NBLDPC_OK:
        raise NbldpcError(st, what)


def nbldpc_status_string(status: int) -> str:
    return lib().nbldpc_status_string(int(status)).decode()


def nbldpc_kernel_launch_count() -> int:
    return int(lib().nbldpc_kernel_launch_count())


NBLDPC_PROBE_ALU = 0
NBLDPC_PROBE_FMA_1_8 = 1
NBLDPC_PROBE_FMA_3_8 = 2
NBLDPC_PROBE_FMA_4_8 = 3
NBLDPC_PROBE_FMA_3_8_SHFL = 4
NBLDPC_PROBE_CONV_64 = 5
NBLDPC_PROBE_CONV_256 = 6


def nbldpc_probe_minmax(form: int, rounds: int, sink, stream=None):
    """Queue one min/max throughput probe launch; returns (min-max pairs of the launch, grid blocks)."""
    pairs, blocks = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(lib().nbldpc_probe_minmax(int(form), int(rounds), ctypes.c_void_p(_ptr(sink)), ctypes.byref(pairs),
                                     ctypes.byref(blocks), ctypes.c_void_p(_stream_ptr(stream))),
           "nbldpc_probe_minmax")
    return pairs.value, blocks.value


def nbldpc_code_create(q: int, prim_poly: int, n_cols: int, n_rows: int, row_ptr, col_idx, coef) -> int:
    """Handle (int) for H in CSR form; raises NbldpcError on a rejected code."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    cf = np.ascontiguousarray(coef, dtype=np.uint8)
    h = ctypes.c_void_p()
    st = lib().nbldpc_code_create(int(q), int(prim_poly), int(n_cols), int(n_rows),
                                  rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  cf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(h))
    _check(st, "nbldpc_code_create")
    return h.value


def nbldpc_code_destroy(handle: int) -> None:
    lib().nbldpc_code_destroy(handle)


def nbldpc_code_info(handle: int):
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().nbldpc_code_info(handle, *[ctypes.byref(x) for x in v]), "nbldpc_code_info")
    return tuple(x.value for x in v)


def nbldpc_decode_workspace_size(handle: int, frames: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nbldpc_decode_workspace_size(handle, int(frames), ctypes.byref(b)),
           "nbldpc_decode_workspace_size")
    return b.value


def nbldpc_decode_host_workspace_size(handle: int, chunk_frames: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nbldpc_decode_host_workspace_size(handle, int(chunk_frames), ctypes.byref(b)),
           "nbldpc_decode_host_workspace_size")
    return b.value


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _stream_ptr(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def nbldpc_decode(handle: int, gamma, frames: int, max_iters: int, early_stop: int, out_sym, out_iters,
                  out_ok, workspace, workspace_bytes: int | None = None, stream=None) -> None:
    """Queue a decode of device buffers on `stream` (default: torch's current stream)."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size()
    st = lib().nbldpc_decode(handle, _ptr(gamma), int(frames), int(max_iters), int(early_stop),
                             _ptr(out_sym), _ptr(out_iters), _ptr(out_ok), _ptr(workspace),
                             int(workspace_bytes), _stream_ptr(stream))
    _check(st, "nbldpc_decode")


def nbldpc_fftspa_workspace_size(handle: int, frames: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nbldpc_fftspa_workspace_size(handle, int(frames), ctypes.byref(b)), "nbldpc_fftspa_workspace_size")
    return b.value


def nbldpc_fftspa_decode(handle: int, prob, frames: int, max_iters: int, early_stop: int, out_sym, out_iters,
                         out_ok, out_app, workspace, workspace_bytes: int | None = None, stream=None) -> None:
    """Queue an FFT-SPA decode of device buffers on `stream` (out_app may be None)."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size()
    st = lib().nbldpc_fftspa_decode(handle, _ptr(prob), int(frames), int(max_iters), int(early_stop),
                                    _ptr(out_sym), _ptr(out_iters), _ptr(out_ok), _ptr(out_app),
                                    _ptr(workspace), int(workspace_bytes), _stream_ptr(stream))
    _check(st, "nbldpc_fftspa_decode")


def nbldpc_fftspa_decode_host_workspace_size(handle: int, chunk_frames: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nbldpc_fftspa_decode_host_workspace_size(handle, int(chunk_frames), ctypes.byref(b)),
           "nbldpc_fftspa_decode_host_workspace_size")
    return b.value


def nbldpc_fftspa_decode_host(handle: int, prob_host, frames: int, max_iters: int, early_stop: int,
                              out_sym_host, out_iters_host, out_ok_host, chunk_frames: int, workspace,
                              workspace_bytes: int | None = None, stream=None) -> None:
    """Queue an FFT-SPA decode of host buffers (pinned for overlap); sync `stream` before reading outputs."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size()
    st = lib().nbldpc_fftspa_decode_host(handle, _ptr(prob_host), int(frames), int(max_iters), int(early_stop),
                                         _ptr(out_sym_host), _ptr(out_iters_host), _ptr(out_ok_host),
                                         int(chunk_frames), _ptr(workspace), int(workspace_bytes),
                                         _stream_ptr(stream))
    _check(st, "nbldpc_fftspa_decode_host")


def nbldpc_decode_host(handle: int, gamma_host, frames: int, max_iters: int, early_stop: int,
                       out_sym_host, out_iters_host, out_ok_host, chunk_frames: int, workspace,
                       workspace_bytes: int | None = None, stream=None) -> None:
    """Queue a decode of host buffers (pinned for overlap); sync `stream` before reading outputs."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size()
    st = lib().nbldpc_decode_host(handle, _ptr(gamma_host), int(frames), int(max_iters), int(early_stop),
                                  _ptr(out_sym_host), _ptr(out_iters_host), _ptr(out_ok_host),
                                  int(chunk_frames), _ptr(workspace), int(workspace_bytes),
                                  _stream_ptr(stream))
    _check(st, "nbldpc_decode_host")


def nbldpc_decode_noalloc(handle: int, gamma, frames: int, max_iters: int, early_stop: int, out_sym,
                          out_iters, out_ok, stream=None) -> None:
    """Queue a decode that uses the library's fixed device scratch instead of a
    caller workspace (for callers that cannot allocate device memory).  Calls
    that overlap on the GPU share that scratch and race; queue them in order."""
    st = lib().nbldpc_decode_noalloc(handle, _ptr(gamma), int(frames), int(max_iters), int(early_stop),
                                     _ptr(out_sym), _ptr(out_iters), _ptr(out_ok), _stream_ptr(stream))
    _check(st, "nbldpc_decode_noalloc")


def _jobs_array(jobs):
    arr = (nbldpc_job * len(jobs))()
    for i, j in enumerate(jobs):
        if isinstance(j, dict):
            j = (j["code"], j["gamma"], j["frames"], j["max_iters"], j["early_stop"], j["out_sym"],
                 j["out_iters"], j["out_ok"])
        code, gamma, frames, mi, es, sym, its, ok = j
        arr[i] = nbldpc_job(code, _ptr(gamma), int(frames), int(mi), int(es), _ptr(sym), _ptr(its), _ptr(ok))
    return arr


def nbldpc_decode_batch_workspace_size(jobs) -> int:
    """Workspace bytes for a batch; jobs: sequence of (handle, gamma, frames, max_iters, early_stop,
    out_sym, out_iters, out_ok) tuples or dicts with those keys."""
    arr = _jobs_array(jobs)
    b = ctypes.c_size_t()
    _check(lib().nbldpc_decode_batch_workspace_size(arr, len(jobs), ctypes.byref(b)),
           "nbldpc_decode_batch_workspace_size")
    return b.value


def nbldpc_decode_batch(jobs, workspace, workspace_bytes: int | None = None, stream=None) -> None:
    """Queue one persistent launch over the frames of every job (mixed codes)."""
    arr = _jobs_array(jobs)
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size()
    _check(lib().nbldpc_decode_batch(arr, len(jobs), _ptr(workspace), int(workspace_bytes), _stream_ptr(stream)),
           "nbldpc_decode_batch")


def nbldpc_code_get_tuning(handle: int):
    v, f = ctypes.c_int(), ctypes.c_int()
    _check(lib().nbldpc_code_get_tuning(handle, ctypes.byref(v), ctypes.byref(f)), "nbldpc_code_get_tuning")
    return v.value, f.value


def nbldpc_code_set_tuning(handle: int, variant: int, frames_per_block: int) -> None:
    _check(lib().nbldpc_code_set_tuning(handle, int(variant), int(frames_per_block)), "nbldpc_code_set_tuning")


def nbldpc_code_set_message_bits(handle: int, bits: int) -> None:
    _check(lib().nbldpc_code_set_message_bits(handle, int(bits)), "nbldpc_code_set_message_bits")


def nbldpc_code_set_cnp_schedule(handle: int, schedule: int) -> None:
    _check(lib().nbldpc_code_set_cnp_schedule(handle, int(schedule)), "nbldpc_code_set_cnp_schedule")


def nbldpc_code_set_work_counter(handle: int, counter) -> None:
    """counter: a torch int64 CUDA tensor of one element (the decodes add to it), or None (off)."""
    ptr = None
    if counter is not None:
        assert counter.is_cuda and counter.dtype == torch.int64 and counter.numel() >= 1
        ptr = counter.data_ptr()
    _check(lib().nbldpc_code_set_work_counter(handle, ptr), "nbldpc_code_set_work_counter")


def nbldpc_code_get_cnp_schedule(handle: int) -> int:
    v = ctypes.c_int()
    _check(lib().nbldpc_code_get_cnp_schedule(handle, ctypes.byref(v)), "nbldpc_code_get_cnp_schedule")
    return v.value


def nbldpc_code_get_message_bits(handle: int) -> int:
    b = ctypes.c_int()
    _check(lib().nbldpc_code_get_message_bits(handle, ctypes.byref(b)), "nbldpc_code_get_message_bits")
    return b.value


def nbldpc_code_autotune_workspace_size(handle: int, frames: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nbldpc_code_autotune_workspace_size(handle, int(frames), ctypes.byref(b)),
           "nbldpc_code_autotune_workspace_size")
    return b.value


def nbldpc_code_autotune(handle: int, gamma, frames: int, max_iters: int, workspace,
                         workspace_bytes: int | None = None, stream=None):
    """Measure every (variant, frames-per-block) pair, keep the fastest; returns the measurements."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size()
    res = (nbldpc_tune_result * 16)()
    n = ctypes.c_int()
    _check(lib().nbldpc_code_autotune(handle, _ptr(gamma), int(frames), int(max_iters), _ptr(workspace),
                                      int(workspace_bytes), _stream_ptr(stream), res, 16, ctypes.byref(n)),
           "nbldpc_code_autotune")
    return [(res[i].variant, res[i].frames_per_block, res[i].ms) for i in range(min(n.value, 16))]


class Decoder:
    """Owns a code handle; allocates outputs and workspace with torch."""

    def __init__(self, q, prim_poly, n_cols, n_rows, row_ptr, col_idx, coef):
        self.handle = nbldpc_code_create(q, prim_poly, n_cols, n_rows, row_ptr, col_idx, coef)
        self.q, self.n, self.m, self.nnz = nbldpc_code_info(self.handle)
        self._ws = None
        self._fws = None

    @classmethod
    def from_code(cls, code):
        return cls(code.q, code.poly, code.n, code.m, code.row_ptr, code.col_idx, code.coef)

    def close(self):
        if self.handle:
            nbldpc_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, gamma: torch.Tensor, max_iters: int, frames: int | None = None):
        f = gamma.shape[0] if frames is None else frames
        ws = torch.empty(nbldpc_code_autotune_workspace_size(self.handle, f), dtype=torch.uint8,
                         device=gamma.device)
        return nbldpc_code_autotune(self.handle, gamma, f, max_iters, ws)

    def set_message_bits(self, bits: int) -> None:
        nbldpc_code_set_message_bits(self.handle, bits)

    def message_bits(self) -> int:
        return nbldpc_code_get_message_bits(self.handle)

    def tuning(self):
        return nbldpc_code_get_tuning(self.handle)

    def set_tuning(self, variant: int, frames_per_block: int) -> None:
        nbldpc_code_set_tuning(self.handle, variant, frames_per_block)

    def workspace(self, frames: int, device) -> torch.Tensor:
        need = nbldpc_decode_workspace_size(self.handle, frames)
        if self._ws is None or self._ws.numel() < need or self._ws.device != torch.device(device):
            self._ws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._ws

    def decode(self, gamma: torch.Tensor, max_iters: int, early_stop: int, stream=None):
        """(symbols [F, N] uint8, iterations [F] int32, ok [F] uint8) on gamma's device."""
        assert gamma.is_cuda and gamma.dtype == torch.uint8 and gamma.is_contiguous()
        f = gamma.shape[0]
        assert gamma.shape[1:] == (self.n, self.q)
        dev = gamma.device
        sym = torch.empty((f, self.n), dtype=torch.uint8, device=dev)
        its = torch.empty((f,), dtype=torch.int32, device=dev)
        ok = torch.empty((f,), dtype=torch.uint8, device=dev)
        ws = self.workspace(f, dev)
        nbldpc_decode(self.handle, gamma, f, max_iters, early_stop, sym, its, ok, ws, stream=stream)
        return sym, its, ok

    def fftspa_workspace(self, frames: int, device) -> torch.Tensor:
        need = nbldpc_fftspa_workspace_size(self.handle, frames)
        if self._fws is None or self._fws.numel() < need or self._fws.device != torch.device(device):
            self._fws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._fws

    def fftspa_decode(self, prob: torch.Tensor, max_iters: int, early_stop: int, want_app: bool = False,
                      stream=None):
        """FFT-SPA (Alg. 1): (symbols, iterations, ok[, app [F, N, q] float32]) on prob's device."""
        assert prob.is_cuda and prob.dtype == torch.float32 and prob.is_contiguous()
        f = prob.shape[0]
        assert prob.shape[1:] == (self.n, self.q)
        dev = prob.device
        sym = torch.empty((f, self.n), dtype=torch.uint8, device=dev)
        its = torch.empty((f,), dtype=torch.int32, device=dev)
        ok = torch.empty((f,), dtype=torch.uint8, device=dev)
        app = torch.empty((f, self.n, self.q), dtype=torch.float32, device=dev) if want_app else None
        ws = self.fftspa_workspace(f, dev)
        nbldpc_fftspa_decode(self.handle, prob, f, max_iters, early_stop, sym, its, ok, app, ws, stream=stream)
        return (sym, its, ok, app) if want_app else (sym, its, ok)

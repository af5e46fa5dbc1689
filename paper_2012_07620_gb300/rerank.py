"""Python binding of the C ABI in ``include/rerank.h`` (ctypes; argument marshalling only).

Every step of the re-ranking runs inside ``librerank.so``.  Tensors are
passed by pointer: CUDA tensors stay on the device, NumPy arrays (or CPU
tensors) are host buffers that the library stages through its own device
workspace.  There is no CPU fallback: without the built library the import
of the symbols fails loudly.
"""
from __future__ import annotations

import ctypes
import pathlib
from typing import Optional

import numpy as np

_LIB_PATH = pathlib.Path(__file__).resolve().parent / "_lib" / "librerank.so"

RERANK_OK = 0
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EBUDGET", 4: "ECUDA", 5: "ETIMEOUT",
                6: "EINTERNAL", 7: "EUNSUPPORTED", 8: "EAGAIN"}
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2}
DTYPE = {"f32": 0, "bf16": 1}
AGGREGATOR = {"sum": 0, "mean": 1, "max": 2}
FEATURE = {"astar": 0, "a": 1, "x": 2}
DEBUG = {"knn_idx": 0, "knn_score": 1, "h0_rowptr": 2, "h0_col": 3, "h0_val": 4,
         "hl_start": 5, "hl_len": 6, "hl_col": 7, "hl_val": 8, "part_s": 9, "part_i": 10, "qerr": 11,
         "hl_dense": 12}


class RerankConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int), ("rescore_m", ctypes.c_int),
                ("alpha", ctypes.c_float), ("aggregator", ctypes.c_int), ("feature_mode", ctypes.c_int),
                ("hbm_budget", ctypes.c_size_t), ("autotune_path", ctypes.c_char_p),
                ("stage_timing", ctypes.c_int)]


class RerankInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("candidates_per_row", ctypes.c_int64),
                ("fp64_rescored", ctypes.c_int64), ("fallback_rows", ctypes.c_int64),
                ("exact_scan_rows", ctypes.c_int64),
                ("h_nnz", ctypes.c_int64 * 9), ("workspace_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64),
                ("error_bits", ctypes.c_int32), ("bad_row", ctypes.c_int32)]


class RerankJob(ctypes.Structure):
    _fields_ = [("xq", ctypes.c_void_p), ("nq", ctypes.c_int64), ("xg", ctypes.c_void_p), ("ng", ctypes.c_int64),
                ("d", ctypes.c_int), ("dtype", ctypes.c_int), ("k1", ctypes.c_int), ("k2", ctypes.c_int),
                ("layers", ctypes.c_int), ("topk_out", ctypes.c_int64), ("out_idx", ctypes.c_void_p),
                ("out_dist", ctypes.c_void_p), ("status", ctypes.c_int)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_query", ctypes.c_int64), ("slots", ctypes.c_int), ("k1", ctypes.c_int), ("k2", ctypes.c_int),
                ("layers", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("xq", ctypes.c_void_p), ("nq", ctypes.c_int64), ("topk_out", ctypes.c_int64),
                ("out_idx", ctypes.c_void_p), ("out_dist", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("queue_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("slot", ctypes.c_int)]


class ServeInfo(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_in_flight", ctypes.c_int), ("completed", ctypes.c_int64),
                ("touched_rows", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("slot_bytes", ctypes.c_int64), ("reuse_layers", ctypes.c_int), ("recomputed_rows", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("sim_chunks", ctypes.c_int), ("prop_warps", ctypes.c_int), ("refine_order", ctypes.c_int),
                ("rescore_m", ctypes.c_int), ("n_bucket", ctypes.c_int), ("ms", ctypes.c_double)]


class RerankError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        text = f"{where}: {STATUS_NAMES.get(status, status)} ({strerror(status)})"
        if status in (2, 4):  # ENOMEM, ECUDA: name the failing CUDA call
            cuda = load_library().rerank_last_cuda_error().decode()
            if cuda:
                text += f" [{cuda}]"
        super().__init__(text)


_lib: Optional[ctypes.CDLL] = None

_SIGS = {
    "rerank_config_init": (None, [ctypes.POINTER(RerankConfig)]),
    "rerank_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(RerankConfig)]),
    "rerank_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "rerank_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rerank_last_cuda_error": (ctypes.c_char_p, []),
    "rerank_check_args": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
    "rerank_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rerank_run_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(RerankJob), ctypes.c_int, ctypes.c_void_p]),
    "rerank_gallery_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(ServeConfig)]),
    "rerank_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "rerank_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(TicketInfo)]),
    "rerank_serve_info_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServeInfo)]),
    "rerank_gallery_unload": (ctypes.c_int, [ctypes.c_void_p]),
    "rerank_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(Tuning), ctypes.c_void_p]),
    "rerank_tuning_lookup": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                            ctypes.POINTER(Tuning)]),
    "rerank_knn": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rerank_last_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(RerankInfo)]),
    "rerank_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_char_p), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    "rerank_debug_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t)]),
}


def library_path() -> pathlib.Path:
    return _LIB_PATH


def load_library() -> ctypes.CDLL:
    """Load librerank.so (built by ``paper_2012_07620_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"{_LIB_PATH} is missing: run paper_2012_07620_gb300.build.build() first")
        lib = ctypes.CDLL(str(_LIB_PATH))
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def strerror(status: int) -> str:
    return load_library().rerank_strerror(status).decode()


def check_args(nq, ng, d, dtype, k1, k2, layers, topk_out) -> int:
    """Host-only argument validation (``rerank_check_args``); returns the status code."""
    return load_library().rerank_check_args(nq, ng, d, DTYPE[dtype] if isinstance(dtype, str) else dtype,
                                            k1, k2, layers, topk_out)


def tuning_lookup(path: str, precision: str, n: int, d: int) -> Optional[dict]:
    """Host-only read of a tuning table file (``rerank_tuning_lookup``); None when
    the file has no entry for (precision, d, bucket of n)."""
    t = Tuning()
    st = load_library().rerank_tuning_lookup(path.encode(), PRECISION[precision], n, d, ctypes.byref(t))
    if st == 8:
        return None
    _check(st, "rerank_tuning_lookup")
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


def _check(status: int, where: str) -> None:
    if status != RERANK_OK:
        raise RerankError(status, where)


def _ptr(x) -> int:
    """Pointer of a torch tensor (device or host) or a C-contiguous NumPy array."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return x.data_ptr()


def _dtype_code(x) -> int:
    if isinstance(x, np.ndarray):
        if x.dtype == np.float32:
            return 0
        raise ValueError("NumPy features must be float32")
    import torch
    if x.dtype == torch.float32:
        return 0
    if x.dtype == torch.bfloat16:
        return 1
    raise ValueError("features must be float32 or bfloat16")


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    return stream if isinstance(stream, int) else stream.cuda_stream


class Reranker:
    """A library context (``rerank_create``) with its device workspace."""

    def __init__(self, device: int = 0, precision: str = "fp32", rescore_m: int = 16, alpha: float = 2.0,
                 aggregator: str = "sum", feature: str = "astar", hbm_budget: int = 0,
                 stage_timing: bool = False, autotune_path: Optional[str] = None):
        lib = load_library()
        cfg = RerankConfig()
        lib.rerank_config_init(ctypes.byref(cfg))
        cfg.device = device
        cfg.precision = PRECISION[precision]
        cfg.rescore_m = rescore_m
        cfg.alpha = alpha
        cfg.aggregator = AGGREGATOR[aggregator]
        cfg.feature_mode = FEATURE[feature]
        cfg.hbm_budget = hbm_budget
        cfg.stage_timing = 1 if stage_timing else 0
        self._path = autotune_path.encode() if autotune_path else None
        cfg.autotune_path = self._path
        h = ctypes.c_void_p()
        _check(lib.rerank_create(ctypes.byref(h), ctypes.byref(cfg)), "rerank_create")
        self._h = h
        self._lib = lib
        self.device = device
        self._live = {}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rerank_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, xq, xg, k1: int, k2: int, layers: int, topk_out: int = 0, out_idx=None, out_dist=None,
            stream=None):
        """Algorithm 1 end to end; returns (out_idx, out_dist) of shape (nq, topk_out or ng).

        Outputs default to the inputs' kind: CUDA tensors for CUDA inputs,
        NumPy arrays for host inputs."""
        nq, d = xq.shape
        ng = xg.shape[0]
        t = topk_out if topk_out else ng
        if out_idx is None:
            out_idx, out_dist = self._alloc_out(xq, (nq, t))
        st = self._lib.rerank_run(self._h, _ptr(xq), nq, _ptr(xg), ng, d, _dtype_code(xq), k1, k2, layers, topk_out,
                                  _ptr(out_idx), _ptr(out_dist), _stream_handle(stream))
        _check(st, "rerank_run")
        return out_idx, out_dist

    def run_batch(self, jobs, stream=None):
        """Many independent instances in one call (``rerank_run_batch``).

        ``jobs``: list of dicts with keys xq, xg, k1, k2, layers and optionally
        topk_out, out_idx, out_dist.  Returns a list of (out_idx, out_dist)."""
        arr = (RerankJob * len(jobs))()
        outs = []
        for i, j in enumerate(jobs):
            xq, xg = j["xq"], j["xg"]
            nq, d = xq.shape
            ng = xg.shape[0]
            topk = j.get("topk_out", 0)
            oi, od = j.get("out_idx"), j.get("out_dist")
            if oi is None:
                oi, od = self._alloc_out(xq, (nq, topk if topk else ng))
            outs.append((oi, od))
            arr[i] = RerankJob(_ptr(xq), nq, _ptr(xg), ng, d, _dtype_code(xq), j["k1"], j["k2"], j["layers"], topk,
                               _ptr(oi), _ptr(od), 0)
        st = self._lib.rerank_run_batch(self._h, arr, len(jobs), _stream_handle(stream))
        self.batch_status = [arr[i].status for i in range(len(jobs))]
        _check(st, "rerank_run_batch")
        return outs

    def autotune(self, xq, xg, k1: int, k2: int, layers: int, stream=None) -> dict:
        """Measure launch shapes on this instance and keep the best (``rerank_autotune``)."""
        nq, d = xq.shape
        ng = xg.shape[0]
        t = Tuning()
        _check(self._lib.rerank_autotune(self._h, _ptr(xq), nq, _ptr(xg), ng, d, _dtype_code(xq), k1, k2, layers,
                                         ctypes.byref(t), _stream_handle(stream)), "rerank_autotune")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    # ---- serving ----
    def load_gallery(self, xg, max_query: int, k1: int, k2: int, layers: int, slots: int = 0) -> None:
        """Make ``xg`` the resident gallery and start the request loop (``rerank_gallery_load``)."""
        ng, d = xg.shape
        sc = ServeConfig(max_query, slots, k1, k2, layers)
        _check(self._lib.rerank_gallery_load(self._h, _ptr(xg), ng, d, _dtype_code(xg), ctypes.byref(sc)),
               "rerank_gallery_load")
        self._gallery_rows = ng

    def submit(self, xq, topk_out: int = 0, out_idx=None, out_dist=None, stream=None) -> tuple:
        """Queue one request; returns (ticket, out_idx, out_dist).  The binding
        keeps the three buffers alive until ``wait`` returns for the ticket; the
        request reads ``xq`` after the work already queued on ``stream``
        (default: the current torch stream)."""
        nq = xq.shape[0]
        t = topk_out if topk_out else self._gallery_rows
        if out_idx is None:
            out_idx, out_dist = self._alloc_out(xq, (nq, t))
        rq = Request(_ptr(xq), nq, topk_out, _ptr(out_idx), _ptr(out_dist), _stream_handle(stream))
        ticket = ctypes.c_uint64()
        _check(self._lib.rerank_submit(self._h, ctypes.byref(rq), ctypes.byref(ticket)), "rerank_submit")
        self._live[ticket.value] = (xq, out_idx, out_dist)
        return ticket.value, out_idx, out_dist

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        """Wait for a request; returns its timings (raises on a failed request,
        returns None while it is still running after ``timeout_ms``)."""
        info = TicketInfo()
        st = self._lib.rerank_wait(self._h, ticket, timeout_ms, ctypes.byref(info))
        if st == 8:
            return None
        self._live.pop(ticket, None)
        _check(st, "rerank_wait")
        return {"queue_ms": info.queue_ms, "total_ms": info.total_ms, "slot": info.slot}

    def serve_info(self) -> dict:
        info = ServeInfo()
        _check(self._lib.rerank_serve_info_get(self._h, ctypes.byref(info)), "rerank_serve_info_get")
        return {f: getattr(info, f) for f, _ in ServeInfo._fields_}

    def unload_gallery(self) -> None:
        _check(self._lib.rerank_gallery_unload(self._h), "rerank_gallery_unload")

    def knn(self, x, k: int, out_idx=None, out_score=None, stream=None):
        """Exact top-k neighbour lists (Eq. 7-8) of every row of x; returns (idx, score)."""
        n, d = x.shape
        if out_idx is None:
            out_idx, out_score = self._alloc_out(x, (n, k))
        st = self._lib.rerank_knn(self._h, _ptr(x), n, d, _dtype_code(x), k, _ptr(out_idx), _ptr(out_score),
                                  _stream_handle(stream))
        _check(st, "rerank_knn")
        return out_idx, out_score

    @staticmethod
    def _alloc_out(like, shape):
        if isinstance(like, np.ndarray):
            return np.empty(shape, np.int32), np.empty(shape, np.float32)
        import torch
        if like.is_cuda:
            return (torch.empty(shape, dtype=torch.int32, device=like.device),
                    torch.empty(shape, dtype=torch.float32, device=like.device))
        return torch.empty(shape, dtype=torch.int32), torch.empty(shape, dtype=torch.float32)

    def last_info(self) -> dict:
        info = RerankInfo()
        _check(self._lib.rerank_last_info(self._h, ctypes.byref(info)), "rerank_last_info")
        out = {f: getattr(info, f) for f, _ in RerankInfo._fields_}
        out["h_nnz"] = list(info.h_nnz)
        return out

    def stage_times(self) -> dict:
        ms = (ctypes.c_float * 32)()
        names = (ctypes.c_char_p * 32)()
        cnt = ctypes.c_int()
        _check(self._lib.rerank_stage_times(self._h, ms, names, 32, ctypes.byref(cnt)), "rerank_stage_times")
        return {names[i].decode(): ms[i] for i in range(min(cnt.value, 32))}

    def debug(self, what: str) -> np.ndarray:
        """Host copy of an intermediate array of the last call (see RERANK_DBG_* in rerank.h)."""
        code = DEBUG[what]
        nb = ctypes.c_size_t()
        _check(self._lib.rerank_debug_copy(self._h, code, None, 0, ctypes.byref(nb)), "rerank_debug_copy")
        dt = {5: np.int64, 1: np.float32, 4: np.float32, 8: np.float32, 9: np.float32, 11: np.float32,
              12: np.float32}.get(code, np.int32)
        arr = np.empty(nb.value // np.dtype(dt).itemsize, dtype=dt)
        _check(self._lib.rerank_debug_copy(self._h, code, arr.ctypes.data, arr.nbytes, ctypes.byref(nb)),
               "rerank_debug_copy")
        return arr

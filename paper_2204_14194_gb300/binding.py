"""Thin ctypes binding of libse.so (the C ABI in include/se.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device buffers and streams come from PyTorch (``data_ptr()``
and ``torch.cuda.Stream.cuda_stream``); the names mirror the C entry points.
If the library cannot be loaded (not built, or no CUDA runtime) every call
raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

SE_OK, SE_PENDING = 0, 1
SE_ERR = {-1: "SE_ERR_INVALID", -2: "SE_ERR_NOMEM", -3: "SE_ERR_CUDA", -4: "SE_ERR_TIMEOUT",
          -5: "SE_ERR_EMPTY_SUPPORT", -6: "SE_ERR_CANCELLED", -7: "SE_ERR_UNKNOWN_TICKET"}
BASIS = {"dct": 1, "wht": 2, "dct_wht": 3, "numeric": 4, "dft": 5, "bdft": 6, "dft_bdft": 7}
PREC = {"fp64": 0, "bf16x6": 1, "bf16x3": 3, "bf16": 4, "certified": 5}
GRAM = {"auto": 0, "full": 1, "lazy": 2}
PRODUCTS = {"auto": 0, "dense": 1, "transform": 2}

# every entry point declared in include/se.h
EXPORTS = ["se_ctx_create", "se_ctx_destroy", "se_plan", "se_plan_destroy", "se_plan_reset_tables",
           "se_extrapolate_batch", "se_extrapolate_strided", "se_extrapolate_host", "se_sync",
           "se_submit", "se_poll", "se_cancel", "se_last_error", "se_stats", "se_set_profiling",
           "se_stage_times", "se_extrapolate_noalloc", "se_plan_autotune", "se_plan_costs",
           "se_set_graphs", "se_tuning_stats", "se_tuned_variant", "se_cert_stats", "se_plan_info",
           "se_check_wait_timeout", "se_check_sample_conversion", "se_extrapolate_host_async",
           "se_host_wait"]
STAGES = ["pack", "tables", "projections", "iterate", "model"]


class SeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {SE_ERR.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(C.Structure):
    _fields_ = [("M", C.c_int), ("N", C.c_int), ("basis", C.c_int), ("K", C.c_int),
                ("dict", C.c_void_p), ("rho_hat", C.c_double), ("rho", C.c_void_p),
                ("support", C.c_void_p), ("gamma", C.c_double), ("iterations", C.c_int),
                ("prec", C.c_int), ("gram", C.c_int), ("products", C.c_int), ("T", C.c_int)]


class Block(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("support", C.c_void_p), ("out", C.c_void_p),
                ("sel_idx", C.c_void_p), ("sel_coef", C.c_void_p), ("iterations", C.c_int)]


class Request(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("support", C.c_void_p), ("out", C.c_void_p),
                ("sel_idx", C.c_void_p), ("sel_coef", C.c_void_p), ("iterations", C.c_int)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libse.so (building it first if it is missing and allowed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"{path} is not built")
            _build.build()
        lib = C.CDLL(path)
        vp, i32, dbl, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64
        sig = {
            "se_ctx_create": ([i32, C.c_size_t, C.POINTER(vp)], i32),
            "se_ctx_destroy": ([vp], i32),
            "se_plan": ([vp, C.POINTER(PlanDesc), C.POINTER(vp)], i32),
            "se_plan_destroy": ([vp], i32),
            "se_plan_reset_tables": ([vp], i32),
            "se_extrapolate_batch": ([vp, vp, i32, C.POINTER(Block), vp], i32),
            "se_extrapolate_strided": ([vp, vp, i32, vp, vp, vp, vp, i32, vp], i32),
            "se_extrapolate_host": ([vp, vp, i32, vp, vp, vp, vp, i32], i32),
            "se_extrapolate_host_async": ([vp, vp, i32, vp, vp, vp, vp, i32, C.POINTER(u64)], i32),
            "se_host_wait": ([vp, u64], i32),
            "se_extrapolate_noalloc": ([vp, vp, i32, vp, vp, vp, vp, i32, vp], i32),
            "se_sync": ([vp, vp], i32),
            "se_submit": ([vp, vp, C.POINTER(Request), C.POINTER(u64)], i32),
            "se_poll": ([vp, u64, C.c_int64, C.POINTER(dbl)], i32),
            "se_cancel": ([vp, u64], i32),
            "se_last_error": ([], C.c_char_p),
            "se_stats": ([vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(u64)], i32),
            "se_set_profiling": ([vp, i32], i32),
            "se_stage_times": ([vp, C.POINTER(dbl), C.POINTER(u64), i32, i32], i32),
            "se_plan_autotune": ([vp, vp, i32, vp], i32),
            "se_plan_costs": ([vp, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl)], i32),
            "se_set_graphs": ([vp, i32], i32),
            "se_tuning_stats": ([vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(u64)], i32),
            "se_tuned_variant": ([vp, C.c_char_p, C.POINTER(i32)], i32),
            "se_check_wait_timeout": ([vp, C.c_uint32, vp], i32),
            "se_check_sample_conversion": ([vp, vp, vp, vp, i32, vp], i32),
            "se_cert_stats": ([vp, C.POINTER(u64), C.POINTER(u64)], i32),
            "se_plan_info": ([vp, C.c_char_p, C.c_size_t], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(status: int, where: str, allow=(SE_OK,)):
    if status in allow:
        return status
    msg = load().se_last_error()
    raise SeError(status, where, msg.decode() if msg else "")


def _ptr(t) -> Optional[int]:
    """Device or host address of a torch tensor / numpy array / int (None passes through)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """An se_ctx_t: one CUDA device, optional HBM budget."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.se_ctx_create(int(device), int(hbm_budget_bytes), C.byref(h)), "se_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self._lib.se_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        _check(self._lib.se_sync(self.handle, _stream_handle(stream)), "se_sync")

    def host_wait(self, ticket: int):
        """Wait for an asynchronous host-buffer call (Plan.extrapolate_host_async)."""
        _check(self._lib.se_host_wait(self.handle, int(ticket)), "se_host_wait")

    def stats(self):
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(self._lib.se_stats(self.handle, C.byref(a), C.byref(b), C.byref(c)), "se_stats")
        return {"kernel_launches": a.value, "table_builds": b.value, "serving_slices": c.value}

    def tuning_stats(self):
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(self._lib.se_tuning_stats(self.handle, C.byref(a), C.byref(b), C.byref(c)), "se_tuning_stats")
        return {"tunings": a.value, "graph_builds": b.value, "graph_replays": c.value}

    def cert_stats(self):
        a, b = C.c_uint64(), C.c_uint64()
        _check(self._lib.se_cert_stats(self.handle, C.byref(a), C.byref(b)), "se_cert_stats")
        return {"blocks": a.value, "recomputed": b.value}

    def check_wait_timeout(self, limit_us: int = 200_000, stream=None):
        """Queue a device wait that runs out after limit_us (se_check_wait_timeout)."""
        _check(self._lib.se_check_wait_timeout(self.handle, int(limit_us), _stream_handle(stream)),
               "se_check_wait_timeout")

    def check_sample_conversion(self, x, out, back=None, stream=None):
        """The projection kernels' fp64 -> fp32 sample conversion on device tensors (and,
        into back, the model kernels' fp32 -> fp64 conversion of the results)."""
        _check(self._lib.se_check_sample_conversion(self.handle, _ptr(x), _ptr(out), _ptr(back), int(x.numel()),
                                                    _stream_handle(stream)), "se_check_sample_conversion")

    def tuned_variant(self, key: str) -> int:
        """The autotuner's kept variant for a shape key, -1 if not tuned."""
        v = C.c_int()
        _check(self._lib.se_tuned_variant(self.handle, key.encode(), C.byref(v)), "se_tuned_variant")
        return v.value

    def set_graphs(self, enable: bool = True):
        _check(self._lib.se_set_graphs(self.handle, int(bool(enable))), "se_set_graphs")

    def set_profiling(self, enable: bool = True):
        _check(self._lib.se_set_profiling(self.handle, int(bool(enable))), "se_set_profiling")

    def stage_times(self, reset: bool = True):
        """{stage: (milliseconds, launches)} accumulated since the last reset."""
        ms = (C.c_double * len(STAGES))()
        cnt = (C.c_uint64 * len(STAGES))()
        _check(self._lib.se_stage_times(self.handle, ms, cnt, len(STAGES), int(bool(reset))), "se_stage_times")
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(len(STAGES))}

    def plan(self, M: int, N: int, basis: str, K: int, rho_hat: float, gamma: float,
             iterations: int, prec: str = "bf16x6", gram: str = "auto",
             dictionary: Optional[np.ndarray] = None, support: Optional[np.ndarray] = None,
             rho: Optional[np.ndarray] = None, products: str = "auto", T: int = 1) -> "Plan":
        """T > 1: a video block of T frames (arrays frame-major, [T][M][N])."""
        return Plan(self, M, N, basis, K, rho_hat, gamma, iterations, prec, gram, dictionary,
                    support, rho, products, T)

    # serving -------------------------------------------------------------
    def submit(self, plan: "Plan", samples: np.ndarray, out: np.ndarray,
               sel_idx: Optional[np.ndarray] = None, sel_coef: Optional[np.ndarray] = None,
               iterations: int = 0, support: Optional[np.ndarray] = None) -> int:
        s = np.ascontiguousarray(samples, dtype=np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous
        sup = None if support is None else np.ascontiguousarray(support, dtype=np.uint8)
        req = Request(s.ctypes.data, _ptr(sup), out.ctypes.data, _ptr(sel_idx), _ptr(sel_coef),
                      int(iterations))
        t = C.c_uint64()
        _check(self._lib.se_submit(self.handle, plan.handle, C.byref(req), C.byref(t)), "se_submit")
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1):
        """Returns (status, latency_s); status SE_OK or SE_PENDING, raises on failure."""
        lat = C.c_double(0.0)
        st = self._lib.se_poll(self.handle, C.c_uint64(ticket), int(timeout_us), C.byref(lat))
        _check(st, "se_poll", allow=(SE_OK, SE_PENDING))
        return st, lat.value

    def cancel(self, ticket: int) -> int:
        st = self._lib.se_cancel(self.handle, C.c_uint64(ticket))
        return _check(st, "se_cancel", allow=(SE_OK, SE_PENDING))


class Plan:
    """An se_plan_t.  Host arrays are copied by the library."""

    def __init__(self, ctx: Context, M, N, basis, K, rho_hat, gamma, iterations, prec, gram,
                 dictionary, support, rho, products="auto", T=1):
        self.ctx = ctx
        self._lib = ctx._lib
        self.M, self.N, self.K, self.iterations = int(M), int(N), int(K), int(iterations)
        self.T = int(T)
        self.prec = prec
        self.products = products
        d = None if dictionary is None else np.ascontiguousarray(dictionary, dtype=np.float64)
        sup = None if support is None else np.ascontiguousarray(support, dtype=np.uint8)
        rh = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        desc = PlanDesc(int(M), int(N), BASIS[basis], int(K), _ptr(d), float(rho_hat), _ptr(rh),
                        _ptr(sup), float(gamma), int(iterations), PREC[prec], GRAM[gram],
                        PRODUCTS[products], int(T))
        h = C.c_void_p()
        _check(self._lib.se_plan(ctx.handle, C.byref(desc), C.byref(h)), "se_plan")
        self.handle = h

    def close(self):
        if self.handle and self.ctx.handle:
            self._lib.se_plan_destroy(self.handle)
        self.handle = None

    def reset_tables(self):
        _check(self._lib.se_plan_reset_tables(self.handle), "se_plan_reset_tables")

    def info(self) -> dict:
        """The forms this plan's batches use (se_plan_info), as a dict."""
        buf = C.create_string_buffer(256)
        _check(self._lib.se_plan_info(self.handle, buf, 256), "se_plan_info")
        out = {}
        for item in buf.value.decode().split():
            k, _, v = item.partition("=")
            out[k] = v or True
        return out

    def autotune(self, n_probe: int = 256, stream=None):
        """Measure table / full / lazy costs on n_probe synthetic blocks (synchronous)."""
        _check(self._lib.se_plan_autotune(self.ctx.handle, self.handle, int(n_probe), _stream_handle(stream)),
               "se_plan_autotune")
        return self.costs()

    def costs(self):
        """{'table_ms', 'full_ms_per_block', 'lazy_ms_per_block'} (0 = not measured yet)."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        _check(self._lib.se_plan_costs(self.handle, C.byref(a), C.byref(b), C.byref(c)), "se_plan_costs")
        return {"table_ms": a.value, "full_ms_per_block": b.value, "lazy_ms_per_block": c.value}

    def extrapolate_strided(self, samples, out, sel_idx=None, sel_coef=None, iterations: int = 0,
                            stream=None):
        """Device tensors samples/out [n, M, N] float64 (contiguous); async on stream."""
        n = int(samples.shape[0])
        _check(self._lib.se_extrapolate_strided(self.ctx.handle, self.handle, n, _ptr(samples),
                                                _ptr(out), _ptr(sel_idx), _ptr(sel_coef),
                                                int(iterations), _stream_handle(stream)),
               "se_extrapolate_strided")

    def extrapolate_noalloc(self, samples, out, sel_idx=None, sel_coef=None, iterations: int = 0,
                            stream=None):
        """Like extrapolate_strided, with all scratch in the library's static device array."""
        n = int(samples.shape[0])
        _check(self._lib.se_extrapolate_noalloc(self.ctx.handle, self.handle, n, _ptr(samples),
                                                _ptr(out), _ptr(sel_idx), _ptr(sel_coef),
                                                int(iterations), _stream_handle(stream)),
               "se_extrapolate_noalloc")

    def extrapolate_batch(self, blocks, stream=None):
        """blocks: list of dicts with device tensors samples/out and optional support,
        sel_idx, sel_coef, iterations."""
        arr = (Block * len(blocks))()
        for i, b in enumerate(blocks):
            arr[i] = Block(_ptr(b["samples"]), _ptr(b.get("support")), _ptr(b["out"]),
                           _ptr(b.get("sel_idx")), _ptr(b.get("sel_coef")),
                           int(b.get("iterations", 0)))
        _check(self._lib.se_extrapolate_batch(self.ctx.handle, self.handle, len(blocks), arr,
                                              _stream_handle(stream)), "se_extrapolate_batch")

    def extrapolate_host_async(self, samples, out, sel_idx=None, sel_coef=None, iterations: int = 0) -> int:
        """Host buffers (pinned torch CPU tensors, or numpy); returns a ticket for
        Context.host_wait.  The buffers must stay unchanged until the wait."""
        n = int(samples.shape[0])
        t = C.c_uint64(0)
        _check(self._lib.se_extrapolate_host_async(self.ctx.handle, self.handle, n, _ptr(samples), _ptr(out),
                                                   _ptr(sel_idx), _ptr(sel_coef), int(iterations), C.byref(t)),
               "se_extrapolate_host_async")
        return int(t.value)

    def extrapolate_host(self, samples: np.ndarray, out: np.ndarray, sel_idx=None, sel_coef=None,
                         iterations: int = 0):
        """Host buffers (numpy, or pinned torch CPU tensors); synchronous."""
        n = int(samples.shape[0])
        _check(self._lib.se_extrapolate_host(self.ctx.handle, self.handle, n, _ptr(samples),
                                             _ptr(out), _ptr(sel_idx), _ptr(sel_coef),
                                             int(iterations)), "se_extrapolate_host")

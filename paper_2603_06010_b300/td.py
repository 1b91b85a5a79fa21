"""Thin ctypes binding of libtd (the C ABI in include/td.h).

Argument marshalling only: every step of the likelihood runs in libtd's CUDA
kernels.  The library is loaded from the package directory; if it is missing
the import of this module's `lib()` raises -- there is no CPU fallback.
Device buffers are torch tensors (PyTorch supplies device memory and
streams); their data pointers are passed through unchanged.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtd.so")

TD_OK, TD_ERR_INVALID, TD_ERR_NOT_PD, TD_ERR_OOM, TD_ERR_CUDA, TD_ERR_TIMEOUT, TD_ERR_NOT_FACTORED, \
    TD_ERR_UNSUPPORTED, TD_ERR_BUSY = range(9)
TD_PREC_FP64, TD_PREC_BF16X6, TD_PREC_BF16X3, TD_PREC_AUTO, TD_PREC_BF16X10 = range(5)
(TD_PATH_AUTO, TD_PATH_TENSOR, TD_PATH_STREAM, TD_PATH_FP64, TD_PATH_STREAM64, TD_PATH_SMALLK,
 TD_PATH_TENSOR128, TD_PATH_STREAM128, TD_PATH_GSCE) = range(9)

STATUS_NAMES = {0: "TD_OK", 1: "TD_ERR_INVALID", 2: "TD_ERR_NOT_PD", 3: "TD_ERR_OOM", 4: "TD_ERR_CUDA",
                5: "TD_ERR_TIMEOUT", 6: "TD_ERR_NOT_FACTORED", 7: "TD_ERR_UNSUPPORTED", 8: "TD_ERR_BUSY"}

# every symbol include/td.h declares, with (restype, argtypes)
_c = ctypes
_vp = _c.c_void_p
_i64 = _c.c_int64
SIGNATURES = {
    "td_options_default": (None, [_vp]),
    "td_segment_create": (_c.c_int, [_vp, _i64, _vp, _vp, _c.POINTER(_vp)]),
    "td_factor": (_c.c_int, [_vp, _vp]),
    "td_logdet": (_c.c_int, [_vp, _c.POINTER(_c.c_double)]),
    "td_kept": (_i64, [_vp]),
    "td_last_pivot": (_i64, [_vp]),
    "td_loglike_batch": (_c.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "td_reserve": (_c.c_int, [_vp, _i64, _vp]),
    "td_loglike_grouped": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _c.c_int, _vp, _vp]),
    "td_check": (_c.c_int, [_vp, _vp]),
    "td_segment_destroy": (None, [_vp]),
    "td_last_error": (_c.c_char_p, []),
    "td_resident_bytes": (_i64, [_vp]),
    "td_debug_bounded_wait": (_c.c_int, [_i64, _vp]),
    "td_debug_plan": (_c.c_int, [_c.POINTER(_i64), _c.POINTER(_i64), _c.c_int, _c.c_int, _c.c_int, _c.c_int,
                                 _c.POINTER(_c.c_int), _c.c_int]),
    "td_loglike_batch_noalloc": (_c.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "td_loglike_batch_host": (_c.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "td_set_data": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "td_data_inner": (_c.c_int, [_vp, _c.POINTER(_c.c_double)]),
    "td_template_batch": (_c.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "td_project_batch": (_c.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "td_segment_save": (_c.c_int, [_vp, _c.c_char_p, _vp]),
    "td_loglike_batch_gather": (_c.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "td_segment_load": (_c.c_int, [_c.c_char_p, _vp, _vp]),
    "td_group_create": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _c.c_int, _vp, _vp, _c.POINTER(_vp)]),
    "td_group_set_joint": (_c.c_int, [_vp, _vp]),
    "td_gs_prepare": (_c.c_int, [_vp, _vp]),
    "td_group_launch": (_c.c_int, [_vp, _vp]),
    "td_group_graph_launch": (_c.c_int, [_vp, _vp]),
    "td_group_tune": (_c.c_int, [_vp, _vp, _c.POINTER(_c.c_double)]),
    "td_group_check": (_c.c_int, [_vp, _vp]),
    "td_group_clock": (_c.c_int, [_vp, _vp, _c.POINTER(_c.c_double)]),
    "td_group_shape": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "td_group_destroy": (None, [_vp]),
    "td_segment_release_fp64": (_c.c_int, [_vp]),
    "td_factor_many": (_c.c_int, [_vp, _c.c_int, _c.c_int, _vp]),
    "td_server_config_default": (None, [_vp]),
    "td_server_create": (_c.c_int, [_vp, _c.POINTER(_vp)]),
    "td_server_add_segment": (_c.c_int, [_vp, _vp, _i64, _vp, _c.POINTER(_i64)]),
    "td_server_prefetch": (_c.c_int, [_vp, _i64]),
    "td_server_submit": (_c.c_int, [_vp, _i64, _vp, _i64, _i64, _vp, _c.POINTER(_i64)]),
    "td_server_poll": (_c.c_int, [_vp, _i64, _c.POINTER(_c.c_int)]),
    "td_server_latency": (_c.c_int, [_vp, _i64, _c.POINTER(_c.c_double)]),
    "td_server_set_budget": (_c.c_int, [_vp, _i64]),
    "td_server_wait": (_c.c_int, [_vp, _i64, _i64]),
    "td_server_cancel": (_c.c_int, [_vp, _i64]),
    "td_server_pause": (_c.c_int, [_vp, _c.c_int]),
    "td_server_drain": (_c.c_int, [_vp, _i64]),
    "td_server_replay": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "td_server_get_stats": (_c.c_int, [_vp, _vp, _c.c_int]),
    "td_server_destroy": (None, [_vp]),
    "td_profile_enable": (_c.c_int, [_vp, _c.c_int]),
    "td_profile_read": (_c.c_int, [_vp, _c.POINTER(_c.c_double), _c.POINTER(_i64), _c.POINTER(_i64)]),
    "td_profile_clock": (_c.c_int, [_vp, _vp, _c.POINTER(_c.c_double)]),
}


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch_cols", ctypes.c_int64), ("max_pending_cols", ctypes.c_int64),
                ("resident_bytes_budget", ctypes.c_int64), ("n_streams", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_kept", ctypes.c_int64), ("gs_gapfree", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("host_spill_bytes", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("evals_per_s", ctypes.c_double), ("requests_done", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("hits", ctypes.c_int64), ("misses", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("refused", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("resident_bytes", ctypes.c_int64), ("reloads", ctypes.c_int64)]


class TemplateOut(ctypes.Structure):
    _fields_ = [("logL", ctypes.c_void_p), ("chi2", ctypes.c_void_p), ("hh", ctypes.c_void_p),
                ("dh", ctypes.c_void_p), ("rho_mf", ctypes.c_void_p), ("rho_eff2", ctypes.c_void_p)]


class TdOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("path", ctypes.c_int), ("refine", ctypes.c_int),
                ("reserved0", ctypes.c_int), ("wait_limit_ns", ctypes.c_int64)]


class TdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libtd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtd.so is not built ({LIB_PATH}); run paper_2603_06010_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != TD_OK:
        raise TdError(code, lib().td_last_error().decode())


def options(precision: int = TD_PREC_AUTO, path: int = TD_PATH_AUTO, refine: int = 0,
            wait_limit_ns: int = 1_000_000_000) -> TdOptions:
    o = TdOptions()
    lib().td_options_default(ctypes.byref(o))
    o.precision, o.path, o.refine, o.wait_limit_ns = precision, path, refine, wait_limit_ns
    return o


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Segment:
    """One analysis segment (td_segment): ACF + gap mask, factored on device."""

    def __init__(self, acf, mask=None, stream=None, factor: bool = True):
        acf = np.ascontiguousarray(acf, dtype=np.float64)
        self.n = int(acf.shape[0])
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        h = ctypes.c_void_p()
        st = _stream_ptr(stream)
        _check(lib().td_segment_create(acf.ctypes.data, self.n, None if m is None else m.ctypes.data,
                                       st, ctypes.byref(h)))
        self.handle = h
        if factor:
            self.factor(stream)

    def factor(self, stream=None):
        _check(lib().td_factor(self.handle, _stream_ptr(stream)))

    def loglike_gather_into(self, R, logL, opt: TdOptions | None = None, chi2=None, stream=None):
        """td_loglike_batch_gather: R CUDA float32 (K, ldr >= n), every sample of the
        segment; the kept rows are gathered on the device."""
        _check(lib().td_loglike_batch_gather(self.handle, R.data_ptr(), int(R.stride(0)), int(R.shape[0]),
                                             logL.data_ptr(), None if opt is None else ctypes.byref(opt),
                                             None if chi2 is None else chi2.data_ptr(), _stream_ptr(stream)))

    def save(self, path, stream=None):
        """td_segment_save: the resident evaluation state to a file."""
        _check(lib().td_segment_save(self.handle, os.fsencode(path), _stream_ptr(stream)))

    @classmethod
    def load(cls, path, stream=None) -> "Segment":
        """td_segment_load: a new segment from a file written by save()."""
        h = ctypes.c_void_p()
        _check(lib().td_segment_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(h)))
        seg = cls.__new__(cls)
        seg.handle = h
        seg.n = None
        return seg

    @property
    def n_kept(self) -> int:
        return int(lib().td_kept(self.handle))

    @property
    def logdet(self) -> float:
        v = ctypes.c_double()
        _check(lib().td_logdet(self.handle, ctypes.byref(v)))
        return v.value

    @property
    def last_pivot(self) -> int:
        return int(lib().td_last_pivot(self.handle))

    @property
    def resident_bytes(self) -> int:
        return int(lib().td_resident_bytes(self.handle))

    def release_fp64(self):
        _check(lib().td_segment_release_fp64(self.handle))

    def gs_prepare(self, stream=None):
        """td_gs_prepare: Gohberg-Semencul spectra for path TD_PATH_GSCE (gap-free, 1024 <= N <= 32768)."""
        _check(lib().td_gs_prepare(self.handle, _stream_ptr(stream)))

    def reserve(self, K: int, opt: TdOptions | None = None):
        _check(lib().td_reserve(self.handle, int(K), None if opt is None else ctypes.byref(opt)))

    def loglike_into(self, R, logL, opt: TdOptions | None = None, chi2=None, stream=None, ldr=None):
        """R: CUDA float32 tensor, shape (K, ldr) row-major == N' x K column-major.
        logL (and chi2): CUDA float64 tensors of K entries."""
        K = int(R.shape[0])
        ld = int(R.stride(0)) if ldr is None else int(ldr)
        _check(lib().td_loglike_batch(self.handle, R.data_ptr(), ld, K, logL.data_ptr(),
                                      None if opt is None else ctypes.byref(opt),
                                      None if chi2 is None else chi2.data_ptr(), _stream_ptr(stream)))

    def loglike(self, R, opt: TdOptions | None = None, with_chi2: bool = False, stream=None):
        import torch
        K = int(R.shape[0])
        logL = torch.empty(K, dtype=torch.float64, device=R.device)
        chi2 = torch.empty(K, dtype=torch.float64, device=R.device) if with_chi2 else None
        self.loglike_into(R, logL, opt, chi2, stream)
        return (logL, chi2) if with_chi2 else logL

    def loglike_noalloc_into(self, R, logL, chi2=None, stream=None):
        """td_loglike_batch_noalloc: default options, scratch in the library's
        fixed device array (no device allocation by this call)."""
        _check(lib().td_loglike_batch_noalloc(self.handle, R.data_ptr(), int(R.stride(0)), int(R.shape[0]),
                                              logL.data_ptr(), None if chi2 is None else chi2.data_ptr(),
                                              _stream_ptr(stream)))

    def loglike_host_into(self, R, logL, opt: TdOptions | None = None, chi2=None, stream=None):
        """td_loglike_batch_host: R a host float32 array/tensor (K, ldr) (row-major
        == N' x K column-major), logL (and chi2) host float64 of K entries.
        Pinned torch tensors let the copies overlap the evaluation."""
        def ptr(x):
            return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        K, ldr = int(R.shape[0]), int(R.stride(0) if hasattr(R, "data_ptr") else R.strides[0] // 4)
        _check(lib().td_loglike_batch_host(self.handle, ptr(R), ldr, K, ptr(logL),
                                           None if opt is None else ctypes.byref(opt),
                                           None if chi2 is None else ptr(chi2), _stream_ptr(stream)))

    def set_data(self, d, opt: TdOptions | None = None, stream=None):
        """td_set_data: the data vector (float64, N' kept samples; numpy or torch)."""
        if hasattr(d, "data_ptr"):
            ptr, keep = d.data_ptr(), d
        else:
            keep = np.ascontiguousarray(d, dtype=np.float64)
            ptr = keep.ctypes.data
        _check(lib().td_set_data(self.handle, ptr, None if opt is None else ctypes.byref(opt), _stream_ptr(stream)))

    @property
    def data_inner(self) -> float:
        v = ctypes.c_double()
        _check(lib().td_data_inner(self.handle, ctypes.byref(v)))
        return v.value

    def template_into(self, H, logL, chi2=None, hh=None, dh=None, rho_mf=None, rho_eff2=None,
                      opt: TdOptions | None = None, stream=None):
        """td_template_batch: H CUDA float32 (K, ldh); outputs CUDA float64 (K,) or None."""
        p = (lambda x: None if x is None else x.data_ptr())
        out = TemplateOut(p(logL), p(chi2), p(hh), p(dh), p(rho_mf), p(rho_eff2))
        _check(lib().td_template_batch(self.handle, H.data_ptr(), int(H.stride(0)), int(H.shape[0]),
                                       ctypes.byref(out), None if opt is None else ctypes.byref(opt),
                                       _stream_ptr(stream)))

    def project_into(self, hp, hc, fp, fc, offset, logL, chi2=None, hh=None, dh=None, rho_mf=None,
                     rho_eff2=None, lw=None, opt: TdOptions | None = None, stream=None):
        """td_project_batch: hp, hc CUDA float32 (K, ldw) (hc may be None);
        fp, fc CUDA float64 (K,); offset CUDA int64 (K,); outputs CUDA float64
        (K,) or None.  lw defaults to hp's row length."""
        p = (lambda x: None if x is None else x.data_ptr())
        out = TemplateOut(p(logL), p(chi2), p(hh), p(dh), p(rho_mf), p(rho_eff2))
        if hc is not None and hc.stride(0) != hp.stride(0):
            raise ValueError("hp and hc need the same leading dimension")
        lw = int(hp.shape[1]) if lw is None else int(lw)
        _check(lib().td_project_batch(self.handle, hp.data_ptr(), p(hc), int(hp.stride(0)), lw, int(hp.shape[0]),
                                      fp.data_ptr(), p(fc), offset.data_ptr(), ctypes.byref(out),
                                      None if opt is None else ctypes.byref(opt), _stream_ptr(stream)))

    def profile(self, enable: bool = True):
        _check(lib().td_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self):
        """(dominant-kernel ms summed, dominant launches, kernels launched)."""
        ms, nd, nk = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().td_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(nd), ctypes.byref(nk)))
        return ms.value, nd.value, nk.value

    def profile_clock(self, stream=None) -> float:
        """SM clock (MHz) the split-product kernel ran at since the last read."""
        mhz = ctypes.c_double()
        _check(lib().td_profile_clock(self.handle, _stream_ptr(stream), ctypes.byref(mhz)))
        return mhz.value

    def check(self, stream=None):
        _check(lib().td_check(self.handle, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().td_segment_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TD_FACTOR_NO_FP64 = 1
TD_FACTOR_FP64_CORES = 2


def factor_many(segments, flags: int = TD_FACTOR_NO_FP64, stream=None):
    """td_factor_many: factor segments created with factor=False (gap-free ones
    by the O(N^2) Levinson-Durbin operator build when flags has NO_FP64)."""
    n = len(segments)
    H = (ctypes.c_void_p * n)(*[s.handle.value for s in segments])
    _check(lib().td_factor_many(H, n, int(flags), _stream_ptr(stream)))


def loglike_grouped(segments, Rs, logLs, opt: TdOptions | None = None, stream=None):
    n = len(segments)
    H = (ctypes.c_void_p * n)(*[s.handle.value for s in segments])
    RP = (ctypes.c_void_p * n)(*[r.data_ptr() for r in Rs])
    LD = (ctypes.c_int64 * n)(*[int(r.stride(0)) for r in Rs])
    KK = (ctypes.c_int64 * n)(*[int(r.shape[0]) for r in Rs])
    LP = (ctypes.c_void_p * n)(*[x.data_ptr() for x in logLs])
    _check(lib().td_loglike_grouped(H, RP, LD, KK, LP, n, None if opt is None else ctypes.byref(opt),
                                    _stream_ptr(stream)))


class Group:
    """A grouped-evaluation plan (td_group): many segments, one launch."""

    def __init__(self, segments, Rs, logLs, chi2s=None, opt: TdOptions | None = None, stream=None):
        n = len(segments)
        self._keep = (list(segments), list(Rs), list(logLs), list(chi2s) if chi2s else None)
        H = (ctypes.c_void_p * n)(*[s.handle.value for s in segments])
        RP = (ctypes.c_void_p * n)(*[r.data_ptr() for r in Rs])
        LD = (ctypes.c_int64 * n)(*[int(r.stride(0)) for r in Rs])
        KK = (ctypes.c_int64 * n)(*[int(r.shape[0]) for r in Rs])
        LP = (ctypes.c_void_p * n)(*[x.data_ptr() for x in logLs])
        CP = None if not chi2s else (ctypes.c_void_p * n)(*[x.data_ptr() for x in chi2s])
        h = ctypes.c_void_p()
        _check(lib().td_group_create(H, RP, LD, KK, LP, CP, n, None if opt is None else ctypes.byref(opt),
                                     _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h

    def set_joint(self, joint):
        """td_group_set_joint: joint = CUDA float64 (K,) summed logL over the segments, or None."""
        self._joint = joint
        _check(lib().td_group_set_joint(self.handle, None if joint is None else joint.data_ptr()))

    def launch(self, stream=None):
        _check(lib().td_group_launch(self.handle, _stream_ptr(stream)))

    def graph_launch(self, stream=None):
        _check(lib().td_group_graph_launch(self.handle, _stream_ptr(stream)))

    def tune(self, stream=None) -> float:
        ms = ctypes.c_double()
        _check(lib().td_group_tune(self.handle, _stream_ptr(stream), ctypes.byref(ms)))
        return ms.value

    def check(self, stream=None):
        _check(lib().td_group_check(self.handle, _stream_ptr(stream)))

    def clock(self, stream=None) -> float:
        """SM clock (MHz) the product launches ran at since the last read."""
        mhz = ctypes.c_double()
        _check(lib().td_group_clock(self.handle, _stream_ptr(stream), ctypes.byref(mhz)))
        return mhz.value

    def shape(self):
        bn, sf, ni = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib().td_group_shape(self.handle, ctypes.byref(bn), ctypes.byref(sf), ctypes.byref(ni))
        return bn.value, sf.value, ni.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().td_group_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """td_server: continuous-batching likelihood server (see include/td.h)."""

    PENDING, RUNNING, DONE, CANCELLED, FAILED = range(5)

    def __init__(self, max_batch_cols=4096, max_pending_cols=1 << 20, resident_bytes_budget=0, n_streams=4,
                 precision=TD_PREC_AUTO, max_kept=32768, gs_gapfree=False, deterministic=False,
                 host_spill_bytes=0):
        c = ServerConfig()
        lib().td_server_config_default(ctypes.byref(c))
        c.max_batch_cols, c.max_pending_cols = max_batch_cols, max_pending_cols
        c.resident_bytes_budget, c.n_streams, c.precision, c.max_kept = (resident_bytes_budget, n_streams,
                                                                         precision, max_kept)
        c.gs_gapfree = 1 if gs_gapfree else 0
        c.deterministic = 1 if deterministic else 0
        c.host_spill_bytes = int(host_spill_bytes)
        h = ctypes.c_void_p()
        _check(lib().td_server_create(ctypes.byref(c), ctypes.byref(h)))
        self.handle = h

    def add_segment(self, acf, mask=None) -> int:
        acf = np.ascontiguousarray(acf, dtype=np.float64)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        sid = ctypes.c_int64()
        _check(lib().td_server_add_segment(self.handle, acf.ctypes.data, int(acf.shape[0]),
                                           None if m is None else m.ctypes.data, ctypes.byref(sid)))
        return sid.value

    def set_budget(self, resident_bytes_budget: int):
        _check(lib().td_server_set_budget(self.handle, int(resident_bytes_budget)))

    def prefetch(self, seg_id: int):
        _check(lib().td_server_prefetch(self.handle, int(seg_id)))

    def submit(self, seg_id: int, R, logL) -> int:
        """R: CUDA float32 (K, ldr); logL: CUDA float64 (K,).  Raises TdError(TD_ERR_BUSY) if refused."""
        t = ctypes.c_int64()
        _check(lib().td_server_submit(self.handle, int(seg_id), R.data_ptr(), int(R.stride(0)), int(R.shape[0]),
                                      logL.data_ptr(), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int()
        _check(lib().td_server_poll(self.handle, int(ticket), ctypes.byref(st)))
        return st.value

    def latency_us(self, ticket: int) -> float:
        """td_server_latency: submission-to-completion time of a finished request."""
        v = ctypes.c_double()
        _check(lib().td_server_latency(self.handle, int(ticket), ctypes.byref(v)))
        return v.value

    def wait(self, ticket: int, timeout_us: int = 60_000_000):
        _check(lib().td_server_wait(self.handle, int(ticket), int(timeout_us)))

    def cancel(self, ticket: int):
        _check(lib().td_server_cancel(self.handle, int(ticket)))

    def pause(self, paused: bool = True):
        _check(lib().td_server_pause(self.handle, 1 if paused else 0))

    def drain(self, timeout_us: int = 120_000_000):
        _check(lib().td_server_drain(self.handle, int(timeout_us)))

    def replay(self, t_submit_s, seg_ids, Rs, logLs):
        n = len(t_submit_s)
        T = np.ascontiguousarray(t_submit_s, dtype=np.float64)
        S = np.ascontiguousarray(seg_ids, dtype=np.int64)
        RP = np.array([r.data_ptr() for r in Rs], dtype=np.uint64)
        LD = np.array([int(r.stride(0)) for r in Rs], dtype=np.int64)
        KK = np.array([int(r.shape[0]) for r in Rs], dtype=np.int64)
        LP = np.array([x.data_ptr() for x in logLs], dtype=np.uint64)
        tickets = np.zeros(n, dtype=np.int64)
        _check(lib().td_server_replay(self.handle, T.ctypes.data, S.ctypes.data, RP.ctypes.data, LD.ctypes.data,
                                      KK.ctypes.data, LP.ctypes.data, n, tickets.ctypes.data))
        return tickets

    def stats(self, reset: bool = False) -> dict:
        s = ServerStats()
        _check(lib().td_server_get_stats(self.handle, ctypes.byref(s), 1 if reset else 0))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().td_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_bounded_wait(limit_ns: int, stream=None) -> int:
    """Run the bounded-wait probe; returns the td_status (TD_ERR_TIMEOUT expected)."""
    return int(lib().td_debug_bounded_wait(int(limit_ns), _stream_ptr(stream)))

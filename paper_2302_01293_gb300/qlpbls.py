"""Thin ctypes binding of libqlpbls (include/qlp_bls.h), same names as the C ABI.

Argument marshalling only: PyTorch supplies device memory and the stream, every
step of the search runs in the library's CUDA kernels. There is no CPU path:
loading fails loudly when the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

PHASE_FP64, PHASE_DF, PHASE_FP32 = 0, 1, 2
SUM_PLAIN, SUM_COMP, SUM_FIXED, SUM_FIXED64 = 0, 1, 2, 3
BIN_SHARED, BIN_PER_Q = 0, 1
MAD_RAW, MAD_RESID = 0, 1
METHOD_AUTO, METHOD_POINTS, METHOD_CELLS = 0, 1, 2
TREND_DOUBLES = 84
CNN_ACT, CNN_GACT, CNN_LOGIT, CNN_DLOGIT = 0, 1, 2, 3
CNN_IN_CH = 6  # network input channels: S/N, mask, S/N at the bins of 2P, P/2, 3P, P/3

STAR_UNSORTED, STAR_TOO_FEW, STAR_EMPTY_GRID, STAR_NBINS_CAP, STAR_ZERO_MAD = 1, 2, 4, 8, 16

BEST_DTYPE = np.dtype([("f_idx", "<i8"), ("f", "<f8"), ("period", "<f8"), ("t0", "<f8"),
                       ("q", "<f8"), ("depth", "<f8"), ("sr", "<f8"), ("snr", "<f8"),
                       ("j", "<i4"), ("k", "<i4"), ("m", "<i4"), ("nbins", "<i4"),
                       ("status", "<i4"), ("pad", "<i4")])
assert BEST_DTYPE.itemsize == 88

# qlp_bls_cand_stats
STATS_DTYPE = np.dtype([("t0", "<f8"), ("depth", "<f8"), ("q", "<f8"), ("q_in", "<f8"), ("z", "<f8"),
                        ("chi2", "<f8"), ("sigma_w", "<f8"), ("sigma_r", "<f8"), ("depth_mean", "<f8"),
                        ("snr_pink", "<f8"), ("n_fit", "<i4"), ("n_in", "<i4"), ("n_before", "<i4"),
                        ("n_after", "<i4"), ("n_transits", "<i4"), ("iterations", "<i4"), ("status", "<i4"),
                        ("detected", "<i4")])
assert STATS_DTYPE.itemsize == 112


class CParams(ctypes.Structure):
    _fields_ = [("samples_per_peak", ctypes.c_double), ("dlogq", ctypes.c_double),
                ("noverlap", ctypes.c_double), ("qmin_fac", ctypes.c_double),
                ("qmax_fac", ctypes.c_double), ("pmin_aR", ctypes.c_double),
                ("gap_days", ctypes.c_double), ("rho_default", ctypes.c_double),
                ("nbins_cap", ctypes.c_int32), ("phase_mode", ctypes.c_int32),
                ("sum_mode", ctypes.c_int32), ("mad_mode", ctypes.c_int32),
                ("chunk_freqs", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("n_threads", ctypes.c_int32), ("tile_points", ctypes.c_int32),
                ("method", ctypes.c_int32), ("grid_mode", ctypes.c_int32),
                ("coarse_bins", ctypes.c_int32), ("cell_window", ctypes.c_int32),
                ("coarse_pmin", ctypes.c_double), ("coarse_pmax", ctypes.c_double),
                ("bin_mode", ctypes.c_int32), ("work_loop_bound", ctypes.c_int32)]


@dataclasses.dataclass
class Params:
    samples_per_peak: float = 2.0
    dlogq: float = 0.1
    noverlap: float = 3.0
    qmin_fac: float = 0.5
    qmax_fac: float = 2.0
    pmin_aR: float = 2.0
    gap_days: float = 27.4
    rho_default: float = 1.41
    nbins_cap: int = 8192
    phase_mode: int = PHASE_DF
    sum_mode: int = SUM_FIXED
    mad_mode: int = MAD_RAW
    chunk_freqs: int = 0
    warps_per_block: int = 0
    n_threads: int = 0
    tile_points: int = 0
    method: int = 0
    grid_mode: int = 0
    coarse_bins: int = 4096
    cell_window: int = 0
    coarse_pmin: float = 0.1
    coarse_pmax: float = 400.0
    bin_mode: int = 0
    work_loop_bound: int = 0

    def to_c(self) -> CParams:
        c = CParams()
        for f in dataclasses.fields(self):
            setattr(c, f.name, getattr(self, f.name))
        return c

    @classmethod
    def from_c(cls, c: CParams) -> "Params":
        return cls(**{f.name: getattr(c, f.name) for f in dataclasses.fields(cls)})


ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_DEVICE, ERR_UNSUPPORTED = -1, -2, -3, -4, -5
DEVERR_QUEUE, DEVERR_NBINS, DEVERR_SNR_BINS, DEVERR_COPY, DEVERR_RANGE = 1, 2, 4, 32, 64


class QlpError(RuntimeError):
    """A library call returned a non-zero status; .code holds it (ERR_*)."""

    def __init__(self, msg: str, code: int = 0):
        super().__init__(msg)
        self.code = code


_lib = None
_lock = threading.Lock()

_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i32, _i64, _d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


def lib():
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            L.qlp_bls_params_default.argtypes = [_P(CParams)]
            L.qlp_bls_params_default.restype = None
            L.qlp_bls_plan.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _P(_vp)]
            L.qlp_bls_plan.restype = ctypes.c_int
            L.qlp_bls_plan_info.argtypes = [_vp, _P(_i64), _vp, _vp, _vp, _P(_i64), _P(_d)]
            L.qlp_bls_plan_info.restype = ctypes.c_int
            L.qlp_bls_plan_stats.argtypes = [_vp, _P(_d), _P(_d), _P(_d), _P(_i32), _P(_i32)]
            L.qlp_bls_plan_stats.restype = ctypes.c_int
            L.qlp_bls_plan_exact_stats.argtypes = [_vp, _P(_i32), _P(_d), _P(_d)]
            L.qlp_bls_plan_exact_stats.restype = ctypes.c_int
            L.qlp_bls_plan_narrow_stats.argtypes = [_vp, _P(_i32), _P(_d), _P(_d)]
            L.qlp_bls_plan_narrow_stats.restype = ctypes.c_int
            L.qlp_bls_plan_launches.argtypes = [_vp, _P(_i32)]
            L.qlp_bls_plan_launches.restype = ctypes.c_int
            L.qlp_bls_plan_times.argtypes = [_vp, _P(_d)]
            L.qlp_bls_plan_times.restype = ctypes.c_int
            L.qlp_bls_kernel_timing.argtypes = [_vp, _i32]
            L.qlp_bls_kernel_timing.restype = ctypes.c_int
            L.qlp_bls_kernel_time.argtypes = [_vp, _P(ctypes.c_float), _P(_i32)]
            L.qlp_bls_kernel_time.restype = ctypes.c_int
            L.qlp_bls_search.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.qlp_bls_search.restype = ctypes.c_int
            L.qlp_bls_snr.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.qlp_bls_snr.restype = ctypes.c_int
            L.qlp_bls_run_host.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                           _vp, _vp, _i64, _vp, _P(_i64)]
            L.qlp_bls_run_host.restype = ctypes.c_int
            L.qlp_bls_device_status.argtypes = [_vp, _vp, _P(_i32)]
            L.qlp_bls_device_status.restype = ctypes.c_int
            L.qlp_bls_plan_destroy.argtypes = [_vp]
            L.qlp_bls_plan_destroy.restype = None
            L.qlp_bls_star_grid.argtypes = [_P(CParams), _i64, _vp, _vp, _vp, _d, _i64, _vp, _vp,
                                            _P(_i32), _P(_d), _P(_d), _P(_d), _P(_d), _vp, _vp, _i64,
                                            _P(_i64)]
            L.qlp_bls_star_grid.restype = ctypes.c_int
            L.qlp_bls_batch_grid.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                             _i64]
            L.qlp_bls_batch_grid.restype = ctypes.c_int
            L.qlp_bls_search_static.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _d, _i32, _vp,
                                                _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.qlp_bls_search_static.restype = ctypes.c_int
            L.qlp_cnn_pack_w64.argtypes = [_vp, _vp, _i32, _vp]
            L.qlp_cnn_pack_w64.restype = ctypes.c_int
            L.qlp_cnn_conv64.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]
            L.qlp_cnn_conv64.restype = ctypes.c_int
            L.qlp_cnn_wgrad64_workspace.argtypes = [_i32, _i32]
            L.qlp_cnn_wgrad64_workspace.restype = _i64
            L.qlp_cnn_conv64_wgrad.argtypes = [_vp, _vp, _vp, _vp, _i32, _i32, _vp, _vp]
            L.qlp_cnn_conv64_wgrad.restype = ctypes.c_int
            L.qlp_cnn_n_params.argtypes = []
            L.qlp_cnn_n_params.restype = ctypes.c_int32
            L.qlp_cnn_create.argtypes = [_i32, _i32, ctypes.c_uint64, _P(_vp)]
            L.qlp_cnn_create.restype = ctypes.c_int
            L.qlp_cnn_destroy.argtypes = [_vp]
            L.qlp_cnn_destroy.restype = None
            L.qlp_cnn_set_params.argtypes = [_vp, _vp, _vp]
            L.qlp_cnn_set_params.restype = ctypes.c_int
            L.qlp_cnn_get_params.argtypes = [_vp, _vp, _vp, _vp]
            L.qlp_cnn_get_params.restype = ctypes.c_int
            L.qlp_cnn_forward.argtypes = [_vp, _vp, _i32, _vp, _vp]
            L.qlp_cnn_forward.restype = ctypes.c_int
            L.qlp_cnn_backward.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, _vp]
            L.qlp_cnn_backward.restype = ctypes.c_int
            L.qlp_cnn_adam_step.argtypes = [_vp, ctypes.c_float, _vp]
            L.qlp_cnn_adam_step.restype = ctypes.c_int
            L.qlp_cnn_train_step.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float, _vp]
            L.qlp_cnn_train_step.restype = ctypes.c_int
            L.qlp_cnn_loss.argtypes = [_vp, _P(ctypes.c_float), _P(_i32), _vp]
            L.qlp_cnn_loss.restype = ctypes.c_int
            L.qlp_cnn_last_error.argtypes = []
            L.qlp_cnn_last_error.restype = ctypes.c_char_p
            L.qlp_bls_plan_windows.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                               _vp, _vp, _vp, _P(_vp)]
            L.qlp_bls_plan_windows.restype = ctypes.c_int
            L.qlp_bls_plan_windows_from.argtypes = [_vp, _P(CParams), _vp, _vp, _vp, _vp, _P(_vp)]
            L.qlp_bls_plan_windows_from.restype = ctypes.c_int
            L.qlp_bls_snr_trend.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.qlp_bls_snr_trend.restype = ctypes.c_int
            L.qlp_bls_coarse_tensor.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp]
            L.qlp_bls_coarse_periods.argtypes = [_P(CParams), _i32, _vp, _vp]
            L.qlp_bls_coarse_periods.restype = ctypes.c_int
            L.qlp_bls_coarse_bins.argtypes = [_P(CParams), _i32, _vp, _vp]
            L.qlp_bls_coarse_bins.restype = ctypes.c_int
            L.qlp_bls_proposal_windows.argtypes = [_P(CParams), _i32, _vp, _i32, _d, _vp, _vp, _vp, _i64]
            L.qlp_bls_proposal_windows.restype = ctypes.c_int
            L.qlp_bls_coarse_tensor.restype = ctypes.c_int
            L.qlp_cnn_topk.argtypes = [_vp, _vp, _i32, _i32, _i32, _vp, _vp]
            L.qlp_cnn_topk.restype = ctypes.c_int
            L.qlp_cnn_shape.argtypes = [_vp, _P(_i32), _P(_i32)]
            L.qlp_cnn_shape.restype = ctypes.c_int
            L.qlp_cnn_get_tensor.argtypes = [_vp, _i32, _i32, _i32, _vp, _i64, _vp]
            L.qlp_cnn_get_tensor.restype = ctypes.c_int
            L.qlp_set_device_budget.argtypes = [_i64]
            L.qlp_set_device_budget.restype = ctypes.c_int
            L.qlp_device_bytes_held.argtypes = []
            L.qlp_device_bytes_held.restype = _i64
            L.qlp_cnn_save.argtypes = [_vp, ctypes.c_char_p, _vp]
            L.qlp_cnn_save.restype = ctypes.c_int
            L.qlp_cnn_load.argtypes = [_vp, ctypes.c_char_p, _vp]
            L.qlp_cnn_load.restype = ctypes.c_int
            L.qlp_bls_search_learned.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                                 _i32, ctypes.c_double, _vp, _vp, _vp]
            L.qlp_bls_search_learned.restype = ctypes.c_int
            L.qlp_bls_autotune.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp,
                                           _P(CParams), _P(_i32)]
            L.qlp_bls_autotune.restype = ctypes.c_int
            L.qlp_bls_graph_capture.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.qlp_bls_graph_capture.restype = ctypes.c_int
            L.qlp_bls_graph_launch.argtypes = [_vp, _i32, _vp]
            L.qlp_bls_graph_launch.restype = ctypes.c_int
            L.qlp_bls_candidate_stats.argtypes = [_vp, _vp, _vp, _vp]
            L.qlp_bls_candidate_stats.restype = ctypes.c_int
            L.qlp_bls_top_peaks.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_double, _vp]
            L.qlp_bls_top_peaks.restype = ctypes.c_int
            L.qlp_bls_search_multi.argtypes = [_P(CParams), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp,
                                               _vp]
            L.qlp_bls_search_multi.restype = ctypes.c_int
            L.qlp_strerror.argtypes = [ctypes.c_int]
            L.qlp_strerror.restype = ctypes.c_char_p
            L.qlp_last_cuda_error.argtypes = []
            L.qlp_last_cuda_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        L = lib()
        msg = L.qlp_strerror(rc).decode()
        cu = L.qlp_last_cuda_error().decode()
        raise QlpError(f"{what}: {msg} ({rc}){' / ' + cu if cu else ''}", rc)


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host_inputs(offsets, t, y, dy, rho, rstar):
    offsets = np.ascontiguousarray(offsets, np.int64)
    t = np.ascontiguousarray(t, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    dy = np.ascontiguousarray(dy, np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
    rstar = None if rstar is None else np.ascontiguousarray(rstar, np.float64)
    return offsets, t, y, dy, rho, rstar


class Plan:
    """A library-owned search plan (qlp_bls_plan) and its sizes."""

    def __init__(self, offsets, t, y, dy, rho=None, rstar=None, params: Params | None = None,
                 stream=None, windows=None):
        """windows: optional (win_offsets int64 [n_stars+1], f_lo, f_hi) restricting
        each star's grid (qlp_bls_plan_windows)."""
        import torch
        self._h = ctypes.c_void_p()
        L = lib()
        offsets, t, y, dy, rho, rstar = _host_inputs(offsets, t, y, dy, rho, rstar)
        self.n_stars = int(offsets.shape[0] - 1)
        self.params = params or Params()
        cp = self.params.to_c()
        self.device = torch.device("cuda", torch.cuda.current_device())
        if windows is None:
            rc = L.qlp_bls_plan(ctypes.byref(cp), self.n_stars, _np_ptr(offsets), _np_ptr(t), _np_ptr(y),
                                _np_ptr(dy), _np_ptr(rho), _np_ptr(rstar), _stream_ptr(stream),
                                ctypes.byref(self._h))
            _check(rc, "qlp_bls_plan")
        else:
            wo = np.ascontiguousarray(windows[0], np.int64)
            wl = np.ascontiguousarray(windows[1], np.float64)
            wh = np.ascontiguousarray(windows[2], np.float64)
            rc = L.qlp_bls_plan_windows(ctypes.byref(cp), self.n_stars, _np_ptr(offsets), _np_ptr(t),
                                        _np_ptr(y), _np_ptr(dy), _np_ptr(rho), _np_ptr(rstar), _np_ptr(wo),
                                        _np_ptr(wl), _np_ptr(wh), _stream_ptr(stream), ctypes.byref(self._h))
            _check(rc, "qlp_bls_plan_windows")
        self._load_info()

    @classmethod
    def windows_from(cls, base: "Plan", windows, params: "Params | None" = None, stream=None) -> "Plan":
        """qlp_bls_plan_windows_from: the windowed plan of base's stars (windows as in the
        constructor) made from base's point analysis and device copy of the points."""
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p()
        self.n_stars = base.n_stars
        self.params = params or Params()
        self.device = base.device
        cp = self.params.to_c()
        wo = np.ascontiguousarray(windows[0], np.int64)
        wl = np.ascontiguousarray(windows[1], np.float64)
        wh = np.ascontiguousarray(windows[2], np.float64)
        rc = lib().qlp_bls_plan_windows_from(base._h, ctypes.byref(cp), _np_ptr(wo), _np_ptr(wl), _np_ptr(wh),
                                             _stream_ptr(stream), ctypes.byref(self._h))
        _check(rc, "qlp_bls_plan_windows_from")
        self._load_info()
        return self

    def _load_info(self):
        L = lib()
        nft = _i64()
        npts = _i64()
        work = _d()
        L.qlp_bls_plan_info(self._h, ctypes.byref(nft), None, None, None, ctypes.byref(npts),
                            ctypes.byref(work))
        self.n_freq_total = int(nft.value)
        self.n_points = int(npts.value)
        self.work = float(work.value)
        self.freq_offsets = np.zeros(self.n_stars + 1, np.int64)
        self.freqs = np.zeros(self.n_freq_total, np.float64)
        self.star_status = np.zeros(self.n_stars, np.int32)
        _check(L.qlp_bls_plan_info(self._h, None, _np_ptr(self.freq_offsets), _np_ptr(self.freqs),
                                   _np_ptr(self.star_status), None, None), "qlp_bls_plan_info")
        wp, wc, ed, nc, nw = _d(), _d(), _d(), _i32(), _i32()
        _check(L.qlp_bls_plan_stats(self._h, ctypes.byref(wp), ctypes.byref(wc), ctypes.byref(ed),
                                    ctypes.byref(nc), ctypes.byref(nw)), "qlp_bls_plan_stats")
        self.work_points, self.work_cells, self.edges = wp.value, wc.value, ed.value
        self.n_cell_stars = int(nc.value)
        self.n_windowed = int(nw.value)
        ne, ee, eb = _i32(), _d(), _d()
        _check(L.qlp_bls_plan_exact_stats(self._h, ctypes.byref(ne), ctypes.byref(ee), ctypes.byref(eb)),
               "qlp_bls_plan_exact_stats")
        self.n_exact_stars = int(ne.value)
        self.exact_edges = ee.value
        self.exact_bins = eb.value
        _check(L.qlp_bls_plan_narrow_stats(self._h, ctypes.byref(ne), ctypes.byref(ee), ctypes.byref(eb)),
               "qlp_bls_plan_narrow_stats")
        self.n_narrow_stars = int(ne.value)
        self.narrow_edges = ee.value
        self.narrow_bins = eb.value
        _check(L.qlp_bls_plan_launches(self._h, ctypes.byref(ne)), "qlp_bls_plan_launches")
        self.search_launches = int(ne.value)

    def alloc_outputs(self):
        import torch
        n = max(self.n_freq_total, 1)
        dev = self.device
        return dict(sr=torch.empty(n, dtype=torch.float32, device=dev),
                    qidx=torch.empty(n, dtype=torch.uint8, device=dev),
                    kbin=torch.empty(n, dtype=torch.int32, device=dev),
                    s=torch.empty(n, dtype=torch.float32, device=dev),
                    r=torch.empty(n, dtype=torch.float32, device=dev),
                    snr=torch.empty(n, dtype=torch.float32, device=dev),
                    best=torch.empty(max(self.n_stars, 1) * BEST_DTYPE.itemsize, dtype=torch.uint8,
                                     device=dev))

    def search(self, out=None, stream=None):
        """qlp_bls_search into `out` (from alloc_outputs); returns `out`."""
        out = out or self.alloc_outputs()
        rc = lib().qlp_bls_search(self._h, _stream_ptr(stream), out["sr"].data_ptr(),
                                  out["qidx"].data_ptr(), out["kbin"].data_ptr(), out["s"].data_ptr(),
                                  out["r"].data_ptr())
        _check(rc, "qlp_bls_search")
        return out

    def snr(self, out, stream=None, trend_in=None, trend_out=None):
        """qlp_bls_snr (or qlp_bls_snr_trend when a trend tensor is given) on the
        arrays of a previous search; returns `out`."""
        if trend_in is None and trend_out is None:
            rc = lib().qlp_bls_snr(self._h, _stream_ptr(stream), out["sr"].data_ptr(),
                                   out["qidx"].data_ptr(), out["kbin"].data_ptr(), out["s"].data_ptr(),
                                   out["r"].data_ptr(), out["snr"].data_ptr(), out["best"].data_ptr())
            _check(rc, "qlp_bls_snr")
        else:
            rc = lib().qlp_bls_snr_trend(self._h, _stream_ptr(stream), out["sr"].data_ptr(),
                                         out["qidx"].data_ptr(), out["kbin"].data_ptr(), out["s"].data_ptr(),
                                         out["r"].data_ptr(),
                                         trend_in.data_ptr() if trend_in is not None else None,
                                         trend_out.data_ptr() if trend_out is not None else None,
                                         out["snr"].data_ptr(), out["best"].data_ptr())
            _check(rc, "qlp_bls_snr_trend")
        return out

    def alloc_trend(self):
        import torch
        return torch.zeros(max(self.n_stars, 1) * TREND_DOUBLES, dtype=torch.float64, device=self.device)

    def coarse_tensor(self, out, stream=None, snr_rows: bool = False):
        """qlp_bls_coarse_tensor: BF16 [n_stars, coarse_bins, CNN_IN_CH] network input; with
        snr_rows also the FP32 S/N per coarse bin [n_stars, coarse_bins]."""
        import torch
        nb = self.params.coarse_bins
        x0 = torch.empty(max(self.n_stars, 1), nb, CNN_IN_CH, dtype=torch.bfloat16, device=self.device)
        rows = torch.empty(max(self.n_stars, 1), nb, dtype=torch.float32, device=self.device) if snr_rows else None
        rc = lib().qlp_bls_coarse_tensor(self._h, _stream_ptr(stream), out["snr"].data_ptr(), nb,
                                         x0.data_ptr(), rows.data_ptr() if rows is not None else None)
        _check(rc, "qlp_bls_coarse_tensor")
        if snr_rows:
            return x0[: self.n_stars], rows[: self.n_stars]
        return x0[: self.n_stars]

    def device_status(self, stream=None) -> int:
        flags = _i32()
        rc = lib().qlp_bls_device_status(self._h, _stream_ptr(stream), ctypes.byref(flags))
        if rc not in (0, -4):
            _check(rc, "qlp_bls_device_status")
        return int(flags.value)

    def graph_capture(self, out, parts: int = 3):
        """qlp_bls_graph_capture: record the search (parts 1), the S/N (2) or both
        (3) into `out` (from alloc_outputs) as a CUDA graph of this plan."""
        _check(lib().qlp_bls_graph_capture(self._h, int(parts), out["sr"].data_ptr(), out["qidx"].data_ptr(),
                                           out["kbin"].data_ptr(), out["s"].data_ptr(), out["r"].data_ptr(),
                                           out["snr"].data_ptr(), out["best"].data_ptr()),
               "qlp_bls_graph_capture")
        return out

    def graph_launch(self, parts: int = 3, stream=None):
        _check(lib().qlp_bls_graph_launch(self._h, int(parts), _stream_ptr(stream)), "qlp_bls_graph_launch")

    def plan_times(self):
        """qlp_bls_plan_times: seconds of the plan's construction phases (host grid,
        host staging, device allocation, upload and plan-time kernels)."""
        v = (ctypes.c_double * 4)()
        _check(lib().qlp_bls_plan_times(self._h, v), "qlp_bls_plan_times")
        return dict(host_grid=v[0], host_staging=v[1], device_alloc=v[2], upload=v[3])

    def kernel_timing(self, enable: bool = True):
        """qlp_bls_kernel_timing: bracket the main search kernel of every later
        search (and graph captured afterwards) with CUDA events."""
        _check(lib().qlp_bls_kernel_timing(self._h, 1 if enable else 0), "qlp_bls_kernel_timing")

    def kernel_time(self):
        """qlp_bls_kernel_time: (milliseconds, kernel id) of the last search's main
        kernel; kernel 0 per-point, 1 compensated cell, 2 exact cell."""
        ms, k = ctypes.c_float(), _i32()
        _check(lib().qlp_bls_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(k)), "qlp_bls_kernel_time")
        return float(ms.value), int(k.value)

    def candidate_stats(self, out, stats=None, stream=None):
        """qlp_bls_candidate_stats on the best records in `out` (after snr); returns
        the device buffer of n_stars STATS_DTYPE records."""
        import torch
        if stats is None:
            stats = torch.empty(max(self.n_stars, 1) * STATS_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        _check(lib().qlp_bls_candidate_stats(self._h, _stream_ptr(stream), out["best"].data_ptr(), stats.data_ptr()),
               "qlp_bls_candidate_stats")
        return stats

    def top_peaks(self, out, n: int, sep: float = 0.01, stream=None):
        """qlp_bls_top_peaks on out["snr"]: device int32 [n_stars, n]."""
        import torch
        idx = torch.empty(max(self.n_stars, 1), int(n), dtype=torch.int32, device=self.device)
        _check(lib().qlp_bls_top_peaks(self._h, _stream_ptr(stream), out["snr"].data_ptr(), int(n), float(sep),
                                       idx.data_ptr()), "qlp_bls_top_peaks")
        return idx

    def stats_host(self, stats) -> np.ndarray:
        raw = stats.cpu().numpy()[: self.n_stars * STATS_DTYPE.itemsize]
        return raw.view(STATS_DTYPE).copy()

    def best_host(self, out) -> np.ndarray:
        raw = out["best"].cpu().numpy()[: self.n_stars * BEST_DTYPE.itemsize]
        return raw.view(BEST_DTYPE).copy()

    def star_slice(self, s: int) -> slice:
        return slice(int(self.freq_offsets[s]), int(self.freq_offsets[s + 1]))

    def close(self):
        if self._h and self._h.value:
            lib().qlp_bls_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_host(offsets, t, y, dy, rho=None, rstar=None, params: Params | None = None,
             sr_capacity: int = 0):
    """qlp_bls_run_host: host arrays in, host results out (best per star, and the
    SR / S/N spectra when sr_capacity >= the number of trial frequencies)."""
    L = lib()
    offsets, t, y, dy, rho, rstar = _host_inputs(offsets, t, y, dy, rho, rstar)
    n_stars = int(offsets.shape[0] - 1)
    cp = (params or Params()).to_c()
    best = np.zeros(max(n_stars, 1), BEST_DTYPE)
    sr = np.zeros(sr_capacity, np.float32) if sr_capacity > 0 else None
    snr = np.zeros(sr_capacity, np.float32) if sr_capacity > 0 else None
    nft = _i64()
    rc = L.qlp_bls_run_host(ctypes.byref(cp), n_stars, _np_ptr(offsets), _np_ptr(t), _np_ptr(y),
                            _np_ptr(dy), _np_ptr(rho), _np_ptr(rstar), _np_ptr(sr), _np_ptr(snr),
                            int(sr_capacity), _np_ptr(best), ctypes.byref(nft))
    _check(rc, "qlp_bls_run_host")
    return dict(best=best[:n_stars], sr=sr, snr=snr, n_freq_total=int(nft.value))


def autotune(offsets, t, y, dy, rho=None, rstar=None, params: Params | None = None,
             sample_stars: int = 256, stream=None):
    """qlp_bls_autotune: (tuned Params, whether the process cache answered)."""
    L = lib()
    offsets, t, y, dy, rho, rstar = _host_inputs(offsets, t, y, dy, rho, rstar)
    cp = (params or Params()).to_c()
    out = CParams()
    cached = _i32()
    rc = L.qlp_bls_autotune(ctypes.byref(cp), int(offsets.shape[0] - 1), _np_ptr(offsets), _np_ptr(t),
                            _np_ptr(y), _np_ptr(dy), _np_ptr(rho), _np_ptr(rstar), int(sample_stars),
                            _stream_ptr(stream), ctypes.byref(out), ctypes.byref(cached))
    _check(rc, "qlp_bls_autotune")
    return Params.from_c(out), bool(cached.value)


def star_grid(t, y, dy, rho=float("nan"), params: Params | None = None, windows=None):
    """qlp_bls_star_grid: the host plan of one star (no device work); windows is an
    optional list of (f_lo, f_hi) frequency windows."""
    L = lib()
    t = np.ascontiguousarray(t, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    dy = np.ascontiguousarray(dy, np.float64)
    cp = (params or Params()).to_c()
    wlo = whi = None
    if windows is not None:
        w = np.asarray(windows, np.float64).reshape(-1, 2)
        wlo, whi = np.ascontiguousarray(w[:, 0]), np.ascontiguousarray(w[:, 1])
    st, pmin, pmax, tref, base, nf = _i32(), _d(), _d(), _d(), _d(), _i64()
    args = [ctypes.byref(cp), t.shape[0], _np_ptr(t), _np_ptr(y), _np_ptr(dy), float(rho),
            0 if wlo is None else wlo.shape[0], _np_ptr(wlo), _np_ptr(whi),
            ctypes.byref(st), ctypes.byref(pmin), ctypes.byref(pmax), ctypes.byref(tref),
            ctypes.byref(base)]
    _check(L.qlp_bls_star_grid(*args, None, None, 0, ctypes.byref(nf)), "qlp_bls_star_grid")
    freqs = np.zeros(nf.value, np.float64)
    qmins = np.zeros(nf.value, np.float64)
    _check(L.qlp_bls_star_grid(*args, _np_ptr(freqs), _np_ptr(qmins), nf.value, ctypes.byref(nf)),
           "qlp_bls_star_grid")
    return dict(status=int(st.value), pmin=pmin.value, pmax=pmax.value, t_ref=tref.value,
                baseline=base.value, freqs=freqs, qmins=qmins)


def batch_grid(offsets, t, y, dy, rho=None, params: Params | None = None):
    """qlp_bls_batch_grid: the trial-frequency grids of a batch from the batch
    planner (host only); returns (star_status, freq_offsets, freqs)."""
    L = lib()
    offsets = np.ascontiguousarray(offsets, np.int64)
    n = offsets.shape[0] - 1
    t = np.ascontiguousarray(t, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    dy = np.ascontiguousarray(dy, np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
    cp = (params or Params()).to_c()
    status = np.zeros(n, np.int32)
    foff = np.zeros(n + 1, np.int64)
    args = [ctypes.byref(cp), n, _np_ptr(offsets), _np_ptr(t), _np_ptr(y), _np_ptr(dy), _np_ptr(rho),
            _np_ptr(status), _np_ptr(foff)]
    _check(L.qlp_bls_batch_grid(*args, None, 0), "qlp_bls_batch_grid")
    freqs = np.zeros(int(foff[-1]), np.float64)
    _check(L.qlp_bls_batch_grid(*args, _np_ptr(freqs), freqs.shape[0]), "qlp_bls_batch_grid")
    return status, foff, freqs


def set_device_budget(nbytes: int):
    """qlp_set_device_budget: cap the device bytes the library's plans and networks
    hold at once (0 = no cap)."""
    _check(lib().qlp_set_device_budget(int(nbytes)), "qlp_set_device_budget")


def device_bytes_held() -> int:
    """qlp_device_bytes_held: device bytes the library's plans and networks hold."""
    return int(lib().qlp_device_bytes_held())


def search_static(tp, y, dy, baseline, freqs, qmins, out, params: Params | None = None, stream=None,
                  flags=None):
    """qlp_bls_search_static: one star's search with no device allocation inside
    the call. tp, y, dy: device float64 tensors (t - t_min sorted, flux, error);
    freqs, qmins: host float64 arrays; out: dict of device tensors sr, qidx, kbin,
    s, r with at least len(freqs) entries (as from Plan.alloc_outputs); flags: an
    optional device int32 tensor that receives the call's device error bits."""
    L = lib()
    freqs = np.ascontiguousarray(freqs, np.float64)
    qmins = np.ascontiguousarray(qmins, np.float64)
    cp = (params or Params()).to_c()
    rc = L.qlp_bls_search_static(ctypes.byref(cp), int(tp.numel()), tp.data_ptr(), y.data_ptr(),
                                 dy.data_ptr(), float(baseline), int(freqs.shape[0]),
                                 _np_ptr(freqs), _np_ptr(qmins), _stream_ptr(stream),
                                 out["sr"].data_ptr(), out["qidx"].data_ptr(), out["kbin"].data_ptr(),
                                 out["s"].data_ptr(), out["r"].data_ptr(),
                                 flags.data_ptr() if flags is not None else None)
    _check(rc, "qlp_bls_search_static")
    return out


class CNN:
    """The proposal network (qlp_cnn_*): BF16 inputs [B][L][CNN_IN_CH] and FP32 labels
    [B][L] as device tensors; parameters as a host float32 array."""

    def __init__(self, max_batch: int, length: int = 4096, seed: int = 0):
        L = lib()
        self._h = ctypes.c_void_p()
        self.max_batch, self.length = int(max_batch), int(length)
        rc = L.qlp_cnn_create(self.max_batch, self.length, int(seed), ctypes.byref(self._h))
        _check(rc, "qlp_cnn_create")
        self.n_params = int(L.qlp_cnn_n_params())

    def _chk(self, rc, what):
        if rc != 0:
            msg = lib().qlp_cnn_last_error().decode()
            raise QlpError(f"{what}: {lib().qlp_strerror(rc).decode()} ({rc}) {msg}")

    def params(self, with_grads: bool = False):
        p = np.zeros(self.n_params, np.float32)
        g = np.zeros(self.n_params, np.float32) if with_grads else None
        self._chk(lib().qlp_cnn_get_params(self._h, _np_ptr(p), _np_ptr(g), _stream_ptr(None)),
                  "qlp_cnn_get_params")
        return (p, g) if with_grads else p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.shape[0] == self.n_params
        self._chk(lib().qlp_cnn_set_params(self._h, _np_ptr(p), _stream_ptr(None)), "qlp_cnn_set_params")

    def forward(self, x0, out=None, stream=None):
        import torch
        B = int(x0.shape[0])
        out = out if out is not None else torch.empty(B, self.length, dtype=torch.float32, device=x0.device)
        self._chk(lib().qlp_cnn_forward(self._h, x0.data_ptr(), B, out.data_ptr(), _stream_ptr(stream)),
                  "qlp_cnn_forward")
        return out

    def backward(self, x0, labels, pos_weight: float, stream=None):
        self._chk(lib().qlp_cnn_backward(self._h, x0.data_ptr(), labels.data_ptr(), int(x0.shape[0]),
                                         float(pos_weight), _stream_ptr(stream)), "qlp_cnn_backward")

    def adam_step(self, lr: float, stream=None):
        self._chk(lib().qlp_cnn_adam_step(self._h, float(lr), _stream_ptr(stream)), "qlp_cnn_adam_step")

    def train_step(self, x0, labels, pos_weight: float, lr: float, stream=None):
        self._chk(lib().qlp_cnn_train_step(self._h, x0.data_ptr(), labels.data_ptr(), int(x0.shape[0]),
                                           float(pos_weight), float(lr), _stream_ptr(stream)),
                  "qlp_cnn_train_step")

    def loss(self, stream=None) -> float:
        v = ctypes.c_float()
        e = _i32()
        rc = lib().qlp_cnn_loss(self._h, ctypes.byref(v), ctypes.byref(e), _stream_ptr(stream))
        self._chk(rc, "qlp_cnn_loss")
        return float(v.value)

    def tensor(self, which: int, layer: int, batch: int, stream=None) -> np.ndarray:
        """qlp_cnn_get_tensor: a kept tensor of the last forward / backward as a host
        array: ACT / GACT layer 1..5 as float32 [batch][len][64] (from BF16),
        LOGIT / DLOGIT as float32 [batch][len]."""
        if which in (CNN_ACT, CNN_GACT):
            raw = np.zeros((batch, self.length, 64), np.uint16)
        else:
            raw = np.zeros((batch, self.length), np.float32)
        self._chk(lib().qlp_cnn_get_tensor(self._h, int(which), int(layer), int(batch), _np_ptr(raw),
                                           raw.nbytes, _stream_ptr(stream)), "qlp_cnn_get_tensor")
        if raw.dtype == np.uint16:
            return (raw.astype(np.uint32) << 16).view(np.float32)
        return raw

    def save(self, path: str, stream=None):
        self._chk(lib().qlp_cnn_save(self._h, os.fsencode(path), _stream_ptr(stream)), "qlp_cnn_save")

    def load(self, path: str, stream=None):
        self._chk(lib().qlp_cnn_load(self._h, os.fsencode(path), _stream_ptr(stream)), "qlp_cnn_load")

    def close(self):
        if self._h and self._h.value:
            lib().qlp_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_w64(w, transpose: bool = False, stream=None):
    """qlp_cnn_pack_w64: FP32 weights [9][64][64] (device) -> the tensor-core
    operand layout (device uint8 [73728])."""
    import torch
    wpack = torch.empty(73728, dtype=torch.uint8, device=w.device)
    _check(lib().qlp_cnn_pack_w64(w.data_ptr(), wpack.data_ptr(), int(transpose), _stream_ptr(stream)),
           "qlp_cnn_pack_w64")
    return wpack


def conv64(x, wpack, bias=None, mask=None, relu: bool = True, out=None, err=None, stream=None):
    """qlp_cnn_conv64: y = conv(x) (+ bias, ReLU) for BF16 x [B][L][64] on the tensor cores."""
    import torch
    y = out if out is not None else torch.empty_like(x)
    err = err if err is not None else torch.zeros(1, dtype=torch.int32, device=x.device)
    _check(lib().qlp_cnn_conv64(x.data_ptr(), wpack.data_ptr(), bias.data_ptr() if bias is not None else None,
                                mask.data_ptr() if mask is not None else None, y.data_ptr(), int(x.shape[0]),
                                int(x.shape[1]), int(relu), err.data_ptr(), _stream_ptr(stream)),
           "qlp_cnn_conv64")
    return y


def conv64_wgrad(dy, x, stream=None):
    """qlp_cnn_conv64_wgrad: (dW [9, 64, 64], db [64]) FP32 of a 64 -> 64 layer."""
    import torch
    B, L = int(x.shape[0]), int(x.shape[1])
    ws = torch.empty(max(int(lib().qlp_cnn_wgrad64_workspace(B, L)), 1), dtype=torch.float32, device=x.device)
    out = torch.empty(9 * 64 * 64 + 64, dtype=torch.float32, device=x.device)
    err = torch.zeros(1, dtype=torch.int32, device=x.device)
    _check(lib().qlp_cnn_conv64_wgrad(dy.data_ptr(), x.data_ptr(), ws.data_ptr(), out.data_ptr(), B, L,
                                      err.data_ptr(), _stream_ptr(stream)), "qlp_cnn_conv64_wgrad")
    if int(err.item()) != 0:
        raise QlpError(f"qlp_cnn_conv64_wgrad: device error flags {int(err.item())}")
    return out[:9 * 64 * 64].view(9, 64, 64), out[9 * 64 * 64:]


def topk(logits, x0, k: int, stream=None):
    """qlp_cnn_topk: device int32 [batch, k] indices of the largest valid logits."""
    import torch
    B, L = int(logits.shape[0]), int(logits.shape[1])
    out = torch.empty(B, k, dtype=torch.int32, device=logits.device)
    rc = lib().qlp_cnn_topk(logits.data_ptr(), x0.data_ptr(), B, L, int(k), out.data_ptr(),
                            _stream_ptr(stream))
    _check(rc, "qlp_cnn_topk")
    return out


def coarse_periods(x, params: Params | None = None) -> np.ndarray:
    """qlp_bls_coarse_periods: the period of (fractional) coarse bin positions x."""
    x = np.ascontiguousarray(np.atleast_1d(x), np.float64)
    out = np.zeros(x.shape[0], np.float64)
    cp = (params or Params()).to_c()
    _check(lib().qlp_bls_coarse_periods(ctypes.byref(cp), int(x.shape[0]), _np_ptr(x), _np_ptr(out)),
           "qlp_bls_coarse_periods")
    return out


def coarse_bins(periods, params: Params | None = None) -> np.ndarray:
    """qlp_bls_coarse_bins: the nearest coarse bin of each period (-1 outside the grid)."""
    per = np.ascontiguousarray(np.atleast_1d(periods), np.float64)
    out = np.zeros(per.shape[0], np.int32)
    cp = (params or Params()).to_c()
    _check(lib().qlp_bls_coarse_bins(ctypes.byref(cp), int(per.shape[0]), _np_ptr(per), _np_ptr(out)),
           "qlp_bls_coarse_bins")
    return out


def proposal_windows(bins, params: Params | None = None, half_width: float = 1.0):
    """qlp_bls_proposal_windows: (win_offsets, f_lo, f_hi) around each star's valid
    proposed coarse bins (int [n_stars, k])."""
    b = np.ascontiguousarray(np.atleast_2d(bins), np.int32)
    n, k = int(b.shape[0]), int(b.shape[1])
    cp = (params or Params()).to_c()
    off = np.zeros(n + 1, np.int64)
    L = lib()
    _check(L.qlp_bls_proposal_windows(ctypes.byref(cp), n, _np_ptr(b), k, float(half_width), _np_ptr(off),
                                      None, None, 0), "qlp_bls_proposal_windows")
    lo = np.zeros(max(int(off[-1]), 1), np.float64)
    hi = np.zeros_like(lo)
    _check(L.qlp_bls_proposal_windows(ctypes.byref(cp), n, _np_ptr(b), k, float(half_width), _np_ptr(off),
                                      _np_ptr(lo), _np_ptr(hi), lo.shape[0]), "qlp_bls_proposal_windows")
    return off, lo[: off[-1]], hi[: off[-1]]


def search_learned(offsets, t, y, dy, rho, rstar, net: CNN | None, k: int = 32, half_width: float = 1.0,
                   params: Params | None = None, stream=None):
    """qlp_bls_search_learned: host light curves in, the learned path's best
    candidate per star and the proposed coarse bins [n_stars, k] out. net=None
    ranks the coarse bins by S/N instead (the path without the network)."""
    L = lib()
    offsets, t, y, dy, rho, rstar = _host_inputs(offsets, t, y, dy, rho, rstar)
    n_stars = int(offsets.shape[0] - 1)
    cp = (params or Params()).to_c()
    best = np.zeros(max(n_stars, 1), BEST_DTYPE)
    bins = np.zeros((max(n_stars, 1), int(k)), np.int32)
    rc = L.qlp_bls_search_learned(ctypes.byref(cp), n_stars, _np_ptr(offsets), _np_ptr(t), _np_ptr(y),
                                  _np_ptr(dy), _np_ptr(rho), _np_ptr(rstar),
                                  net._h if net is not None else None, int(k),
                                  float(half_width), _stream_ptr(stream), _np_ptr(best), _np_ptr(bins))
    _check(rc, "qlp_bls_search_learned")
    return best[:n_stars], bins[:n_stars]


def search_multi(offsets, t, y, dy, rho=None, rstar=None, n_planets: int = 3, params: Params | None = None,
                 stream=None):
    """qlp_bls_search_multi: (best [n_planets, n_stars], stats [n_planets, n_stars], n_found [n_stars])."""
    L = lib()
    offsets, t, y, dy, rho, rstar = _host_inputs(offsets, t, y, dy, rho, rstar)
    n_stars = int(offsets.shape[0] - 1)
    cp = (params or Params()).to_c()
    best = np.zeros((int(n_planets), max(n_stars, 1)), BEST_DTYPE)
    stats = np.zeros((int(n_planets), max(n_stars, 1)), STATS_DTYPE)
    found = np.zeros(max(n_stars, 1), np.int32)
    rc = L.qlp_bls_search_multi(ctypes.byref(cp), n_stars, _np_ptr(offsets), _np_ptr(t), _np_ptr(y), _np_ptr(dy),
                                _np_ptr(rho), _np_ptr(rstar), int(n_planets), _stream_ptr(stream), _np_ptr(best),
                                _np_ptr(stats), _np_ptr(found))
    _check(rc, "qlp_bls_search_multi")
    return best[:, :n_stars], stats[:, :n_stars], found[:n_stars]

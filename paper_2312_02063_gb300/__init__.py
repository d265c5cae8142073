"""Python binding of libgpfc.so: the GPFC fold + score path on one GB300 (sm_103a).

Thin ctypes marshalling over the C ABI in include/gpfc.h, with the same names
(gpfc_fold, gpfc_score_box, gpfc_best_period, gpfc_search, ...). PyTorch provides the
device buffers and the stream; every step of the path runs in the library's kernels.
There is no CPU fallback: importing works anywhere, but every call needs the compiled
library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np
import torch

from . import _build

__all__ = [
    "GpfcError", "Context", "load_library", "library_path",
    "gpfc_fold", "gpfc_score_box", "gpfc_score_cnn", "gpfc_best_period", "gpfc_search",
    "gpfc_best_period_noalloc", "gpfc_probe_smem_rmw", "gpfc_search_batched", "gpfc_fold_equal_count", "gpfc_peaks", "peaks_to_numpy", "gpfc_roc", "gpfc_detrend", "gpfc_synth_vectors", "gpfc_autotune", "FoldConfig",
    "SCORER_BOX", "SCORER_CNN",
]

SCORER_BOX = 0
SCORER_CNN = 1
BOX_AUTO = 0       # from 256 bins the one-kernel search, else the fold's epilogue
BOX_EPILOGUE = 1   # box search inside the fold kernel
BOX_WARP = 2       # separate box kernel, one warp per profile
BOX_FUSED = 3      # one kernel: an extra warp per fold block scores the block's previous task

STATUS = {0: "GPFC_OK", -1: "GPFC_EINVAL", -2: "GPFC_ENOMEM", -3: "GPFC_ECUDA", -4: "GPFC_ERANGE",
          -5: "GPFC_ETIMEOUT", -6: "GPFC_ENOTSUP"}


class GpfcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class FoldConfig(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int32), ("layout", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("streams", ctypes.c_int32)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


LAYOUT_PAIRED16 = 1
LAYOUT_PACKED64 = 2
LAYOUT_RED32 = 3


class CnnWeights(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("conv1_w", "conv1_b", "conv2_w", "conv2_b", "conv3_w",
                                               "conv3_b", "fc1_w", "fc1_b", "fc2_w", "fc2_b")]


CNN_PARAM_NAMES = ["conv1.w", "conv1.b", "conv2.w", "conv2.b", "conv3.w", "conv3.b",
                   "fc1.w", "fc1.b", "fc2.w", "fc2.b"]
CNN_PARAM_SHAPES = {"conv1.w": (16, 1, 5), "conv1.b": (16,), "conv2.w": (32, 16, 5), "conv2.b": (32,),
                    "conv3.w": (64, 32, 5), "conv3.b": (64,), "fc1.w": (256, 2048), "fc1.b": (256,),
                    "fc2.w": (1, 256), "fc2.b": (1,)}


class BoxParams(ctypes.Structure):
    _fields_ = [("w_min", ctypes.c_int32), ("w_max", ctypes.c_int32), ("sigma", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libgpfc.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise GpfcError(-3, f"libgpfc.so not found at {_build.LIB}; run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        L.gpfc_version.restype = ctypes.c_int
        L.gpfc_strerror.restype = ctypes.c_char_p
        L.gpfc_strerror.argtypes = [ctypes.c_int]
        L.gpfc_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp]
        L.gpfc_destroy.argtypes = [_vp]
        L.gpfc_destroy.restype = None
        L.gpfc_set_stream.argtypes = [_vp, _vp]
        L.gpfc_last_error.argtypes = [_vp]
        L.gpfc_last_error.restype = ctypes.c_char_p
        L.gpfc_sync.argtypes = [_vp]
        L.gpfc_num_sms.argtypes = [_vp]
        L.gpfc_set_fold_config.argtypes = [_vp, ctypes.POINTER(FoldConfig)]
        L.gpfc_fold_max_warps.argtypes = [ctypes.c_int32, ctypes.c_int32]
        L.gpfc_set_timing.argtypes = [_vp, ctypes.c_int]
        L.gpfc_kernel_time_ms.argtypes = [_vp, ctypes.POINTER(ctypes.c_float)]
        L.gpfc_fold.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_double, _vp, _vp]
        L.gpfc_score_box.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.POINTER(BoxParams), _vp, _vp, _vp]
        L.gpfc_best_period.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
        L.gpfc_best_period_noalloc.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp]
        L.gpfc_score_cnn.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(CnnWeights), _vp]
        L.gpfc_cnn_logits.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(CnnWeights), _vp]
        L.gpfc_search.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_double, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.gpfc_search_batched.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp,
                                          ctypes.c_int64, _vp, ctypes.c_int32, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.gpfc_set_graph.argtypes = [_vp, ctypes.c_int]
        L.gpfc_set_box_path.argtypes = [_vp, ctypes.c_int]
        L.gpfc_fold_launch_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)]
        L.gpfc_peaks.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                 ctypes.c_double, ctypes.c_int32, _vp, _vp]
        L.gpfc_fold_equal_count.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_double, _vp]
        L.gpfc_check_wait_timeout.argtypes = [_vp, ctypes.c_int64]
        L.gpfc_set_autotune.argtypes = [_vp, ctypes.c_int]
        L.gpfc_autotune.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int, _vp, ctypes.POINTER(FoldConfig)]
        L.gpfc_last_fold_plan.argtypes = [_vp, ctypes.POINTER(FoldConfig)]
        L.gpfc_workspace_size.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_size_t)]
        L.gpfc_probe_smem_rmw.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        _lib = L
        return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, device, name, numel=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t


class Context:
    """A gpfc_ctx bound to one CUDA device and a stream (torch's current stream by default)."""

    def __init__(self, device=0, stream=None):
        if not torch.cuda.is_available():
            raise GpfcError(-3, "no CUDA device: the GPFC path runs only on the GPU")
        self.lib = load_library()
        self.device = torch.device("cuda", device if isinstance(device, int) else torch.device(device).index or 0)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        h = _vp()
        with torch.cuda.device(self.device):
            rc = self.lib.gpfc_create(ctypes.byref(h), self.device.index, _vp(s.cuda_stream))
        if rc != 0:
            raise GpfcError(rc, self.lib.gpfc_last_error(None).decode() or self.lib.gpfc_strerror(rc).decode())
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gpfc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise GpfcError(rc, self.lib.gpfc_last_error(self.handle).decode() or
                            self.lib.gpfc_strerror(rc).decode())

    def set_stream(self, stream):
        self._check(self.lib.gpfc_set_stream(self.handle, _vp(stream.cuda_stream)))
        self.stream = stream

    def sync(self):
        self._check(self.lib.gpfc_sync(self.handle))

    def set_fold_config(self, warps=0, layout=0, chunk=0, tile=0, blocks_per_sm=0, streams=0):
        """Fold launch configuration; 0 means automatic for each field."""
        cfg = FoldConfig(int(warps), int(layout), int(chunk), int(tile), int(blocks_per_sm), int(streams))
        self._check(self.lib.gpfc_set_fold_config(self.handle, ctypes.byref(cfg)))

    def last_fold_plan(self) -> dict:
        """Launch config of the most recent fold plan (warps, layout, chunk, tile, blocks_per_sm)."""
        cfg = FoldConfig()
        self._check(self.lib.gpfc_last_fold_plan(self.handle, ctypes.byref(cfg)))
        return cfg.as_dict()

    def set_autotune(self, enable: int = 1):
        """1: use and make tuned fold configs; 0: do not; -1: off and forget the tuned configs."""
        self._check(self.lib.gpfc_set_autotune(self.handle, int(enable)))

    def set_graph(self, enable: bool):
        """Capture gpfc_search_batched into a CUDA graph and replay it (default on)."""
        self._check(self.lib.gpfc_set_graph(self.handle, int(bool(enable))))

    def set_box_path(self, path: int):
        """Where the box-SNR search runs: BOX_AUTO, BOX_EPILOGUE or BOX_WARP."""
        self._check(self.lib.gpfc_set_box_path(self.handle, int(path)))

    def check_wait_timeout(self, limit_cycles: int = 2_000_000):
        """Run the bounded-wait self-test: the next sync raises GpfcError(GPFC_ETIMEOUT)."""
        self._check(self.lib.gpfc_check_wait_timeout(self.handle, int(limit_cycles)))

    def workspace_size(self, n: int, n_periods: int, nbins: int) -> int:
        v = ctypes.c_size_t()
        self._check(self.lib.gpfc_workspace_size(self.handle, int(n), int(n_periods), int(nbins), ctypes.byref(v)))
        return int(v.value)

    def reset_fold_config(self):
        self._check(self.lib.gpfc_set_fold_config(self.handle, None))

    def fold_max_warps(self, nbins, layout):
        return int(self.lib.gpfc_fold_max_warps(int(nbins), int(layout)))

    def set_timing(self, enable: bool):
        self._check(self.lib.gpfc_set_timing(self.handle, int(bool(enable))))

    def kernel_time_ms(self) -> float:
        v = ctypes.c_float()
        self._check(self.lib.gpfc_kernel_time_ms(self.handle, ctypes.byref(v)))
        return float(v.value)

    def fold_launch_times(self) -> tuple[float, int]:
        """(summed ms, count) of the fold launches of the last timed warp-path box search."""
        ms, n = ctypes.c_float(), ctypes.c_int32()
        self._check(self.lib.gpfc_fold_launch_times(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    @property
    def num_sms(self):
        return self.lib.gpfc_num_sms(self.handle)


def gpfc_fold(ctx: Context, times, flux, periods, nbins: int, t0: float = math.nan, folded=None,
              counts=None, want_folded=True, want_counts=True):
    """Fold (times f64, flux f32) at every period (f64) into nbins equal-width bins.

    Returns (folded f32 [P][nbins] or None, counts i32 [P][nbins] or None); outputs are
    allocated on the context's device unless given.
    """
    dev = ctx.device
    n, npd = times.numel(), periods.numel()
    _need(times, torch.float64, dev, "times")
    _need(flux, torch.float32, dev, "flux", n)
    _need(periods, torch.float64, dev, "periods")
    if folded is None and want_folded:
        folded = torch.empty((npd, nbins), dtype=torch.float32, device=dev)
    if counts is None and want_counts:
        counts = torch.empty((npd, nbins), dtype=torch.int32, device=dev)
    if folded is not None:
        _need(folded, torch.float32, dev, "folded", npd * nbins)
    if counts is not None:
        _need(counts, torch.int32, dev, "counts", npd * nbins)
    ctx._check(ctx.lib.gpfc_fold(ctx.handle, _ptr(times), _ptr(flux), n, _ptr(periods), npd, int(nbins),
                                 float(t0), _ptr(folded), _ptr(counts)))
    return folded, counts


def gpfc_fold_equal_count(ctx: Context, times, flux, periods, nbins: int = 256, nfine: int = 4096,
                          t0: float = math.nan, folded=None):
    """The paper's two-tier fold: nfine equal-width fine bins merged into nbins bins of
    n/nbins samples each. Returns folded f32 [P][nbins] (means)."""
    dev = ctx.device
    n, npd = times.numel(), periods.numel()
    _need(times, torch.float64, dev, "times")
    _need(flux, torch.float32, dev, "flux", n)
    _need(periods, torch.float64, dev, "periods")
    if folded is None:
        folded = torch.empty((npd, nbins), dtype=torch.float32, device=dev)
    _need(folded, torch.float32, dev, "folded", npd * nbins)
    ctx._check(ctx.lib.gpfc_fold_equal_count(ctx.handle, _ptr(times), _ptr(flux), n, _ptr(periods), npd,
                                             int(nfine), int(nbins), float(t0), _ptr(folded)))
    return folded


def gpfc_score_box(ctx: Context, folded, counts, w_min: int, w_max: int, sigma: float = 0.0,
                   score=None, best_s=None, best_w=None, want_best=True):
    """Box-SNR of each profile ([P][nbins] means + counts). Returns (score, best_s, best_w)."""
    dev = ctx.device
    npd, nbins = folded.shape
    _need(folded, torch.float32, dev, "folded")
    _need(counts, torch.int32, dev, "counts", folded.numel())
    if score is None:
        score = torch.empty(npd, dtype=torch.float32, device=dev)
    if want_best and best_s is None:
        best_s = torch.empty(npd, dtype=torch.int32, device=dev)
    if want_best and best_w is None:
        best_w = torch.empty(npd, dtype=torch.int32, device=dev)
    bp = BoxParams(int(w_min), int(w_max), float(sigma))
    ctx._check(ctx.lib.gpfc_score_box(ctx.handle, _ptr(folded), _ptr(counts), npd, int(nbins),
                                      ctypes.byref(bp), _ptr(score), _ptr(best_s), _ptr(best_w)))
    return score, best_s, best_w


def _cnn_weights(ctx, weights):
    ptrs = []
    for n in CNN_PARAM_NAMES:
        t = weights[n]
        _need(t, torch.float32, ctx.device, n, int(torch.Size(CNN_PARAM_SHAPES[n]).numel()))
        ptrs.append(ctypes.c_void_p(t.data_ptr()))
    return CnnWeights(*ptrs)


def gpfc_score_cnn(ctx: Context, folded, weights, counts=None, score=None):
    """CNN score of each 256-bin profile. weights: dict name -> FP32 CUDA tensor (PyTorch layout)."""
    dev = ctx.device
    _need(folded, torch.float32, dev, "folded")
    npd = folded.shape[0]
    if counts is not None:
        _need(counts, torch.int32, dev, "counts", folded.numel())
    if score is None:
        score = torch.empty(npd, dtype=torch.float32, device=dev)
    w = _cnn_weights(ctx, weights)
    ctx._check(ctx.lib.gpfc_score_cnn(ctx.handle, _ptr(folded), _ptr(counts), npd, int(folded.shape[1]),
                                      ctypes.byref(w), _ptr(score)))
    return score


def gpfc_cnn_logits(ctx: Context, folded, weights, counts=None, logit=None):
    """Pre-sigmoid CNN outputs of each 256-bin profile."""
    dev = ctx.device
    _need(folded, torch.float32, dev, "folded")
    npd = folded.shape[0]
    if counts is not None:
        _need(counts, torch.int32, dev, "counts", folded.numel())
    if logit is None:
        logit = torch.empty(npd, dtype=torch.float32, device=dev)
    w = _cnn_weights(ctx, weights)
    ctx._check(ctx.lib.gpfc_cnn_logits(ctx.handle, _ptr(folded), _ptr(counts), npd, int(folded.shape[1]),
                                       ctypes.byref(w), _ptr(logit)))
    return logit


def gpfc_best_period(ctx: Context, score, best_index=None, best_score=None):
    """argmax of score (ties -> smaller index, NaN never wins). Returns (index i64[1], score f32[1])."""
    dev = ctx.device
    _need(score, torch.float32, dev, "score")
    if best_index is None:
        best_index = torch.empty(1, dtype=torch.int64, device=dev)
    if best_score is None:
        best_score = torch.empty(1, dtype=torch.float32, device=dev)
    ctx._check(ctx.lib.gpfc_best_period(ctx.handle, _ptr(score), score.numel(), _ptr(best_index),
                                        _ptr(best_score)))
    return best_index, best_score


def gpfc_probe_smem_rmw(word_bytes: int = 8, nbins: int = 32, warps: int = 16, blocks_per_sm: int = 1,
                        iters: int = 20000, stream=None, op: int = 0):
    """Measured rate of lane-private shared-memory read-modify-writes (see include/gpfc.h):
    returns (updates per second, updates per SM clock cycle). Runs on the current device."""
    lib = load_library()
    if not torch.cuda.is_available():
        raise GpfcError(-3, "no CUDA device: libgpfc runs on the GPU only")
    s = stream if stream is not None else torch.cuda.current_stream()
    ups, upc = ctypes.c_double(), ctypes.c_double()
    rc = lib.gpfc_probe_smem_rmw(word_bytes, op, nbins, warps, blocks_per_sm, iters, _vp(s.cuda_stream),
                                 ctypes.byref(ups), ctypes.byref(upc))
    if rc != 0:
        raise GpfcError(rc, lib.gpfc_strerror(rc).decode())
    return ups.value, upc.value


def gpfc_best_period_noalloc(score, best_index, best_score, stream=None):
    """Allocation-free argmax of score (see include/gpfc.h). No context: runs on the current
    device and the given torch stream (default: torch's current stream). The outputs must be
    preallocated device tensors (int64 [1], float32 [1]); this call allocates nothing."""
    lib = load_library()
    if not (isinstance(score, torch.Tensor) and score.is_cuda and score.dtype == torch.float32
            and score.is_contiguous()):
        raise TypeError("score must be a contiguous float32 CUDA tensor")
    dev = score.device
    _need(best_index, torch.int64, dev, "best_index", 1)
    _need(best_score, torch.float32, dev, "best_score", 1)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        rc = lib.gpfc_best_period_noalloc(_ptr(score), score.numel(), _ptr(best_index), _ptr(best_score),
                                          _vp(s.cuda_stream))
    if rc != 0:
        raise GpfcError(rc, lib.gpfc_strerror(rc).decode())
    return best_index, best_score


def gpfc_search(ctx: Context, times, flux, periods, nbins: int, t0: float = math.nan, scorer: int = SCORER_BOX,
                w_min: int = 1, w_max: int | None = None, sigma: float = 0.0, score=None, best_index=None,
                best_score=None, weights=None):
    """Fold + score without materialising profiles. Returns (score [P], best_index [1], best_score [1])."""
    dev = ctx.device
    n, npd = times.numel(), periods.numel()
    _need(times, torch.float64, dev, "times")
    _need(flux, torch.float32, dev, "flux", n)
    _need(periods, torch.float64, dev, "periods")
    if score is None:
        score = torch.empty(npd, dtype=torch.float32, device=dev)
    if best_index is None:
        best_index = torch.empty(1, dtype=torch.int64, device=dev)
    if best_score is None:
        best_score = torch.empty(1, dtype=torch.float32, device=dev)
    if scorer == SCORER_BOX:
        if w_max is None:
            w_max = int(math.ceil(0.125 * nbins))
        params = BoxParams(int(w_min), int(w_max), float(sigma))
        pp = ctypes.cast(ctypes.pointer(params), _vp)
    elif scorer == SCORER_CNN:
        if weights is None:
            raise ValueError("the CNN scorer needs weights")
        params = _cnn_weights(ctx, weights)
        pp = ctypes.cast(ctypes.pointer(params), _vp)
    else:
        raise GpfcError(-6, f"unknown scorer {scorer}")
    ctx._check(ctx.lib.gpfc_search(ctx.handle, _ptr(times), _ptr(flux), n, _ptr(periods), npd, int(nbins),
                                   float(t0), int(scorer), pp, _ptr(score), _ptr(best_index),
                                   _ptr(best_score)))
    return score, best_index, best_score


def _scorer_params(ctx, scorer, nbins, w_min, w_max, sigma, weights):
    if scorer == SCORER_BOX:
        if w_max is None:
            w_max = int(math.ceil(0.125 * nbins))
        params = BoxParams(int(w_min), int(w_max), float(sigma))
    elif scorer == SCORER_CNN:
        if weights is None:
            raise ValueError("the CNN scorer needs weights")
        params = _cnn_weights(ctx, weights)
    else:
        raise GpfcError(-6, f"unknown scorer {scorer}")
    return params, ctypes.cast(ctypes.pointer(params), _vp)


def gpfc_search_batched(ctx: Context, lc_offsets, times, flux, grid_offsets, periods, nbins: int = 256, t0s=None,
                        scorer: int = SCORER_BOX, w_min: int = 1, w_max: int | None = None, sigma: float = 0.0,
                        weights=None, score=None, best_index=None, best_score=None):
    """Fold + score many stars in one launch sequence (CSR offsets, all on the device).

    lc_offsets [S+1] int64 into times f64 / flux f32; grid_offsets [S+1] int64 into periods
    f64; t0s [S] f64 or None. Returns (score [sum of grid lengths] f32, best_index [S] int64
    as an index into each star's own grid, best_score [S] f32).
    """
    dev = ctx.device
    S = lc_offsets.numel() - 1
    if S < 1:
        raise ValueError("lc_offsets needs at least two entries")
    _need(lc_offsets, torch.int64, dev, "lc_offsets")
    _need(grid_offsets, torch.int64, dev, "grid_offsets", S + 1)
    n, npd = times.numel(), periods.numel()
    _need(times, torch.float64, dev, "times")
    _need(flux, torch.float32, dev, "flux", n)
    _need(periods, torch.float64, dev, "periods")
    if t0s is not None:
        _need(t0s, torch.float64, dev, "t0s", S)
    if score is None:
        score = torch.empty(npd, dtype=torch.float32, device=dev)
    if best_index is None:
        best_index = torch.empty(S, dtype=torch.int64, device=dev)
    if best_score is None:
        best_score = torch.empty(S, dtype=torch.float32, device=dev)
    params, pp = _scorer_params(ctx, scorer, nbins, w_min, w_max, sigma, weights)
    ctx._check(ctx.lib.gpfc_search_batched(ctx.handle, S, _ptr(lc_offsets), _ptr(times), _ptr(flux), n,
                                           _ptr(grid_offsets), _ptr(periods), npd, _ptr(t0s), int(nbins),
                                           int(scorer), pp, _ptr(score), _ptr(best_index), _ptr(best_score)))
    return score, best_index, best_score


STAR_SUMMARY_DTYPE = np.dtype([("sde", "<f8"), ("mean", "<f8"), ("sd", "<f8"), ("best_index", "<i8"),
                               ("best_score", "<f4"), ("n_peaks", "<i4"), ("truncated", "<i4"), ("n_listed", "<i4")])
PEAK_DTYPE = np.dtype([("index", "<i8"), ("height", "<f4"), ("width", "<i4"), ("harmonic", "<i4"),
                       ("reserved", "<i4")])


def gpfc_peaks(ctx: Context, score, periods, grid_offsets=None, k_sigma: float = 3.0, min_width: int = 4,
               harmonic_tol: float = 1e-3, max_peaks: int = 8):
    """Per-star decision over periodograms (SDE of Eq. 3, the peak rule of Sec. 4.2,
    harmonic flags). Returns device byte tensors (summary [S] records, peaks [S][max_peaks]
    records); `peaks_to_numpy` decodes them."""
    dev = ctx.device
    npd = score.numel()
    _need(score, torch.float32, dev, "score")
    _need(periods, torch.float64, dev, "periods", npd)
    S = 1 if grid_offsets is None else grid_offsets.numel() - 1
    if grid_offsets is not None:
        _need(grid_offsets, torch.int64, dev, "grid_offsets")
    summary = torch.empty(S * STAR_SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    peaks = torch.empty(max(1, S * max_peaks * PEAK_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    ctx._check(ctx.lib.gpfc_peaks(ctx.handle, _ptr(score), _ptr(periods), S, _ptr(grid_offsets), npd,
                                  float(k_sigma), int(min_width), float(harmonic_tol), int(max_peaks),
                                  _ptr(summary), _ptr(peaks) if max_peaks > 0 else None))
    return summary, peaks


class DetrendParams(ctypes.Structure):
    _fields_ = [("time_gap", ctypes.c_double), ("flux_gap_sigma", ctypes.c_double), ("clip_sigma", ctypes.c_double),
                ("ridge", ctypes.c_double), ("edge", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("n_spacings", ctypes.c_int32), ("reserved", ctypes.c_int32), ("spacings", ctypes.c_double * 8)]


def gpfc_detrend(ctx: Context, times, flux, mask=None, spacings=(), edge: int = 30, **kw):
    """Pre-processing of Sec. 2.2 (see include/gpfc.h): returns device tensors (times f64,
    detrended flux f32, segment index i32), each of the output length."""
    L = ctx.lib
    if not getattr(L, "_gpfc_detrend_bound", False):
        L.gpfc_detrend.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(DetrendParams), _vp, _vp, _vp,
                                   _vp]
        L._gpfc_detrend_bound = True
    dev = ctx.device
    n = times.numel()
    _need(times, torch.float64, dev, "times")
    _need(flux, torch.float32, dev, "flux", n)
    if mask is not None:
        _need(mask, torch.uint8, dev, "mask", n)
    prm = DetrendParams(**kw)
    prm.edge = edge if edge > 0 else -1
    prm.n_spacings = len(spacings)
    for i, v in enumerate(spacings):
        prm.spacings[i] = float(v)
    t_out = torch.empty(n, dtype=torch.float64, device=dev)
    f_out = torch.empty(n, dtype=torch.float32, device=dev)
    s_out = torch.empty(n, dtype=torch.int32, device=dev)
    n_out = torch.empty(1, dtype=torch.int64, device=dev)
    ctx._check(L.gpfc_detrend(ctx.handle, _ptr(times), _ptr(flux), _ptr(mask), n, ctypes.byref(prm), _ptr(t_out),
                              _ptr(f_out), _ptr(s_out), _ptr(n_out)))
    k = int(n_out.item())
    return t_out[:k], f_out[:k], s_out[:k]


def gpfc_roc(ctx: Context, pos, neg, fprs=()):
    """ROC statistics of labelled scores (see include/gpfc.h): returns device tensors
    (u2 int64 [1], thr float32 [n_fpr], tp int64 [n_fpr]); AUC = u2 / (2 n_pos n_neg)."""
    L = ctx.lib
    if not getattr(L, "_gpfc_roc_bound", False):
        L.gpfc_roc.argtypes = [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_double), _vp, _vp, _vp]
        L._gpfc_roc_bound = True
    dev = ctx.device
    _need(pos, torch.float32, dev, "pos")
    _need(neg, torch.float32, dev, "neg")
    f = (ctypes.c_double * max(1, len(fprs)))(*[float(x) for x in fprs])
    u2 = torch.empty(1, dtype=torch.int64, device=dev)
    thr = torch.empty(max(1, len(fprs)), dtype=torch.float32, device=dev)
    tp = torch.empty(max(1, len(fprs)), dtype=torch.int64, device=dev)
    ctx._check(L.gpfc_roc(ctx.handle, _ptr(pos), pos.numel(), _ptr(neg), neg.numel(), len(fprs), f, _ptr(u2),
                          _ptr(thr), _ptr(tp)))
    return u2, thr[: len(fprs)], tp[: len(fprs)]


def peaks_to_numpy(summary, peaks, max_peaks: int = 8):
    """Copy gpfc_peaks' outputs to the host as numpy record arrays (summary [S], peaks [S][max_peaks])."""
    sm = np.frombuffer(summary.cpu().numpy().tobytes(), dtype=STAR_SUMMARY_DTYPE)
    pk = np.frombuffer(peaks.cpu().numpy().tobytes()[: len(sm) * max_peaks * PEAK_DTYPE.itemsize], dtype=PEAK_DTYPE)
    return sm, pk.reshape(len(sm), max_peaks)


def gpfc_autotune(ctx: Context, times, flux, periods, nbins: int, scorer: int = SCORER_BOX, w_min: int = 1,
                  w_max: int | None = None, sigma: float = 0.0) -> dict:
    """Time the fold's launch configs on this star and keep the fastest in the context."""
    dev = ctx.device
    n = times.numel()
    _need(times, torch.float64, dev, "times")
    _need(flux, torch.float32, dev, "flux", n)
    _need(periods, torch.float64, dev, "periods")
    if scorer == SCORER_BOX:
        params, pp = _scorer_params(ctx, scorer, nbins, w_min, w_max, sigma, None)
    else:
        params, pp = None, None
    out = FoldConfig()
    ctx._check(ctx.lib.gpfc_autotune(ctx.handle, _ptr(times), _ptr(flux), n, _ptr(periods), periods.numel(),
                                     int(nbins), int(scorer), pp, ctypes.byref(out)))
    return out.as_dict()


# ---------------------------------------------------------------- training


class CnnGrads(ctypes.Structure):
    _fields_ = CnnWeights._fields_


def _bind_training(L):
    if getattr(L, "_gpfc_train_bound", False):
        return
    L.gpfc_cnn_saved_bytes.argtypes = [ctypes.c_int64]
    L.gpfc_cnn_saved_bytes.restype = ctypes.c_size_t
    L.gpfc_cnn_forward_train.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(CnnWeights),
                                         _vp, _vp]
    L.gpfc_cnn_backward.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.POINTER(CnnWeights), _vp,
                                    ctypes.POINTER(CnnGrads)]
    L.gpfc_bce_with_logits.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp]
    L.gpfc_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, ctypes.c_int64]
    L._gpfc_train_bound = True


def gpfc_cnn_forward_train(ctx: Context, folded, weights, counts=None):
    """Training forward: returns (logit [B], saved activations uint8 buffer)."""
    _bind_training(ctx.lib)
    dev = ctx.device
    _need(folded, torch.float32, dev, "folded")
    B = folded.shape[0]
    if counts is not None:
        _need(counts, torch.int32, dev, "counts", folded.numel())
    saved = torch.empty(int(ctx.lib.gpfc_cnn_saved_bytes(B)), dtype=torch.uint8, device=dev)
    logit = torch.empty(B, dtype=torch.float32, device=dev)
    w = _cnn_weights(ctx, weights)
    ctx._check(ctx.lib.gpfc_cnn_forward_train(ctx.handle, _ptr(folded), _ptr(counts), B, int(folded.shape[1]),
                                              ctypes.byref(w), _ptr(logit), _ptr(saved)))
    return logit, saved


def gpfc_cnn_backward(ctx: Context, dlogit, weights, saved, grads=None):
    """Backward pass: dict of FP32 gradients (PyTorch layout) for dL/dlogit."""
    _bind_training(ctx.lib)
    dev = ctx.device
    _need(dlogit, torch.float32, dev, "dlogit")
    if grads is None:
        grads = {n: torch.empty(CNN_PARAM_SHAPES[n], dtype=torch.float32, device=dev) for n in CNN_PARAM_NAMES}
    g = CnnGrads(*[ctypes.c_void_p(grads[n].data_ptr()) for n in CNN_PARAM_NAMES])
    w = _cnn_weights(ctx, weights)
    ctx._check(ctx.lib.gpfc_cnn_backward(ctx.handle, _ptr(dlogit), dlogit.numel(), ctypes.byref(w), _ptr(saved),
                                         ctypes.byref(g)))
    return grads


def gpfc_bce_with_logits(ctx: Context, logit, label, want_grad=True):
    """Mean BCE-with-logits loss (device scalar) and dL/dlogit."""
    _bind_training(ctx.lib)
    dev = ctx.device
    _need(logit, torch.float32, dev, "logit")
    _need(label, torch.float32, dev, "label", logit.numel())
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    dlogit = torch.empty_like(logit) if want_grad else None
    ctx._check(ctx.lib.gpfc_bce_with_logits(ctx.handle, _ptr(logit), _ptr(label), logit.numel(), _ptr(loss),
                                            _ptr(dlogit)))
    return loss, dlogit


def gpfc_adam(ctx: Context, param, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One in-place Adam step on an FP32 tensor."""
    _bind_training(ctx.lib)
    for t, n in ((param, "param"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t, torch.float32, ctx.device, n, param.numel())
    ctx._check(ctx.lib.gpfc_adam(ctx.handle, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), float(lr),
                                 float(beta1), float(beta2), float(eps), int(step)))


class CNNFunction(torch.autograd.Function):
    """CNN scorer as an autograd function: forward and backward run in libgpfc's kernels.

    CNNFunction.apply(gctx, folded, counts_or_None, *params) -> logits [B]; params in the
    order of CNN_PARAM_NAMES (FP32 CUDA tensors, PyTorch layout).
    """

    @staticmethod
    def forward(fctx, gctx, folded, counts, *params):
        weights = dict(zip(CNN_PARAM_NAMES, params))
        logit, saved = gpfc_cnn_forward_train(gctx, folded, weights, counts)
        fctx.gctx = gctx
        fctx.saved_buffer = saved
        fctx.weights = weights
        return logit

    @staticmethod
    def backward(fctx, grad_logit):
        grads = gpfc_cnn_backward(fctx.gctx, grad_logit.contiguous().float(), fctx.weights, fctx.saved_buffer)
        return (None, None, None) + tuple(grads[n] for n in CNN_PARAM_NAMES)


class SynthParams(ctypes.Structure):
    _fields_ = [("n_cadences", ctypes.c_int32), ("cadence", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("depth_min", ctypes.c_double), ("depth_max", ctypes.c_double),
                ("dur_min_h", ctypes.c_double), ("dur_max_h", ctypes.c_double),
                ("p_min", ctypes.c_double), ("p_max", ctypes.c_double), ("drift_bins", ctypes.c_double)]


# Training-set recipe: 65,536-cadence light curves at 29.4 min, transits with depth
# log-uniform 30-2,000 ppm, duration 0.5-3 h, period 0.2-1 d, folded at the true period
# with up to half a bin of drift; white noise log-uniform 1e-4..1e-3.
TRAINING_SET = dict(n_cadences=65536, cadence=29.4 / 1440.0, sigma_min=1e-4, sigma_max=1e-3,
                    depth_min=30e-6, depth_max=2000e-6, dur_min_h=0.5, dur_max_h=3.0, p_min=0.2, p_max=1.0,
                    drift_bins=0.5)


def gpfc_synth_profiles(ctx: Context, seed: int, first: int, n: int, nbins: int = 256, params=None,
                        want_counts=True, want_period=False, want_std=False):
    """Generate n training profiles j = first..first+n-1.

    Returns (folded, counts, label, period, flux_std); unrequested outputs are None.
    """
    L = ctx.lib
    if not getattr(L, "_gpfc_synth_bound", False):
        L.gpfc_synth_profiles.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(SynthParams), _vp, _vp, _vp, _vp, _vp]
        L._gpfc_synth_bound = True
    sp = SynthParams(**(params or TRAINING_SET))
    dev = ctx.device
    folded = torch.empty((n, nbins), dtype=torch.float32, device=dev)
    counts = torch.empty((n, nbins), dtype=torch.int32, device=dev) if want_counts else None
    label = torch.empty(n, dtype=torch.float32, device=dev)
    period = torch.empty(n, dtype=torch.float64, device=dev) if want_period else None
    std = torch.empty(n, dtype=torch.float32, device=dev) if want_std else None
    ctx._check(L.gpfc_synth_profiles(ctx.handle, ctypes.c_uint64(seed), first, n, nbins, ctypes.byref(sp),
                                     _ptr(folded), _ptr(counts), _ptr(label), _ptr(period), _ptr(std)))
    return folded, counts, label, period, std


class VectorParams(ctypes.Structure):
    _fields_ = [("alpha_pos_min", ctypes.c_double), ("alpha_pos_max", ctypes.c_double),
                ("alpha_neg_max", ctypes.c_double), ("q_min", ctypes.c_double), ("q_max", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("sigma_max", ctypes.c_double), ("n_points", ctypes.c_int32)]


# The paper's training-set recipe (Sec. 2.6-2.7): SNR 6-10 positives, noise-only and
# SNR < 5 negatives, trapezoids with duration/period 0.04-0.12 (Table 2), per-point noise
# 1e-4..5e-4, 65,536-point light curves behind each 256-bin vector.
PAPER_VECTORS = dict(alpha_pos_min=6.0, alpha_pos_max=10.0, alpha_neg_max=5.0, q_min=0.04, q_max=0.12,
                     sigma_min=1e-4, sigma_max=5e-4, n_points=65536)


def gpfc_synth_vectors(ctx: Context, seed: int, first: int, n: int, nbins: int = 256, params=None):
    """Generate n paper-recipe vectors j = first..first+n-1.

    Returns (folded [n][nbins], label [n], alpha [n], sigma_bin [n]) on the device.
    """
    L = ctx.lib
    if not getattr(L, "_gpfc_vec_bound", False):
        L.gpfc_synth_vectors.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.POINTER(VectorParams), _vp, _vp, _vp, _vp]
        L._gpfc_vec_bound = True
    vp = VectorParams(**(params or PAPER_VECTORS))
    dev = ctx.device
    folded = torch.empty((n, nbins), dtype=torch.float32, device=dev)
    label = torch.empty(n, dtype=torch.float32, device=dev)
    alpha = torch.empty(n, dtype=torch.float32, device=dev)
    sb = torch.empty(n, dtype=torch.float32, device=dev)
    ctx._check(L.gpfc_synth_vectors(ctx.handle, ctypes.c_uint64(seed), first, n, nbins, ctypes.byref(vp),
                                    _ptr(folded), _ptr(label), _ptr(alpha), _ptr(sb)))
    return folded, label, alpha, sb

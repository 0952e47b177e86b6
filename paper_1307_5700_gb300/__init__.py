"""GB300 multibeam dedispersion search -- Python binding of ``libtpdd.so``.

A thin ctypes layer over the C ABI declared in ``include/tp_dedisp.h``: every
function here has the name of the C entry point it calls and only marshals
arguments (numpy arrays and host buffers as host pointers, torch CUDA tensors
as device pointers, torch streams as ``cudaStream_t``).  All computation runs
in the library's CUDA kernels; there is no CPU path.  Importing works without a
GPU; calling an entry point needs the built library (``build()``), and the
library needs a CUDA device.

Negative status codes raise ``TpError`` carrying the code and the library's
error text.  ``TP_ETRUNC`` / ``TP_EOVERFLOW`` from ``tp_get_candidates`` are
reported in its return value instead, since the records are still valid.
"""
import ctypes
import os

import numpy as np

from . import build as _build

# TP_DEBUG_BOUNDS=1 in the environment selects the bounds-checking build
DEBUG_BOUNDS = os.environ.get("TP_DEBUG_BOUNDS", "") == "1"
LIB_PATH = _build.LIB_DEBUG if DEBUG_BOUNDS else _build.LIB

TP_OK = 0
TP_EINVAL = -1
TP_ENOMEM = -2
TP_EADMIT = -3
TP_EBUSY = -4
TP_ENOTREADY = -5
TP_ETRUNC = -6
TP_ECUDA = -7
TP_ETIMEOUT = -8
TP_EBOUNDS = -9
TP_EOVERFLOW = -10

TP_U8, TP_F16, TP_BF16, TP_F32 = 0, 1, 2, 3
TP_C16 = 4
DTYPES = {"u8": TP_U8, "f16": TP_F16, "bf16": TP_BF16, "f32": TP_F32, "c16": TP_C16}
TP_STATS_BLOCK, TP_STATS_EXTERNAL = 0, 1

# Every entry point of include/tp_dedisp.h (checked by the tests).
EXPORTS = (
    "tp_rfi_defaults", "tp_engine_create", "tp_engine_destroy", "tp_sync", "tp_engine_memory",
    "tp_create_plan", "tp_plan_destroy", "tp_plan_info", "tp_get_delay_table", "tp_beam_open",
    "tp_beam_close", "tp_beam_footprint", "tp_beam_set_stream", "tp_beam_set_bandpass",
    "tp_push_block", "tp_dedisperse", "tp_detect", "tp_get_candidates", "tp_beam_info",
    "tp_get_series", "tp_get_bandpass", "tp_get_masks", "tp_get_series_stats",
    "tp_set_profiling", "tp_get_stage_times", "tp_engine_launches", "tp_last_error_string",
    "tp_version", "tp_plan_shapes", "tp_plan_set_shape", "tp_autotune", "tp_channel_stats_noalloc",
    "tp_run_ready", "tp_engine_stream", "tp_server_create", "tp_server_add_stream", "tp_server_submit",
    "tp_server_end_stream", "tp_server_run", "tp_server_results", "tp_server_candidates", "tp_server_destroy",
    "tp_beam_rewind", "tp_autotune_batch", "tp_plan_set_postprocess", "tp_get_processed_series",
    "tp_get_detrend", "tp_plan_set_bandpass_fit", "tp_get_bandpass_fit", "tp_plan_set_clustering",
    "tp_get_clusters", "tp_get_candidate_labels", "tp_prefetch_block", "tp_push_prefetched",
    "tp_get_batch_times", "tp_engine_set_wait_limit", "tp_plan_set_running_stats", "tp_engine_set_batch_grid",
    "tp_beam_export", "tp_beam_import", "tp_engine_set_tuning_cache", "tp_engine_set_canaries",
    "tp_engine_check_canaries", "tp_debug_bounds", "tp_debug_limit_staged", "tp_push_inplace",
    "tp_export_candidates",
)


class TpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class tp_rfi_params(ctypes.Structure):
    _fields_ = [("enable_channel", ctypes.c_int32), ("enable_spectrum", ctypes.c_int32),
                ("chunk_width", ctypes.c_int32), ("dilate_channels", ctypes.c_int32),
                ("tau_channel", ctypes.c_double), ("tau_spectrum", ctypes.c_double),
                ("stats_mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tp_candidate(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("dm_idx", ctypes.c_int32), ("t_abs", ctypes.c_int64),
                ("snr", ctypes.c_float), ("value", ctypes.c_float)]


CAND_DTYPE = np.dtype([("beam", np.int32), ("dm_idx", np.int32), ("t_abs", np.int64),
                       ("snr", np.float32), ("value", np.float32)])


class tp_cluster_params(ctypes.Structure):
    _fields_ = [("t_eps", ctypes.c_int32), ("dm_eps", ctypes.c_int32), ("snr_eps", ctypes.c_double),
                ("min_pts", ctypes.c_int32), ("smooth", ctypes.c_int32), ("rmse_max", ctypes.c_double),
                ("dm_min", ctypes.c_double)]


CLUSTER_DTYPE = np.dtype([("label", np.int32), ("n", np.int32), ("d_lo", np.int32), ("d_hi", np.int32),
                          ("d_star", np.int32), ("flags", np.int32), ("t_first", np.int64), ("t_last", np.int64),
                          ("snr_max", np.float32), ("width_ms", np.float32), ("rmse", np.float32),
                          ("reserved", np.float32)])

_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
_d = ctypes.c_double

_SIGS = {
    "tp_rfi_defaults": (None, [_vp]),
    "tp_engine_create": (_i, [_i, _sz, _vp, _vp]),
    "tp_engine_destroy": (_i, [_vp]),
    "tp_sync": (_i, [_vp]),
    "tp_engine_memory": (_i, [_vp, _vp, _vp]),
    "tp_create_plan": (_i, [_vp, _i, _d, _d, _d, _vp, _i, _i, _vp, _d, _vp]),
    "tp_plan_destroy": (_i, [_vp]),
    "tp_plan_info": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "tp_get_delay_table": (_i, [_vp, _vp, _sz]),
    "tp_beam_open": (_i, [_vp, _vp, _i, _i, _vp]),
    "tp_beam_close": (_i, [_vp, _i]),
    "tp_beam_footprint": (_i, [_vp, _i, _i, _vp]),
    "tp_beam_set_stream": (_i, [_vp, _i, _vp]),
    "tp_beam_set_bandpass": (_i, [_vp, _i, _vp, _vp, _i]),
    "tp_push_block": (_i, [_vp, _i, _vp, _i, _i]),
    "tp_prefetch_block": (_i, [_vp, _i, _vp, _i]),
    "tp_push_prefetched": (_i, [_vp, _i]),
    "tp_push_inplace": (_i, [_vp, _i, _vp, ctypes.c_int64, _i]),
    "tp_dedisperse": (_i, [_vp, _i]),
    "tp_detect": (_i, [_vp, _i]),
    "tp_get_candidates": (_i, [_vp, _i, _vp, _i, _vp]),
    "tp_export_candidates": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "tp_beam_info": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "tp_get_series": (_i, [_vp, _i, _vp, _sz, _i]),
    "tp_get_bandpass": (_i, [_vp, _i, _vp, _vp, _i]),
    "tp_get_masks": (_i, [_vp, _i, _vp, _vp, _vp]),
    "tp_get_series_stats": (_i, [_vp, _i, _vp, _vp, _i]),
    "tp_set_profiling": (_i, [_vp, _i]),
    "tp_get_stage_times": (_i, [_vp, _i, _vp, _vp]),
    "tp_get_batch_times": (_i, [_vp, _vp, _vp]),
    "tp_engine_set_wait_limit": (_i, [_vp, ctypes.c_longlong]),
    "tp_plan_set_running_stats": (_i, [_vp, _d]),
    "tp_engine_set_batch_grid": (_i, [_vp, _i]),
    "tp_beam_export": (_i, [_vp, _i, _vp, _sz, _vp]),
    "tp_beam_import": (_i, [_vp, _i, _vp, _sz]),
    "tp_engine_set_tuning_cache": (_i, [_vp, ctypes.c_char_p]),
    "tp_engine_set_canaries": (_i, [_vp, _i]),
    "tp_engine_check_canaries": (_i, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "tp_debug_bounds": (_i, []),
    "tp_debug_limit_staged": (_i, [_vp, _i, ctypes.c_int64]),
    "tp_engine_launches": (_i, [_vp, _vp]),
    "tp_plan_shapes": (_i, [_vp, _vp, _vp, _i]),
    "tp_plan_set_shape": (_i, [_vp, _i]),
    "tp_autotune": (_i, [_vp, _i, _i, _vp, _vp, _i]),
    "tp_autotune_batch": (_i, [_vp, _i, _vp, _vp, _i]),
    "tp_plan_set_postprocess": (_i, [_vp, _i, _i]),
    "tp_get_processed_series": (_i, [_vp, _i, _vp, ctypes.c_size_t, _i]),
    "tp_get_detrend": (_i, [_vp, _i, _vp, _vp, _vp, _i]),
    "tp_plan_set_bandpass_fit": (_i, [_vp, _i, _d]),
    "tp_plan_set_clustering": (_i, [_vp, _vp]),
    "tp_get_clusters": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "tp_get_candidate_labels": (_i, [_vp, _i, _vp, _i, _vp]),
    "tp_get_bandpass_fit": (_i, [_vp, _i, _vp, _vp, _vp, _i]),
    "tp_channel_stats_noalloc": (_i, [_vp, _i, _i, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                                     _vp]),
    "tp_run_ready": (_i, [_vp, _i, _vp]),
    "tp_engine_stream": (_i, [_vp, _vp]),
    "tp_server_create": (_i, [_vp, _vp, _d, _i, _vp]),
    "tp_server_add_stream": (_i, [_vp, _vp, _vp]),
    "tp_server_submit": (_i, [_vp, _i, _vp, _i, _d]),
    "tp_server_end_stream": (_i, [_vp, _i]),
    "tp_server_run": (_i, [_vp, _d]),
    "tp_server_results": (_i, [_vp, _vp, _i, _vp]),
    "tp_server_candidates": (_i, [_vp, _i, _vp, _i, _vp]),
    "tp_server_destroy": (_i, [_vp]),
    "tp_beam_rewind": (_i, [_vp, _i]),
    "tp_last_error_string": (ctypes.c_char_p, []),
    "tp_version": (_i, []),
}


def build(force=False, debug=None):
    """Compile the CUDA library for sm_103a (in-tree) and return its path
    (debug: the bounds-checking variant; None: the one this process loads)."""
    return _build.build(force=force, debug=DEBUG_BOUNDS if debug is None else debug)


def lib():
    """The loaded library.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; call "
                               "paper_1307_5700_gb300.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise TpError(rc, lib().tp_last_error_string().decode(errors="replace"))
    return rc


def _addr(obj):
    """Address of a buffer: numpy array (host), torch tensor (its device or
    host address), ctypes object, int, or None."""
    if obj is None:
        return None
    if isinstance(obj, int):
        return obj
    if isinstance(obj, np.ndarray):
        if not obj.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return obj.ctypes.data
    if hasattr(obj, "data_ptr"):
        if hasattr(obj, "is_contiguous") and not obj.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return obj.data_ptr()
    return ctypes.addressof(obj)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


# ---- entry points ------------------------------------------------------------------

def tp_rfi_defaults():
    p = tp_rfi_params()
    lib().tp_rfi_defaults(ctypes.byref(p))
    return p


def tp_version():
    return lib().tp_version()


def tp_last_error_string():
    return lib().tp_last_error_string().decode(errors="replace")


def tp_engine_create(device=0, hbm_budget_bytes=0, cuda_stream=None):
    h = ctypes.c_void_p()
    _check(lib().tp_engine_create(device, hbm_budget_bytes, _stream(cuda_stream), ctypes.byref(h)))
    return h


def tp_engine_destroy(e):
    return _check(lib().tp_engine_destroy(e))


def tp_sync(e):
    return _check(lib().tp_sync(e))


def tp_engine_memory(e):
    used, budget = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().tp_engine_memory(e, ctypes.byref(used), ctypes.byref(budget)))
    return used.value, budget.value


def tp_create_plan(e, nchan, f_lo_mhz, bw_mhz, t_samp_s, dm_list, dtype, rfi=None, nsigma=5.0):
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    h = ctypes.c_void_p()
    _check(lib().tp_create_plan(e, nchan, f_lo_mhz, bw_mhz, t_samp_s, dm.ctypes.data, len(dm), dtype,
                                ctypes.byref(rfi) if rfi is not None else None, nsigma, ctypes.byref(h)))
    return h


def tp_plan_destroy(p):
    return _check(lib().tp_plan_destroy(p))


def tp_plan_info(p):
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().tp_plan_info(p, *[ctypes.byref(x) for x in v]))
    return dict(nchan=v[0].value, ndm=v[1].value, max_delay=v[2].value, dtype=v[3].value)


def tp_get_delay_table(p):
    info = tp_plan_info(p)
    out = np.empty((info["ndm"], info["nchan"]), np.int32)
    _check(lib().tp_get_delay_table(p, out.ctypes.data, out.size))
    return out


def tp_beam_footprint(p, block_nsamp, cand_capacity):
    n = ctypes.c_size_t()
    _check(lib().tp_beam_footprint(p, block_nsamp, cand_capacity, ctypes.byref(n)))
    return n.value


def tp_beam_open(e, p, block_nsamp, cand_capacity):
    b = ctypes.c_int()
    _check(lib().tp_beam_open(e, p, block_nsamp, cand_capacity, ctypes.byref(b)))
    return b.value


def tp_beam_close(e, beam):
    return _check(lib().tp_beam_close(e, beam))


def tp_beam_set_stream(e, beam, cuda_stream):
    return _check(lib().tp_beam_set_stream(e, beam, _stream(cuda_stream)))


def tp_beam_set_bandpass(e, beam, mu, sigma):
    mu = np.ascontiguousarray(mu, np.float64)
    sigma = np.ascontiguousarray(sigma, np.float64)
    return _check(lib().tp_beam_set_bandpass(e, beam, mu.ctypes.data, sigma.ctypes.data, len(mu)))


def tp_push_block(e, beam, buf, nsamp=None, buf_is_device=None):
    """``buf``: (nchan, nsamp) numpy array (host) or torch tensor (device or
    host), in the plan's sample format (bfloat16 as uint16 bits on the host)."""
    if nsamp is None:
        nsamp = buf.shape[-1]
    if buf_is_device is None:
        buf_is_device = bool(getattr(buf, "is_cuda", False))
    return _check(lib().tp_push_block(e, beam, _addr(buf), int(nsamp), int(bool(buf_is_device))))


def tp_push_inplace(e, beam, buf, nsamp, pitch=None):
    """``buf``: a (nchan, pitch) torch CUDA tensor (or device address with
    ``pitch`` given) whose columns [max_delay, max_delay + nsamp) hold the
    block; the engine fills columns [0, max_delay) and reads it in place."""
    if pitch is None:
        pitch = buf.shape[-1]
    return _check(lib().tp_push_inplace(e, beam, _addr(buf), int(pitch), int(nsamp)))


def tp_prefetch_block(e, beam, host_buf, nsamp=None):
    """Start the copy of the next block from ``host_buf`` (a host numpy array
    or pinned torch tensor, (nchan, nsamp)); the caller keeps it unchanged
    until the block has been pushed and processed."""
    if nsamp is None:
        nsamp = host_buf.shape[-1]
    if getattr(host_buf, "is_cuda", False):
        raise ValueError("tp_prefetch_block takes a host buffer")
    return _check(lib().tp_prefetch_block(e, beam, _addr(host_buf), int(nsamp)))


def tp_push_prefetched(e, beam):
    return _check(lib().tp_push_prefetched(e, beam))


def tp_dedisperse(e, beam):
    return _check(lib().tp_dedisperse(e, beam))


def tp_detect(e, beam):
    return _check(lib().tp_detect(e, beam))


def tp_get_candidates(e, beam, cap):
    """Returns (records as a CAND_DTYPE array, n_total, status)."""
    out = np.zeros(max(int(cap), 1), CAND_DTYPE)
    n = ctypes.c_int()
    rc = lib().tp_get_candidates(e, beam, out.ctypes.data, int(cap), ctypes.byref(n))
    if rc < 0 and rc not in (TP_ETRUNC, TP_EOVERFLOW):
        _check(rc)
    return out[:min(n.value, int(cap))], n.value, rc


def tp_export_candidates(e, beam, out, cap, n_total, status=None):
    """Enqueue the stream-ordered export of the beam's candidates into
    ``out`` (cap records, CAND_DTYPE layout), the count into ``n_total`` (one
    uint64) and the status word into ``status`` (one int32, or None): page-
    locked host or device buffers, e.g. torch tensors made with
    pin_memory=True; they hold the results once the stream has passed the
    export."""
    _check(lib().tp_export_candidates(e, beam, _addr(out) if cap else None, int(cap), _addr(n_total),
                                      _addr(status) if status is not None else None))


def tp_beam_info(e, beam):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    k = ctypes.c_int()
    _check(lib().tp_beam_info(e, beam, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(k)))
    return dict(nsamp_window=a.value, nout=b.value, t0_abs=c.value, nchunk=k.value)


def tp_get_series(e, beam, out=None, ndm=None, is_int=False):
    """D (ndm x nout) into ``out`` (numpy or torch), allocated on the host if
    None."""
    info = tp_beam_info(e, beam)
    if out is None:
        out = np.empty((ndm, info["nout"]), np.int32 if is_int else np.float32)
    nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    is_dev = bool(getattr(out, "is_cuda", False))
    _check(lib().tp_get_series(e, beam, _addr(out), nbytes, int(is_dev)))
    return out


def tp_get_bandpass(e, beam, nchan):
    mu = np.empty(nchan, np.float64)
    sigma = np.empty(nchan, np.float64)
    _check(lib().tp_get_bandpass(e, beam, mu.ctypes.data, sigma.ctypes.data, nchan))
    return mu, sigma


def tp_get_masks(e, beam, nchan):
    info = tp_beam_info(e, beam)
    cf = np.empty((nchan, info["nchunk"]), np.uint8)
    cr = np.empty((nchan, info["nchunk"]), np.uint8)
    sf = np.empty(info["nsamp_window"], np.uint8)
    _check(lib().tp_get_masks(e, beam, cf.ctypes.data, cr.ctypes.data, sf.ctypes.data))
    return cf, cr, sf


def tp_get_series_stats(e, beam, ndm):
    mu = np.empty(ndm, np.float64)
    sigma = np.empty(ndm, np.float64)
    _check(lib().tp_get_series_stats(e, beam, mu.ctypes.data, sigma.ctypes.data, ndm))
    return mu, sigma


def tp_set_profiling(e, enable=True):
    return _check(lib().tp_set_profiling(e, int(bool(enable))))


def tp_get_stage_times(e, beam):
    """(ms[4]: push, A1-A3, A4-A5, A6-A7 accumulated; number of blocks)."""
    ms = np.zeros(4, np.float64)
    n = ctypes.c_int64()
    _check(lib().tp_get_stage_times(e, beam, ms.ctypes.data, ctypes.byref(n)))
    return ms, n.value


def tp_get_batch_times(e):
    """(ms of the batched dedispersion launches timed since profiling was
    enabled, number of batches)."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().tp_get_batch_times(e, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def tp_plan_set_running_stats(p, alpha):
    """Exponential average of the bandpass statistics across blocks, weight
    alpha on the new block (1 = per block)."""
    return _check(lib().tp_plan_set_running_stats(p, float(alpha)))


def tp_engine_set_tuning_cache(e, path):
    """Autotuner cache file (None: off)."""
    return _check(lib().tp_engine_set_tuning_cache(e, None if path is None else os.fsencode(path)))


def tp_engine_set_canaries(e, enable):
    """Canary padding around the buffers of beams opened from now on."""
    return _check(lib().tp_engine_set_canaries(e, int(bool(enable))))


def tp_engine_check_canaries(e):
    """Number of damaged canary pads over the engine's open beams."""
    n = ctypes.c_int()
    _check(lib().tp_engine_check_canaries(e, ctypes.byref(n)))
    return n.value


def tp_debug_bounds():
    """True when the loaded library is the bounds-checking build."""
    return bool(lib().tp_debug_bounds())


def tp_debug_limit_staged(e, beam, nbytes):
    """Bounds-checking build: the staged-series extent the checks of `beam`
    use (negative: the real one)."""
    return _check(lib().tp_debug_limit_staged(e, beam, int(nbytes)))


def tp_beam_export(e, beam):
    """The beam's stream state (bytes) for tp_beam_import."""
    n = ctypes.c_size_t()
    _check(lib().tp_beam_export(e, beam, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().tp_beam_export(e, beam, buf, n.value, ctypes.byref(n)))
    return buf.raw


def tp_beam_import(e, beam, state):
    """Continue a stream in a fresh beam from a state of tp_beam_export."""
    return _check(lib().tp_beam_import(e, beam, state, len(state)))


def tp_engine_set_batch_grid(e, ctas=0):
    """Batched dedispersion grid: 0 persistent (default), > 0 at most that
    many CTAs, < 0 one CTA per work item."""
    return _check(lib().tp_engine_set_batch_grid(e, int(ctas)))


def tp_engine_set_wait_limit(e, tries=-1):
    """Attempts of the dedispersion kernel's waits before it reports
    TP_ETIMEOUT (-1: the default; 0: give up at once)."""
    return _check(lib().tp_engine_set_wait_limit(e, int(tries)))


def tp_engine_launches(e):
    n = ctypes.c_uint64()
    _check(lib().tp_engine_launches(e, ctypes.byref(n)))
    return n.value


def tp_plan_shapes(p):
    """(current shape, feasible flags per shape)."""
    sh = ctypes.c_int()
    n = _check(lib().tp_plan_shapes(p, ctypes.byref(sh), None, 0))
    feas = np.zeros(n, np.int32)
    _check(lib().tp_plan_shapes(p, ctypes.byref(sh), feas.ctypes.data, n))
    return sh.value, feas.astype(bool)


def tp_plan_set_shape(p, shape):
    return _check(lib().tp_plan_set_shape(p, int(shape)))


def tp_autotune(e, beam, reps=3):
    """(best shape, ms per launch for every shape; -1 where infeasible)."""
    best = ctypes.c_int()
    ms = np.full(128, -1.0, np.float32)
    _check(lib().tp_autotune(e, beam, int(reps), ctypes.byref(best), ms.ctypes.data, len(ms)))
    return best.value, ms


def tp_plan_set_postprocess(p, median_width=1, detrend=False):
    """Median filter width (odd, 1 = off) and detrending for the plan's beams
    (before any beam is opened; see tp_dedisp.h)."""
    return _check(lib().tp_plan_set_postprocess(p, int(median_width), int(bool(detrend))))


def tp_get_processed_series(e, beam, out=None, ndm=None, is_int=False):
    """The series the detection ran on (median-filtered, or D)."""
    info = tp_beam_info(e, beam)
    if out is None:
        out = np.empty((ndm, info["nout"]), np.int32 if is_int else np.float32)
    nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    is_dev = bool(getattr(out, "is_cuda", False))
    _check(lib().tp_get_processed_series(e, beam, _addr(out), nbytes, int(is_dev)))
    return out


def tp_get_detrend(e, beam, ndm):
    """(mean, beta, sigma) of the detrending line mean + beta (2t - (T - 1))."""
    mean = np.empty(ndm, np.float64)
    beta = np.empty(ndm, np.float64)
    sigma = np.empty(ndm, np.float64)
    _check(lib().tp_get_detrend(e, beam, mean.ctypes.data, beta.ctypes.data, sigma.ctypes.data, ndm))
    return mean, beta, sigma


def tp_plan_set_bandpass_fit(p, order, tau_mask=5.0):
    """Fitted bandpass of polynomial order ``order`` (-1: off) for the plan's
    beams (before any beam is opened; see tp_dedisp.h)."""
    return _check(lib().tp_plan_set_bandpass_fit(p, int(order), float(tau_mask)))


def tp_get_bandpass_fit(e, beam, nchan):
    """(b_c, masked channels, rmse) of the beam's current block."""
    b = np.empty(nchan, np.float64)
    m = np.empty(nchan, np.uint8)
    r = ctypes.c_double()
    _check(lib().tp_get_bandpass_fit(e, beam, b.ctypes.data, m.ctypes.data, ctypes.byref(r), nchan))
    return b, m.astype(bool), r.value


def tp_plan_set_clustering(p, t_eps=20, dm_eps=3, snr_eps=5.0, min_pts=5, smooth=3, rmse_max=0.4, dm_min=1.0,
                           enable=True):
    """Clustering and classification of every block's detections (Sec. 2.3;
    see tp_dedisp.h); enable=False turns it off."""
    if not enable:
        return _check(lib().tp_plan_set_clustering(p, None))
    prm = tp_cluster_params(int(t_eps), int(dm_eps), float(snr_eps), int(min_pts), int(smooth), float(rmse_max),
                            float(dm_min))
    return _check(lib().tp_plan_set_clustering(p, ctypes.byref(prm)))


def tp_get_clusters(e, beam, cap=1 << 16):
    """(cluster records, number of clusters, truncated)."""
    out = np.zeros(max(int(cap), 1), CLUSTER_DTYPE)
    n = ctypes.c_int()
    tr = ctypes.c_int()
    _check(lib().tp_get_clusters(e, beam, out.ctypes.data, int(cap), ctypes.byref(n), ctypes.byref(tr)))
    return out[:min(n.value, cap)], n.value, bool(tr.value)


def tp_get_candidate_labels(e, beam, cap=1 << 20):
    """Cluster number (-1: noise) of each stored detection, in record order."""
    out = np.zeros(max(int(cap), 1), np.int32)
    n = ctypes.c_int()
    _check(lib().tp_get_candidate_labels(e, beam, out.ctypes.data, int(cap), ctypes.byref(n)))
    return out[:min(n.value, cap)]


def tp_autotune_batch(e, reps=2):
    """(best shape, ms per batched launch for every shape; -1 where not timed)."""
    best = ctypes.c_int()
    ms = np.full(128, -1.0, np.float32)
    _check(lib().tp_autotune_batch(e, int(reps), ctypes.byref(best), ms.ctypes.data, len(ms)))
    return best.value, ms


def tp_channel_stats_noalloc(x, dtype, mu, sigma, chunk_flag, chunk_raw, rfi=None, nsamp=None, stream=None):
    """A1-A2 of a device block ``x`` (nchan, pitch) into caller-provided device
    outputs, with no allocation by the library (see tp_dedisp.h)."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    nchan, pitch = x.shape
    nsamp = pitch if nsamp is None else nsamp
    return _check(lib().tp_channel_stats_noalloc(
        _addr(x), dtype, nchan, nsamp, pitch, ctypes.byref(rfi) if rfi is not None else None, _addr(mu),
        _addr(sigma), _addr(chunk_flag), _addr(chunk_raw), _stream(stream)))


def tp_run_ready(e, use_graph=False):
    """A1-A7 for every beam holding a new block, batched (see tp_dedisp.h);
    returns the number of beams processed."""
    n = ctypes.c_int()
    _check(lib().tp_run_ready(e, int(bool(use_graph)), ctypes.byref(n)))
    return n.value


class tp_stream_desc(ctypes.Structure):
    _fields_ = [("nchan", ctypes.c_int32), ("ndm", ctypes.c_int32), ("f_lo_mhz", ctypes.c_double),
                ("bw_mhz", ctypes.c_double), ("t_samp_s", ctypes.c_double), ("dm_list", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("block_nsamp", ctypes.c_int32), ("cand_capacity", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


SERVE_RESULT_DTYPE = np.dtype([("stream", np.int32), ("seq", np.int32), ("arrival_s", np.float64),
                               ("start_s", np.float64), ("done_s", np.float64), ("n_candidates", np.int64),
                               ("status", np.int32), ("reserved", np.int32)])


def tp_engine_stream(e):
    v = ctypes.c_void_p()
    _check(lib().tp_engine_stream(e, ctypes.byref(v)))
    return v.value


def tp_server_create(e, rfi=None, nsigma=5.0, keep_candidates=False):
    h = ctypes.c_void_p()
    _check(lib().tp_server_create(e, ctypes.byref(rfi) if rfi is not None else None, nsigma,
                                  int(bool(keep_candidates)), ctypes.byref(h)))
    return h


_server_keep = {}


def tp_server_add_stream(s, nchan, f_lo_mhz, bw_mhz, t_samp_s, dm_list, dtype, block_nsamp, cand_capacity):
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    d = tp_stream_desc(nchan, len(dm), f_lo_mhz, bw_mhz, t_samp_s, dm.ctypes.data, dtype, block_nsamp,
                       cand_capacity, 0)
    sid = ctypes.c_int()
    _check(lib().tp_server_add_stream(s, ctypes.byref(d), ctypes.byref(sid)))
    return sid.value


def tp_server_submit(s, stream_id, block, arrival_s, nsamp=None):
    """``block`` must stay alive until the request is done (keep a reference)."""
    if nsamp is None:
        nsamp = block.shape[-1]
    rid = _check(lib().tp_server_submit(s, stream_id, _addr(block), int(nsamp), float(arrival_s)))
    _server_keep.setdefault(s.value, []).append(block)
    return rid


def tp_server_end_stream(s, stream_id):
    return _check(lib().tp_server_end_stream(s, stream_id))


def tp_server_run(s, time_limit_s=1e9):
    return _check(lib().tp_server_run(s, float(time_limit_s)))


def tp_server_results(s):
    n = ctypes.c_int()
    _check(lib().tp_server_results(s, None, 0, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), SERVE_RESULT_DTYPE)
    _check(lib().tp_server_results(s, out.ctypes.data, n.value, ctypes.byref(n)))
    return out[:n.value]


def tp_server_candidates(s, request, cap=1 << 20):
    out = np.zeros(max(cap, 1), CAND_DTYPE)
    n = ctypes.c_int()
    _check(lib().tp_server_candidates(s, request, out.ctypes.data, cap, ctypes.byref(n)))
    return out[:min(n.value, cap)]


def tp_server_destroy(s):
    rc = _check(lib().tp_server_destroy(s))
    _server_keep.pop(s.value, None)
    return rc


def tp_beam_rewind(e, beam):
    return _check(lib().tp_beam_rewind(e, beam))

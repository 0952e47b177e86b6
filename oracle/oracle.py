"""Python face of the CPU oracle (test infrastructure only).

The arithmetic lives in ``tp_oracle.c``; this module only marshals numpy
arrays into it and strings the steps together in the paper's order
(Sec. 2.2.1 RFI thresholding -> Sec. 2.2.2 dedispersion -> Sec. 2.2.3
normalisation -> Sec. 2.3 detection).  Only the tests, the package smoke
check and the benchmark's CPU-baseline leg may import it.

Input blocks are numpy arrays of shape (nchan, nsamp) in channel-major order
(the paper's beam/channel/time organisation, Sec. 2.1): ``uint8``,
``float16``, ``float32``, or ``uint16`` holding bfloat16 bit patterns
(pass ``dtype="bf16"``).
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

DTYPE_CODES = {"u8": 0, "f16": 1, "bf16": 2, "f32": 3, "c16": 4}
# complex voltage samples: int16 real part, then int16 imaginary part
C16 = np.dtype([("re", "<i2"), ("im", "<i2")])

STATS_BLOCK = 0
STATS_EXTERNAL = 1

_lib = None

_p = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double


class Candidate(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("dm_idx", ctypes.c_int32), ("t_abs", ctypes.c_int64),
                ("snr", ctypes.c_float), ("value", ctypes.c_float)]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "orc_set_threads": (None, [_i]),
            "orc_get_threads": (_i, []),
            "orc_has_openmp": (_i, []),
            "orc_channel_freqs": (None, [_i, _d, _d, _p]),
            "orc_delay_exact": (None, [_i, _d, _d, _d, _p, _i, _p]),
            "orc_delay_table": (_i64, [_i, _d, _d, _d, _p, _i, _p]),
            "orc_delay_ties": (_i64, [_i, _d, _d, _d, _p, _i, _d, _p, _p, _p, _i64]),
            "orc_bandpass_float": (None, [_p, _i, _i, _i64, _i64, _p, _p]),
            "orc_bandpass_u8": (None, [_p, _i, _i64, _i64, _p, _p, _p, _p, _p, _p]),
            "orc_channel_mask_float": (None, [_p, _i, _i, _i64, _i64, _i, _d, _i, _p, _p, _p, _p]),
            "orc_channel_mask_u8": (None, [_p, _i, _i64, _i64, _i, _d, _i, _p, _p, _p, _p]),
            "orc_channel_mask_u8_ext": (None, [_p, _i, _i64, _i64, _i, _d, _i, _p, _p, _p, _p]),
            "orc_spectrum_mask_float": (None, [_p, _i, _i, _i64, _i64, _i, _d, _p, _p, _p, _p]),
            "orc_spectrum_mask_u8": (None, [_p, _i, _i64, _i64, _i, _d, _p, _p, _p, _p]),
            "orc_spectrum_mask_u8_ext": (None, [_p, _i, _i64, _i64, _i, _d, _p, _p, _p, _p]),
            "orc_corrected_float": (None, [_p, _i, _i, _i64, _i64, _p, _p, _p, _i, _p]),
            "orc_dedisperse_float": (None, [_p, _i, _i, _i64, _i64, _p, _p, _p, _i, _p, _i, _i64, _p]),
            "orc_dedisperse_u8": (None, [_p, _i, _i64, _i64, _p, _p, _p, _i, _p, _i, _i64, _p]),
            "orc_dedisperse_points_float": (None, [_p, _i, _i, _i64, _i64, _p, _p, _p, _i, _p, _p, _p, _i64, _p]),
            "orc_dedisperse_points_u8": (None, [_p, _i, _i64, _i64, _p, _p, _p, _i, _p, _p, _p, _i64, _p]),
            "orc_abs_mass_points_float": (None, [_p, _i, _i, _i64, _i64, _p, _p, _p, _i, _p, _p, _p, _i64, _p]),
            "orc_storage_bandpass": (None, [_i, _p, _i, _p]),
            "orc_stored_mass_points": (None, [_p, _i, _i, _i64, _i64, _p, _p, _p, _i, _p, _p, _p, _i64, _p]),
            "orc_series_stats_float": (None, [_p, _i, _i64, _p, _p]),
            "orc_series_stats_int": (None, [_p, _i, _i64, _p, _p, _p, _p]),
            "orc_candidates_float": (_i64, [_p, _i, _i64, _p, _p, _d, _i, _i64, _p, _i64]),
            "orc_candidates_int": (_i64, [_p, _i, _i64, _p, _p, _d, _i, _i64, _p, _i64]),
            "orc_median_float": (None, [_p, _i, _i64, _i, _p]),
            "orc_channel_mask_fit": (None, [_p, _i, _i, _i64, _i64, _i, _d, _i, _p, _d, _p, _p]),
            "orc_median_int": (None, [_p, _i, _i64, _i, _p]),
            "orc_detrend_float": (None, [_p, _i, _i64, _p, _p, _p]),
            "orc_detrend_int": (None, [_p, _i, _i64, _p, _p, _p, _p]),
            "orc_candidates_detrend": (_i64, [_p, _i, _i, _i64, _p, _p, _p, _d, _i, _i64, _p, _i64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def set_threads(n):
    """Threads used by the dedispersion loop (1 unless OpenMP is available)."""
    lib().orc_set_threads(int(n))
    return lib().orc_get_threads() if lib().orc_has_openmp() else 1


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _input(x, dtype):
    code = DTYPE_CODES[dtype]
    want = {"u8": np.uint8, "f16": np.float16, "bf16": np.uint16, "f32": np.float32, "c16": C16}[dtype]
    x = np.ascontiguousarray(x)
    if x.dtype != want:
        raise TypeError(f"dtype {dtype} needs a {np.dtype(want)} array, got {x.dtype}")
    if x.ndim != 2:
        raise ValueError("input must be (nchan, nsamp)")
    return x, code


@dataclass
class RfiParams:
    """Thresholding parameters of Sec. 2.2.1 (readings R5, R6)."""
    enable_channel: bool = True
    enable_spectrum: bool = True
    chunk_width: int = 256          # W_c
    tau_channel: float = 5.0        # channel threshold, in sigma_c sqrt(n) units
    tau_spectrum: float = 6.0       # spectrum threshold, in sqrt(sum sigma_c^2) units
    dilate_channels: bool = False   # also flag the same chunk of adjacent channels


# ---- plan ----------------------------------------------------------------------

def channel_freqs(nchan, f_lo, bw):
    f = np.empty(nchan, np.float64)
    lib().orc_channel_freqs(nchan, f_lo, bw, _ptr(f))
    return f


def delay_exact(nchan, f_lo, bw, t_samp, dm):
    dm = _c(dm, np.float64)
    out = np.empty((len(dm), nchan), np.float64)
    lib().orc_delay_exact(nchan, f_lo, bw, t_samp, _ptr(dm), len(dm), _ptr(out))
    return out


def delay_table(nchan, f_lo, bw, t_samp, dm):
    """Integer delay table (ndm, nchan) int32 and its maximum (Eq. 1, R1-R3)."""
    dm = _c(dm, np.float64)
    out = np.zeros((max(len(dm), 1), max(nchan, 1)), np.int32)
    dmax = lib().orc_delay_table(nchan, f_lo, bw, t_samp, _ptr(dm), len(dm), _ptr(out))
    if dmax < 0:
        raise ValueError("invalid plan arguments")
    return out, int(dmax)


def delay_ties(nchan, f_lo, bw, t_samp, dm, eps=1e-9):
    """Tie log of Eq. 1's rounding (R3): the (d, c) pairs whose unrounded
    delay lies within ``eps`` of a half-integer, as a list of (d, c, value),
    so that a delay mismatch against another implementation can be traced to
    a rounding tie."""
    dm = _c(dm, np.float64)
    cap = 1 << 16
    od = np.zeros(cap, np.int32)
    oc = np.zeros(cap, np.int32)
    ov = np.zeros(cap, np.float64)
    n = lib().orc_delay_ties(nchan, f_lo, bw, t_samp, _ptr(dm), len(dm), float(eps), _ptr(od), _ptr(oc),
                             _ptr(ov), cap)
    if n < 0:
        raise ValueError("invalid plan arguments")
    if n > cap:
        raise ValueError(f"{n} ties: more than the log holds")
    return [(int(od[i]), int(oc[i]), float(ov[i])) for i in range(n)]


# ---- A1-A3 ---------------------------------------------------------------------

def bandpass(x, dtype):
    """Block bandpass statistics (R4).  For 8-bit input also the exact sums."""
    x, code = _input(x, dtype)
    nchan, nsamp = x.shape
    mu = np.empty(nchan, np.float64)
    sigma = np.empty(nchan, np.float64)
    if dtype == "u8":
        S, Q, V, b = (np.empty(nchan, np.int64) for _ in range(4))
        lib().orc_bandpass_u8(_ptr(x), nchan, nsamp, nsamp, _ptr(S), _ptr(Q), _ptr(V), _ptr(b),
                              _ptr(mu), _ptr(sigma))
        return dict(mu=mu, sigma=sigma, S=S, Q=Q, V=V, b=b, external=False)
    lib().orc_bandpass_float(_ptr(x), code, nchan, nsamp, nsamp, _ptr(mu), _ptr(sigma))
    return dict(mu=mu, sigma=sigma, b=storage_bandpass(dtype, mu), external=False)


def storage_bandpass(dtype, mu):
    """Bandpass value in the data's storage format (R7): binary16 / bfloat16
    round mu to nearest even, binary32 keeps mu (8-bit: see bandpass())."""
    mu = _c(mu, np.float64)
    b = np.empty_like(mu)
    lib().orc_storage_bandpass(DTYPE_CODES[dtype], _ptr(mu), len(mu), _ptr(b))
    return b


def external_stats(dtype, mu, sigma):
    """Statistics supplied by the caller instead of measured on the block.
    For 8-bit input the bandpass value is the integer floor(mu + 1/2)."""
    mu = _c(mu, np.float64)
    sigma = _c(sigma, np.float64)
    st = dict(mu=mu, sigma=sigma, external=True)
    if dtype == "u8":
        st["b"] = np.floor(mu + 0.5).astype(np.int64)
    else:
        st["b"] = storage_bandpass(dtype, mu)
    return st


def running_stats(prev, x, dtype, alpha):
    """Running bandpass statistics across the blocks of a stream (Sec. 2.2.1
    averages the bandpass over each processing iteration; reading R15): the block's own
    mean mu and variance sigma^2 (R4) are folded into an exponential average
    with weight alpha on the new block,
        mu_run = alpha * mu + (1 - alpha) * mu_run_prev,
        var_run = alpha * sigma^2 + (1 - alpha) * var_run_prev,
    starting from the first block's own values; alpha = 1 is per-block
    statistics.  Returns (state, stats): the state (mu_run, var_run) for the
    next block, and the statistics the block is thresholded and corrected
    with, in the form of external statistics (mu_run, sqrt(var_run))."""
    st = bandpass(x, dtype)
    mu, var = st["mu"], st["sigma"] * st["sigma"]
    if prev is not None:
        mu = alpha * mu + (1.0 - alpha) * prev[0]
        var = alpha * var + (1.0 - alpha) * prev[1]
    return (mu, var), external_stats(dtype, mu, np.sqrt(var))


def bandpass_fit(mu, order, tau_mask):
    """Fitted bandpass of Sec. 2.2.1 "Bandpass Correction", reading R13.

    1. The averaged bandpass is the block means mu_c.
    2. High-power channels are masked before the fit: the local excess
       e_c = mu_c - (mu_{c-1} + mu_{c+1}) / 2 (one neighbour at the band
       edges) above tau_mask times 1.4826 * median_c |e_c| (the lower middle
       element of the sorted values); a masked channel takes the mean of its
       nearest unmasked neighbours on each side (one side at the edges).
    3. Least squares with Legendre polynomials P_0 .. P_order of
       x_c = (2c - (N - 1)) / (N - 1) (x = 0 for N = 1) gives b_c.
    4. RMSE = sqrt(mean_c (b_c - interpolated mu_c)^2).
    Returns dict(b, rmse, masked, mu_interp)."""
    mu = _c(mu, np.float64)
    n = len(mu)
    if n == 1:
        e = np.zeros(1)
    else:
        e = np.empty(n)
        e[0] = mu[0] - mu[1]
        e[-1] = mu[-1] - mu[-2]
        e[1:-1] = mu[1:-1] - (mu[:-2] + mu[2:]) / 2.0
    srt = np.sort(np.abs(e))
    scale = 1.4826 * srt[(n - 1) // 2]
    masked = e > tau_mask * scale
    if masked.all():
        masked[:] = False
    mi = mu.copy()
    good = np.nonzero(~masked)[0]
    for c in np.nonzero(masked)[0]:
        left = good[good < c]
        right = good[good > c]
        vals = ([mu[left[-1]]] if len(left) else []) + ([mu[right[0]]] if len(right) else [])
        mi[c] = sum(vals) / len(vals)
    xc = np.zeros(n) if n == 1 else (2.0 * np.arange(n) - (n - 1)) / (n - 1)
    V = np.polynomial.legendre.legvander(xc, order)
    coef = np.linalg.lstsq(V, mi, rcond=None)[0]
    b = V @ coef
    rmse = float(np.sqrt(np.mean((b - mi) ** 2)))
    return dict(b=b, rmse=rmse, masked=masked, mu_interp=mi, coef=coef)


def fit_stats(x, dtype, order, tau_mask):
    """Block statistics with the fitted bandpass (R13): mu, sigma as measured,
    b = the fit (8-bit data: the integer floor(fit + 1/2); 16-bit data: the fit
    in the storage format), plus the fit products."""
    st = bandpass(x, dtype)
    fit = bandpass_fit(st["mu"], order, tau_mask)
    out = dict(mu=st["mu"], sigma=st["sigma"], external=True, fit=fit)
    if dtype == "u8":
        out["b"] = np.floor(fit["b"] + 0.5).astype(np.int64)
    else:
        out["b"] = storage_bandpass(dtype, fit["b"])
    return out


def channel_mask(x, dtype, stats, rfi):
    x, code = _input(x, dtype)
    nchan, nsamp = x.shape
    W = int(rfi.chunk_width)
    nchunk = (nsamp + W - 1) // W
    raw = np.zeros((nchan, nchunk), np.uint8)
    flag = np.zeros((nchan, nchunk), np.uint8)
    if not rfi.enable_channel:
        return raw, flag
    dil = int(bool(rfi.dilate_channels))
    if "fit" in stats:
        lib().orc_channel_mask_fit(_ptr(x), code, nchan, nsamp, nsamp, W, rfi.tau_channel, dil,
                                   _ptr(_c(stats["fit"]["b"], np.float64)), stats["fit"]["rmse"], _ptr(raw),
                                   _ptr(flag))
    elif dtype == "u8" and not stats["external"]:
        lib().orc_channel_mask_u8(_ptr(x), nchan, nsamp, nsamp, W, rfi.tau_channel, dil,
                                  _ptr(stats["S"]), _ptr(stats["V"]), _ptr(raw), _ptr(flag))
    elif dtype == "u8":
        lib().orc_channel_mask_u8_ext(_ptr(x), nchan, nsamp, nsamp, W, rfi.tau_channel, dil,
                                      _ptr(stats["b"]), _ptr(stats["sigma"]), _ptr(raw), _ptr(flag))
    else:
        lib().orc_channel_mask_float(_ptr(x), code, nchan, nsamp, nsamp, W, rfi.tau_channel, dil,
                                     _ptr(stats["mu"]), _ptr(stats["sigma"]), _ptr(raw), _ptr(flag))
    return raw, flag


def spectrum_mask(x, dtype, stats, rfi, chunk_flag):
    x, code = _input(x, dtype)
    nchan, nsamp = x.shape
    W = int(rfi.chunk_width)
    spec = np.zeros(nsamp, np.uint8)
    if not rfi.enable_spectrum:
        return spec
    cf = _c(chunk_flag, np.uint8)
    if dtype == "u8" and not stats["external"]:
        lib().orc_spectrum_mask_u8(_ptr(x), nchan, nsamp, nsamp, W, rfi.tau_spectrum,
                                   _ptr(stats["S"]), _ptr(stats["V"]), _ptr(cf), _ptr(spec))
    elif dtype == "u8":
        lib().orc_spectrum_mask_u8_ext(_ptr(x), nchan, nsamp, nsamp, W, rfi.tau_spectrum,
                                       _ptr(stats["b"]), _ptr(stats["sigma"]), _ptr(cf), _ptr(spec))
    else:
        # the spectrum stage subtracts the bandpass: the fitted one when fitted
        ref = _c(stats["fit"]["b"], np.float64) if "fit" in stats else stats["mu"]
        lib().orc_spectrum_mask_float(_ptr(x), code, nchan, nsamp, nsamp, W, rfi.tau_spectrum,
                                      _ptr(ref), _ptr(stats["sigma"]), _ptr(cf), _ptr(spec))
    return spec


def corrected(x, dtype, stats, chunk_flag, spec_flag, W):
    """Substituted, bandpass-corrected samples y[c][t] = x~ - b_c (R7),
    float64; b_c is the bandpass value in the storage format."""
    x, code = _input(x, dtype)
    nchan, nsamp = x.shape
    cf = _c(chunk_flag, np.uint8)
    sf = _c(spec_flag, np.uint8)
    if dtype == "u8":
        b = stats["b"]
        flag = cf[:, np.arange(nsamp) // W].astype(bool) | sf.astype(bool)[None, :]
        return np.where(flag, 0, x.astype(np.int64) - b[:, None]).astype(np.float64)
    y = np.empty((nchan, nsamp), np.float64)
    lib().orc_corrected_float(_ptr(x), code, nchan, nsamp, nsamp, _ptr(stats["b"]), _ptr(cf),
                              _ptr(sf), W, _ptr(y))
    return y


# ---- A5 ------------------------------------------------------------------------

def dedisperse(x, dtype, stats, chunk_flag, spec_flag, W, delay, T):
    """D[d][t] for 0 <= t < T: float64 for float input, int64 for 8-bit input."""
    x, code = _input(x, dtype)
    nchan, nsamp = x.shape
    delay = _c(delay, np.int32)
    ndm = delay.shape[0]
    cf = _c(chunk_flag, np.uint8)
    sf = _c(spec_flag, np.uint8)
    if T <= 0:
        raise ValueError("block shorter than the largest delay")
    if dtype == "u8":
        D = np.empty((ndm, T), np.int64)
        lib().orc_dedisperse_u8(_ptr(x), nchan, nsamp, nsamp, _ptr(stats["b"]), _ptr(cf), _ptr(sf),
                                W, _ptr(delay), ndm, T, _ptr(D))
    else:
        D = np.empty((ndm, T), np.float64)
        lib().orc_dedisperse_float(_ptr(x), code, nchan, nsamp, nsamp, _ptr(stats["b"]), _ptr(cf),
                                   _ptr(sf), W, _ptr(delay), ndm, T, _ptr(D))
    return D


def dedisperse_points(x, dtype, stats, chunk_flag, spec_flag, W, delay, d_idx, t_idx):
    """D at selected (d, t) pairs, plus (float input) the sum of |y| there."""
    x, code = _input(x, dtype)
    nchan, nsamp = x.shape
    delay = _c(delay, np.int32)
    d_idx = _c(d_idx, np.int32)
    t_idx = _c(t_idx, np.int64)
    n = len(d_idx)
    cf = _c(chunk_flag, np.uint8)
    sf = _c(spec_flag, np.uint8)
    if dtype == "u8":
        out = np.empty(n, np.int64)
        lib().orc_dedisperse_points_u8(_ptr(x), nchan, nsamp, nsamp, _ptr(stats["b"]), _ptr(cf),
                                       _ptr(sf), W, _ptr(delay), _ptr(d_idx), _ptr(t_idx), n, _ptr(out))
        return out, None
    out = np.empty(n, np.float64)
    mass = np.empty(n, np.float64)
    args = (_ptr(x), code, nchan, nsamp, nsamp, _ptr(stats["b"]), _ptr(cf), _ptr(sf), W,
            _ptr(delay), _ptr(d_idx), _ptr(t_idx), n)
    lib().orc_dedisperse_points_float(*args, _ptr(out))
    if dtype in ("f32", "c16"):
        lib().orc_abs_mass_points_float(*args, _ptr(mass))
    else:  # FP32 accumulation of the stored 16-bit samples: bounded by sum |x~|
        lib().orc_stored_mass_points(*args, _ptr(mass))
    return out, mass


# ---- A6-A7 ---------------------------------------------------------------------

def series_stats(D):
    D = np.ascontiguousarray(D)
    ndm, T = D.shape
    mu = np.empty(ndm, np.float64)
    sigma = np.empty(ndm, np.float64)
    if D.dtype == np.int64:
        SD = np.empty(ndm, np.int64)
        SD2 = np.empty(ndm, np.int64)
        lib().orc_series_stats_int(_ptr(D), ndm, T, _ptr(SD), _ptr(SD2), _ptr(mu), _ptr(sigma))
        return dict(mu=mu, sigma=sigma, SD=SD, SD2=SD2)
    D = _c(D, np.float64)
    lib().orc_series_stats_float(_ptr(D), ndm, T, _ptr(mu), _ptr(sigma))
    return dict(mu=mu, sigma=sigma)


CAND_DTYPE = np.dtype([("beam", np.int32), ("dm_idx", np.int32), ("t_abs", np.int64),
                       ("snr", np.float32), ("value", np.float32)])


def candidates(D, mu, sigma, nsigma, beam=0, t0=0, cap=None):
    """Candidates in (d, t) order as a structured array, and the total count."""
    D = np.ascontiguousarray(D)
    ndm, T = D.shape
    if cap is None:
        cap = ndm * T
    out = np.zeros(max(int(cap), 1), CAND_DTYPE)
    mu = _c(mu, np.float64)
    sigma = _c(sigma, np.float64)
    if D.dtype == np.int64:
        n = lib().orc_candidates_int(_ptr(D), ndm, T, _ptr(mu), _ptr(sigma), nsigma, beam, t0,
                                     _ptr(out), cap)
    else:
        D = _c(D, np.float64)
        n = lib().orc_candidates_float(_ptr(D), ndm, T, _ptr(mu), _ptr(sigma), nsigma, beam, t0,
                                       _ptr(out), cap)
    return out[:min(n, cap)], int(n)


# ---- post-processing (Sec. 2.2.3) ------------------------------------------------

def median_filter(D, w):
    """Eq. 2 with the median: each value replaced by the median of the w values
    centred on it, the ends of the series repeating (R11).  w odd, 1 <= w <= 63."""
    if w % 2 != 1 or not 1 <= w <= 63:
        raise ValueError("median width must be odd, 1..63")
    D = np.ascontiguousarray(D)
    ndm, T = D.shape
    if D.dtype == np.int64:
        out = np.empty_like(D)
        lib().orc_median_int(_ptr(D), ndm, T, w, _ptr(out))
        return out
    D = _c(D, np.float64)
    out = np.empty_like(D)
    lib().orc_median_float(_ptr(D), ndm, T, w, _ptr(out))
    return out


def detrend(D):
    """Least-squares line mean + beta * (2t - (T - 1)) per series and the
    residual's population deviation (R11); for int64 series also the exact
    sums (Sy, Suy, Syy)."""
    D = np.ascontiguousarray(D)
    ndm, T = D.shape
    mean = np.empty(ndm, np.float64)
    beta = np.empty(ndm, np.float64)
    sigma = np.empty(ndm, np.float64)
    if D.dtype == np.int64:
        sums = np.empty((ndm, 3), np.int64)
        lib().orc_detrend_int(_ptr(D), ndm, T, _ptr(sums), _ptr(mean), _ptr(beta), _ptr(sigma))
        return dict(mean=mean, beta=beta, sigma=sigma, sums=sums)
    D = _c(D, np.float64)
    lib().orc_detrend_float(_ptr(D), ndm, T, _ptr(mean), _ptr(beta), _ptr(sigma))
    return dict(mean=mean, beta=beta, sigma=sigma)


def candidates_detrend(D, mean, beta, sigma, nsigma, beam=0, t0=0, cap=None):
    """Candidates of detrended series: residual >= nsigma * sigma, (d, t) order."""
    D = np.ascontiguousarray(D)
    ndm, T = D.shape
    if cap is None:
        cap = ndm * T
    out = np.zeros(max(int(cap), 1), CAND_DTYPE)
    is_int = D.dtype == np.int64
    if not is_int:
        D = _c(D, np.float64)
    n = lib().orc_candidates_detrend(_ptr(D), int(is_int), ndm, T, _ptr(_c(mean, np.float64)),
                                     _ptr(_c(beta, np.float64)), _ptr(_c(sigma, np.float64)), nsigma, beam, t0,
                                     _ptr(out), cap)
    return out[:min(n, cap)], int(n)


def post_process(D, median_width=1, detrend_on=False, nsigma=5.0, beam=0, t0=0, cap=None):
    """A6-A7 with the optional post-processing of Sec. 2.2.3: the median
    filter, then either the detrended detection or the plain one."""
    Y = median_filter(D, median_width) if median_width > 1 else D
    if detrend_on:
        st = detrend(Y)
        cands, n = candidates_detrend(Y, st["mean"], st["beta"], st["sigma"], nsigma, beam=beam, t0=t0, cap=cap)
    else:
        st = series_stats(Y)
        cands, n = candidates(Y, st["mu"], st["sigma"], nsigma, beam=beam, t0=t0, cap=cap)
    return dict(Y=Y, stats=st, candidates=cands, n_candidates=n)


# ---- the whole block -------------------------------------------------------------

def search_block(x, dtype, delay, max_delay, rfi=None, nsigma=5.0, beam=0, t0=0, stats=None,
                 cand_cap=None, keep_series=True, fit=None):
    """Run A1-A7 on one block window x (nchan, nsamp).  ``stats`` replaces the
    measured bandpass when given (see ``external_stats``); ``fit`` = (order,
    tau_mask) uses the fitted bandpass (``fit_stats``).  Returns every
    intermediate product."""
    rfi = rfi or RfiParams()
    x, _ = _input(x, dtype)
    nchan, nsamp = x.shape
    T = nsamp - max_delay
    if fit is not None:
        st = fit_stats(x, dtype, fit[0], fit[1])
    else:
        st = stats if stats is not None else bandpass(x, dtype)
    raw, cflag = channel_mask(x, dtype, st, rfi)
    sflag = spectrum_mask(x, dtype, st, rfi, cflag)
    D = dedisperse(x, dtype, st, cflag, sflag, rfi.chunk_width, delay, T)
    ss = series_stats(D)
    cands, n = candidates(D, ss["mu"], ss["sigma"], nsigma, beam=beam, t0=t0, cap=cand_cap)
    out = dict(stats=st, chunk_raw=raw, chunk_flag=cflag, spec_flag=sflag, series=ss,
               candidates=cands, n_candidates=n, T=T)
    if keep_series:
        out["D"] = D
    return out


# ---- clustering and classification of the detections (Sec. 2.3) -------------------

@dataclass
class ClusterParams:
    """Parameters of the clustering and classification stage (reading R14)."""
    t_eps: int = 20          # T_t: neighbourhood half-extent in samples
    dm_eps: int = 3          # DM_t: neighbourhood half-extent in DM trials
    snr_eps: float = 5.0     # SNR_t: neighbourhood half-extent in SNR
    min_pts: int = 5         # MinPts (the point itself included)
    smooth: int = 3          # k of the moving average of the DM-SNR signature (odd)
    rmse_max: float = 0.4    # largest RMSE of the normalised signature against Eq. 3
    dm_min: float = 1.0      # clusters peaking below this DM are broadband RFI


def dbscan(d, t, snr, prm):
    """DBSCAN (Sec. 2.3, Ester et al.) of detections (d, t, snr) with the box
    neighbourhood |d_q - d_p| <= dm_eps, |t_q - t_p| <= t_eps,
    |snr_q - snr_p| <= snr_eps (the point itself included).  Core points have
    at least min_pts neighbours; clusters are the connected groups of core
    points (core points in each other's neighbourhood); a border point (not
    core, with a core neighbour) joins the cluster of its lowest-index core
    neighbour; the rest is noise (-1).  Clusters are numbered 0, 1, ... in
    the order of their lowest-index core point.  Plain O(N^2) search.
    Returns (labels, core)."""
    d = np.asarray(d, np.int64)
    t = np.asarray(t, np.int64)
    s = np.asarray(snr, np.float64)
    n = len(d)
    nb = []
    for p in range(n):
        m = (np.abs(d - d[p]) <= prm.dm_eps) & (np.abs(t - t[p]) <= prm.t_eps) & \
            (np.abs(s - s[p]) <= prm.snr_eps)
        nb.append(np.nonzero(m)[0])
    core = np.array([len(x) >= prm.min_pts for x in nb], bool)
    comp = -np.ones(n, np.int64)
    for p in range(n):                       # components of the core graph, by search
        if not core[p] or comp[p] >= 0:
            continue
        comp[p] = p
        stack = [p]
        while stack:
            q = stack.pop()
            for r in nb[q]:
                if core[r] and comp[r] < 0:
                    comp[r] = p
                    stack.append(r)
    labels = -np.ones(n, np.int64)
    roots = sorted({int(comp[p]) for p in range(n) if core[p]})
    rank = {r: i for i, r in enumerate(roots)}
    for p in range(n):
        if core[p]:
            labels[p] = rank[int(comp[p])]
        else:
            cn = [int(q) for q in nb[p] if core[q]]
            if cn:
                labels[p] = rank[int(comp[min(cn)])]
    return labels, core


def eq3_ratio(ddm, width_ms, bw_mhz, f_ghz):
    """Eq. 3-4: measured / true peak flux of a Gaussian pulse of FWHM width_ms
    dedispersed with a DM error ddm, rectangular band of bw_mhz at f_ghz:
    (sqrt(pi) / 2) erf(zeta) / zeta, zeta = 6.91e-3 ddm bw / (W f^3); 1 at 0."""
    from math import erf, pi, sqrt
    z = 6.91e-3 * abs(ddm) * bw_mhz / (width_ms * (f_ghz * f_ghz * f_ghz))
    if z == 0.0:
        return 1.0
    return sqrt(pi) / 2.0 * erf(z) / z


def classify(d, t, snr, labels, dm_list, t_samp, bw_mhz, f_ghz, prm):
    """The classification steps of Sec. 2.3 for every cluster (reading R14):
    1. the DM-SNR signature: per DM trial of the cluster, its largest SNR;
    2. a centred moving average of prm.smooth trials over the trials from the
       cluster's lowest to its highest (trials without detections count 0;
       at the ends the average is over the trials available);
    3. d* = the trial with the most detections (ties: the lowest trial), and
       its largest SNR; d* with DM below prm.dm_min is broadband RFI;
    4. the width: (last - first detection time at d* + 1) samples, in ms;
    5. the smoothed signature divided by its largest value;
    6. Eq. 3 with dDM = DM_d - DM_{d*};
    7. the RMSE of 5 against 6 over the cluster's trials;
    8. a candidate when not broadband RFI and RMSE <= prm.rmse_max.
    Returns one dict per cluster, in cluster order."""
    d = np.asarray(d, np.int64)
    t = np.asarray(t, np.int64)
    s = np.asarray(snr, np.float64)
    out = []
    k = prm.smooth
    for c in range(int(labels.max()) + 1 if len(labels) else 0):
        m = labels == c
        dc, tc, sc = d[m], t[m], s[m]
        lo, hi = int(dc.min()), int(dc.max())
        nd = hi - lo + 1
        sig = np.zeros(nd)
        cnt = np.zeros(nd, np.int64)
        for di, si in zip(dc, sc):
            sig[di - lo] = max(sig[di - lo], si)
            cnt[di - lo] += 1
        sm = np.empty(nd)
        for i in range(nd):
            a, b = max(0, i - k // 2), min(nd, i + k // 2 + 1)
            sm[i] = sig[a:b].sum() / (b - a)
        ds = lo + int(np.argmax(cnt))
        rfi = dm_list[ds] < prm.dm_min
        ts = tc[dc == ds]
        width_ms = float(ts.max() - ts.min() + 1) * t_samp * 1e3
        norm = sm / sm.max()
        model = np.array([eq3_ratio(dm_list[lo + i] - dm_list[ds], width_ms, bw_mhz, f_ghz) for i in range(nd)])
        rmse = float(np.sqrt(np.mean((norm - model) ** 2)))
        out.append(dict(cluster=c, n=int(m.sum()), d_lo=lo, d_hi=hi, d_star=ds, snr_max=float(sc.max()),
                        t_first=int(tc.min()), t_last=int(tc.max()), width_ms=width_ms, rmse=rmse,
                        broadband=bool(rfi), candidate=bool((not rfi) and rmse <= prm.rmse_max)))
    return out

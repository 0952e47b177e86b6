"""A second, independently written statement of the search method in plain
Python (lists, ``math``, ``fractions``), for tiny inputs only.

It re-derives every step from the paper -- Eq. 1 delays, the bandpass and
thresholding stages of Sec. 2.2.1, the dedispersion sum of Sec. 2.2.2, the
series normalisation of Sec. 2.2.3 and the n-sigma detection of Sec. 2.3 --
without looking at the C oracle, and the tests require the two to agree
exactly (integers) or to 1e-12 (binary64).
"""
import math
from fractions import Fraction

K_DM = Fraction("4148.808")  # s MHz^2, the constant of Eq. 1


def freqs(nchan, f_lo, bw):
    return [f_lo + (c + 0.5) * (bw / nchan) for c in range(nchan)]


def delays_exact(nchan, f_lo, bw, t_samp, dms):
    """Exact rational delays (no rounding anywhere)."""
    df = Fraction(bw) / nchan
    f = [Fraction(f_lo) + (c + Fraction(1, 2)) * df for c in range(nchan)]
    fref = max(f)
    ts = Fraction(t_samp)
    return [[K_DM * Fraction(dm) * (1 / (fc * fc) - 1 / (fref * fref)) / ts for fc in f] for dm in dms]


def delays_float(nchan, f_lo, bw, t_samp, dms):
    """Integer delays, binary64 evaluated left to right, rounded half up."""
    f = freqs(nchan, f_lo, bw)
    fref = max(f)
    out = []
    for dm in dms:
        row = []
        for fc in f:
            v = 4148.808 * dm * (1.0 / (fc * fc) - 1.0 / (fref * fref)) / t_samp
            row.append(int(math.floor(v + 0.5)))
        out.append(row)
    return out


def storage_round(v, kind):
    """mu in the storage format, nearest with ties to even (R7)."""
    if kind == "f32" or v == 0:
        return v
    sig, emin = (11, -14) if kind == "f16" else (8, -126)
    m, e = math.frexp(abs(v))
    q = max(e - sig, emin - sig + 1)
    r = round(abs(v) / 2.0 ** q) * 2.0 ** q     # round() ties to even
    return math.copysign(r, v)


def _chunks(n, W):
    return [(lo, min(lo + W, n)) for lo in range(0, n, W)]


def search(x, is_u8, W, tau_c, tau_s, chan_on, spec_on, delays, nsigma, dilate_channels=False, kind="f32"):
    """x: list of channel lists.  Returns (flags, spec, D, mu_d, sigma_d, cands).
    kind: storage format of float data ("f32", "f16", "bf16")."""
    nchan, n = len(x), len(x[0])
    # bandpass
    if is_u8:
        S = [sum(r) for r in x]
        Q = [sum(v * v for v in r) for r in x]
        V = [n * q - s * s for s, q in zip(S, Q)]
        b = [(2 * s + n) // (2 * n) for s in S]
        mu = [s / n for s in S]
        sig = [math.sqrt(v) / n for v in V]
    else:
        mu = [math.fsum(r) / n for r in x]
        sig = [math.sqrt(math.fsum((v - m) ** 2 for v in r) / n) for r, m in zip(x, mu)]
    ch = _chunks(n, W)
    # channel thresholding
    raw = [[False] * len(ch) for _ in range(nchan)]
    if chan_on:
        for c in range(nchan):
            for k, (lo, hi) in enumerate(ch):
                if is_u8:
                    e = sum(n * x[c][t] - S[c] for t in range(lo, hi))
                    raw[c][k] = float(e) > tau_c * math.sqrt(float(V[c]) * float(hi - lo))
                else:
                    e = math.fsum(x[c][t] - mu[c] for t in range(lo, hi))
                    raw[c][k] = e > tau_c * sig[c] * math.sqrt(hi - lo)
    flags = [[False] * len(ch) for _ in range(nchan)]
    for c in range(nchan):
        for k in range(len(ch)):
            nb = [raw[c][j] for j in (k - 1, k, k + 1) if 0 <= j < len(ch)]
            if dilate_channels:
                nb += [raw[j][k] for j in (c - 1, c + 1) if 0 <= j < nchan]
            flags[c][k] = any(nb)
    # spectrum thresholding
    spec = [False] * n
    if spec_on:
        for t in range(n):
            # only the channels whose chunk at t is not flagged take part,
            # in the sum and in its spread
            keep = [c for c in range(nchan) if not flags[c][t // W]]
            if is_u8:
                thr = tau_s * math.sqrt(float(sum(V[c] for c in keep)))
                m = sum(n * x[c][t] - S[c] for c in keep)
                spec[t] = float(m) > thr
            else:
                thr = tau_s * math.sqrt(math.fsum(sig[c] * sig[c] for c in keep))
                m = math.fsum(x[c][t] - mu[c] for c in keep)
                spec[t] = m > thr

    if not is_u8:
        b = [storage_round(m, kind) for m in mu]

    def y(c, t):
        if flags[c][t // W] or spec[t]:
            return 0
        return x[c][t] - b[c]

    dmax = max(max(r) for r in delays)
    T = n - dmax
    D = [[(sum if is_u8 else math.fsum)(y(c, t + delays[d][c]) for c in range(nchan)) for t in range(T)]
         for d in range(len(delays))]
    mu_d, sig_d = [], []
    for row in D:
        if is_u8:
            s = sum(row)
            q = sum(v * v for v in row)
            m = s / T
            var = q / T - m * m
            mu_d.append(m)
            sig_d.append(math.sqrt(var if var > 0 else 0.0))
        else:
            m = math.fsum(row) / T
            mu_d.append(m)
            sig_d.append(math.sqrt(math.fsum((v - m) ** 2 for v in row) / T))
    cands = []
    for d, row in enumerate(D):
        if not sig_d[d] > 0:
            continue
        for t, v in enumerate(row):
            if float(v) - mu_d[d] >= nsigma * sig_d[d]:
                cands.append((d, t))
    return dict(flags=flags, raw=raw, spec=spec, D=D, mu_d=mu_d, sigma_d=sig_d, cands=cands, T=T,
                mu=mu, sigma=sig)

"""Pins of the CPU oracle to facts fixed outside itself: closed forms, the
paper's equations, invariants of the dedispersion sum, and an independently
written brute force.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import oracle as O
from tests import bruteforce as BF

BAND = dict(nchan=1024, f_lo=398.0, bw=20.0, t_samp=51.2e-6)


# ---- Eq. 1: the delay table ------------------------------------------------------

def test_delay_spot_values_config1():
    """Lowest channel of the 398-418 MHz / 1024-channel / 51.2 us band: the
    exact closed form gives 47.73, 1432.03 and 3007.25 samples at DM 1, 30, 63."""
    ex = BF.delays_exact(1024, 398, 20, "51.2e-6", [1, 30, 63])
    assert [round(float(r[0]), 2) for r in ex] == [47.73, 1432.03, 3007.25]
    tab, dmax = O.delay_table(**BAND, dm=np.arange(64, dtype=np.float64))
    assert tab[1, 0] == 48 and tab[30, 0] == 1432 and tab[63, 0] == 3007
    assert dmax == 3007
    assert np.all(tab[:, -1] == 0)          # the top channel is the reference (R2)
    assert np.all(tab[0] == 0)              # DM 0 has no delay


@pytest.mark.parametrize("nchan,f_lo,bw,ts,dms", [
    (1024, 398.0, 20.0, "51.2e-6", [0.2 * i for i in range(0, 640, 37)]),
    (4096, 1200.0, 300.0, "64e-6", [float(i) for i in range(0, 2048, 97)]),
    (256, 398.0, 20.0, "51.2e-6", [0.0, 0.2, 5.4, 127.8]),
    (37, 100.0, 3.3, "1e-3", [0.0, 1.0, 2.5, 10.0]),
])
def test_delay_table_matches_exact_rational(nchan, f_lo, bw, ts, dms):
    """Rounded binary64 delays equal the exactly rounded rational closed form
    except where the exact value lies within 1e-6 of a half-integer tie."""
    dms = np.array(dms, dtype=np.float64)
    tab, _ = O.delay_table(nchan, f_lo, bw, float(ts), dms)
    ex = BF.delays_exact(nchan, Fraction(f_lo), Fraction(bw), ts, [Fraction(float(d)) for d in dms])
    near = 0
    for d in range(len(dms)):
        for c in range(nchan):
            v = ex[d][c]
            r = math.floor(v + Fraction(1, 2))
            frac = v - math.floor(v)
            if abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 6):
                near += 1
                assert tab[d, c] in (r - 1, r)
            else:
                assert tab[d, c] == r, (d, c, float(v))
    assert near <= 2


def test_delay_tie_log_finds_planted_and_exact_ties():
    """The tie log (R3) lists exactly the (d, c) pairs whose unrounded delay,
    computed as an exact rational, lies within 1e-9 of a half-integer.  Two
    trials are planted on ties of channel 0 (their DM makes the exact delay
    n + 1/2 up to the binary64 rounding of the DM itself)."""
    nchan, f_lo, bw, ts = 16, 400.0, 16.0, "1e-3"
    unit = BF.delays_exact(nchan, Fraction(f_lo), Fraction(bw), ts, [Fraction(1)])[0][0]  # delay at DM 1
    planted = [float(Fraction(2 * n + 1, 2) / unit) for n in (3, 40)]
    dms = np.array([0.0, 1.0, planted[0], 7.3, planted[1], 55.55], dtype=np.float64)
    ties = O.delay_ties(nchan, f_lo, bw, float(ts), dms, eps=1e-9)
    ex = BF.delays_exact(nchan, Fraction(f_lo), Fraction(bw), ts, [Fraction(float(d)) for d in dms])
    want = {(d, c) for d in range(len(dms)) for c in range(nchan)
            if abs(ex[d][c] - math.floor(ex[d][c]) - Fraction(1, 2)) <= Fraction(1, 10 ** 9)}
    got = {(d, c) for d, c, _ in ties}
    assert (2, 0) in want and (4, 0) in want
    assert got == want
    for d, c, v in ties:
        assert abs(v - float(ex[d][c])) < 1e-9
    # a plan of the benchmark's band: its ties (if any) are what the exact
    # rational form finds within the same distance
    dms = np.arange(0, 640, 7) * 0.2
    ties = {(d, c) for d, c, _ in O.delay_ties(1024, 398.0, 20.0, 51.2e-6, dms)}
    ex = BF.delays_exact(1024, Fraction(398), Fraction(20), "51.2e-6", [Fraction(float(d)) for d in dms])
    want = {(d, c) for d in range(len(dms)) for c in range(1024)
            if abs(ex[d][c] - math.floor(ex[d][c]) - Fraction(1, 2)) <= Fraction(1, 10 ** 9)}
    assert ties == want


def test_delay_uses_4148_808_not_rounded_constant():
    """The binding constant is 4148.808 s MHz^2; Eq. 1's printed 4.15e6 ms
    differs by 0.03 %, which moves the large delays by about one sample."""
    tab, dmax = O.delay_table(4096, 1200.0, 300.0, 64e-6, np.array([2047.0]))
    assert dmax == 33166
    ex_415 = 4150.0 * 2047 * (1 / (1200 + 0.5 * 300 / 4096) ** 2 - 1 / (1500 - 0.5 * 300 / 4096) ** 2) / 64e-6
    assert round(ex_415) != dmax


def test_delay_descending_band_mirrors_ascending():
    dms = np.linspace(0, 100, 11)
    up, m1 = O.delay_table(512, 398.0, 20.0, 51.2e-6, dms)
    down, m2 = O.delay_table(512, 418.0, -20.0, 51.2e-6, dms)
    assert m1 == m2
    assert np.array_equal(up, down[:, ::-1])


def test_delay_monotone_and_python_float_agree():
    dms = np.arange(0, 128, 0.2)[:640]
    tab, _ = O.delay_table(**BAND, dm=dms)
    assert np.all(np.diff(tab, axis=0) >= 0)       # grows with DM
    assert np.all(np.diff(tab, axis=1) <= 0)       # shrinks towards the top of the band
    pyf = BF.delays_float(1024, 398.0, 20.0, 51.2e-6, list(dms[::41]))
    assert np.array_equal(tab[::41], np.array(pyf))


@pytest.mark.parametrize("args", [
    (0, 398.0, 20.0, 51.2e-6, [1.0]),
    (16, 398.0, 20.0, 0.0, [1.0]),
    (16, 398.0, 20.0, 51.2e-6, [-1.0]),
    (16, 398.0, 20.0, 51.2e-6, [float("nan")]),
    (16, 398.0, 0.0, 51.2e-6, [1.0]),
    (16, -10.0, 5.0, 51.2e-6, [1.0]),
])
def test_delay_rejects_invalid(args):
    with pytest.raises(ValueError):
        O.delay_table(*args[:4], np.array(args[4]))


# ---- whole-chain brute force on tiny inputs -------------------------------------------

def _tiny(dtype, seed, nchan, nsamp):
    g = synth.rng(seed)
    xf = g.standard_normal((nchan, nsamp)).astype(np.float32)
    # a few strong features so that both thresholding stages fire
    xf[1, 8:40] += 6.0
    xf[:, nsamp // 2] += 8.0
    xf[nchan - 1, nsamp - 5:] += 9.0
    if dtype == "u8":
        return synth.to_u8(xf * 16 + 128)
    if dtype == "f16":
        return synth.to_f16(xf)
    if dtype == "bf16":
        return synth.to_bf16_bits(xf)
    return xf


def _as_lists(x, dtype):
    if dtype == "u8":
        return [[int(v) for v in r] for r in x]
    if dtype == "bf16":
        return synth.bf16_bits_to_f32(x).astype(np.float64).tolist()
    return x.astype(np.float64).tolist()


@pytest.mark.parametrize("dtype", ["u8", "f32", "f16", "bf16"])
@pytest.mark.parametrize("seed,nchan,nsamp,W,dil", [(1, 7, 200, 16, False), (2, 16, 256, 24, True),
                                                    (3, 3, 97, 10, False)])
def test_bruteforce_agrees(dtype, seed, nchan, nsamp, W, dil):
    x = _tiny(dtype, seed, nchan, nsamp)
    dms = np.array([0.0, 3.0, 7.5, 12.0, 20.0, 33.0, 40.0, 47.0][: 8 if nchan > 3 else 4])
    f_lo, bw = 398.0, 20.0 * nchan / 1024 * 40
    ts = float(O.delay_exact(nchan, f_lo, bw, 1.0, np.array([dms[-1]])).max()) / (nsamp / 3.0)
    tab, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    assert dmax < nsamp // 2
    rfi = O.RfiParams(chunk_width=W, tau_channel=3.0, tau_spectrum=3.0, dilate_channels=dil)
    r = O.search_block(x, dtype, tab, dmax, rfi=rfi, nsigma=2.0)
    bf = BF.search(_as_lists(x, dtype), dtype == "u8", W, 3.0, 3.0, True, True, tab.tolist(), 2.0,
                   dilate_channels=dil, kind=dtype if dtype != "u8" else "f32")
    assert np.array_equal(r["chunk_raw"].astype(bool), np.array(bf["raw"]))
    assert np.array_equal(r["chunk_flag"].astype(bool), np.array(bf["flags"]))
    assert np.array_equal(r["spec_flag"].astype(bool), np.array(bf["spec"]))
    assert r["chunk_flag"].any() and r["spec_flag"].any()
    D = r["D"]
    if dtype == "u8":
        assert D.dtype == np.int64
        assert np.array_equal(D, np.array(bf["D"], dtype=np.int64))
        assert np.array_equal(r["series"]["mu"], np.array(bf["mu_d"]))
        assert np.array_equal(r["series"]["sigma"], np.array(bf["sigma_d"]))
    else:
        np.testing.assert_allclose(D, np.array(bf["D"]), rtol=0, atol=1e-12 * max(1.0, np.abs(D).max()))
        np.testing.assert_allclose(r["series"]["mu"], bf["mu_d"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["series"]["sigma"], bf["sigma_d"], rtol=1e-12, atol=1e-12)
    got = [(int(c["dm_idx"]), int(c["t_abs"])) for c in r["candidates"]]
    assert got == bf["cands"]
    assert r["n_candidates"] == len(bf["cands"]) > 0


# ---- invariants of the dedispersion sum --------------------------------------------------

def _plan(dms, nchan=64, nsamp=2048):
    bw = 20.0 * nchan / 1024 * 8
    tab, dmax = O.delay_table(nchan, 398.0, bw, 51.2e-6, np.asarray(dms, np.float64))
    return tab, dmax


def test_dm0_row_is_plain_channel_sum():
    x = synth.noise(64, 2048, 7)
    x[5, 100:700] += 20
    x[:, 999] += 8
    tab, dmax = _plan([0.0, 5.0, 10.0, 20.0])
    r = O.search_block(x, "f32", tab, dmax, rfi=O.RfiParams(chunk_width=64))
    assert r["chunk_flag"].any() and r["spec_flag"].any()
    mu = x.astype(np.float64).mean(axis=1)
    W = 64
    flag = r["chunk_flag"][:, np.arange(2048) // W].astype(bool) | r["spec_flag"].astype(bool)[None, :]
    y = np.where(flag, 0.0, x.astype(np.float64) - mu[:, None])
    T = r["T"]
    np.testing.assert_allclose(r["D"][0], y[:, :T].sum(axis=0), rtol=0, atol=1e-9)


def test_flagged_samples_contribute_nothing():
    """Garbage written into flagged samples leaves D unchanged (R7)."""
    x = synth.noise(64, 2048, 8)
    x[10:12, 300:900] += 25
    x[:, 1500] += 9
    tab, dmax = _plan([0.0, 4.0, 9.0, 15.0])
    rfi = O.RfiParams(chunk_width=64)
    st = O.bandpass(x, "f32")
    _, cf = O.channel_mask(x, "f32", st, rfi)
    sf = O.spectrum_mask(x, "f32", st, rfi, cf)
    assert cf.sum() > 0 and sf.sum() > 0
    T = 2048 - dmax
    D1 = O.dedisperse(x, "f32", st, cf, sf, 64, tab, T)
    g = synth.rng(99)
    flag = cf[:, np.arange(2048) // 64].astype(bool) | sf.astype(bool)[None, :]
    x2 = x.copy()
    x2[flag] = g.uniform(-1e6, 1e6, flag.sum()).astype(np.float32)
    D2 = O.dedisperse(x2, "f32", st, cf, sf, 64, tab, T)
    assert np.array_equal(D1, D2)


def test_linearity_and_impulse_response():
    tab, dmax = _plan([0.0, 3.0, 11.0, 30.0])
    zero = O.external_stats("f32", np.zeros(64), np.ones(64))
    off = O.RfiParams(enable_channel=False, enable_spectrum=False, chunk_width=64)
    T = 2048 - dmax

    def D(x):
        return O.dedisperse(x, "f32", zero, np.zeros((64, 32), np.uint8), np.zeros(2048, np.uint8), 64, tab, T)

    a = synth.noise(64, 2048, 1)
    b = synth.noise(64, 2048, 2)
    np.testing.assert_allclose(D(a + b), D(a) + D(b), rtol=0, atol=1e-5)
    imp = np.zeros((64, 2048), np.float32)
    c0, t0 = 17, 1000
    imp[c0, t0] = 1.0
    Di = D(imp)
    for d in range(4):
        t = t0 - tab[d, c0]
        assert Di[d, t] == 1.0
        assert Di[d].sum() == 1.0
    _ = off


def test_pulse_peaks_at_its_dm_and_time():
    """Noise-free 1 ms Gaussian pulse swept with the DM-30 delays peaks at
    exactly (d = 30, t0); with N(0,1) noise at SNR 20 it is recovered within
    one trial and half a FWHM."""
    dms = np.arange(64, dtype=np.float64)
    tab, dmax = O.delay_table(**BAND, dm=dms)
    t0, nsamp = 12000, 32768
    fwhm = 1e-3 / 51.2e-6
    x = np.zeros((1024, nsamp), np.float32)
    synth.add_pulse(x, tab[30].astype(np.float64) + t0, fwhm, 0.625)
    zero = O.external_stats("f32", np.zeros(1024), np.ones(1024))
    W = 256
    T = nsamp - dmax
    nk = (nsamp + W - 1) // W
    sub = np.arange(t0 - 400, t0 + 400)
    dd = np.repeat(np.arange(64), len(sub)).astype(np.int32)
    tt = np.tile(sub, 64).astype(np.int64)
    v, _ = O.dedisperse_points(x, "f32", zero, np.zeros((1024, nk), np.uint8), np.zeros(nsamp, np.uint8),
                               W, tab, dd, tt)
    i = int(np.argmax(v))
    assert (dd[i], tt[i]) == (30, t0)
    # with noise, through the whole chain
    x = synth.single_block_workload(lambda: tab[30].astype(np.float64), seed=1000)
    r = O.search_block(x, "f32", tab, dmax, keep_series=True)
    D = r["D"]
    d, t = np.unravel_index(np.argmax(D), D.shape)
    assert abs(d - 30) <= 1 and abs(t - t0) <= math.ceil(fwhm / 2)
    snr = (D[d, t] - r["series"]["mu"][d]) / r["series"]["sigma"][d]
    assert 17 < snr < 23
    assert T == r["T"]


def test_dm_response_follows_eq3():
    """Peak of a dedispersed Gaussian pulse at a wrong DM relative to the right
    one follows Eq. 3-4 (rectangular band approximation) within 15 %."""
    dms = np.array([30.0, 30.2, 30.6, 31.0, 29.0, 32.0])
    tab, dmax = O.delay_table(**BAND, dm=dms)
    x = np.zeros((1024, 8192), np.float32)
    fwhm = 1e-3 / 51.2e-6
    # a continuous sweep for DM 30 (the sky), not the rounded table
    ex = BF.delays_exact(1024, 398, 20, "51.2e-6", [30])[0]
    synth.add_pulse(x, np.array([float(v) for v in ex]) + 1000, fwhm, 1.0)
    zero = O.external_stats("f32", np.zeros(1024), np.ones(1024))
    D = O.dedisperse(x, "f32", zero, np.zeros((1024, 32), np.uint8), np.zeros(8192, np.uint8), 256, tab,
                     8192 - dmax)
    peak = D.max(axis=1)
    for i, dm in enumerate(dms[1:], start=1):
        ddm = abs(dm - 30.0)
        zeta = 6.91e-3 * ddm * 20.0 / (1.0 * 0.408 ** 3)
        pred = math.sqrt(math.pi) / 2 / zeta * math.erf(zeta)
        assert abs(peak[i] / peak[0] - pred) <= 0.15 * pred, (dm, peak[i] / peak[0], pred)


# ---- statistics -------------------------------------------------------------------------

def test_bandpass_float_matches_numpy():
    x = synth.noise(32, 5000, 3, mean=128.0, std=16.0)
    st = O.bandpass(x, "f32")
    xd = x.astype(np.float64)
    np.testing.assert_allclose(st["mu"], xd.mean(axis=1), rtol=1e-13)
    np.testing.assert_allclose(st["sigma"], xd.std(axis=1), rtol=1e-12)


def test_bandpass_u8_exact():
    x = synth.to_u8(synth.noise(16, 3001, 4, mean=128, std=16))
    x[3] = 0          # a dropped-packet gap channel
    st = O.bandpass(x, "u8")
    xi = x.astype(np.int64)
    assert np.array_equal(st["S"], xi.sum(axis=1))
    assert np.array_equal(st["Q"], (xi * xi).sum(axis=1))
    assert np.array_equal(st["b"], np.floor(xi.mean(axis=1) + 0.5).astype(np.int64))
    np.testing.assert_allclose(st["sigma"], xi.std(axis=1), rtol=1e-12)
    assert st["sigma"][3] == 0.0 and st["b"][3] == 0


def test_series_stats_and_candidates_against_numpy():
    g = synth.rng(5)
    D = g.standard_normal((6, 4000))
    D[2, 1234] = 12.0
    D[4, 10] = 9.0
    D[5, :] = 3.0                   # sigma = 0: no candidates
    ss = O.series_stats(D)
    np.testing.assert_allclose(ss["mu"], D.mean(axis=1), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ss["sigma"], D.std(axis=1), rtol=1e-12, atol=1e-15)
    c, n = O.candidates(D, ss["mu"], ss["sigma"], 5.0, beam=3, t0=100)
    ref = [(d, t) for d in range(5) for t in range(4000) if D[d, t] - ss["mu"][d] >= 5 * ss["sigma"][d]]
    assert [(int(a["dm_idx"]), int(a["t_abs"]) - 100) for a in c] == ref
    assert (2, 1234) in ref and (4, 10) in ref
    assert all(int(a["beam"]) == 3 for a in c)
    c2, n2 = O.candidates(D, ss["mu"], ss["sigma"], 5.0, cap=1)
    assert len(c2) == 1 and n2 == n


def test_all_zero_gap_spectra_are_not_flagged():
    """Dropped-packet gaps (Sec. 2.1) are all-zero spectra; they fall below the
    mean, and the upward-only thresholds of Sec. 2.2.1 do not flag them."""
    x = synth.to_u8(synth.noise(32, 1024, 6, mean=128, std=16))
    x[:, 300:340] = 0
    st = O.bandpass(x, "u8")
    rfi = O.RfiParams(chunk_width=32)
    raw, cf = O.channel_mask(x, "u8", st, rfi)
    sf = O.spectrum_mask(x, "u8", st, rfi, cf)
    assert not sf[300:340].any()
    assert not raw[:, 300 // 32: 340 // 32 + 1].any()


def test_storage_bandpass_matches_library_conversions():
    """The 16-bit bandpass value (R7) is mu rounded to nearest even in the
    storage format: numpy's binary16 and torch's bfloat16 conversions agree."""
    import torch
    g = synth.rng(11)
    mu = np.concatenate([g.standard_normal(2000) * 10 ** g.uniform(-8, 4, 2000),
                         [0.0, -0.0, 65504.0, 6.1e-5, 5.96e-8, 1 + 2 ** -11, 1 + 3 * 2 ** -11, 128.3]])
    b16 = O.storage_bandpass("f16", mu)
    assert np.array_equal(b16, mu.astype(np.float16).astype(np.float64))
    bbf = O.storage_bandpass("bf16", mu)
    ref = torch.tensor(mu, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bbf, ref)
    assert np.array_equal(O.storage_bandpass("f32", mu), mu)


@pytest.mark.parametrize("lo,hi", [(64.0, 1024.0), (1024.0, 4096.0)])
def test_storage_bandpass_cost_is_a_series_offset(lo, hi):
    """Cost of R7 for binary16 data against a binary64 bandpass value: every
    unflagged sample of channel c moves by mu_c - b_c, so D moves by the sum
    of (mu_c - b_c) over the channels unflagged at (c, t + delay[d][c]): with
    nothing flagged one constant per block, which the series normalisation
    removes exactly; a flagged sample contributes 0 under both readings, so
    each flagged term shifts D by at most max |mu_c - b_c| (half an ulp of
    the level)."""
    g = synth.rng(7)
    nchan, nsamp, W = 64, 4096, 256
    mu_c = g.uniform(lo, hi, nchan)
    x = synth.to_f16(synth.noise(nchan, nsamp, 11, std=16.0) + mu_c[:, None].astype(np.float32))
    tab, dmax = _plan([0.0, 4.0, 9.0, 15.0])
    T = nsamp - dmax
    st = O.bandpass(x, "f16")
    st64 = dict(st, b=st["mu"].copy())
    dev = st["mu"] - st["b"]
    assert 0 < np.abs(dev).max() <= 2.0 ** (np.floor(np.log2(hi)) - 11)
    cf = np.zeros((nchan, nsamp // W), np.uint8)
    sf = np.zeros(nsamp, np.uint8)
    D = O.dedisperse(x, "f16", st, cf, sf, W, tab, T)
    D64 = O.dedisperse(x, "f16", st64, cf, sf, W, tab, T)
    scale = np.abs(x.astype(np.float64)).sum(axis=0).max()
    assert np.allclose(D - D64, dev.sum(), rtol=0, atol=1e-12 * scale)
    z = (D - D.mean(1, keepdims=True)) / D.std(1, keepdims=True)
    z64 = (D64 - D64.mean(1, keepdims=True)) / D64.std(1, keepdims=True)
    assert np.abs(z - z64).max() < 1e-9
    # a flagged chunk and a flagged spectrum: the offset then varies with
    # the flags, by at most max |mu_c - b_c| per flagged term
    cf[5, 3] = 1
    sf[1000:1010] = 1
    D = O.dedisperse(x, "f16", st, cf, sf, W, tab, T)
    D64 = O.dedisperse(x, "f16", st64, cf, sf, W, tab, T)
    off = D - D64 - dev.sum()
    assert np.abs(off).max() > 0
    assert np.abs(off).max() <= nchan * np.abs(dev).max() + 1e-12 * scale


# ---- running bandpass statistics (reading R15) -------------------------------------

def test_running_stats_alpha_one_is_per_block_and_closed_form():
    """alpha = 1 gives each block's own statistics; otherwise the running mean
    and variance after k blocks equal the closed form of the exponential
    average, sum_i w_i m_i with w_1 = (1 - alpha)^(k - 1) and
    w_i = alpha (1 - alpha)^(k - i) for i > 1 (weights summing to 1)."""
    blocks = [synth.noise(8, 512, 40 + k, mean=1.0 + k, std=1.0 + 0.5 * k) for k in range(4)]
    st = None
    for x in blocks:
        st, s = O.running_stats(st, x, "f32", 1.0)
        b = O.bandpass(x, "f32")
        assert np.array_equal(s["mu"], b["mu"]) and np.allclose(s["sigma"], b["sigma"], rtol=1e-15)
        assert s["external"]
    a = 0.3
    st = None
    for k, x in enumerate(blocks, 1):
        st, s = O.running_stats(st, x, "f32", a)
        w = [(1 - a) ** (k - 1)] + [a * (1 - a) ** (k - i) for i in range(2, k + 1)]
        assert abs(sum(w) - 1.0) < 1e-12
        mus = [O.bandpass(blocks[i], "f32")["mu"] for i in range(k)]
        vs = [O.bandpass(blocks[i], "f32")["sigma"] ** 2 for i in range(k)]
        np.testing.assert_allclose(s["mu"], sum(wi * m for wi, m in zip(w, mus)), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(s["sigma"] ** 2, sum(wi * v for wi, v in zip(w, vs)), rtol=1e-12)


def test_running_stats_u8_hand_values():
    """Two 8-bit blocks of constant channels 10 and 20 (variance 0, then a
    channel alternating 18/22: variance 4): with alpha = 1/2 the running mean
    is 15, the running variance 2, the integer bandpass floor(15 + 1/2) = 15."""
    x1 = np.full((2, 8), 10, np.uint8)
    x2 = np.full((2, 8), 20, np.uint8)
    x2[1, 0::2], x2[1, 1::2] = 18, 22
    st, s1 = O.running_stats(None, x1, "u8", 0.5)
    assert np.array_equal(s1["mu"], [10.0, 10.0]) and np.array_equal(s1["sigma"], [0.0, 0.0])
    st, s2 = O.running_stats(st, x2, "u8", 0.5)
    assert np.array_equal(s2["mu"], [15.0, 15.0])
    assert np.array_equal(st[1], [0.0, 2.0]) and np.array_equal(s2["sigma"], np.sqrt([0.0, 2.0]))
    assert np.array_equal(s2["b"], [15, 15])

"""Post-processing (Sec. 2.2.3: the median filter of Eq. 2, detrending and
normalisation) through the C ABI against the oracle.

Bars: 8-bit data bit-exact (filtered series, detrending line and deviation,
candidate records); float data: the filtered series is exactly the median of
the GPU's own dedispersed series (a selection, no arithmetic) and within the
dedispersion bound of the oracle's (the median is 1-Lipschitz in the sup
norm), the line and deviation within 1e-6 relative of the oracle's, and the
candidate set equal to the oracle's outside a borderline band; the
candidates are in every case exactly the binary64 decisions on the GPU's own
filtered series and line."""
import os

import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O
from tests.gpu_run import GpuBeam

pytestmark = pytest.mark.gpu

TOL = 1e-5
NCHAN, F_LO, BW, TS = 128, 398.0, 20.0, 51.2e-6


@pytest.fixture(scope="module", autouse=True)
def _setup():
    tp.build()
    O.set_threads(os.cpu_count() or 1)


def _block(dtype, nsamp, seed, od):
    xf = synth.noise(NCHAN, nsamp, seed)
    # a slow drift common to all channels (what detrending removes) and a pulse
    xf += (np.linspace(-1.0, 1.0, nsamp, dtype=np.float32) * 0.6)[None, :]
    synth.add_pulse(xf, od[30].astype(np.float64) + nsamp // 2, 12.0, 0.9)
    if dtype == "u8":
        return synth.to_u8(xf * 16.0 + 128.0)
    if dtype == "f16":
        return synth.to_f16(xf)
    return xf


def _decide(Y, mean, beta, sigma, nsigma, detrend):
    """The detection predicate in binary64, the oracle's operation order."""
    Yd = Y.astype(np.float64)
    T = Y.shape[1]
    if detrend:
        u = (2 * np.arange(T, dtype=np.int64) - (T - 1)).astype(np.float64)
        lin = mean[:, None] + beta[:, None] * u[None, :]
        hit = (Yd - lin) >= (nsigma * sigma)[:, None]
    else:
        hit = (Yd - mean[:, None]) >= (nsigma * sigma)[:, None]
    hit &= (sigma > 0)[:, None]
    return hit


def _run(dtype, w, detrend, nsamp=8999, nsigma=4.5, seed=6100):
    dms = np.arange(48) * 1.0
    od, dmax = O.delay_table(NCHAN, F_LO, BW, TS, dms)
    x = _block(dtype, nsamp, seed, od)
    rfi = O.RfiParams()
    g = GpuBeam(NCHAN, F_LO, BW, TS, dms, dtype, rfi=rfi, nsigma=nsigma, cap=1 << 20)
    try:
        tp.tp_plan_set_postprocess(g.plan, w, detrend)
        r = g.run(x)
        Y = tp.tp_get_processed_series(g.e, g.beam, ndm=len(dms), is_int=dtype == "u8")
        mu, sig = tp.tp_get_series_stats(g.e, g.beam, len(dms))
        beta = tp.tp_get_detrend(g.e, g.beam, len(dms))[1] if detrend else np.zeros(len(dms))
    finally:
        g.close()
    o = O.search_block(x, dtype, od, dmax, rfi=rfi, nsigma=nsigma)
    return x, r, Y, mu, sig, beta, o, od


@pytest.mark.parametrize("w,detrend", [(5, True), (9, False), (1, True), (3, True)])
def test_post_u8_bit_exact(w, detrend):
    x, r, Y, mu, sig, beta, o, od = _run("u8", w, detrend)
    D = r["D"].astype(np.int64)
    assert np.array_equal(D, o["D"])
    p = O.post_process(o["D"], median_width=w, detrend_on=detrend, nsigma=4.5)
    assert np.array_equal(Y.astype(np.int64), p["Y"])
    if detrend:
        assert np.array_equal(mu, p["stats"]["mean"])
        assert np.array_equal(beta, p["stats"]["beta"])
        assert np.array_equal(sig, p["stats"]["sigma"])
    else:
        assert np.array_equal(mu, p["stats"]["mu"]) and np.array_equal(sig, p["stats"]["sigma"])
    assert r["n_candidates"] == p["n_candidates"] > 0
    got, want = r["candidates"], p["candidates"]
    for f in ("dm_idx", "t_abs", "snr", "value"):
        assert np.array_equal(got[f], want[f]), f


@pytest.mark.parametrize("dtype,w,detrend", [("f32", 5, True), ("f32", 3, False), ("f16", 7, True),
                                             ("f32", 1, True)])
def test_post_float(dtype, w, detrend):
    x, r, Y, mu, sig, beta, o, od = _run(dtype, w, detrend)
    Dg = r["D"].astype(np.float64)
    # exactly the median of the GPU's own series
    assert np.array_equal(Y.astype(np.float64), O.median_filter(Dg, w) if w > 1 else Dg)
    # within the dedispersion bound of the oracle's filtered series
    ndm, T = Dg.shape
    dd = np.repeat(np.arange(ndm, dtype=np.int32), T)
    tt = np.tile(np.arange(T, dtype=np.int64), ndm)
    _, mass = O.dedisperse_points(x, dtype, o["stats"], o["chunk_flag"], o["spec_flag"], 256, od, dd, tt)
    bound = TOL * mass.reshape(ndm, T).max()
    p = O.post_process(o["D"], median_width=w, detrend_on=detrend, nsigma=4.5)
    assert np.abs(Y.astype(np.float64) - p["Y"]).max() <= bound
    st = p["stats"]
    m_o = st["mean"] if detrend else st["mu"]
    scale = st["sigma"]
    assert np.all(np.abs(mu - m_o) <= 1e-6 * scale + bound)
    assert np.all(np.abs(sig - st["sigma"]) <= 1e-6 * scale + bound)
    if detrend:
        assert np.all(np.abs(beta - st["beta"]) * (T - 1) <= 1e-6 * scale + bound)
    # the GPU's candidates are exactly its binary64 decisions
    hit = _decide(Y, mu, beta, sig, 4.5, detrend)
    keys = {(int(c["dm_idx"]), int(c["t_abs"])) for c in r["candidates"]}
    assert keys == {(int(d), int(t)) for d, t in zip(*np.nonzero(hit))}
    assert r["n_candidates"] == int(hit.sum()) > 0
    # and equal to the oracle's outside the band the float differences can move
    mine = _decide(p["Y"], m_o, st["beta"] if detrend else np.zeros(ndm), st["sigma"], 4.5, detrend)
    if detrend:
        u = (2 * np.arange(T) - (T - 1)).astype(np.float64)
        marg = p["Y"] - (m_o[:, None] + st["beta"][:, None] * u[None, :]) - 4.5 * st["sigma"][:, None]
    else:
        marg = p["Y"] - m_o[:, None] - 4.5 * st["sigma"][:, None]
    band = np.abs(marg) <= 2 * bound + 1e-5 * st["sigma"][:, None] * 5.5
    assert np.array_equal(hit & ~band, mine & ~band)
    assert band.sum() <= max(5, 1e-4 * hit.size)


def test_post_fullsize_stream_f32():
    """The benchmark's block (1024 channels, 640 DMs, 2^17 samples) with a
    5-wide median and detrending: the filtered series is exactly the median
    of the GPU's series, the line and deviation match the oracle's on it, and
    the candidates are exactly the binary64 decisions on it."""
    nchan, B, dms = 1024, 1 << 17, np.arange(640) * 0.2
    od, dmax = O.delay_table(nchan, F_LO, BW, TS, dms)
    x = synth.noise(nchan, B + dmax, 990)
    synth.add_pulse(x, od[300].astype(np.float64) + 70000, 20.0, 0.5)
    x += (np.linspace(-1.0, 1.0, B + dmax, dtype=np.float32) * 0.3)[None, :]
    g = GpuBeam(nchan, F_LO, BW, TS, dms, "f32", nsigma=5.0, cap=1 << 21)
    try:
        tp.tp_plan_set_postprocess(g.plan, 5, True)
        r = g.run(x)
        Y = tp.tp_get_processed_series(g.e, g.beam, ndm=len(dms))
        mean, beta, sig = tp.tp_get_detrend(g.e, g.beam, len(dms))
    finally:
        g.close()
    D = r["D"].astype(np.float64)
    assert np.array_equal(Y.astype(np.float64), O.median_filter(D, 5))
    st = O.detrend(Y.astype(np.float64))
    np.testing.assert_allclose(mean, st["mean"], rtol=0, atol=1e-7 * st["sigma"].max())
    np.testing.assert_allclose(sig, st["sigma"], rtol=1e-6)
    np.testing.assert_allclose(beta * (B - 1), st["beta"] * (B - 1), rtol=0, atol=1e-6 * st["sigma"].max())
    hit = _decide(Y, mean, beta, sig, 5.0, True)
    assert r["n_candidates"] == int(hit.sum()) > 0
    c = r["candidates"]
    assert np.all(hit[c["dm_idx"], c["t_abs"] - r["info"]["t0_abs"]])


def test_postprocess_arguments():
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, 64, F_LO, BW, TS, np.arange(8) * 1.0, "f32", None, 5.0)
        for bad in (0, 2, 11, -1):
            with pytest.raises(tp.TpError):
                tp.tp_plan_set_postprocess(p, bad, False)
        tp.tp_plan_set_postprocess(p, 9, True)
        b = tp.tp_beam_open(e, p, 4000, 1024)
        with pytest.raises(tp.TpError) as ei:
            tp.tp_plan_set_postprocess(p, 3, False)
        assert ei.value.code == tp.TP_EBUSY
        with pytest.raises(tp.TpError):  # no detected block yet
            tp.tp_get_detrend(e, b, 8)
        tp.tp_beam_close(e, b)
        tp.tp_plan_set_postprocess(p, 1, False)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)

"""Full-size checks in the launch configuration the benchmark times: the
1024-channel / 640-DM / 2^17-sample FP32 stream (second block, with the
overlap tail carried on the device) under every kernel shape the plan admits,
and the 4096-channel / 2048-DM / 2^18-sample 8-bit wide-band block.  The
oracle computes the statistics and masks of the whole window, D at sampled
points one by one, and complete D rows (with their detections) for 18 DM
trials spread over the range, first and last included; series statistics
and the full candidate list are also checked through properties that hold
at any size."""
import os

import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _sample_points(ndm, T, n, seed):
    g = synth.rng(seed)
    d = np.concatenate([[0, 0, ndm - 1, ndm - 1], g.integers(0, ndm, n)]).astype(np.int32)
    t = np.concatenate([[0, T - 1, 0, T - 1], g.integers(0, T, n)]).astype(np.int64)
    return d, t


def _check_candidates(D, cands, n_total, row_mu, row_sigma, nsigma, t0):
    """Every record is a detection of the series it came from, in (d, t)
    order, and the count equals the number of detections in D."""
    Dd = D.astype(np.float64)
    thr = row_mu + nsigma * row_sigma
    hits = (Dd - row_mu[:, None]) >= nsigma * row_sigma[:, None]
    assert int(hits.sum()) == n_total
    keys = np.stack([cands["dm_idx"].astype(np.int64), cands["t_abs"]], axis=1)
    assert np.all(np.diff(keys[:, 0] * (1 << 40) + keys[:, 1]) > 0)
    d = cands["dm_idx"]
    t = cands["t_abs"] - t0
    assert np.all(hits[d, t])
    assert np.all(cands["value"] == D[d, t].astype(np.float32))
    assert np.all(Dd[d, t] >= thr[d] - 1e-9 * np.abs(thr[d]))


def _oracle_rows(window, dtype, st, cf, sf, W, od, sel, T):
    """Complete oracle rows D[sel[i]][0..T) (binary64 or exact integers), the
    magnitude sum_c |y| of every element (float data), and the oracle's
    candidates of those rows (Sec. 2.3 on each row's own statistics)."""
    D = O.dedisperse(window, dtype, st, cf, sf, W, od[sel], T)
    mass = None
    if dtype != "u8":
        ya = np.abs(O.corrected(window, dtype, st, cf, sf, W))
        mass = np.zeros((len(sel), T))
        for i, d in enumerate(sel):
            for c in range(window.shape[0]):
                o = int(od[d, c])
                mass[i] += ya[c, o:o + T]
    ss = O.series_stats(D)
    cands, _ = O.candidates(D, ss["mu"], ss["sigma"], 5.0)
    return D, mass, ss, cands


def _check_rows(Dg, sel, Do, mass, ss, ocands, gcands, t0, exact):
    """The GPU's rows equal the oracle's (bit-exact for integers, within
    TOL * sum|y| for floats) and so do its detections in those rows (floats:
    outside the band where the oracle's statistic lies within the series and
    statistics bounds of its threshold)."""
    got = Dg[sel].astype(np.float64 if not exact else np.int64)
    if exact:
        assert np.array_equal(got, Do.astype(np.int64))
    else:
        err = np.abs(got - Do)
        assert np.all(err <= TOL * mass), float((err / mass).max())
    want = {(int(sel[c["dm_idx"]]), int(c["t_abs"])) for c in ocands}
    rows = set(int(d) for d in sel)
    have = {(int(c["dm_idx"]), int(c["t_abs"]) - t0) for c in gcands if int(c["dm_idx"]) in rows}
    diff = want ^ have
    if exact:
        assert not diff, sorted(diff)[:5]
        return
    pos = {int(d): i for i, d in enumerate(sel)}
    for d, t in diff:
        i = pos[d]
        thr = ss["mu"][i] + 5.0 * ss["sigma"][i]
        band = TOL * mass[i, t] + 1e-5 * ss["sigma"][i]
        assert abs(Do[i, t] - thr) <= band, (d, t, Do[i, t], thr, band)


ROW_SEL_640 = np.unique(np.concatenate([np.linspace(0, 639, 16).astype(int), [1, 638]]))


def test_stream1024_640dm_f32_fullsize_all_shapes():
    tp.build()
    O.set_threads(os.cpu_count() or 1)
    nchan, B, dms = 1024, 1 << 17, np.arange(640) * 0.2
    f_lo, bw, ts = 398.0, 20.0, 51.2e-6
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    g = synth.rng(77)
    blocks = []
    for k in range(2):
        x = synth.noise(nchan, B, 770 + k)
        for _ in range(8):
            d = int(g.integers(25, 600))
            synth.add_pulse(x, od[d].astype(np.float64) + int(g.integers(0, B - dmax - 200)), 40.0,
                            float(g.uniform(8, 30)) / 32)
        synth.apply_bursts(x, synth.poisson_bursts(nchan, B, 780 + k))
        blocks.append(x)
    window = np.ascontiguousarray(np.concatenate([blocks[0][:, B - dmax:], blocks[1]], axis=1))
    rfi = O.RfiParams()
    st = O.bandpass(window, "f32")
    raw, cf = O.channel_mask(window, "f32", st, rfi)
    sf = O.spectrum_mask(window, "f32", st, rfi, cf)
    assert cf.any()
    dd, tt = _sample_points(len(dms), B, 3000, 5)
    want, mass = O.dedisperse_points(window, "f32", st, cf, sf, rfi.chunk_width, od, dd, tt)
    sel = ROW_SEL_640
    Drow, mrow, ssrow, crow = _oracle_rows(window, "f32", st, cf, sf, rfi.chunk_width, od, sel, B)
    assert len(crow) > 0

    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, nchan, f_lo, bw, ts, dms, "f32", tp.tp_rfi_defaults(), 5.0)
        b = tp.tp_beam_open(e, p, B, 1 << 21)
        tp.tp_push_block(e, b, blocks[0])
        tp.tp_dedisperse(e, b)
        tp.tp_detect(e, b)
        tp.tp_get_candidates(e, b, 0)
        tp.tp_push_block(e, b, blocks[1])
        tp.tp_dedisperse(e, b)
        best, ms = tp.tp_autotune(e, b, reps=1)
        _, feasible = tp.tp_plan_shapes(p)
        shapes = [s for s in np.nonzero(feasible)[0]]
        assert best in shapes and len(shapes) >= 2
        info = tp.tp_beam_info(e, b)
        assert info["nout"] == B and info["t0_abs"] == B - dmax
        for sh in shapes:
            tp.tp_plan_set_shape(p, int(sh))
            tp.tp_beam_rewind(e, b)  # the window is still the second block's
            tp.tp_dedisperse(e, b)
            cfg, crg, sfg = tp.tp_get_masks(e, b, nchan)
            assert np.array_equal(cfg, cf) and np.array_equal(crg, raw) and np.array_equal(sfg, sf)
            D = tp.tp_get_series(e, b, ndm=len(dms))
            got = D[dd, tt].astype(np.float64)
            err = np.abs(got - want)
            assert np.all(err <= TOL * mass), (sh, float((err / mass).max()))
            tp.tp_detect(e, b)
            cands, n, rc = tp.tp_get_candidates(e, b, 1 << 21)
            mu, sigma = tp.tp_get_series_stats(e, b, len(dms))
            Dd = D.astype(np.float64)
            np.testing.assert_allclose(mu, Dd.mean(axis=1), rtol=0, atol=1e-6 * np.abs(Dd).mean())
            np.testing.assert_allclose(sigma, Dd.std(axis=1), rtol=1e-5)
            _check_candidates(D, cands, n, mu, sigma, 5.0, info["t0_abs"])
            _check_rows(D, sel, Drow, mrow, ssrow, crow, cands, info["t0_abs"], exact=False)
        tp.tp_plan_set_shape(p, int(best))
        tp.tp_beam_close(e, b)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)


def test_wideband_4096ch_2048dm_u8_fullsize():
    tp.build()
    O.set_threads(os.cpu_count() or 1)
    nchan, B, dms = 4096, 1 << 18, np.arange(2048) * 1.0
    f_lo, bw, ts = 1200.0, 300.0, 64e-6
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    assert dmax == 33166
    g = synth.rng(55)
    xf = g.standard_normal((nchan, B + dmax), dtype=np.float32)
    for _ in range(6):
        d = int(g.integers(100, 2000))
        synth.add_pulse(xf, od[d].astype(np.float64) + int(g.integers(0, B - 2000)), 20.0, 25.0 / 64)
    bad = g.choice(nchan, nchan // 20, replace=False)          # 5 % of channels carry RFI
    for c in bad:
        t0 = int(g.integers(0, B))
        xf[c, t0:t0 + 4096] += 15.0
    x = synth.to_u8(xf * 16 + 128)
    rfi = O.RfiParams()
    st = O.bandpass(x, "u8")
    raw, cf = O.channel_mask(x, "u8", st, rfi)
    sf = O.spectrum_mask(x, "u8", st, rfi, cf)
    dd, tt = _sample_points(len(dms), B, 3000, 6)
    want, _ = O.dedisperse_points(x, "u8", st, cf, sf, rfi.chunk_width, od, dd, tt)
    sel = np.unique(np.concatenate([np.linspace(0, 2047, 16).astype(int), [1, 2046]]))
    Drow, _, ssrow, crow = _oracle_rows(x, "u8", st, cf, sf, rfi.chunk_width, od, sel, B)
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, nchan, f_lo, bw, ts, dms, "u8", tp.tp_rfi_defaults(), 5.0)
        assert np.array_equal(tp.tp_get_delay_table(p), od)
        b = tp.tp_beam_open(e, p, B + dmax, 1 << 21)
        tp.tp_push_block(e, b, x)
        tp.tp_dedisperse(e, b)
        best, ms = tp.tp_autotune(e, b, reps=1)
        tp.tp_dedisperse(e, b)
        tp.tp_detect(e, b)
        cfg, crg, sfg = tp.tp_get_masks(e, b, nchan)
        assert np.array_equal(cfg, cf) and np.array_equal(crg, raw) and np.array_equal(sfg, sf)
        assert cf[bad].any(axis=1).mean() > 0.9
        D = tp.tp_get_series(e, b, ndm=len(dms), is_int=True)
        assert np.array_equal(D[dd, tt].astype(np.int64), want)
        cands, n, rc = tp.tp_get_candidates(e, b, 1 << 21)
        mu, sigma = tp.tp_get_series_stats(e, b, len(dms))
        Di = D.astype(np.int64)
        T = Di.shape[1]
        s1, s2 = Di.sum(axis=1), (Di * Di).sum(axis=1)
        m = s1 / T
        assert np.array_equal(mu, m)                                    # exact integer sums
        assert np.array_equal(sigma, np.sqrt(np.maximum(s2 / T - m * m, 0.0)))
        _check_candidates(D, cands, n, mu, sigma, 5.0, 0)
        _check_rows(D, sel, Drow, None, ssrow, crow, cands, 0, exact=True)
        tp.tp_beam_close(e, b)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)

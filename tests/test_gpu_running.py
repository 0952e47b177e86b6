"""Running bandpass statistics across a stream's blocks (reading R15) on the
GPU against the oracle: each block's window (overlap tail + new samples) is
thresholded, substituted and dedispersed with the exponential average of the
blocks' means and variances, kept on the device between blocks.  alpha = 1
is bit-identical to per-block statistics, and processing a window again
(tp_beam_rewind) repeats the same update."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O
from tests.gpu_run import GpuBeam
from tests.test_gpu_parity import check_block

pytestmark = pytest.mark.gpu

NCHAN, B = 192, 6000
BAND = (398.0, 20.0, 51.2e-6)
DMS = np.arange(40) * 0.2


def _stream(dtype, n):
    od, dmax = O.delay_table(NCHAN, *BAND, DMS)
    g = synth.rng(4242)
    out = []
    for k in range(n):
        # a bandpass that drifts from block to block, so that the running
        # average differs from each block's own statistics
        x = synth.noise(NCHAN, B, 4300 + k, mean=0.3 * k, std=1.0 + 0.2 * k)
        synth.add_pulse(x, od[int(g.integers(10, 38))].astype(np.float64) + int(g.integers(200, B - 600)), 15.0,
                        12.0 / np.sqrt(NCHAN))
        synth.apply_bursts(x, synth.poisson_bursts(NCHAN, B, 4400 + k, rate_per_sample=1 / 2000.0))
        out.append(synth.to_u8(x * 16 + 128) if dtype == "u8" else x)
    return out, od, dmax


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_running_stats_match_oracle_over_a_stream(dtype):
    tp.build()
    blocks, od, dmax = _stream(dtype, 4)
    rfi = O.RfiParams()
    alpha = 0.25
    g = GpuBeam(NCHAN, *BAND, DMS, dtype, rfi=rfi, nsigma=5.0, cap=1 << 16)
    try:
        tp.tp_plan_set_running_stats(g.plan, alpha)
        state, win = None, None
        for k, x in enumerate(blocks):
            win = x if win is None else np.ascontiguousarray(np.concatenate([win[:, -dmax:], x], axis=1))
            state, st = O.running_stats(state, win, dtype, alpha)
            res = g.run(x)
            t0 = res["info"]["t0_abs"]
            o = O.search_block(win, dtype, od, dmax, rfi=rfi, nsigma=5.0, stats=st, t0=t0)
            if k > 0:
                assert not np.allclose(st["mu"], O.bandpass(win, dtype)["mu"])
            check_block(res, o, win, dtype, od, rfi, 5.0, t0=t0)
            if k == 2:
                # the same window again: the same running values and results
                tp.tp_beam_rewind(g.e, g.beam)
                tp.tp_dedisperse(g.e, g.beam)
                tp.tp_detect(g.e, g.beam)
                mu2, sg2 = tp.tp_get_bandpass(g.e, g.beam, NCHAN)
                assert np.array_equal(mu2, res["mu"]) and np.array_equal(sg2, res["sigma"])
                D2 = tp.tp_get_series(g.e, g.beam, ndm=len(DMS), is_int=dtype == "u8")
                assert np.array_equal(D2, res["D"])
    finally:
        g.close()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_running_stats_alpha_one_is_per_block(dtype):
    tp.build()
    blocks, od, dmax = _stream(dtype, 3)
    rfi = O.RfiParams()
    a = GpuBeam(NCHAN, *BAND, DMS, dtype, rfi=rfi, nsigma=5.0, cap=1 << 16)
    b = GpuBeam(NCHAN, *BAND, DMS, dtype, rfi=rfi, nsigma=5.0, cap=1 << 16)
    try:
        tp.tp_plan_set_running_stats(b.plan, 1.0)
        for x in blocks:
            ra, rb = a.run(x), b.run(x)
            for key in ("mu", "sigma", "chunk_flag", "spec_flag", "D", "row_mu", "row_sigma"):
                assert np.array_equal(ra[key], rb[key]), key
            assert np.array_equal(ra["candidates"], rb["candidates"])
    finally:
        a.close()
        b.close()


def test_running_stats_rejects_bad_settings():
    tp.build()
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, "f32", None, 5.0)
        for bad in (0.0, -0.5, 1.5, float("nan")):
            with pytest.raises(tp.TpError) as err:
                tp.tp_plan_set_running_stats(p, bad)
            assert err.value.code == tp.TP_EINVAL
        tp.tp_plan_set_bandpass_fit(p, 2, 5.0)
        with pytest.raises(tp.TpError):
            tp.tp_plan_set_running_stats(p, 0.5)
        tp.tp_plan_set_bandpass_fit(p, -1, 5.0)
        tp.tp_plan_set_running_stats(p, 0.5)
        with pytest.raises(tp.TpError):
            tp.tp_plan_set_bandpass_fit(p, 2, 5.0)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)

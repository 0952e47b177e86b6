"""The fitted bandpass of Sec. 2.2.1 ("Bandpass Correction", reading R13)
through the C ABI against the oracle: the channels masked before the fit, the
fit and its RMSE, then the whole block (masks identical, 8-bit series exact,
float series within the dedispersion bound, candidates as in the other parity
tests)."""
import os

import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O
from tests.gpu_run import GpuBeam
from tests.test_gpu_parity import check_block

pytestmark = pytest.mark.gpu

NCHAN, F_LO, BW, TS = 192, 398.0, 20.0, 51.2e-6


@pytest.fixture(scope="module", autouse=True)
def _setup():
    tp.build()
    O.set_threads(os.cpu_count() or 1)


def _block(dtype, nsamp, od, seed):
    x = synth.noise(NCHAN, nsamp, seed)
    x += (3.0 + 1.5 * np.linspace(-1, 1, NCHAN) ** 2 - 0.5 * np.linspace(-1, 1, NCHAN) ** 3)[:, None].astype(
        np.float32)
    x[40] += 6.0                                        # a high-power channel
    x[150:152] += 4.0                                   # two adjacent ones
    synth.add_narrowband(x, [90, 91], 2000, 2600, 6.0)  # a burst
    synth.add_broadband(x, [5000], 3.0)
    synth.add_pulse(x, od[30].astype(np.float64) + 3500, 15.0, 1.5)
    if dtype == "u8":
        return synth.to_u8(x * 16.0 + 40.0)
    if dtype == "f16":
        return synth.to_f16(x)
    return x


@pytest.mark.parametrize("dtype,order", [("f32", 2), ("u8", 3), ("f16", 4), ("f32", 0)])
def test_fitted_bandpass_block(dtype, order):
    dms = np.arange(48) * 0.5
    od, dmax = O.delay_table(NCHAN, F_LO, BW, TS, dms)
    nsamp = 7001
    x = _block(dtype, nsamp, od, 4100 + order)
    rfi = O.RfiParams(tau_channel=40.0)
    o = O.search_block(x, dtype, od, dmax, rfi=rfi, nsigma=5.0, fit=(order, 5.0))
    fit = o["stats"]["fit"]
    assert fit["masked"].sum() >= 3
    if order > 0:  # (a constant cannot follow the curved bandpass: its RMSE hides the RFI)
        assert o["chunk_flag"].any()
    g = GpuBeam(NCHAN, F_LO, BW, TS, dms, dtype, rfi=rfi, nsigma=5.0, cap=1 << 18)
    try:
        tp.tp_plan_set_bandpass_fit(g.plan, order, 5.0)
        r = g.run(x)
        bfit, masked, rmse = tp.tp_get_bandpass_fit(g.e, g.beam, NCHAN)
    finally:
        g.close()
    assert np.array_equal(masked, fit["masked"])
    scale = np.abs(fit["b"]).max()
    assert np.abs(bfit - fit["b"]).max() <= 1e-10 * scale
    assert abs(rmse - fit["rmse"]) <= 1e-8 * fit["rmse"] + 1e-12 * scale
    check_block(r, o, x, dtype, od, rfi, 5.0)


def test_fit_arguments():
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, 64, F_LO, BW, TS, np.arange(8) * 1.0, "f32", None, 5.0)
        for order, tau in ((9, 5.0), (-2, 5.0), (2, 0.0), (2, float("nan"))):
            with pytest.raises(tp.TpError):
                tp.tp_plan_set_bandpass_fit(p, order, tau)
        tp.tp_plan_set_bandpass_fit(p, 3, 5.0)
        b = tp.tp_beam_open(e, p, 4000, 1024)
        with pytest.raises(tp.TpError) as ei:
            tp.tp_plan_set_bandpass_fit(p, -1, 5.0)
        assert ei.value.code == tp.TP_EBUSY
        tp.tp_beam_close(e, b)
        tp.tp_plan_set_bandpass_fit(p, -1, 5.0)
        tp.tp_plan_destroy(p)
        rp = tp.tp_rfi_defaults()
        rp.stats_mode = tp.TP_STATS_EXTERNAL
        p2 = tp.tp_create_plan(e, 64, F_LO, BW, TS, np.arange(8) * 1.0, "f32", rp, 5.0)
        with pytest.raises(tp.TpError):
            tp.tp_plan_set_bandpass_fit(p2, 2, 5.0)
        tp.tp_plan_destroy(p2)
    finally:
        tp.tp_engine_destroy(e)

"""Clustering and classification of detections on the device (Sec. 2.3,
reading R14) against the oracle run on the same detection records: cluster
labels identical, every cluster's integer fields, largest SNR and width
identical, its RMSE within float rounding, and its classification identical
(the records themselves are checked against the oracle by the other parity
tests)."""
import os

import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O
from tests.gpu_run import GpuBeam

pytestmark = pytest.mark.gpu

F_LO, BW, TS = 398.0, 20.0, 51.2e-6


@pytest.fixture(scope="module", autouse=True)
def _setup():
    tp.build()
    O.set_threads(os.cpu_count() or 1)


def _run(x, dtype, nchan, dms, prm, nsigma, rfi):
    g = GpuBeam(nchan, F_LO, BW, TS, dms, dtype, rfi=rfi, nsigma=nsigma, cap=1 << 18)
    try:
        tp.tp_plan_set_clustering(g.plan, prm.t_eps, prm.dm_eps, prm.snr_eps, prm.min_pts, prm.smooth, prm.rmse_max,
                                  prm.dm_min)
        r = g.run(x, fetch=False)
        labels = tp.tp_get_candidate_labels(g.e, g.beam)
        cl, ncl, trunc = tp.tp_get_clusters(g.e, g.beam)
    finally:
        g.close()
    return r, labels, cl, ncl, trunc


def _compare(r, labels, cl, ncl, dms, prm):
    c = r["candidates"]
    assert r["n_candidates"] == len(c) == len(labels)
    want, _ = O.dbscan(c["dm_idx"], c["t_abs"], c["snr"], prm)
    assert np.array_equal(labels, want)
    ref = O.classify(c["dm_idx"], c["t_abs"], c["snr"], want, dms, TS, BW, (F_LO + BW / 2) / 1e3, prm)
    assert ncl == len(ref) == len(cl)
    for g, o in zip(cl, ref):
        assert g["label"] == o["cluster"]
        for f in ("n", "d_lo", "d_hi", "d_star", "t_first", "t_last"):
            assert int(g[f]) == o[f], (f, g, o)
        assert g["snr_max"] == np.float32(o["snr_max"])
        assert g["width_ms"] == np.float32(o["width_ms"])
        assert abs(float(g["rmse"]) - o["rmse"]) <= 1e-6 * max(1.0, o["rmse"])
        if abs(o["rmse"] - prm.rmse_max) > 1e-9:
            assert bool(g["flags"] & 1) == o["candidate"], (g, o)
        assert bool(g["flags"] & 2) == o["broadband"]
    return ref


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_pulse_and_rfi_clusters(dtype):
    nchan, nsamp = 256, 16000
    dms = np.arange(80) * 0.5
    od, dmax = O.delay_table(nchan, F_LO, BW, TS, dms)
    x = synth.noise(nchan, nsamp, 5)
    synth.add_pulse(x, od[50].astype(np.float64) + 7000, 19.5, 25.0 / np.sqrt(nchan))
    synth.add_broadband(x, list(range(3000, 3008)), 3.0)
    x[100, 11000:11060] += 150.0
    if dtype == "u8":
        x = synth.to_u8(x * 2.0 + 100.0)
    rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
    prm = O.ClusterParams()
    r, labels, cl, ncl, trunc = _run(x, dtype, nchan, dms, prm, 5.0, rfi)
    assert not trunc
    ref = _compare(r, labels, cl, ncl, dms, prm)
    pulse = [k for k in ref if k["t_first"] <= 7000 <= k["t_last"] and k["d_lo"] > 20]
    assert len(pulse) == 1 and abs(pulse[0]["d_star"] - 50) <= 4


def test_many_small_clusters():
    """A noisy block detected at a low threshold: thousands of detections in
    many small clusters and noise points."""
    nchan, nsamp = 128, 20000
    dms = np.arange(40) * 1.0
    od, dmax = O.delay_table(nchan, F_LO, BW, TS, dms)
    x = synth.noise(nchan, nsamp, 77)
    for k in range(6):
        synth.add_pulse(x, od[5 + 6 * k].astype(np.float64) + 2500 + 2700 * k, 10.0 + 5 * k, 0.9)
    rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
    prm = O.ClusterParams(t_eps=4, dm_eps=1, snr_eps=2.0, min_pts=3, smooth=5, rmse_max=0.3)
    r, labels, cl, ncl, trunc = _run(x, "f32", nchan, dms, prm, 3.2, rfi)
    assert r["n_candidates"] > 1000 and ncl > 15 and (labels < 0).sum() > 100
    _compare(r, labels, cl, ncl, dms, prm)


def test_wide_cluster():
    """A strong pulse over 400 fine DM trials: one cluster spans more trials
    (263) than a classification CTA has threads."""
    nchan, nsamp = 256, 16000
    dms = np.arange(400) * 0.1
    od, dmax = O.delay_table(nchan, F_LO, BW, TS, dms)
    x = synth.noise(nchan, nsamp, 9)
    synth.add_pulse(x, od[200].astype(np.float64) + 6000, 20.0, 120.0 / np.sqrt(nchan))
    rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
    prm = O.ClusterParams()
    r, labels, cl, ncl, trunc = _run(x, "f32", nchan, dms, prm, 5.0, rfi)
    ref = _compare(r, labels, cl, ncl, dms, prm)
    assert max(k["d_hi"] - k["d_lo"] + 1 for k in ref) > 256


def test_clustering_arguments():
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, 64, F_LO, BW, TS, np.arange(8) * 1.0, "f32", None, 5.0)
        for bad in (dict(t_eps=-1), dict(min_pts=0), dict(smooth=2), dict(snr_eps=float("nan"))):
            with pytest.raises(tp.TpError):
                tp.tp_plan_set_clustering(p, **bad)
        big = tp.tp_create_plan(e, 64, F_LO, BW, TS, np.arange(14337) * 0.01, "f32", None, 5.0)
        with pytest.raises(tp.TpError):  # more DM trials than the classification holds
            tp.tp_plan_set_clustering(big)
        tp.tp_plan_destroy(big)
        b = tp.tp_beam_open(e, p, 4000, 1024)
        with pytest.raises(tp.TpError) as ei:
            tp.tp_plan_set_clustering(p)
        assert ei.value.code == tp.TP_EBUSY
        with pytest.raises(tp.TpError):  # the plan does not cluster
            tp.tp_get_clusters(e, b)
        tp.tp_beam_close(e, b)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)

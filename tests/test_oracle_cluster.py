"""Pins of the oracle's clustering and classification of detections (Sec. 2.3,
reading R14): DBSCAN on hand-made point sets and against the connected
components of the core graph computed by a graph library, the Eq. 3-4 model
against its closed form, and the classification of a dispersed pulse, a
broadband spike and a narrowband burst."""
from math import erf, pi, sqrt

import numpy as np
import pytest

import synth
from oracle import oracle as O


def test_dbscan_hand_cases():
    p = O.ClusterParams(t_eps=2, dm_eps=1, snr_eps=5.0, min_pts=3)
    d = np.array([0, 0, 1, 1, 10, 10, 11, 30])
    t = np.array([5, 6, 5, 7, 100, 101, 100, 500])
    s = np.array([6, 7, 6, 8, 6, 6, 7, 9.0])
    lab, core = O.dbscan(d, t, s, p)
    assert lab.tolist() == [0, 0, 0, 0, 1, 1, 1, -1]
    # extents are inclusive; MinPts counts the point itself
    lab, core = O.dbscan([0, 1, 2], [0, 2, 4], [5, 5, 5.0], O.ClusterParams(t_eps=2, dm_eps=1, snr_eps=0.0,
                                                                             min_pts=3))
    assert core.tolist() == [False, True, False] and lab.tolist() == [0, 0, 0]
    lab, core = O.dbscan([0, 1, 2], [0, 2, 4], [5, 5, 5.0], O.ClusterParams(t_eps=1, dm_eps=1, snr_eps=0.0,
                                                                             min_pts=3))
    assert lab.tolist() == [-1, -1, -1]
    # the SNR extent separates points close in (t, DM)
    lab, _ = O.dbscan([0, 0, 0, 0], [0, 1, 2, 3], [6, 6.5, 20, 20.5], O.ClusterParams(t_eps=3, dm_eps=0,
                                                                                      snr_eps=2.0, min_pts=2))
    assert lab.tolist() == [0, 0, 1, 1]


def test_dbscan_border_and_noise_points():
    """Points within reach of a core point but not core themselves join its
    cluster; an isolated point is noise (the lowest-index rule for border
    points within reach of several clusters is checked on random sets
    against the graph library below)."""
    p = O.ClusterParams(t_eps=1, dm_eps=0, snr_eps=100.0, min_pts=3)
    d = np.zeros(7, int)
    s = np.full(7, 6.0)
    t = np.array([0, 1, 2, 4, 6, 7, 8])
    lab, core = O.dbscan(d, t, s, p)
    assert core.tolist() == [False, True, False, False, False, True, False]
    assert lab.tolist() == [0, 0, 0, -1, 1, 1, 1]


def test_dbscan_equals_core_graph_components():
    nx = pytest.importorskip("networkx")
    g = np.random.default_rng(2)
    n = 400
    d = g.integers(0, 20, n)
    t = g.integers(0, 300, n)
    s = g.uniform(5, 15, n)
    p = O.ClusterParams(t_eps=6, dm_eps=2, snr_eps=4.0, min_pts=4)
    lab, core = O.dbscan(d, t, s, p)
    nb = lambda a, b: abs(d[a] - d[b]) <= 2 and abs(t[a] - t[b]) <= 6 and abs(s[a] - s[b]) <= 4.0
    G = nx.Graph()
    cores = [i for i in range(n) if core[i]]
    G.add_nodes_from(cores)
    for i in cores:
        for j in cores:
            if i < j and nb(i, j):
                G.add_edge(i, j)
    comps = sorted((sorted(c) for c in nx.connected_components(G)), key=lambda c: c[0])
    assert int(lab.max()) + 1 == len(comps)
    for k, comp in enumerate(comps):
        assert set(np.nonzero((lab == k) & core)[0]) == set(comp)
    for i in range(n):
        if not core[i]:
            cn = [j for j in cores if nb(i, j)]
            assert lab[i] == (lab[min(cn)] if cn else -1)


def test_eq3_model_closed_form():
    assert O.eq3_ratio(0.0, 1.0, 20.0, 0.408) == 1.0
    # zeta = 1: (sqrt(pi)/2) erf(1)
    f = 0.408
    ddm = 1.0 * f ** 3 / (6.91e-3 * 20.0)
    assert abs(O.eq3_ratio(ddm, 1.0, 20.0, f) - sqrt(pi) / 2 * erf(1.0)) < 1e-15
    vals = [O.eq3_ratio(x, 1.0, 20.0, f) for x in np.linspace(0, 10, 50)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    assert O.eq3_ratio(-2.5, 1.0, 20.0, f) == O.eq3_ratio(2.5, 1.0, 20.0, f)


def test_classification_of_pulse_and_rfi():
    nchan, nsamp = 256, 16000
    dms = np.arange(80) * 0.5
    f_lo, bw, ts = 398.0, 20.0, 51.2e-6
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    x = synth.noise(nchan, nsamp, 5)
    synth.add_pulse(x, od[50].astype(np.float64) + 7000, 19.5, 25.0 / np.sqrt(nchan))
    synth.add_broadband(x, list(range(3000, 3008)), 3.0)
    x[100, 11000:11060] += 150.0
    rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
    o = O.search_block(x, "f32", od, dmax, rfi=rfi, nsigma=5.0)
    c = o["candidates"]
    p = O.ClusterParams()
    lab, core = O.dbscan(c["dm_idx"], c["t_abs"], c["snr"], p)
    cl = O.classify(c["dm_idx"], c["t_abs"], c["snr"], lab, dms, ts, bw, (f_lo + bw / 2) / 1e3, p)
    pulse = [r for r in cl if r["t_first"] <= 7000 <= r["t_last"] and r["d_lo"] > 20]
    assert len(pulse) == 1 and pulse[0]["candidate"] and abs(pulse[0]["d_star"] - 50) <= 4
    spike = [r for r in cl if r["d_hi"] == 0]
    assert len(spike) == 1 and spike[0]["broadband"] and not spike[0]["candidate"]
    burst = [r for r in cl if r["t_last"] >= 11000 and r["d_hi"] - r["d_lo"] > 40]
    assert len(burst) == 1 and burst[0]["rmse"] > 0.6 and not burst[0]["candidate"]


def test_classification_hand_worked_fixture():
    """Every classification product of two small clusters against the values
    worked out by hand in tests/golden/classify_two_clusters.txt (Sec. 2.3,
    steps 1-8, Eq. 3-4): the signature's largest SNR per trial, the 3-trial
    average with its shortened end windows, d* by detection count (not by
    SNR), the width at d*, the RMSE over the cluster's trial range and the
    broadband / candidate decisions."""
    from tests.golden_io import load
    g = load("classify_two_clusters.txt")
    m = g["meta"]
    pts = g["points"]
    d, t, snr, lab = pts[:, 0].astype(np.int64), pts[:, 1].astype(np.int64), pts[:, 2], pts[:, 3].astype(np.int64)
    dms = np.arange(int(m["ndm"])) * float(m["dm_step"])
    p = O.ClusterParams(smooth=int(m["smooth"]), dm_min=float(m["dm_min"]), rmse_max=float(m["rmse_max"]))
    cl = O.classify(d, t, snr, lab, dms, float(m["t_samp"]), float(m["bw_mhz"]), float(m["f_ghz"]), p)
    assert len(cl) == len(g["expected"])
    for r, e in zip(cl, g["expected"]):
        assert r["cluster"] == int(e[0]) and r["n"] == int(e[1])
        assert (r["d_lo"], r["d_hi"], r["d_star"]) == (int(e[2]), int(e[3]), int(e[4]))
        assert r["snr_max"] == e[5] and (r["t_first"], r["t_last"]) == (int(e[6]), int(e[7]))
        assert abs(r["width_ms"] - e[8]) < 1e-12
        assert abs(r["rmse"] - e[9]) < 1e-11, (r["rmse"], e[9])
        assert r["broadband"] == bool(e[10]) and r["candidate"] == bool(e[11])

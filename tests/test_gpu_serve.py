"""Serving loop: streams of different channel counts, DM ranges and block
lengths, Poisson arrivals, admission by HBM budget, continuous batching.
Every block's candidates equal those of the same stream run alone."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth

pytestmark = pytest.mark.gpu

STREAMS = [  # (nchan, block, ndm, dm step)
    (256, 6000, 48, 0.5),
    (512, 8192, 64, 0.4),
    (1024, 5000, 32, 1.0),
    (256, 9000, 24, 2.0),
    (512, 6000, 40, 0.5),
    (1024, 7000, 56, 0.2),
]


def _blocks(i, nchan, B, nblk):
    out = []
    for k in range(nblk):
        xf = synth.noise(nchan, B, 4000 + 10 * i + k, mean=128.0, std=16.0)
        synth.add_narrowband(xf, [nchan // 3], 100, 900, 200.0)
        synth.add_broadband(xf, [B // 2], 60.0)
        out.append(synth.to_u8(xf))
    return out


def _solo(nchan, B, dms, blocks):
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, nchan, 398.0, 20.0, 51.2e-6, dms, "u8", None, 4.0)
        b = tp.tp_beam_open(e, p, B, 1 << 16)
        out = []
        for x in blocks:
            tp.tp_push_block(e, b, x)
            tp.tp_dedisperse(e, b)
            tp.tp_detect(e, b)
            c, n, rc = tp.tp_get_candidates(e, b, 1 << 16)
            out.append(c.copy())
        tp.tp_beam_close(e, b)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)
    return out


def test_serving_mix_equals_solo_and_admission_waits():
    import torch
    tp.build()
    nblk = 3
    data = [_blocks(i, nc, B, nblk) for i, (nc, B, nd, st) in enumerate(STREAMS)]
    dms = [np.arange(nd) * st for (nc, B, nd, st) in STREAMS]
    # budget: the three largest streams fit together, all six do not
    probe = tp.tp_engine_create(0)
    foot = []
    for (nc, B, nd, st), dm in zip(STREAMS, dms):
        p = tp.tp_create_plan(probe, nc, 398.0, 20.0, 51.2e-6, dm, "u8", None, 4.0)
        foot.append(tp.tp_beam_footprint(p, B, 1 << 16))
        tp.tp_plan_destroy(p)
    tp.tp_engine_destroy(probe)
    budget = sum(sorted(foot)[-3:]) + (4 << 20)  # + the delay tables of the plans
    assert budget < sum(foot)
    stream = torch.cuda.Stream()
    e = tp.tp_engine_create(0, budget, stream.cuda_stream)
    try:
        srv = tp.tp_server_create(e, nsigma=4.0, keep_candidates=True)
        g = synth.rng(7)
        rids = {}
        for i, (nc, B, nd, st) in enumerate(STREAMS):
            sid = tp.tp_server_add_stream(srv, nc, 398.0, 20.0, 51.2e-6, dms[i], "u8", B, 1 << 16)
            t = float(g.exponential(0.01))
            for k in range(nblk):
                rids[(i, k)] = tp.tp_server_submit(srv, sid, data[i][k], t)
                t += float(g.exponential(0.01))
            tp.tp_server_end_stream(srv, sid)
        tp.tp_server_run(srv, time_limit_s=600.0)
        res = tp.tp_server_results(srv)
        assert len(res) == len(STREAMS) * nblk
        assert np.all(res["done_s"] >= res["start_s"]) and np.all(res["start_s"] >= res["arrival_s"])
        # admission made some stream wait for another to end
        first_start = [res[res["stream"] == i]["start_s"].min() for i in range(len(STREAMS))]
        last_done = [res[res["stream"] == i]["done_s"].max() for i in range(len(STREAMS))]
        assert any(fs > min(last_done) for fs in first_start)
        # blocks of a stream run in order
        for i in range(len(STREAMS)):
            r = np.sort(res[res["stream"] == i], order="seq")
            assert np.all(np.diff(r["start_s"]) >= 0)
        mix = {key: tp.tp_server_candidates(srv, rid) for key, rid in rids.items()}
        used, _ = tp.tp_engine_memory(e)
        tp.tp_server_destroy(srv)
    finally:
        tp.tp_engine_destroy(e)
    for i, (nc, B, nd, st) in enumerate(STREAMS):
        solo = _solo(nc, B, dms[i], data[i])
        for k in range(nblk):
            a, b = solo[k], mix[(i, k)]
            assert len(a) > 0
            assert np.array_equal(a["dm_idx"], b["dm_idx"]) and np.array_equal(a["t_abs"], b["t_abs"])
            assert np.array_equal(a["snr"], b["snr"]) and np.array_equal(a["value"], b["value"])
            assert np.all(b["beam"] == b["beam"][0])

"""Several beams of different plans in one batched launch (and through a
cached CUDA graph) give exactly the results of their solo runs, block after
block, whatever the grid that drains the batch's work items; one beam is
also checked against the oracle."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

NCHAN, F_LO, BW, TS = 256, 398.0, 20.0, 51.2e-6
PLANS = [np.arange(40) * 0.4, np.arange(80) * 0.2, np.arange(120) * 0.2, np.arange(24) * 1.0]


def _blocks(dtype, seed, nblk, B):
    out = []
    for k in range(nblk):
        x = synth.noise(NCHAN, B, seed + k)
        synth.add_narrowband(x, [7, 8], 1000, 1600, 9.0)
        synth.add_broadband(x, [2500], 7.0)
        if dtype == "f16":
            x = synth.to_f16(x)
        elif dtype == "u8":
            x = synth.to_u8(x * 16 + 128)
        out.append(x)
    return out


def _run(mode, dtype, blocks_per_beam, B, stream=None, grid=None):
    """mode: 'solo' (per-beam calls), 'batch' (beam = -1), 'graph'; grid:
    the batched launch's CTA count (None: the default persistent grid)."""
    e = tp.tp_engine_create(0, 0, stream)
    res = []
    try:
        if grid is not None:
            tp.tp_engine_set_batch_grid(e, grid)
        plans = [tp.tp_create_plan(e, NCHAN, F_LO, BW, TS, dms, dtype, None, 4.0) for dms in PLANS]
        beams = [tp.tp_beam_open(e, p, B, 1 << 16) for p in plans]
        nblk = len(blocks_per_beam[0])
        for k in range(nblk):
            for b, blocks in zip(beams, blocks_per_beam):
                tp.tp_push_block(e, b, blocks[k])
            if mode == "solo":
                for b in beams:
                    tp.tp_dedisperse(e, b)
                    tp.tp_detect(e, b)
            elif mode == "batch":
                tp.tp_dedisperse(e, -1)
                tp.tp_detect(e, -1)
            else:
                assert tp.tp_run_ready(e, use_graph=True) == len(beams)
            step = []
            for b, dms in zip(beams, PLANS):
                c, n, rc = tp.tp_get_candidates(e, b, 1 << 16)
                D = tp.tp_get_series(e, b, ndm=len(dms), is_int=dtype == "u8")
                step.append((c.copy(), D))
            res.append(step)
        for b in beams:
            tp.tp_beam_close(e, b)
        for p in plans:
            tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)
    return res


@pytest.mark.parametrize("dtype", ["f16", "u8", "f32"])
def test_batch_and_graph_equal_solo(dtype):
    import torch
    tp.build()
    B = 6000
    blocks = [_blocks(dtype, 100 * (i + 1), 3, B) for i in range(len(PLANS))]
    stream = torch.cuda.Stream()
    solo = _run("solo", dtype, blocks, B)
    batch = _run("batch", dtype, blocks, B)
    graph = _run("graph", dtype, blocks, B, stream=stream.cuda_stream)
    for k in range(3):
        for i in range(len(PLANS)):
            for other in (batch, graph):
                assert np.array_equal(solo[k][i][1], other[k][i][1]), (dtype, k, i)
                assert np.array_equal(solo[k][i][0], other[k][i][0]), (dtype, k, i)
    # beam 1, first block, against the oracle
    od, dmax = O.delay_table(NCHAN, F_LO, BW, TS, PLANS[1])
    o = O.search_block(blocks[1][0], dtype, od, dmax, nsigma=4.0)
    D = solo[0][1][1]
    if dtype == "u8":
        assert np.array_equal(D.astype(np.int64), o["D"])
    else:
        dd = np.repeat(np.arange(len(PLANS[1]), dtype=np.int32), o["T"])
        tt = np.tile(np.arange(o["T"], dtype=np.int64), len(PLANS[1]))
        _, mass = O.dedisperse_points(blocks[1][0], dtype, o["stats"], o["chunk_flag"], o["spec_flag"], 256,
                                      od, dd, tt)
        assert np.all(np.abs(D.astype(np.float64) - o["D"]).ravel() <= 1e-5 * mass)


@pytest.mark.parametrize("dtype", ["f32", "u8"])
@pytest.mark.parametrize("grid", [-1, 1, 7, 300])
def test_batched_grid_sizes_equal_solo(dtype, grid):
    """The batched kernel drains its work items with any grid: one CTA per
    item (-1), a single CTA taking every item (1), a few CTAs taking many
    items each (7), and more CTAs than items of the smaller beams (300);
    every beam's series and candidates equal its solo run exactly."""
    import torch
    tp.build()
    B = 6000
    blocks = [_blocks(dtype, 700 * (i + 1), 2, B) for i in range(len(PLANS))]
    solo = _run("solo", dtype, blocks, B)
    stream = torch.cuda.Stream()
    for mode in ("batch", "graph"):
        other = _run(mode, dtype, blocks, B, stream=stream.cuda_stream, grid=grid)
        for k in range(2):
            for i in range(len(PLANS)):
                assert np.array_equal(solo[k][i][1], other[k][i][1]), (mode, grid, k, i)
                assert np.array_equal(solo[k][i][0], other[k][i][0]), (mode, grid, k, i)


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_batch_autotune_keeps_results(dtype):
    """tp_autotune_batch picks for each plan a shape it admits (the heaviest
    plan's is returned); the batch run with them gives the solo series exactly
    (every shape adds each output's channels in index order, FP32 or exact
    integers) and the same candidates."""
    import torch
    tp.build()
    B = 6000
    blocks = [_blocks(dtype, 300 * (i + 1), 1, B) for i in range(len(PLANS))]
    solo = _run("solo", dtype, blocks, B)
    stream = torch.cuda.Stream()
    e = tp.tp_engine_create(0, 0, stream.cuda_stream)
    try:
        plans = [tp.tp_create_plan(e, NCHAN, F_LO, BW, TS, dms, dtype, None, 4.0) for dms in PLANS]
        beams = [tp.tp_beam_open(e, p, B, 1 << 16) for p in plans]
        for b, bl in zip(beams, blocks):
            tp.tp_push_block(e, b, bl[0])
        tp.tp_run_ready(e, use_graph=False)
        best, ms = tp.tp_autotune_batch(e, reps=1)
        work = [len(dms) for dms in PLANS]
        for p, w in zip(plans, work):
            cur, feas = tp.tp_plan_shapes(p)
            assert feas[cur]
            if w == max(work):
                assert cur == best
        assert tp.tp_run_ready(e, use_graph=True) == len(beams)
        for i, (b, dms) in enumerate(zip(beams, PLANS)):
            c, n, rc = tp.tp_get_candidates(e, b, 1 << 16)
            D = tp.tp_get_series(e, b, ndm=len(dms), is_int=dtype == "u8")
            assert np.array_equal(D, solo[0][i][1]), i
            # the row statistics sum per-time-tile partials, whose grouping
            # follows the shape's tile length: snr may differ in the last bits
            ref = solo[0][i][0]
            for f in ("beam", "dm_idx", "t_abs", "value"):
                assert np.array_equal(c[f], ref[f]), (i, f)
            np.testing.assert_allclose(c["snr"], ref["snr"], rtol=1e-6)
        for b in beams:
            tp.tp_beam_close(e, b)
        for p in plans:
            tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)

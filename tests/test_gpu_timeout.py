"""The dedispersion kernel's bounded waits report a timeout instead of
hanging: with the engine's wait limit at 0 every wait for staged data or a
free stage buffer gives up at once, each CTA lets its own copies in flight
land and leaves, and tp_get_candidates returns TP_ETIMEOUT.  The engine then
processes the next block normally, with results identical to an engine that
never timed out.  Covers the form with a producer warp, the rotating forms
(FP32 and 8-bit) and the threaded 8-bit form."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

NCHAN, NSAMP = 256, 16384
DMS = np.arange(48) * 0.2
BAND = (398.0, 20.0, 51.2e-6)


def _block(dtype, seed):
    od, _ = O.delay_table(NCHAN, *BAND, DMS)
    x = synth.noise(NCHAN, NSAMP, seed)
    synth.add_pulse(x, od[30].astype(np.float64) + 9000, 19.5, 15.0 / np.sqrt(NCHAN))
    return synth.to_u8(x * 16 + 128) if dtype == "u8" else x


def _run(e, b, x):
    tp.tp_beam_rewind(e, b) if x is None else tp.tp_push_block(e, b, x)
    tp.tp_dedisperse(e, b)
    tp.tp_detect(e, b)
    return tp.tp_get_candidates(e, b, 1 << 16)


@pytest.mark.parametrize("dtype,shapes", [("f32", (33, 53, 55)), ("u8", (57, 59))])
def test_zero_wait_limit_reports_timeout_and_engine_recovers(dtype, shapes):
    tp.build()
    blocks = [_block(dtype, 900 + k) for k in range(3)]
    e = tp.tp_engine_create(0)
    ref = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, dtype, None, 5.0)
        pr = tp.tp_create_plan(ref, NCHAN, *BAND, DMS, dtype, None, 5.0)
        _, feasible = tp.tp_plan_shapes(p)
        todo = [s for s in shapes if feasible[s]]
        assert todo, "none of the shapes is feasible on this plan"
        for sh in todo:
            tp.tp_plan_set_shape(p, sh)
            tp.tp_plan_set_shape(pr, sh)
            b = tp.tp_beam_open(e, p, NSAMP, 1 << 16)
            br = tp.tp_beam_open(ref, pr, NSAMP, 1 << 16)
            # a normal first block, so that the series the timed-out launch
            # leaves untouched hold finite values
            _run(e, b, blocks[0])
            _run(ref, br, blocks[0])
            tp.tp_engine_set_wait_limit(e, 0)
            with pytest.raises(tp.TpError) as err:
                _run(e, b, blocks[1])
            assert err.value.code == tp.TP_ETIMEOUT, (sh, err.value)
            tp.tp_engine_set_wait_limit(e, -1)
            # the same block again, now with the default limit: the results
            # match the engine that never timed out, bit for bit
            got, n, _ = _run(e, b, None)
            want, nw, _ = _run(ref, br, blocks[1])
            assert n == nw and np.array_equal(got, want), sh
            Dg = tp.tp_get_series(e, b, ndm=len(DMS), is_int=dtype == "u8")
            Dr = tp.tp_get_series(ref, br, ndm=len(DMS), is_int=dtype == "u8")
            assert np.array_equal(Dg, Dr), sh
            got, n, _ = _run(e, b, blocks[2])
            want, nw, _ = _run(ref, br, blocks[2])
            assert n == nw and np.array_equal(got, want), sh
            tp.tp_beam_close(e, b)
            tp.tp_beam_close(ref, br)
        tp.tp_plan_destroy(p)
        tp.tp_plan_destroy(pr)
    finally:
        tp.tp_engine_destroy(e)
        tp.tp_engine_destroy(ref)


@pytest.mark.parametrize("grid", [0, 3])
def test_timeout_in_a_persistent_batch_flags_every_beam(grid):
    """A batch drained by a persistent grid (0: the default, 3: three CTAs
    taking many items each) with the wait limit at 0: the CTAs give up on
    their first items and record TP_ETIMEOUT for the beams of every item they
    leave undone, so that each beam of the batch reports the timeout; the next
    batch with the default limit equals a batch that never timed out."""
    tp.build()
    import torch
    plans_dms = [DMS, np.arange(80) * 0.2, np.arange(24) * 1.0]
    blocks = [_block("f32", 950 + k) for k in range(3)]
    stream = torch.cuda.Stream()
    e = tp.tp_engine_create(0, 0, stream.cuda_stream)
    ref = tp.tp_engine_create(0, 0, stream.cuda_stream)
    try:
        tp.tp_engine_set_batch_grid(e, grid)
        ps = [tp.tp_create_plan(e, NCHAN, *BAND, d, "f32", None, 5.0) for d in plans_dms]
        pr = [tp.tp_create_plan(ref, NCHAN, *BAND, d, "f32", None, 5.0) for d in plans_dms]
        bs = [tp.tp_beam_open(e, p, NSAMP, 1 << 16) for p in ps]
        br = [tp.tp_beam_open(ref, p, NSAMP, 1 << 16) for p in pr]

        def batch(eng, beams, k):
            for b in beams:
                tp.tp_push_block(eng, b, blocks[k])
            tp.tp_run_ready(eng, use_graph=False)
            return [tp.tp_get_candidates(eng, b, 1 << 16) for b in beams]

        batch(e, bs, 0)
        batch(ref, br, 0)
        tp.tp_engine_set_wait_limit(e, 0)
        for b in bs:
            tp.tp_push_block(e, b, blocks[1])
        tp.tp_run_ready(e, use_graph=False)
        for b in bs:
            with pytest.raises(tp.TpError) as err:
                tp.tp_get_candidates(e, b, 1 << 16)
            assert err.value.code == tp.TP_ETIMEOUT
        tp.tp_engine_set_wait_limit(e, -1)
        for b in bs:
            tp.tp_beam_rewind(e, b)
        tp.tp_run_ready(e, use_graph=False)
        got = [tp.tp_get_candidates(e, b, 1 << 16) for b in bs]
        for b in br:
            tp.tp_push_block(ref, b, blocks[1])
        tp.tp_run_ready(ref, use_graph=False)
        want = [tp.tp_get_candidates(ref, b, 1 << 16) for b in br]
        for (cg, ng, _), (cw, nw, _) in zip(got, want):
            assert ng == nw and np.array_equal(cg, cw)
        for b in bs:
            tp.tp_beam_close(e, b)
        for b in br:
            tp.tp_beam_close(ref, b)
    finally:
        tp.tp_engine_destroy(e)
        tp.tp_engine_destroy(ref)

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

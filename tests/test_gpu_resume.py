"""Checkpoint and resume of a stream (tp_beam_export / tp_beam_import): the
state saved between blocks, loaded into a fresh beam of another engine,
continues the stream with series, statistics and candidates identical to the
stream that was never interrupted (per-block and running statistics)."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth

pytestmark = pytest.mark.gpu

NCHAN, B = 192, 5000
BAND = (398.0, 20.0, 51.2e-6)
DMS = np.arange(40) * 0.3


def _blocks(dtype, n):
    out = []
    for k in range(n):
        x = synth.noise(NCHAN, B, 6100 + k, mean=0.2 * k)
        synth.add_narrowband(x, [20, 21], 1000 + 200 * k, 1800 + 200 * k, 8.0)
        out.append(synth.to_u8(x * 16 + 128) if dtype == "u8" else x)
    return out


def _open(dtype, alpha):
    e = tp.tp_engine_create(0)
    p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, dtype, None, 4.0)
    if alpha < 1.0:
        tp.tp_plan_set_running_stats(p, alpha)
    b = tp.tp_beam_open(e, p, B, 1 << 16)
    return e, p, b


def _step(e, b, x, dtype):
    tp.tp_push_block(e, b, x)
    tp.tp_dedisperse(e, b)
    tp.tp_detect(e, b)
    c, n, _ = tp.tp_get_candidates(e, b, 1 << 16)
    D = tp.tp_get_series(e, b, ndm=len(DMS), is_int=dtype == "u8")
    mu, sg = tp.tp_get_bandpass(e, b, NCHAN)
    return c.copy(), n, D, mu, sg, tp.tp_beam_info(e, b)["t0_abs"]


@pytest.mark.parametrize("dtype,alpha", [("f32", 1.0), ("u8", 1.0), ("f32", 0.5), ("u8", 0.25)])
def test_resume_equals_continuous(dtype, alpha):
    tp.build()
    blocks = _blocks(dtype, 5)
    e, p, b = _open(dtype, alpha)
    try:
        cont = [_step(e, b, x, dtype) for x in blocks]
    finally:
        tp.tp_engine_destroy(e)
    e1, p1, b1 = _open(dtype, alpha)
    e2, p2, b2 = _open(dtype, alpha)
    try:
        for x in blocks[:2]:
            _step(e1, b1, x, dtype)
        state = tp.tp_beam_export(e1, b1)
        tp.tp_engine_destroy(e1)
        e1 = None
        tp.tp_beam_import(e2, b2, state)
        for k in range(2, 5):
            got = _step(e2, b2, blocks[k], dtype)
            want = cont[k]
            assert got[1] == want[1] and np.array_equal(got[0], want[0]), k
            for i in (2, 3, 4):
                assert np.array_equal(got[i], want[i]), (k, i)
            assert got[5] == want[5], k
    finally:
        if e1 is not None:
            tp.tp_engine_destroy(e1)
        tp.tp_engine_destroy(e2)


def test_import_checks_the_plan():
    tp.build()
    blocks = _blocks("f32", 1)
    e, p, b = _open("f32", 1.0)
    other = tp.tp_engine_create(0)
    try:
        _step(e, b, blocks[0], "f32")
        state = tp.tp_beam_export(e, b)
        q = tp.tp_create_plan(other, NCHAN, *BAND, DMS * 1.1, "f32", None, 4.0)
        bq = tp.tp_beam_open(other, q, B, 1 << 16)
        with pytest.raises(tp.TpError) as err:
            tp.tp_beam_import(other, bq, state)
        assert err.value.code == tp.TP_EINVAL
        with pytest.raises(tp.TpError):
            tp.tp_beam_import(other, bq, state[:40])
    finally:
        tp.tp_engine_destroy(e)
        tp.tp_engine_destroy(other)

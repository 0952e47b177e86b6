"""The autotuner cache (tp_engine_set_tuning_cache): a choice timed once is
written to the file and applied by a later engine without timing runs; a
different plan misses the cache and adds its own entry."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth

pytestmark = pytest.mark.gpu

NCHAN, B = 256, 12000
BAND = (398.0, 20.0, 51.2e-6)


def _tune(path, dms, x):
    e = tp.tp_engine_create(0)
    try:
        tp.tp_engine_set_tuning_cache(e, path)
        p = tp.tp_create_plan(e, NCHAN, *BAND, dms, "f32", None, 5.0)
        b = tp.tp_beam_open(e, p, B, 1 << 16)
        tp.tp_push_block(e, b, x)
        tp.tp_dedisperse(e, b)
        best, ms = tp.tp_autotune(e, b, reps=1)
        cur, feas = tp.tp_plan_shapes(p)
        tp.tp_dedisperse(e, b)
        tp.tp_detect(e, b)
        c, n, _ = tp.tp_get_candidates(e, b, 1 << 16)
        D = tp.tp_get_series(e, b, ndm=len(dms))
        return best, ms, cur, feas, c.copy(), D
    finally:
        tp.tp_engine_destroy(e)


def test_tuning_cache_reuses_and_extends(tmp_path):
    tp.build()
    path = str(tmp_path / "shapes.txt")
    x = synth.noise(NCHAN, B, 77)
    dms = np.arange(48) * 0.2
    b1, ms1, cur1, feas1, c1, D1 = _tune(path, dms, x)
    assert cur1 == b1 and feas1[b1] and np.count_nonzero(ms1 >= 0) >= 2
    lines = [ln for ln in open(path) if ln.startswith('"')]
    assert len(lines) == 1 and lines[0].split()[-2] == str(b1)
    b2, ms2, cur2, feas2, c2, D2 = _tune(path, dms, x)
    assert b2 == b1 and cur2 == b1
    assert np.count_nonzero(ms2 >= 0) == 1 and ms2[b1] > 0       # no timing runs
    assert np.array_equal(D2, D1) and np.array_equal(c2, c1)
    b3, ms3, *_ = _tune(path, np.arange(40) * 0.25, x)
    assert np.count_nonzero(ms3 >= 0) >= 2
    assert len([ln for ln in open(path) if ln.startswith('"')]) == 2

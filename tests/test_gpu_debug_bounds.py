"""The bounds-checking build of the library (libtpdd_debug.so) and the canary
padding around a beam's device buffers.

Each case runs in a child process, since the binding loads one library per
process (TP_DEBUG_BOUNDS=1 selects the debug one).  The child pushes blocks
of 8-bit, binary16 and binary32 data through every feasible kernel shape,
singly and batched on a persistent grid, with canary padding on, and writes
the series and candidates to a file.  The parent checks that (a) no check
fired and no canary was touched, (b) the debug build's results equal the
release build's bit for bit, and (c) a staged-series extent declared too
small (every access still inside the real buffer) makes the checks fire:
the block reports TP_EBOUNDS, and the next block is clean again."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NCHAN, B = 256, 12000
BAND = (398.0, 20.0, 51.2e-6)
DMS = np.arange(48) * 0.35


def _blocks(dtype, n):
    import synth
    out = []
    for k in range(n):
        x = synth.noise(NCHAN, B, 8200 + k)
        synth.add_narrowband(x, [30, 31], 2000 + 300 * k, 2600 + 300 * k, 9.0)
        synth.add_broadband(x, [5000 + 50 * k], 5.0)
        out.append({"f32": lambda a: a, "f16": synth.to_f16, "u8": lambda a: synth.to_u8(a * 16 + 128)}[dtype](x))
    return out


def _child(out_path):
    import paper_1307_5700_gb300 as tp
    res = {"debug": np.array(tp.tp_debug_bounds())}
    e = tp.tp_engine_create(0)
    try:
        tp.tp_engine_set_canaries(e, 1)
        for dtype in ("f32", "u8", "f16"):
            p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, dtype, None, 4.0)
            b = tp.tp_beam_open(e, p, B, 1 << 16)
            shapes = [int(s) for s in np.nonzero(tp.tp_plan_shapes(p)[1])[0]]
            res[f"{dtype}_shapes"] = np.array(shapes)
            for k, x in enumerate(_blocks(dtype, 2)):
                tp.tp_push_block(e, b, x)
                for sh in shapes:
                    tp.tp_plan_set_shape(p, sh)
                    tp.tp_beam_rewind(e, b)
                    tp.tp_dedisperse(e, b)
                    tp.tp_detect(e, b)
                    c, n, rc = tp.tp_get_candidates(e, b, 1 << 16)
                    assert rc == 0, (dtype, k, sh, rc)
                    res[f"{dtype}_{k}_{sh}_D"] = tp.tp_get_series(e, b, ndm=len(DMS), is_int=dtype == "u8")
                    res[f"{dtype}_{k}_{sh}_c"] = c
            tp.tp_beam_close(e, b)
            tp.tp_plan_destroy(p)
        # three uneven beams batched on a persistent grid of few CTAs, so that
        # every CTA takes several work items
        tp.tp_engine_set_batch_grid(e, 8)
        plans = [tp.tp_create_plan(e, NCHAN, *BAND, DMS[:nd], "f32", None, 4.0) for nd in (16, 32, 48)]
        beams = [tp.tp_beam_open(e, p, B, 1 << 16) for p in plans]
        x = _blocks("f32", 1)[0]
        for b in beams:
            tp.tp_push_block(e, b, x)
        tp.tp_run_ready(e)
        for i, b in enumerate(beams):
            c, n, rc = tp.tp_get_candidates(e, b, 1 << 16)
            assert rc == 0, ("batch", i, rc)
            res[f"batch_{i}_D"] = tp.tp_get_series(e, b, ndm=len(DMS[:[16, 32, 48][i]]))
            res[f"batch_{i}_c"] = c
        res["canaries_bad"] = np.array(tp.tp_engine_check_canaries(e))
        for b in beams:
            tp.tp_beam_close(e, b)
        for p in plans:
            tp.tp_plan_destroy(p)
        if tp.tp_debug_bounds():
            # a staged series declared 1 KB long: the dedispersion kernel's
            # copies beyond it fail their checks and are skipped
            p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, "f32", None, 4.0)
            b = tp.tp_beam_open(e, p, B, 1 << 16)
            blocks = _blocks("f32", 2)
            tp.tp_push_block(e, b, blocks[0])
            tp.tp_debug_limit_staged(e, b, 1024)
            tp.tp_dedisperse(e, b)
            tp.tp_detect(e, b)
            try:
                tp.tp_get_candidates(e, b, 1 << 16)
                res["fired"] = np.array(0)
            except tp.TpError as exc:
                res["fired"] = np.array(exc.code)
            tp.tp_debug_limit_staged(e, b, -1)
            tp.tp_push_block(e, b, blocks[1])
            tp.tp_dedisperse(e, b)
            tp.tp_detect(e, b)
            res["after"] = np.array(tp.tp_get_candidates(e, b, 1 << 16)[2])
            res["canaries_bad_after"] = np.array(tp.tp_engine_check_canaries(e))
            tp.tp_beam_close(e, b)
            tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)
    np.savez(out_path, **res)


def _run(debug, tmp_path):
    out = str(tmp_path / f"res_{int(debug)}.npz")
    env = dict(os.environ, TP_DEBUG_BOUNDS="1" if debug else "0")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


def test_debug_build_matches_release_and_checks_fire(tmp_path):
    import paper_1307_5700_gb300 as tp
    tp.build(debug=False)
    tp.build(debug=True)
    rel = _run(False, tmp_path)
    dbg = _run(True, tmp_path)
    assert int(rel["debug"]) == 0 and int(dbg["debug"]) == 1
    assert int(rel["canaries_bad"]) == 0 and int(dbg["canaries_bad"]) == 0
    keys = sorted(k for k in rel if k not in ("debug",))
    assert keys == sorted(k for k in dbg if k not in ("debug", "fired", "after", "canaries_bad_after"))
    for k in keys:
        assert np.array_equal(rel[k], dbg[k]), k
    assert len(rel["f32_shapes"]) >= 2 and len(rel["u8_shapes"]) >= 2
    assert int(dbg["fired"]) == tp.TP_EBOUNDS
    assert int(dbg["after"]) == 0
    assert int(dbg["canaries_bad_after"]) == 0


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    _child(sys.argv[1])

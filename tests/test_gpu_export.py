"""Stream-ordered export of the candidates (tp_export_candidates): into
page-locked host buffers, the count, records and status equal what
tp_get_candidates returns, for whole and truncated lists, with the next
block's work enqueued before the host reads anything; pageable buffers are
refused."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth

pytestmark = pytest.mark.gpu

NCHAN, B = 128, 5000
BAND = (398.0, 20.0, 51.2e-6)
DMS = np.arange(24) * 0.5


def _pinned(cap):
    import torch
    out = torch.zeros(max(cap, 1) * 24, dtype=torch.uint8, pin_memory=True)
    cnt = torch.zeros(1, dtype=torch.int64, pin_memory=True)
    st = torch.full((1,), -7, dtype=torch.int32, pin_memory=True)
    return out, cnt, st


def _records(out, n):
    return out.numpy()[: 24 * n].view(tp.CAND_DTYPE)


def _blocks(n):
    out = []
    for k in range(n):
        x = synth.noise(NCHAN, B, 8100 + k)
        synth.add_narrowband(x, [30, 31], 600 + 300 * k, 1200 + 300 * k, 9.0)
        out.append(x)
    return out


def test_export_equals_get_candidates():
    import torch
    tp.build()
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, "f32", None, 3.5)
        b = tp.tp_beam_open(e, p, B, 1 << 15)
        blocks = _blocks(3)
        bufs = [_pinned(1 << 15) for _ in blocks]
        small = _pinned(5)
        # every block's work and export are enqueued before the host reads any
        for k, x in enumerate(blocks):
            tp.tp_push_block(e, b, x)
            tp.tp_dedisperse(e, b)
            tp.tp_detect(e, b)
            tp.tp_export_candidates(e, b, bufs[k][0], 1 << 15, bufs[k][1], bufs[k][2])
            if k == 2:
                tp.tp_export_candidates(e, b, small[0], 5, small[1], None)
        tp.tp_sync(e)
        torch.cuda.synchronize()
        want, n, rc = tp.tp_get_candidates(e, b, 1 << 15)  # the last block
        assert rc == 0 and n > 5
        got = _records(bufs[2][0], int(bufs[2][1].item()))
        assert int(bufs[2][1].item()) == n and int(bufs[2][2].item()) == 0
        assert got.tobytes() == want.tobytes()
        # truncated: the first 5 records, the full count
        assert int(small[1].item()) == n
        assert _records(small[0], 5).tobytes() == want[:5].tobytes()
        # the earlier blocks' exports kept their own results
        for k in range(2):
            nk = int(bufs[k][1].item())
            assert nk > 0 and int(bufs[k][2].item()) == 0
            rk = _records(bufs[k][0], nk)
            assert np.all(np.diff(rk["dm_idx"].astype(np.int64) * (1 << 40) + rk["t_abs"]) > 0)
            assert np.all(rk["beam"] == b)
        # a fresh run of block 0 alone gives the same records as its export
        e2 = tp.tp_engine_create(0)
        try:
            p2 = tp.tp_create_plan(e2, NCHAN, *BAND, DMS, "f32", None, 3.5)
            b2 = tp.tp_beam_open(e2, p2, B, 1 << 15)
            tp.tp_push_block(e2, b2, blocks[0])
            tp.tp_dedisperse(e2, b2)
            tp.tp_detect(e2, b2)
            w0, n0, _ = tp.tp_get_candidates(e2, b2, 1 << 15)
            assert n0 == int(bufs[0][1].item())
            assert _records(bufs[0][0], n0).tobytes() == w0.tobytes()
        finally:
            tp.tp_engine_destroy(e2)
    finally:
        tp.tp_engine_destroy(e)


def test_export_refuses_pageable_buffers():
    tp.build()
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, NCHAN, *BAND, DMS, "f32", None, 3.5)
        b = tp.tp_beam_open(e, p, B, 1 << 12)
        out, cnt, st = _pinned(16)
        with pytest.raises(tp.TpError) as ex:  # nothing detected yet
            tp.tp_export_candidates(e, b, out, 16, cnt, st)
        assert ex.value.code == tp.TP_ENOTREADY
        tp.tp_push_block(e, b, _blocks(1)[0])
        tp.tp_dedisperse(e, b)
        tp.tp_detect(e, b)
        pageable = np.zeros(16 * 24, np.uint8)
        pcount = np.zeros(1, np.uint64)
        for args in ((pageable, 16, cnt, st), (out, 16, pcount, st), (out, -1, cnt, st)):
            with pytest.raises(tp.TpError) as ex:
                tp.tp_export_candidates(e, b, *args)
            assert ex.value.code == tp.TP_EINVAL
        # the beam is unharmed
        tp.tp_export_candidates(e, b, out, 16, cnt, st)
        tp.tp_sync(e)
        import torch
        torch.cuda.synchronize()
        _, n, _ = tp.tp_get_candidates(e, b, 16)
        assert int(cnt.item()) == n
    finally:
        tp.tp_engine_destroy(e)

"""In-place push (tp_push_inplace): a block that a device-side producer wrote
into its own buffer is processed where it lies, the engine writing only the
overlap tail into the buffer's first max_delay columns.  The series,
statistics, masks and candidates equal those of the same stream pushed by
copy (tp_push_block), for each sample format, mixed with copy pushes and
prefetched host blocks, batched and replayed from graphs, and across an
export / import of the stream state; invalid buffers are refused."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth

pytestmark = pytest.mark.gpu

NCHAN, B = 160, 6000
BAND = (398.0, 20.0, 51.2e-6)
DMS = np.arange(36) * 0.4


def _blocks(dtype, n, seed=7300):
    out = []
    for k in range(n):
        x = synth.noise(NCHAN, B, seed + k, mean=0.1 * k)
        synth.add_narrowband(x, [12, 13], 900 + 250 * k, 1700 + 250 * k, 9.0)
        synth.add_broadband(x, [3000 + 40 * k], 6.0)
        out.append({"f32": lambda a: a, "f16": synth.to_f16, "u8": lambda a: synth.to_u8(a * 16 + 128)}[dtype](x))
    return out


def _open(dtype, ndm=len(DMS)):
    e = tp.tp_engine_create(0)
    p = tp.tp_create_plan(e, NCHAN, *BAND, DMS[:ndm], dtype, None, 4.0)
    b = tp.tp_beam_open(e, p, B, 1 << 16)
    return e, p, b


def _dmax(p):
    return tp.tp_plan_info(p)["max_delay"]


def _buffer(x, dmax, extra=40):
    """A producer's buffer: (nchan, pitch) with the block in columns
    [dmax, dmax + nsamp) and garbage elsewhere."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    es = t.element_size()
    pitch = dmax + x.shape[1] + extra
    pitch += (-pitch * es) % 16 // es
    buf = torch.full((x.shape[0], pitch), 77, dtype=t.dtype, device="cuda")
    buf[:, dmax:dmax + x.shape[1]] = t
    torch.cuda.synchronize()  # the engine's streams do not wait for torch's
    return buf


def _results(e, b, dtype, ndm=len(DMS)):
    tp.tp_dedisperse(e, b)
    tp.tp_detect(e, b)
    return _read(e, b, dtype, ndm)


def _read(e, b, dtype, ndm=len(DMS)):
    c, n, rc = tp.tp_get_candidates(e, b, 1 << 16)
    D = tp.tp_get_series(e, b, ndm=ndm, is_int=dtype == "u8")
    mu, sg = tp.tp_get_bandpass(e, b, NCHAN)
    return dict(c=c.copy(), n=n, rc=rc, D=D, mu=mu, sg=sg, t0=tp.tp_beam_info(e, b)["t0_abs"])


def _same(got, want, tag):
    for k in want:
        assert np.array_equal(got[k], want[k]), (tag, k)


def _reference(dtype, blocks):
    e, p, b = _open(dtype)
    try:
        out = []
        for x in blocks:
            tp.tp_push_block(e, b, x)
            out.append(_results(e, b, dtype))
        return out
    finally:
        tp.tp_engine_destroy(e)


@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_inplace_equals_copy(dtype):
    tp.build()
    blocks = _blocks(dtype, 5)
    want = _reference(dtype, blocks)
    e, p, b = _open(dtype)
    try:
        dmax = _dmax(p)
        bufs = [_buffer(x, dmax) for x in blocks]
        for k in range(5):
            tp.tp_push_inplace(e, b, bufs[k], B)
            _same(_results(e, b, dtype), want[k], (dtype, k))
            # the engine wrote the previous block's last dmax samples
            if k > 0:
                assert bool((bufs[k][:, :dmax] == bufs[k - 1][:, B:dmax + B]).all())
    finally:
        tp.tp_engine_destroy(e)


def test_inplace_mixed_with_copy_prefetch_and_export():
    tp.build()
    dtype = "f32"
    blocks = _blocks(dtype, 6, seed=7400)
    want = _reference(dtype, blocks)
    e, p, b = _open(dtype)
    e2 = None
    try:
        dmax = _dmax(p)
        bufs = [_buffer(x, dmax) for x in blocks]
        tp.tp_push_inplace(e, b, bufs[0], B)              # the first block: copied
        _same(_results(e, b, dtype), want[0], 0)
        tp.tp_push_inplace(e, b, bufs[1], B)
        _same(_results(e, b, dtype), want[1], 1)
        tp.tp_push_block(e, b, bufs[2][:, dmax:dmax + B].contiguous())  # copy after in place
        _same(_results(e, b, dtype), want[2], 2)
        tp.tp_push_inplace(e, b, bufs[3], B)
        r3 = _results(e, b, dtype)
        _same(r3, want[3], 3)
        tp.tp_prefetch_block(e, b, blocks[4])              # prefetched after in place
        tp.tp_push_prefetched(e, b)
        _same(_results(e, b, dtype), want[4], 4)
        # export after an in-place block, resume in another engine
        e2, p2, b2 = _open(dtype)
        e3, p3, b3 = _open(dtype)
        try:
            for k in range(3):
                tp.tp_push_block(e3, b3, blocks[k])
                _results(e3, b3, dtype)
            tp.tp_push_inplace(e3, b3, _buffer(blocks[3], dmax), B)
            _results(e3, b3, dtype)
            state = tp.tp_beam_export(e3, b3)
        finally:
            tp.tp_engine_destroy(e3)
        tp.tp_beam_import(e2, b2, state)
        tp.tp_push_block(e2, b2, blocks[4])
        _same(_results(e2, b2, dtype), want[4], "resumed")
    finally:
        tp.tp_engine_destroy(e)
        if e2 is not None:
            tp.tp_engine_destroy(e2)


def test_inplace_batched_graphs():
    tp.build()
    dtype = "f32"
    blocks = _blocks(dtype, 5, seed=7500)
    ndms = (20, 36)
    wants = []
    for nd in ndms:
        e, p, b = _open(dtype, nd)
        try:
            out = []
            for x in blocks:
                tp.tp_push_block(e, b, x)
                out.append(_results(e, b, dtype, nd))
            wants.append(out)
        finally:
            tp.tp_engine_destroy(e)
    import torch
    stream = torch.cuda.Stream()  # graphs are captured on the engine's own stream
    e = tp.tp_engine_create(0, 0, stream.cuda_stream)
    try:
        plans = [tp.tp_create_plan(e, NCHAN, *BAND, DMS[:nd], dtype, None, 4.0) for nd in ndms]
        beams = [tp.tp_beam_open(e, p, B, 1 << 16) for p in plans]
        # three buffers per beam in rotation, so the graphs replay
        bufs = [[_buffer(x, _dmax(p)) for x in blocks[:3]] for p in plans]
        for k in range(5):
            for i, b in enumerate(beams):
                buf = bufs[i][k % 3]
                dmax = _dmax(plans[i])
                buf[:, dmax:dmax + B] = torch.from_numpy(blocks[k]).cuda()
                torch.cuda.synchronize()
                tp.tp_push_inplace(e, b, buf, B)
            tp.tp_run_ready(e, use_graph=True)
            for i, b in enumerate(beams):
                got = _read(e, b, dtype, ndms[i])
                # the records name the beam that produced them: beam i here,
                # beam 0 in the one-beam engines
                assert np.all(got["c"]["beam"] == b)
                got["c"]["beam"] = wants[i][k]["c"]["beam"]
                _same(got, wants[i][k], (i, k))
    finally:
        tp.tp_engine_destroy(e)


def test_inplace_rejects_invalid_buffers():
    import torch
    tp.build()
    blocks = _blocks("f32", 3)
    e, p, b = _open("f32")
    try:
        dmax = _dmax(p)
        for x in blocks[:2]:
            last = _buffer(x, dmax)
            tp.tp_push_inplace(e, b, last, B)
            _results(e, b, "f32")
        ok = dmax + B + (-(dmax + B)) % 4
        short = torch.zeros((NCHAN, dmax + B - 4), dtype=torch.float32, device="cuda")
        odd = torch.zeros((NCHAN, ok + 1), dtype=torch.float32, device="cuda")
        host = np.zeros((NCHAN, ok), np.float32)
        # too short, a row pitch that is not a multiple of 16 bytes, the
        # previous block's buffer, host memory
        for bad, pitch in ((short, None), (odd, None), (last, None), (host, ok)):
            with pytest.raises(tp.TpError) as ex:
                tp.tp_push_inplace(e, b, bad, B, pitch)
            assert ex.value.code == tp.TP_EINVAL
        # the beam is unharmed: the next valid block goes through
        tp.tp_push_inplace(e, b, _buffer(blocks[2], dmax), B)
        assert _results(e, b, "f32")["rc"] == 0
    finally:
        tp.tp_engine_destroy(e)

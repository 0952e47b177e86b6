"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: bit-exact delay tables, masks, 8-bit int32 series and candidate sets;
FP32 series within |D_gpu - D_oracle| <= 1e-5 * sum_c |y| (the magnitude of the
terms summed at that point); binary16 / bfloat16 storage judged against the
binary64 oracle run on the same quantised input, with the same bound.  Float
candidate sets must match except entries whose oracle statistic lies within
that bound of the threshold (reported; the seeded inputs keep them rare)."""
import math
import os

import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth
from oracle import oracle as O
from tests.gpu_run import GpuBeam

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _setup():
    tp.build()
    O.set_threads(os.cpu_count() or 1)


def _mass_all(x, dtype, st, cf, sf, W, delay, T):
    ndm = delay.shape[0]
    dd = np.repeat(np.arange(ndm, dtype=np.int32), T)
    tt = np.tile(np.arange(T, dtype=np.int64), ndm)
    _, mass = O.dedisperse_points(x, dtype, st, cf, sf, W, delay, dd, tt)
    return mass.reshape(ndm, T)


def _as_f64(x, dtype):
    if dtype == "bf16":
        return synth.bf16_bits_to_f32(x).astype(np.float64)
    if dtype == "c16":  # power of the complex voltages
        return x["re"].astype(np.float64) ** 2 + x["im"].astype(np.float64) ** 2
    return x.astype(np.float64)


def _cand_set(c):
    return {(int(r["dm_idx"]), int(r["t_abs"])) for r in c}


def check_block(g, o, x, dtype, delay, rfi, nsigma, t0=0):
    """Compare one block's GPU products with the oracle's."""
    T = o["T"]
    assert g["info"]["nout"] == T
    assert np.array_equal(g["chunk_raw"], o["chunk_raw"]), "channel exceedances differ"
    assert np.array_equal(g["chunk_flag"], o["chunk_flag"]), "chunk flags differ"
    assert np.array_equal(g["spec_flag"], o["spec_flag"]), "spectrum flags differ"
    # float statistics are summed in FP32 inside 256-sample sub-chunks (13
    # roundings deep) and in FP64 above: |d mu| <= ~13 u mean|x - p| << 1e-6 mean|x|
    scale = np.abs(_as_f64(x, dtype)).mean(axis=1) + np.abs(o["stats"]["mu"])
    assert np.all(np.abs(g["mu"] - o["stats"]["mu"]) <= 1e-6 * scale + 1e-12), "bandpass mean"
    np.testing.assert_allclose(g["sigma"], o["stats"]["sigma"], rtol=2e-6, atol=1e-12)
    Dg, Do = g["D"], o["D"]
    if dtype == "u8":
        assert Dg.dtype == np.int32
        assert np.array_equal(Dg.astype(np.int64), Do), "int32 series differ"
        assert np.array_equal(g["row_mu"], o["series"]["mu"])
        assert np.array_equal(g["row_sigma"], o["series"]["sigma"])
        got = g["candidates"]
        want = o["candidates"]
        assert g["n_candidates"] == o["n_candidates"]
        assert np.array_equal(got["dm_idx"], want["dm_idx"]) and np.array_equal(got["t_abs"], want["t_abs"])
        assert np.array_equal(got["snr"], want["snr"]) and np.array_equal(got["value"], want["value"])
        return
    mass = _mass_all(x, dtype, o["stats"], o["chunk_flag"], o["spec_flag"], rfi.chunk_width, delay, T)
    err = np.abs(Dg.astype(np.float64) - Do)
    bound = TOL * mass + 1e-30
    worst = float((err / np.maximum(mass, 1e-300)).max())
    assert np.all(err <= bound), f"max |dD|/mass = {worst:.3e}"
    np.testing.assert_allclose(g["row_mu"], o["series"]["mu"], rtol=0,
                               atol=1e-5 * float(np.abs(Do).mean()) + 1e-9)
    np.testing.assert_allclose(g["row_sigma"], o["series"]["sigma"], rtol=1e-5)
    # candidates, except entries within the D bound of the threshold
    stat = Do - o["series"]["mu"][:, None] - nsigma * o["series"]["sigma"][:, None]
    border = np.abs(stat) <= TOL * mass + 1e-6 * nsigma * o["series"]["sigma"][:, None]
    bset = {(int(d), int(t) + t0) for d, t in zip(*np.nonzero(border))}
    gs, os_ = _cand_set(g["candidates"]), _cand_set(o["candidates"])
    assert gs - bset == os_ - bset, f"candidate sets differ: {sorted((gs ^ os_) - bset)[:10]}"
    assert len(bset) <= max(5, 1e-4 * Do.size)
    # records: (dm, t) order, values and snr consistent with the oracle
    keys = [(int(r["dm_idx"]), int(r["t_abs"])) for r in g["candidates"]]
    assert keys == sorted(keys)
    for r in g["candidates"][:2000]:
        d, t = int(r["dm_idx"]), int(r["t_abs"]) - t0
        assert abs(r["value"] - Do[d, t]) <= TOL * mass[d, t] + 1e-6 * abs(Do[d, t])
        snr = (Do[d, t] - o["series"]["mu"][d]) / o["series"]["sigma"][d]
        assert abs(r["snr"] - snr) <= 1e-4 * max(1.0, abs(snr))


def run_both(x, dtype, nchan, f_lo, bw, t_samp, dms, rfi, nsigma=5.0, ox=None):
    g = GpuBeam(nchan, f_lo, bw, t_samp, dms, dtype, rfi=rfi, nsigma=nsigma)
    try:
        delay = g.delays()
        od, dmax = O.delay_table(nchan, f_lo, bw, t_samp, dms)
        assert np.array_equal(delay, od), "delay tables differ"
        res = g.run(x)
    finally:
        g.close()
    o = O.search_block(ox if ox is not None else x, dtype, od, dmax, rfi=rfi, nsigma=nsigma)
    return res, o, od


# ---- A0 -----------------------------------------------------------------------------

@pytest.mark.parametrize("nchan,f_lo,bw,ts,dms", [
    (1024, 398.0, 20.0, 51.2e-6, np.arange(64, dtype=np.float64)),
    (1024, 398.0, 20.0, 51.2e-6, np.arange(640) * 0.2),
    (4096, 1200.0, 300.0, 64e-6, np.arange(2048, dtype=np.float64)),
    (1024, 418.0, -20.0, 51.2e-6, np.arange(320) * 0.2),
    (37, 100.0, 3.3, 1e-3, np.array([0.0, 1.0, 2.5, 10.0, 10.0, 77.7])),
    (256, 1400.0, 0.5, 1e-4, np.array([0.0, 1e4])),
])
def test_delay_table_bit_exact(nchan, f_lo, bw, ts, dms):
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, nchan, f_lo, bw, ts, dms, "f32")
        got = tp.tp_get_delay_table(p)
        info = tp.tp_plan_info(p)
        want, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
        assert np.array_equal(got, want)
        assert info["max_delay"] == dmax
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)


def test_plan_rejects_invalid():
    e = tp.tp_engine_create(0)
    try:
        for args in [(0, 398.0, 20.0, 51.2e-6, [1.0]), (16, 398.0, 20.0, 0.0, [1.0]),
                     (16, 398.0, 20.0, 51.2e-6, [-1.0]), (16, 398.0, 20.0, 51.2e-6, [2.0, 1.0]),
                     (16, -30.0, 20.0, 51.2e-6, [1.0]), (16, 398.0, 0.0, 51.2e-6, [1.0])]:
            with pytest.raises(tp.TpError) as ei:
                tp.tp_create_plan(e, *args[:4], np.array(args[4]), "f32")
            assert ei.value.code == tp.TP_EINVAL
    finally:
        tp.tp_engine_destroy(e)


# ---- whole blocks ------------------------------------------------------------------------

def test_config1_single_block_f32():
    """1024 channels over 398-418 MHz, 32768 FP32 samples, DM 0..63: pulse at
    DM 30 / t 12000 (SNR 20), narrowband and broadband RFI."""
    dms = np.arange(64, dtype=np.float64)
    od, dmax = O.delay_table(1024, 398.0, 20.0, 51.2e-6, dms)
    x = synth.single_block_workload(lambda: od[30].astype(np.float64), seed=1000)
    rfi = O.RfiParams()
    g, o, _ = run_both(x, "f32", 1024, 398.0, 20.0, 51.2e-6, dms, rfi)
    assert o["chunk_flag"][[300, 301, 700, 701]].any(axis=1).all()
    assert o["spec_flag"][[5000, 20000, 26000]].all()
    check_block(g, o, x, "f32", od, rfi, 5.0)
    D = g["D"]
    d, t = np.unravel_index(np.argmax(D), D.shape)
    assert abs(d - 30) <= 1 and abs(t - 12000) <= 10


def test_u8_block_exact():
    nchan, nsamp = 256, 40000
    dms = np.arange(96) * 0.5
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    xf = synth.noise(nchan, nsamp, 5001, mean=128.0, std=16.0)
    synth.add_pulse(xf, od[40].astype(np.float64) + 20000, 19.5, 16 * 25 / math.sqrt(nchan))
    synth.add_narrowband(xf, [17, 18, 19], 3000, 7000, 160.0)
    synth.add_broadband(xf, [15000, 31000], 100.0)
    x = synth.to_u8(xf)
    rfi = O.RfiParams(chunk_width=128)
    g, o, _ = run_both(x, "u8", nchan, 398.0, 20.0, 51.2e-6, dms, rfi, nsigma=4.0)
    assert o["chunk_flag"].any() and o["spec_flag"].any() and o["n_candidates"] > 0
    check_block(g, o, x, "u8", od, rfi, 4.0)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_half_precision_storage(dtype):
    nchan, nsamp = 512, 20000
    dms = np.arange(80) * 0.4
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    xf = synth.noise(nchan, nsamp, 6001)
    synth.add_pulse(xf, od[50].astype(np.float64) + 9000, 19.5, 20 / math.sqrt(nchan))
    synth.add_narrowband(xf, [100, 101], 2000, 4000, 8.0)
    x = synth.to_f16(xf) if dtype == "f16" else synth.to_bf16_bits(xf)
    rfi = O.RfiParams()
    g, o, _ = run_both(x, dtype, nchan, 398.0, 20.0, 51.2e-6, dms, rfi)
    check_block(g, o, x, dtype, od, rfi, 5.0)
    # error against the FP32 original, in sigma_D units (quantisation dominated)
    o32 = O.search_block(xf, "f32", od, dmax, rfi=rfi)
    sd = float(np.median(o32["series"]["sigma"]))
    q = float(np.abs(g["D"].astype(np.float64) - o32["D"]).max()) / sd
    assert q < (0.05 if dtype == "f16" else 0.4), q


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_ragged_shapes(dtype):
    """37 channels, 33 DMs with a wide step (the planner splits DM tiles by
    delay spread), window not a multiple of 512 or of W = 100."""
    nchan, nsamp = 37, 9999
    dms = np.concatenate([np.arange(20) * 3.0, 60 + np.arange(13) * 12.0])
    f_lo, bw, ts = 398.0, 20.0, 1e-4
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    assert dmax < nsamp
    xf = synth.noise(nchan, nsamp, 7001, mean=128.0 if dtype == "u8" else 0.0, std=16.0 if dtype == "u8" else 1.0)
    xf[5, 1000:1700] += 200.0 if dtype == "u8" else 12.0
    x = synth.to_u8(xf) if dtype == "u8" else xf
    rfi = O.RfiParams(chunk_width=100, dilate_channels=True)
    g, o, _ = run_both(x, dtype, nchan, f_lo, bw, ts, dms, rfi, nsigma=3.5)
    assert o["chunk_flag"].any()
    check_block(g, o, x, dtype, od, rfi, 3.5)


@pytest.mark.parametrize("dtype,step", [("f32", 0.2), ("f16", 0.2), ("bf16", 0.2), ("u8", 0.2),
                                        ("f32", 0.18), ("f16", 0.18)])
def test_every_shape_elementwise(dtype, step):
    """Every kernel shape the plan admits, element by element against the
    oracle: 256 channels over 398-418 MHz, 62 DM trials (the last group of
    four trials is incomplete), a window that is not a multiple of any tile
    and spans several DM tiles and time tiles.  At DM step 0.2 the last
    group's single delay step (10 samples in the lowest channel) exceeds the
    FP32 DM quads' bound of 9, so those shapes are not admitted; step 0.18
    admits them."""
    nchan, nsamp = 256, 7777
    dms = np.arange(62) * step
    f_lo, bw, ts = 398.0, 20.0, 51.2e-6
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    xf = synth.noise(nchan, nsamp, 7101, mean=128.0 if dtype == "u8" else 0.0, std=16.0 if dtype == "u8" else 1.0)
    synth.add_pulse(xf, od[40].astype(np.float64) + 2500, 20.0, 160.0 if dtype == "u8" else 10.0 / 16)
    xf[17, 3000:3400] += 200.0 if dtype == "u8" else 12.0
    x = {"f32": lambda a: a, "u8": synth.to_u8, "f16": synth.to_f16, "bf16": synth.to_bf16_bits}[dtype](xf)
    rfi = O.RfiParams()
    o = O.search_block(x, dtype, od, dmax, rfi=rfi)
    g = GpuBeam(nchan, f_lo, bw, ts, dms, dtype, rfi=rfi)
    try:
        g.open(nsamp)
        first = g.run(x)
        _, feasible = tp.tp_plan_shapes(g.plan)
        shapes = [int(s) for s in np.nonzero(feasible)[0]]
        assert len(shapes) >= 2
        if step == 0.18 and dtype == "f32":
            assert {53, 55, 46, 33} <= set(shapes)  # the FP32 quad families
        for sh in shapes:
            tp.tp_plan_set_shape(g.plan, sh)
            tp.tp_beam_rewind(g.e, g.beam)
            tp.tp_dedisperse(g.e, g.beam)
            tp.tp_detect(g.e, g.beam)
            cands, n, rc = tp.tp_get_candidates(g.e, g.beam, g.cap)
            r = dict(first, candidates=cands, n_candidates=n, rc=rc,
                     D=tp.tp_get_series(g.e, g.beam, ndm=len(dms), is_int=dtype == "u8"))
            r["row_mu"], r["row_sigma"] = tp.tp_get_series_stats(g.e, g.beam, len(dms))
            try:
                check_block(r, o, x, dtype, od, rfi, 5.0)
            except AssertionError as exc:
                raise AssertionError(f"shape {sh}: {exc}") from exc
    finally:
        g.close()


def _voltage_block(nchan, nsamp, od, seed):
    env = np.ones((nchan, nsamp), np.float32)
    d = min(40, od.shape[0] - 1)
    synth.add_pulse(env, od[d].astype(np.float64) + nsamp // 2, 20.0, 2.5)
    env[33:35, 1000:1700] += 30.0     # narrowband RFI
    env[:, 3333] += 10.0              # broadband spike
    return synth.complex_voltage(env, seed, sigma=30.0)


def test_u8_extreme_values():
    """8-bit samples at the ends of their range over 4096 channels, the most
    the shared-parameter staging kernel takes (its packed 16-bit lanes then sum
    128 values of up to 255 each): mostly 255 with a tenth of the samples 0,
    a block of zeros, channels held at 255 throughout (sigma_c = 0) and
    whole spectra at 255 (flagged, the last one in the window's ragged last
    32-sample tile); the exact statistics, masks, series and candidates
    equal the oracle's."""
    nchan, nsamp = 4096, 2600
    dms = np.arange(6) * 1.0
    f_lo, bw, ts = 1200.0, 300.0, 64e-6
    g = synth.rng(7301)
    x = np.full((nchan, nsamp), 255, np.uint8)
    x[g.random((nchan, nsamp)) < 0.1] = 0
    x[100:140, 1000:1300] = 0
    x[2000:2010] = 255
    x[:, [500, 1777, 2599]] = 255  # spectra at the top of the range: flagged
    rfi = O.RfiParams()
    res, o, od = run_both(x, "u8", nchan, f_lo, bw, ts, dms, rfi, nsigma=3.0)
    assert o["spec_flag"].sum() >= 3
    check_block(res, o, x, "u8", od, rfi, 3.0)


def test_power_detection_c16():
    """Complex int16 voltages detected as power on the device, against the
    oracle (float bars: masks identical, D within 1e-5 of the summed
    magnitude, candidates outside the borderline band)."""
    nchan, nsamp = 192, 7001
    dms = np.arange(62) * 0.2
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    x = _voltage_block(nchan, nsamp, od, 8123)
    rfi = O.RfiParams()
    g, o, _ = run_both(x, "c16", nchan, 398.0, 20.0, 51.2e-6, dms, rfi, nsigma=5.0)
    assert o["chunk_flag"].any() and o["n_candidates"] > 0
    check_block(g, o, x, "c16", od, rfi, 5.0)


def test_power_detection_equals_float_on_power():
    """The device's power of complex voltages (exact below 2^24) makes the
    whole chain bit-identical to the binary32 chain on that power."""
    nchan, nsamp = 160, 6000
    dms = np.arange(40) * 0.4
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    x = _voltage_block(nchan, nsamp, od, 8124)
    p = (x["re"].astype(np.int64) ** 2 + x["im"].astype(np.int64) ** 2)
    assert p.max() < 2 ** 24
    pf = p.astype(np.float32)
    out = []
    for dtype, data in (("c16", x), ("f32", pf)):
        gb = GpuBeam(nchan, 398.0, 20.0, 51.2e-6, dms, dtype, nsigma=4.5, cap=1 << 18)
        try:
            tp.tp_plan_set_shape(gb.plan, int(np.nonzero(tp.tp_plan_shapes(gb.plan)[1])[0][-1]))
            out.append(gb.run(data))
        finally:
            gb.close()
    a, b = out
    for k in ("D", "mu", "sigma", "chunk_flag", "chunk_raw", "spec_flag", "row_mu", "row_sigma"):
        assert np.array_equal(a[k], b[k]), k
    assert a["n_candidates"] == b["n_candidates"] > 0
    assert np.array_equal(a["candidates"], b["candidates"])


def test_degenerate_dm0_single_channel():
    for nchan, dms in [(1, np.array([0.0])), (64, np.array([0.0])), (3, np.array([0.0, 0.0, 1.0]))]:
        x = synth.noise(nchan, 1500, 8001 + nchan)
        rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
        g, o, od = run_both(x, "f32", nchan, 398.0, 20.0, 51.2e-6, dms, rfi, nsigma=2.5)
        check_block(g, o, x, "f32", od, rfi, 2.5)
        if dms.max() == 0:
            y = x.astype(np.float64) - x.astype(np.float64).mean(axis=1, keepdims=True)
            np.testing.assert_allclose(g["D"][0], y.sum(axis=0), rtol=0, atol=1e-4 * nchan)


def test_streaming_equals_long_block():
    """Blocks pushed one after another (overlap tail carried on the device)
    give the same series as one long block, with a fixed bandpass."""
    nchan, B, nblk = 128, 3000, 4
    dms = np.arange(40) * 1.0
    f_lo, bw, ts = 398.0, 20.0, 51.2e-6
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    for dtype in ("f32", "u8"):
        xf = synth.noise(nchan, B * nblk, 9001, mean=128.0 if dtype == "u8" else 0.5,
                         std=16.0 if dtype == "u8" else 1.0)
        x = synth.to_u8(xf) if dtype == "u8" else xf
        mu = x.astype(np.float64).mean(axis=1)
        sig = x.astype(np.float64).std(axis=1)
        rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
        g = GpuBeam(nchan, f_lo, bw, ts, dms, dtype, rfi=rfi, external=True, nsigma=3.0)
        try:
            g.open(B)
            tp.tp_beam_set_bandpass(g.e, g.beam, mu, sig)
            outs, t0s = [], []
            for k in range(nblk):
                r = g.run(x[:, k * B:(k + 1) * B].copy())
                outs.append(r["D"])
                t0s.append(r["info"]["t0_abs"])
                assert r["info"]["nout"] == (B - dmax if k == 0 else B)
        finally:
            g.close()
        assert t0s == [0] + [k * B - dmax for k in range(1, nblk)]
        Dcat = np.concatenate(outs, axis=1)
        st = O.external_stats(dtype, mu, sig)
        T = B * nblk - dmax
        Do = O.dedisperse(x, dtype, st, np.zeros((nchan, 1 + (B * nblk) // 256), np.uint8),
                          np.zeros(B * nblk, np.uint8), 256, od, T)
        assert Dcat.shape == Do.shape
        if dtype == "u8":
            assert np.array_equal(Dcat.astype(np.int64), Do)
        else:
            mass = _mass_all(x, dtype, st, np.zeros((nchan, 1 + (B * nblk) // 256), np.uint8),
                             np.zeros(B * nblk, np.uint8), 256, od, T)
            assert np.all(np.abs(Dcat - Do) <= TOL * mass)


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_prefetched_stream_equals_pushed_stream(dtype):
    """Double-buffered ingest: each block's copy is started while the
    previous block is still being processed (its candidates not yet read);
    every block's series, masks and candidates are bit-identical to the same
    stream pushed block by block, and the stream matches the oracle."""
    torch = pytest.importorskip("torch")
    nchan, B, nblk = 128, 3000, 5
    dms = np.arange(40) * 1.0
    f_lo, bw, ts = 398.0, 20.0, 51.2e-6
    od, dmax = O.delay_table(nchan, f_lo, bw, ts, dms)
    xf = synth.noise(nchan, B * nblk, 9301, mean=128.0 if dtype == "u8" else 0.0, std=16.0 if dtype == "u8" else 1.0)
    synth.add_pulse(xf, od[25].astype(np.float64) + 2 * B + 700, 15.0, 80.0 if dtype == "u8" else 5.0 / 8)
    x = synth.to_u8(xf) if dtype == "u8" else xf
    blocks = [np.ascontiguousarray(x[:, k * B:(k + 1) * B]) for k in range(nblk)]
    # pinned host copies for the prefetching run (the first two pageable)
    host = [b if k < 2 else torch.from_numpy(b).pin_memory() for k, b in enumerate(blocks)]

    def collect(g):
        cands, n, rc = tp.tp_get_candidates(g.e, g.beam, g.cap)
        out = dict(candidates=cands, n_candidates=n, rc=rc, info=tp.tp_beam_info(g.e, g.beam),
                   D=tp.tp_get_series(g.e, g.beam, ndm=len(dms), is_int=dtype == "u8"))
        out["mu"], out["sigma"] = tp.tp_get_bandpass(g.e, g.beam, nchan)
        out["chunk_flag"], out["chunk_raw"], out["spec_flag"] = tp.tp_get_masks(g.e, g.beam, nchan)
        out["row_mu"], out["row_sigma"] = tp.tp_get_series_stats(g.e, g.beam, len(dms))
        return out

    ref = []
    g = GpuBeam(nchan, f_lo, bw, ts, dms, dtype)
    try:
        g.open(B)
        for b in blocks:
            tp.tp_push_block(g.e, g.beam, b)
            tp.tp_dedisperse(g.e, g.beam)
            tp.tp_detect(g.e, g.beam)
            ref.append(collect(g))
    finally:
        g.close()

    got = []
    g = GpuBeam(nchan, f_lo, bw, ts, dms, dtype)
    try:
        g.open(B)
        with pytest.raises(tp.TpError) as ei:
            tp.tp_push_prefetched(g.e, g.beam)
        assert ei.value.code == tp.TP_ENOTREADY
        tp.tp_prefetch_block(g.e, g.beam, host[0])
        with pytest.raises(tp.TpError) as ei:
            tp.tp_prefetch_block(g.e, g.beam, host[1])
        assert ei.value.code == tp.TP_EBUSY
        with pytest.raises(tp.TpError) as ei:
            tp.tp_push_block(g.e, g.beam, blocks[0])
        assert ei.value.code == tp.TP_EBUSY
        tp.tp_push_prefetched(g.e, g.beam)
        tp.tp_dedisperse(g.e, g.beam)
        tp.tp_detect(g.e, g.beam)
        for k in range(1, nblk + 1):
            if k < nblk:
                tp.tp_prefetch_block(g.e, g.beam, host[k])  # overlaps block k - 1
            got.append(collect(g))
            if k < nblk:
                tp.tp_push_prefetched(g.e, g.beam)
                tp.tp_dedisperse(g.e, g.beam)
                tp.tp_detect(g.e, g.beam)
    finally:
        g.close()

    for k, (r, q) in enumerate(zip(ref, got)):
        assert r["info"]["t0_abs"] == q["info"]["t0_abs"], k
        for f in ("D", "mu", "sigma", "chunk_flag", "chunk_raw", "spec_flag", "row_mu", "row_sigma"):
            assert np.array_equal(r[f], q[f]), (k, f)
        assert r["n_candidates"] == q["n_candidates"], k
        for f in ("dm_idx", "t_abs", "snr", "value"):
            assert np.array_equal(r["candidates"][f], q["candidates"][f]), (k, f)
    # and the stream's last block against the oracle's search of its window
    assert sum(r["n_candidates"] for r in got) > 0
    last = got[-1]
    w0 = last["info"]["t0_abs"]
    win = np.ascontiguousarray(x[:, w0:w0 + dmax + B])
    o = O.search_block(win, dtype, od, dmax, rfi=O.RfiParams(), t0=w0)
    check_block(last, o, win, dtype, od, O.RfiParams(), 5.0, t0=w0)


def test_candidate_capacity_and_truncation():
    nchan = 64
    dms = np.arange(16) * 2.0
    x = synth.noise(nchan, 6000, 9101)
    rfi = O.RfiParams(enable_channel=False, enable_spectrum=False)
    g = GpuBeam(nchan, 398.0, 20.0, 51.2e-6, dms, "f32", rfi=rfi, nsigma=2.0, cap=10)
    try:
        r = g.run(x)
        assert r["rc"] == tp.TP_EOVERFLOW and r["n_candidates"] > 10
        assert len(r["candidates"]) == 10
        c2, n2, rc2 = tp.tp_get_candidates(g.e, g.beam, 3)
        assert len(c2) == 3 and n2 == r["n_candidates"]
        assert np.array_equal(c2, r["candidates"][:3])
    finally:
        g.close()
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    o = O.search_block(x, "f32", od, dmax, rfi=rfi, nsigma=2.0)
    first = [(int(c["dm_idx"]), int(c["t_abs"])) for c in o["candidates"][:10]]
    assert [(int(c["dm_idx"]), int(c["t_abs"])) for c in r["candidates"]] == first


def test_device_buffer_push_and_errors():
    import torch
    nchan = 32
    dms = np.arange(8) * 4.0
    x = synth.noise(nchan, 4000, 9201)
    rfi = O.RfiParams()
    g = GpuBeam(nchan, 398.0, 20.0, 51.2e-6, dms, "f32", rfi=rfi)
    try:
        g.open(4000)
        with pytest.raises(tp.TpError) as ei:
            tp.tp_dedisperse(g.e, g.beam)
        assert ei.value.code == tp.TP_ENOTREADY
        with pytest.raises(tp.TpError) as ei:
            tp.tp_push_block(g.e, g.beam, x[:, :10].copy())
        assert ei.value.code == tp.TP_EINVAL
        xt = torch.from_numpy(x).cuda()
        tp.tp_push_block(g.e, g.beam, xt)
        with pytest.raises(tp.TpError) as ei:
            tp.tp_push_block(g.e, g.beam, xt)
        assert ei.value.code == tp.TP_EBUSY
        tp.tp_dedisperse(g.e, g.beam)
        tp.tp_detect(g.e, g.beam)
        c, n, rc = tp.tp_get_candidates(g.e, g.beam, 100)
        D = tp.tp_get_series(g.e, g.beam, ndm=8)
    finally:
        g.close()
    r2, o, od = run_both(x, "f32", nchan, 398.0, 20.0, 51.2e-6, dms, rfi)
    assert np.array_equal(D, r2["D"])


def test_admission_by_footprint():
    budget = 256 << 20
    e = tp.tp_engine_create(0, hbm_budget_bytes=budget)
    try:
        p = tp.tp_create_plan(e, 1024, 398.0, 20.0, 51.2e-6, np.arange(64) * 1.0, "f32")
        need = tp.tp_beam_footprint(p, 32768, 1000)
        small = tp.tp_beam_footprint(p, 4000, 10)
        assert small < budget < need
        with pytest.raises(tp.TpError) as ei:
            tp.tp_beam_open(e, p, 32768, 1000)
        assert ei.value.code == tp.TP_EADMIT
        used, b_ = tp.tp_engine_memory(e)
        assert used < b_ == budget
        b = tp.tp_beam_open(e, p, 4000, 10)
        assert tp.tp_engine_memory(e)[0] == used + small
        tp.tp_beam_close(e, b)
        assert tp.tp_engine_memory(e)[0] == used
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)

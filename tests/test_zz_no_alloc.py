"""The statistics entry point that allocates nothing (tp_channel_stats_noalloc)
agrees with the engine's own A1-A2 results (tp_dedisperse on a beam, read back
with tp_get_bandpass / tp_get_masks) on two calls in a row, each on a new
block, so that the second call runs on scratch holding the first call's data.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import paper_1307_5700_gb300 as tp
import synth

pytestmark = pytest.mark.gpu


def _block(dtype, seed, nchan, nsamp):
    if dtype == "c16":
        # complex voltages whose power carries the same narrowband burst
        env = np.ones((nchan, nsamp))
        env[[3, 4, 40], 2000:6000] += 3.0
        env[:, [9000, 15000]] += 6.0
        return synth.complex_voltage(env, seed, sigma=30.0)
    xf = synth.noise(nchan, nsamp, seed, mean=128.0 if dtype == "u8" else 0.0, std=16.0 if dtype == "u8" else 1.0)
    scale = 16.0 if dtype == "u8" else 1.0
    synth.add_narrowband(xf, [3, 4, 40], 2000, 6000, 12.0 * scale)
    synth.add_broadband(xf, [9000, 15000], 6.0 * scale)
    return {"u8": synth.to_u8, "f32": lambda a: a, "f16": synth.to_f16, "bf16": synth.to_bf16_bits}[dtype](xf)


def _to_device(x):
    """The block as a device tensor of the same bytes (bfloat16 bit patterns
    as int16, complex int16 pairs as one int32 per sample)."""
    import torch
    if x.dtype == synth.C16:
        x = x.view(np.int32)
    elif x.dtype == np.uint16:
        x = x.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _engine_stats(x, dtype, rfi):
    """A1-A2 through the existing path: one beam, one block."""
    nchan, nsamp = x.shape
    e = tp.tp_engine_create(0)
    try:
        p = tp.tp_create_plan(e, nchan, 398.0, 20.0, 51.2e-6, np.arange(8) * 1.0, dtype, rfi, 5.0)
        b = tp.tp_beam_open(e, p, nsamp, 16)
        tp.tp_push_block(e, b, x)
        tp.tp_dedisperse(e, b)
        mu, sigma = tp.tp_get_bandpass(e, b, nchan)
        cf, cr, _ = tp.tp_get_masks(e, b, nchan)
        tp.tp_beam_close(e, b)
        tp.tp_plan_destroy(p)
    finally:
        tp.tp_engine_destroy(e)
    return mu, sigma, cf, cr


@pytest.mark.parametrize("dtype", ["f32", "u8", "f16", "bf16", "c16"])
def test_noalloc_stats_match_engine_twice(dtype):
    import torch
    tp.build()
    nchan, nsamp = 256, 20000
    rfi = tp.tp_rfi_defaults()
    rfi.dilate_channels = 1
    nchunk = (nsamp + rfi.chunk_width - 1) // rfi.chunk_width
    mu = torch.empty(nchan, dtype=torch.float64, device="cuda")
    sigma = torch.empty_like(mu)
    cf = torch.empty((nchan, nchunk), dtype=torch.uint8, device="cuda")
    cr = torch.empty_like(cf)
    for call, seed in enumerate((301, 302)):
        x = _block(dtype, seed, nchan, nsamp)
        want_mu, want_sigma, want_cf, want_cr = _engine_stats(x, dtype, rfi)
        assert want_cf.any()
        xd = _to_device(x)
        tp.tp_channel_stats_noalloc(xd, dtype, mu, sigma, cf, cr, rfi=rfi)
        torch.cuda.synchronize()
        np.testing.assert_allclose(mu.cpu().numpy(), want_mu, rtol=1e-12, atol=1e-12, err_msg=f"call {call}")
        np.testing.assert_allclose(sigma.cpu().numpy(), want_sigma, rtol=1e-12, atol=1e-12, err_msg=f"call {call}")
        assert np.array_equal(cf.cpu().numpy(), want_cf), f"chunk flags, call {call}"
        assert np.array_equal(cr.cpu().numpy(), want_cr), f"exceedances, call {call}"


def test_noalloc_rejects_oversized_block():
    """Sizes beyond the fixed scratch are refused on the host, before any
    kernel runs (x is never read)."""
    import ctypes

    import torch
    tp.build()
    x = torch.zeros((4096, 8), dtype=torch.float32, device="cuda")
    out = torch.zeros(4096, dtype=torch.float64, device="cuda")
    flags = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    rfi = tp.tp_rfi_defaults()
    rfi.chunk_width = 1
    # 4096 channels x 2^20 one-sample chunks: 64 GiB of chunk sums
    rc = tp.lib().tp_channel_stats_noalloc(x.data_ptr(), tp.TP_F32, 4096, 1 << 20, 1 << 20, ctypes.byref(rfi),
                                           out.data_ptr(), out.data_ptr(), flags.data_ptr(), flags.data_ptr(),
                                           None)
    assert rc == tp.TP_EINVAL
    assert "scratch" in tp.tp_last_error_string()

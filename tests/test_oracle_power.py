"""Pins of the oracle's power detection (reading R12: complex voltages, 16 bits
per component, detected as |v|^2 = re^2 + im^2 before the float path): the
power of single samples, the bandpass against numpy, and the whole chain on
complex voltages equal to the binary32 chain on their power."""
import numpy as np

import synth
from oracle import oracle as O


def _power(x):
    return x["re"].astype(np.int64) ** 2 + x["im"].astype(np.int64) ** 2


def test_power_of_single_samples():
    x = np.zeros((1, 4), O.C16)
    x["re"] = [3, -32768, 0, 7]
    x["im"] = [-4, -32768, 0, 0]
    mu = O.bandpass(x, "c16")["mu"][0]
    assert mu == (25 + 2 ** 31 + 0 + 49) / 4


def test_power_bandpass_against_numpy():
    env = np.ones((5, 3001), np.float32)
    x = synth.complex_voltage(env, 31, sigma=50.0)
    st = O.bandpass(x, "c16")
    p = _power(x).astype(np.float64)
    np.testing.assert_allclose(st["mu"], p.mean(axis=1), rtol=1e-13)
    np.testing.assert_allclose(st["sigma"], p.std(axis=1), rtol=1e-11)
    # the expected power of the generator is 2 sigma^2 (one sigma^2 per part)
    assert np.all(np.abs(st["mu"] / (2 * 50.0 ** 2) - 1) < 0.05)


def test_chain_on_voltages_equals_chain_on_power():
    nchan, nsamp = 48, 3000
    dms = np.arange(12) * 2.0
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    env = np.ones((nchan, nsamp), np.float32)
    synth.add_pulse(env, od[7].astype(np.float64) + 1500, 15.0, 3.0)
    env[10:12, 400:700] += 20.0      # narrowband RFI
    env[:, 2200] += 8.0              # a broadband spike
    x = synth.complex_voltage(env, 77, sigma=25.0)
    p = _power(x)
    assert p.max() < 2 ** 24          # exact in binary32
    pf = p.astype(np.float32)
    rfi = O.RfiParams(chunk_width=100)
    a = O.search_block(x, "c16", od, dmax, rfi=rfi, nsigma=4.0)
    b = O.search_block(pf, "f32", od, dmax, rfi=rfi, nsigma=4.0)
    for k in ("chunk_raw", "chunk_flag", "spec_flag", "D"):
        assert np.array_equal(a[k], b[k]), k
    assert a["chunk_flag"].any() and a["spec_flag"].any()
    assert np.array_equal(a["candidates"], b["candidates"]) and a["n_candidates"] > 0
    d, t = np.unravel_index(np.argmax(a["D"]), a["D"].shape)
    assert abs(d - 7) <= 1 and abs(t - 1500) <= 8

"""Pins of the oracle's fitted bandpass (Sec. 2.2.1 "Bandpass Correction",
reading R13): an exact polynomial is reproduced, the Legendre least squares
agree with an independent monomial fit, high-power channels are masked and
interpolated before the fit, and the channel stage compares chunk means with
the fit plus tau times its RMSE."""
import numpy as np

import synth
from oracle import oracle as O


def test_exact_polynomial_is_reproduced():
    n = 300
    c = np.arange(n, dtype=np.float64)
    mu = 2.0 + 0.01 * c - 3e-5 * c ** 2 + 1e-8 * c ** 3
    f = O.bandpass_fit(mu, 3, 5.0)
    assert not f["masked"].any()
    np.testing.assert_allclose(f["b"], mu, rtol=1e-12, atol=1e-12)
    assert f["rmse"] < 1e-12


def test_legendre_fit_equals_monomial_fit():
    g = np.random.default_rng(4)
    n = 257
    mu = np.cos(np.arange(n) / 40.0) + 0.05 * g.standard_normal(n) + 10.0
    for order in (1, 2, 4, 6):
        f = O.bandpass_fit(mu, order, 50.0)
        assert not f["masked"].any()
        x = (2.0 * np.arange(n) - (n - 1)) / (n - 1)
        ref = np.polyval(np.polyfit(x, mu, order), x)
        np.testing.assert_allclose(f["b"], ref, rtol=0, atol=1e-9)
        assert abs(f["rmse"] - np.sqrt(np.mean((ref - mu) ** 2))) < 1e-9


def test_high_power_channels_are_masked_and_interpolated():
    g = np.random.default_rng(5)
    n = 200
    base = 5.0 + 0.002 * np.arange(n) + 0.01 * g.standard_normal(n)
    mu = base.copy()
    mu[50] += 3.0            # one channel of strong RFI
    mu[120:122] += 2.0       # two adjacent ones
    mu[0] += 1.5             # a band edge
    f = O.bandpass_fit(mu, 2, 6.0)
    assert set(np.nonzero(f["masked"])[0]) == {0, 50, 120, 121}
    assert f["mu_interp"][50] == (mu[49] + mu[51]) / 2
    assert f["mu_interp"][120] == (mu[119] + mu[122]) / 2
    assert f["mu_interp"][121] == (mu[119] + mu[122]) / 2
    assert f["mu_interp"][0] == mu[1]
    # the fit is that of the interpolated bandpass, so the RFI does not move it
    clean = O.bandpass_fit(f["mu_interp"], 2, 1e9)
    np.testing.assert_allclose(f["b"], clean["b"], rtol=0, atol=1e-12)
    assert np.abs(f["b"] - (5.0 + 0.002 * np.arange(n))).max() < 0.01


def test_channel_test_against_fit_plus_rmse():
    # 3 channels x 4 chunks of W = 10: chunk means chosen around b + tau rmse
    W, tau = 10, 3.0
    mu = np.array([1.0, 1.0, 1.0])
    x = np.ones((3, 40), np.float32)
    fit = O.bandpass_fit(np.array([1.0, 1.0, 1.0]), 0, 5.0)
    assert fit["rmse"] == 0.0
    fit["rmse"] = 0.5                       # threshold: chunk mean > 1 + 1.5
    x[0, 0:10] = 2.6                        # above: flagged
    x[1, 10:20] = 2.4                       # below: not flagged
    x[2, 30:40] = 2.5                       # equal: not flagged ("exceeds")
    st = dict(mu=mu, sigma=np.ones(3), external=True, fit=fit, b=np.ones(3))
    rfi = O.RfiParams(chunk_width=W, tau_channel=tau)
    raw, flag = O.channel_mask(x, "f32", st, rfi)
    assert raw.tolist() == [[1, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]]
    assert flag.tolist() == [[1, 1, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]]


def test_search_block_with_fit_flags_rfi_and_finds_pulse():
    nchan, nsamp = 96, 6000
    dms = np.arange(24) * 1.0
    od, dmax = O.delay_table(nchan, 398.0, 20.0, 51.2e-6, dms)
    x = synth.noise(nchan, nsamp, 12)
    x += (3.0 + np.linspace(-1, 1, nchan) ** 2)[:, None].astype(np.float32)   # a curved bandpass
    x[30] += 6.0                                                               # a high-power channel
    synth.add_narrowband(x, [70, 71], 2000, 2600, 4.0)                         # a burst
    synth.add_pulse(x, od[12].astype(np.float64) + 3500, 15.0, 1.2)
    rfi = O.RfiParams(tau_channel=40.0)
    o = O.search_block(x, "f32", od, dmax, rfi=rfi, nsigma=6.0, fit=(2, 5.0))
    st = o["stats"]
    # the high-power channel and the burst's channels (their block means rise
    # well above their neighbours') are masked before the fit
    assert np.nonzero(st["fit"]["masked"])[0].tolist() == [30, 70, 71]
    W = rfi.chunk_width
    assert o["chunk_flag"][70, 2000 // W + 1] and o["chunk_flag"][71, 2000 // W + 1]
    assert o["chunk_flag"][30].all()
    d, t = np.unravel_index(np.argmax(o["D"]), o["D"].shape)
    assert abs(d - 12) <= 1 and abs(t - 3500) <= 10
    # u8: the same chain with the integer bandpass value floor(fit + 1/2)
    xu = synth.to_u8(x * 16.0 + 64.0)
    ou = O.search_block(xu, "u8", od, dmax, rfi=rfi, nsigma=6.0, fit=(2, 5.0))
    assert np.array_equal(ou["stats"]["b"], np.floor(ou["stats"]["fit"]["b"] + 0.5).astype(np.int64))
    assert ou["chunk_flag"][30].all()

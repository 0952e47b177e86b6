"""Pins of the oracle's post-processing (Sec. 2.2.3, reading R11): the median
filter of Eq. 2 against a brute force and the filter's defining properties,
the detrending against a library least-squares fit and a direct two-pass
residual, and the detrended detection against a brute force."""
import numpy as np
import pytest

from oracle import oracle as O


def _median_brute(row, w):
    h = w // 2
    T = len(row)
    out = []
    for m in range(T):
        vals = sorted(row[min(max(m + i, 0), T - 1)] for i in range(-h, h + 1))
        out.append(vals[h])
    return out


@pytest.mark.parametrize("w", [1, 3, 5, 7, 9])
def test_median_matches_brute_force(w):
    g = np.random.default_rng(11 + w)
    Df = g.standard_normal((3, 57))
    Di = g.integers(-1000, 1000, (3, 57)).astype(np.int64)
    for D in (Df, Di):
        got = O.median_filter(D, w)
        assert got.dtype == D.dtype
        for d in range(D.shape[0]):
            assert list(got[d]) == _median_brute(list(D[d]), w)


def test_median_defining_properties():
    g = np.random.default_rng(5)
    x = g.standard_normal((1, 200))
    # w = 1 is the identity; a monotone series and a constant one are roots
    assert np.array_equal(O.median_filter(x, 1), x)
    mono = np.sort(x, axis=1)
    assert np.array_equal(O.median_filter(mono, 7), mono)
    const = np.full((2, 30), 4.25)
    assert np.array_equal(O.median_filter(const, 5), const)
    # an isolated outlier of up to h samples disappears; a plateau of h + 1
    # samples survives (the edge-preserving property that motivates the median)
    base = np.zeros((1, 60))
    spike = base.copy()
    spike[0, 30:32] = 100.0
    assert np.array_equal(O.median_filter(spike, 5), base)
    plateau = base.copy()
    plateau[0, 30:33] = 100.0
    assert np.array_equal(O.median_filter(plateau, 5), plateau)
    # the output is always one of the window's own values (no arithmetic)
    y = O.median_filter(x, 9)
    assert np.isin(y, x).all()


def test_median_rejects_even_or_oversized_width():
    with pytest.raises(ValueError):
        O.median_filter(np.zeros((1, 10)), 4)
    with pytest.raises(ValueError):
        O.median_filter(np.zeros((1, 10)), 65)


def test_detrend_matches_least_squares_and_direct_residual():
    g = np.random.default_rng(21)
    T = 5001
    t = np.arange(T, dtype=np.float64)
    D = np.stack([3.5 - 0.002 * t + g.standard_normal(T) * 2.0,
                  g.standard_normal(T) * 7.0 + 40.0,
                  1e-3 * t + 0.5 * np.sin(t / 37.0)])
    st = O.detrend(D)
    for d in range(D.shape[0]):
        slope, icpt = np.polyfit(t, D[d], 1)
        # the oracle's line is mean + beta (2t - (T - 1))
        assert abs(2.0 * st["beta"][d] - slope) <= 1e-10 * (abs(slope) + 1e-6)
        assert abs(st["mean"][d] - st["beta"][d] * (T - 1) - icpt) <= 1e-9 * (abs(icpt) + 1.0)
        r = D[d] - (icpt + slope * t)
        assert abs(st["sigma"][d] - np.sqrt(np.mean(r * r))) <= 1e-9 * st["sigma"][d]


def test_detrend_integer_sums_are_exact():
    g = np.random.default_rng(8)
    T = 777
    D = g.integers(-300000, 300000, (4, T)).astype(np.int64)
    st = O.detrend(D)
    u = [2 * t - (T - 1) for t in range(T)]
    for d in range(4):
        row = [int(v) for v in D[d]]
        assert st["sums"][d][0] == sum(row)
        assert st["sums"][d][1] == sum(ui * v for ui, v in zip(u, row))
        assert st["sums"][d][2] == sum(v * v for v in row)
    sf = O.detrend(D.astype(np.float64))
    np.testing.assert_allclose(st["mean"], sf["mean"], rtol=1e-12)
    np.testing.assert_allclose(st["beta"], sf["beta"], rtol=1e-12)
    np.testing.assert_allclose(st["sigma"], sf["sigma"], rtol=1e-9)


def test_detrended_detection():
    T = 4000
    t = np.arange(T, dtype=np.float64)
    g = np.random.default_rng(3)
    # a pure line has no residual: nothing is detected
    line = np.stack([2.0 + 0.01 * t])
    st = O.detrend(line)
    assert st["sigma"][0] <= 1e-9
    assert O.candidates_detrend(line, st["mean"], st["beta"], np.zeros(1), 5.0)[1] == 0
    # a pulse on a strong drift: found after detrending, hidden without it
    y = 0.05 * t + g.standard_normal(T)
    y[2500:2504] += 12.0
    Y = y[None, :]
    st = O.detrend(Y)
    c, n = O.candidates_detrend(Y, st["mean"], st["beta"], st["sigma"], 6.0)
    assert n >= 1 and set(c["t_abs"]) <= set(range(2500, 2504))
    ss = O.series_stats(Y)
    plain, _ = O.candidates(Y, ss["mu"], ss["sigma"], 6.0)
    assert not any(2500 <= tt < 2504 for tt in plain["t_abs"])
    # against a brute force on a small case, ints and floats
    for D in (g.integers(-50, 50, (3, 64)).astype(np.int64), g.standard_normal((3, 64))):
        st = O.detrend(D)
        cands, n = O.candidates_detrend(D, st["mean"], st["beta"], st["sigma"], 1.5, beam=2, t0=100)
        want = []
        for d in range(3):
            for tt in range(64):
                lin = st["mean"][d] + st["beta"][d] * float(2 * tt - 63)
                r = float(D[d, tt]) - lin
                if st["sigma"][d] > 0 and r >= 1.5 * st["sigma"][d]:
                    want.append((d, 100 + tt, np.float32(r / st["sigma"][d])))
        assert n == len(want)
        assert [(int(c["dm_idx"]), int(c["t_abs"]), c["snr"]) for c in cands] == want
        assert np.all(cands["beam"] == 2)


def test_post_process_composition():
    g = np.random.default_rng(9)
    D = g.integers(-40, 40, (2, 300)).astype(np.int64)
    out = O.post_process(D, median_width=5, detrend_on=True, nsigma=2.0)
    Y = O.median_filter(D, 5)
    assert np.array_equal(out["Y"], Y)
    st = O.detrend(Y)
    assert np.array_equal(out["stats"]["sigma"], st["sigma"])
    plain = O.post_process(D, nsigma=2.0)
    assert np.array_equal(plain["Y"], D)
    ss = O.series_stats(D)
    assert plain["n_candidates"] == O.candidates(D, ss["mu"], ss["sigma"], 2.0)[1]

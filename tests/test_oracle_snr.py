"""Pins of the oracle's spectral S/N (Sec. 2.2 item 1, Eq. 1 and its footnote).

The trend and the robust sigma are checked against NumPy/SciPy library
reductions (histogram, median, interp, median_abs_deviation) on crafted
spectra; the Sturges bin count against hand-computed values.
"""
import math

import numpy as np
import pytest
from scipy.stats import median_abs_deviation

import oracle
from oracle import snr as osn


@pytest.mark.parametrize("n,expect", [(2, 2), (10, 4), (100, 8), (1000, 11), (4436, 13),
                                       (20000, 15), (650000, 20)])
def test_sturges_hand_values(n, expect):
    # N = 1 + 3.322 log10(n), rounded: 4436 -> 13.11 -> 13, 1000 -> 10.97 -> 11
    assert osn.sturges_nbins(n) == expect


def _crafted(n, seed):
    rng = np.random.default_rng(seed)
    f = np.sort(rng.uniform(0.05, 3.0, n))
    sr = 1e-7 * (3.0 - f) + rng.gamma(2.0, 1e-8, n)
    spikes = rng.choice(n, 5, replace=False)
    sr[spikes] += 5e-6
    return f, sr


@pytest.mark.parametrize("n,seed", [(997, 1), (4436, 2), (5000, 3)])
def test_trend_matches_library_median_interp(n, seed):
    f, sr = _crafted(n, seed)
    nb = osn.sturges_nbins(n)
    trend, xs, ys = osn.trend_curve(f, sr)
    counts, edges = np.histogram(f, bins=nb, range=(f[0], f[-1]))
    # same membership as equal-width bins (f sorted -> contiguous runs)
    idx = osn.bin_index(f, nb)
    assert np.array_equal(np.bincount(idx, minlength=nb), counts)
    starts = np.concatenate([[0], np.cumsum(counts)])
    centres = 0.5 * (edges[:-1] + edges[1:])
    lib_x, lib_y = [], []
    for i in range(nb):
        if counts[i]:
            lib_x.append(centres[i])
            lib_y.append(np.median(sr[starts[i]:starts[i + 1]]))
    np.testing.assert_allclose(xs, lib_x, rtol=1e-13)
    np.testing.assert_allclose(ys, lib_y, rtol=1e-13)
    np.testing.assert_allclose(trend, np.interp(f, lib_x, lib_y), rtol=1e-10)


def test_sigma_is_scaled_mad():
    f, sr = _crafted(3001, 7)
    snr, trend, sigma = osn.spectral_snr(f, sr)
    # SciPy's normal-consistent MAD scale is 1/Phi^-1(3/4) = 1.482602...
    assert sigma == pytest.approx(median_abs_deviation(sr, scale="normal"), rel=1e-5)
    np.testing.assert_allclose(snr, (sr - trend) / sigma, rtol=1e-12)
    _, _, s2 = osn.spectral_snr(f, sr, mad_mode="resid")
    assert s2 == pytest.approx(median_abs_deviation(sr - trend, scale="normal"), rel=1e-5)


def test_empty_bins_are_skipped():
    f = np.concatenate([np.linspace(0.1, 0.2, 50), np.linspace(0.9, 1.0, 50)])
    sr = np.concatenate([np.full(50, 2.0), np.full(50, 4.0)])
    trend, xs, ys = osn.trend_curve(f, sr)
    assert len(xs) < osn.sturges_nbins(100)
    assert trend[0] == 2.0 and trend[-1] == 4.0
    mid = (f > xs[0]) & (f < xs[-1])
    assert np.all((trend[mid] >= 2.0) & (trend[mid] <= 4.0))


def test_zero_mad_gives_no_candidate():
    f = np.linspace(0.1, 1.0, 100)
    sr = np.full(100, 3e-8)
    snr, _, sigma = osn.spectral_snr(f, sr)
    assert sigma == 0.0 and np.all(snr == 0)


def test_linear_spectrum_detrends_to_spikes():
    # a perfectly linear spectrum is reproduced by the binned-median trend away
    # from the ends, so only the spikes stand out
    f = np.linspace(0.1, 2.0, 4001)
    sr = 1e-7 * (2.5 - f)
    sr[[500, 2000, 3500]] += 1e-6
    rng = np.random.default_rng(3)
    sr += rng.normal(0, 1e-10, f.shape[0])
    snr, trend, sigma = osn.spectral_snr(f, sr, mad_mode="resid")
    top = np.argsort(snr)[-3:]
    assert sorted(top.tolist()) == [500, 2000, 3500]


def test_top_peaks_separated_bumps_and_invariants():
    from oracle import snr as osn
    f = np.linspace(0.1, 3.0, 20000)
    centres = [0.35, 0.9, 1.7, 2.6]
    heights = [12.0, 30.0, 18.0, 9.0]
    v = sum(h * np.exp(-0.5 * ((f - c) / 0.004) ** 2) for c, h in zip(centres, heights))
    picks = osn.top_peaks(f, v, 4, sep=0.01)
    # the bumps' maxima in order of height
    order = np.argsort(heights)[::-1]
    assert [round(f[k], 2) for k in picks] == [round(centres[i], 2) for i in order]
    rng = np.random.default_rng(2)
    for _ in range(20):
        v = rng.normal(size=3000)
        f = np.sort(rng.uniform(0.1, 3, 3000))
        picks = osn.top_peaks(f, v, 8, sep=0.02)
        assert picks[0] == int(np.argmax(v))
        for a_ in range(len(picks)):
            for b_ in range(a_ + 1, len(picks)):
                assert abs(f[picks[b_]] / f[picks[a_]] - 1) >= 0.02
        # every pick is the maximum of what its predecessors left
        alive = np.ones(3000, bool)
        for k in picks:
            assert v[k] == v[alive].max()
            alive &= ~(np.abs(f / f[k] - 1) < 0.02)

"""Pins of the oracle's search plan (Sec. 2.1) against physics and closed forms.

None of these re-types the oracle's formulas: Kepler's third law is written
here with the stellar mass in SI units, the grid length is checked against a
numerical integral, and bin counts against hand-derived values.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle import plan as op

G = 6.67430e-11
RSUN = 6.957e8


def a_over_r_si(period_days, rho_gcc, r_rsun):
    """a/R* from a^3 = G M P^2 / (4 pi^2), M = 4/3 pi R^3 rho, in SI units."""
    r = r_rsun * RSUN
    mass = 4.0 / 3.0 * math.pi * r ** 3 * rho_gcc * 1000.0
    p = period_days * 86400.0
    return (G * mass * p * p / (4.0 * math.pi ** 2)) ** (1.0 / 3.0) / r


@pytest.mark.parametrize("rho", [0.1, 1.41, 10.0])
@pytest.mark.parametrize("a_r", [2.0, 3.0])
@pytest.mark.parametrize("r_rsun", [0.5, 1.0, 3.0])
def test_pmin_is_where_a_equals_pmin_aR_radii(rho, a_r, r_rsun):
    p = op.Params(pmin_aR=a_r)
    pmin = op.pmin_days(rho * 1000.0, p)
    assert a_over_r_si(pmin, rho, r_rsun) == pytest.approx(a_r, rel=1e-12)


def test_pmin_solar_density_value():
    # a = 2 R_sun around a solar-density star: P = 0.3276 d (7.86 h)
    assert op.pmin_days(1410.0, op.Params()) == pytest.approx(0.32761, abs=5e-5)


@pytest.mark.parametrize("a_r,expect", [(2.0, 1.0 / 6.0), (3.0, math.asin(1.0 / 3.0) / math.pi)])
def test_qcirc_at_pmin(a_r, expect):
    # central chord across the star seen from a = a_r R*: half-angle asin(R*/a)
    p = op.Params(pmin_aR=a_r)
    for rho in (0.3, 1.41, 7.0):
        pmin = op.pmin_days(rho * 1000.0, p)
        assert op.q_min(1.0 / pmin, rho * 1000.0, p) / p.qmin_fac == pytest.approx(expect, rel=1e-12)


def test_earth_transit_duration():
    # Earth seen transiting the Sun centrally lasts about 13 hours
    q = op.q_min(1.0 / 365.25, 1408.0, op.Params()) / 0.5
    assert q * 365.25 * 24.0 == pytest.approx(13.0, rel=0.02)


def test_qcirc_against_si_geometry():
    for period in (0.5, 3.7, 13.0, 80.0):
        for rho in (0.1, 1.41, 10.0):
            a_r = a_over_r_si(period, rho, 1.7)
            expect = math.asin(min(1.0, 1.0 / a_r)) / math.pi
            got = op.q_min(1.0 / period, rho * 1000.0, op.Params()) / 0.5
            assert got == pytest.approx(expect, rel=1e-10)


def _tp(*stretches, cadence=0.02):
    parts = [np.arange(a, b, cadence) for a, b in stretches]
    return np.concatenate(parts)


def test_pmax_single_stretch_is_half_baseline():
    tp = _tp((0.0, 27.4))
    assert op.pmax_days(tp, op.Params()) == pytest.approx((tp[-1] - tp[0]) / 2)
    # a 1-day mid-sector gap is not longer than a sector: still one stretch
    tp = _tp((0.0, 13.0), (14.0, 27.4))
    assert op.pmax_days(tp, op.Params()) == pytest.approx((tp[-1] - tp[0]) / 2)


def test_pmax_longest_stretch_when_long_gap():
    tp = _tp((0.0, 20.0), (50.0, 60.0))            # 30-day gap
    assert op.pmax_days(tp, op.Params()) == pytest.approx(tp[tp < 25][-1] - 0.0)
    tp = _tp((0.0, 5.0), (40.0, 70.0), (100.0, 110.0))
    seg = tp[(tp >= 40) & (tp < 70)]
    assert op.pmax_days(tp, op.Params()) == pytest.approx(seg[-1] - seg[0])


def test_pmax_gap_exactly_one_sector_is_not_a_split():
    tp = np.array([0.0, 1.0, 28.4, 29.0])          # gap of exactly 27.4 d
    assert op.pmax_days(tp, op.Params()) == pytest.approx(29.0 / 2)


def _qmin_si(f, rho, p):
    a_r = a_over_r_si(1.0 / f, rho, 1.0)
    return p.qmin_fac * math.asin(min(1.0, 1.0 / a_r)) / math.pi


@pytest.mark.parametrize("rho,baseline", [(1.41, 27.0), (0.1, 27.0), (10.0, 27.0), (1.41, 120.0)])
def test_grid_length_matches_integral(rho, baseline):
    # steps of q_min/(spp T): the count is the integral of spp T / q_min(f) df
    p = op.Params()
    pmin = op.pmin_days(rho * 1000.0, p)
    pmax = baseline / 2
    freqs = op.freq_grid(pmin, pmax, baseline, rho * 1000.0, p)
    integral, _ = quad(lambda f: p.samples_per_peak * baseline / _qmin_si(f, rho, p),
                       1.0 / pmax, 1.0 / pmin, limit=400)
    assert abs(len(freqs) - integral) <= 0.005 * integral + 2


def test_grid_endpoints_and_spacing_direction():
    p = op.Params()
    rho = 1410.0
    pmin = op.pmin_days(rho, p)
    freqs = op.freq_grid(pmin, 13.7, 27.4, rho, p)
    assert freqs[0] == 1.0 / 13.7
    assert freqs[-1] <= 1.0 / pmin
    assert np.all(np.diff(freqs) > 0)
    # the last step would have crossed 1/Pmin
    nxt = freqs[-1] + _qmin_si(freqs[-1], 1.41, p) / (2 * 27.4)
    assert nxt > 1.0 / pmin * (1 - 1e-9)


def test_single_star_grid_size():
    # one 27.4-d sector with a mid gap at 30-min cadence, solar density: ~4.4k frequencies
    import synth
    b = synth.single_star()
    pl = oracle.plan_batch(b)[0]
    assert pl.status == 0
    assert pl.pmax == pytest.approx(13.6875, abs=1e-9)     # half of 27.375 d baseline
    assert 4300 < pl.freqs.shape[0] < 4600


def test_nbins_and_duration_grid():
    p = op.Params()
    assert op.n_q(p) == 14                           # ln(4)/0.1 = 13.86 -> j = 0..13
    for qmin in (1.0 / 12.0, 0.03, 0.0071, 0.00123):
        nb = op.nbins_of(qmin, p)
        assert 3.0 <= qmin * nb < 3.0 + qmin + 1e-15
        m = op.m_of(qmin, nb, p)
        for j, mj in enumerate(m):
            qj = qmin * math.exp(0.1 * j)
            assert abs(mj - qj * nb) <= 0.5 + 1e-12
        assert m == sorted(m)
    # q_min * nbins just above 3: hand-derived widths round(3 e^{0.1 j})
    nb = 4000
    qmin = 3.0 / nb * (1 + 1e-9)
    assert op.m_of(qmin, op.nbins_of(qmin, p), p) == [3, 3, 4, 4, 4, 5, 5, 6, 7, 7, 8, 9, 10, 11]


def test_status_flags():
    p = op.Params()
    t = np.linspace(0, 10, 50) + 2000.0
    y = np.ones(50)
    dy = np.full(50, 1e-3)
    assert op.plan_star(t[::-1], y, dy, 1.41, 1.0, p).status == op.ST_UNSORTED
    assert op.plan_star(t[:1], y[:1], dy[:1], 1.41, 1.0, p).status == op.ST_TOO_FEW
    # a baseline too short for any period above Pmin
    assert op.plan_star(t[:3] * 0 + np.array([0, 0.1, 0.2]) + 2000, y[:3], dy[:3], 1.41, 1.0,
                        p).status == op.ST_EMPTY_GRID
    # non-finite values and dy <= 0 are dropped before anything else
    y2 = y.copy(); y2[3] = np.nan
    dy2 = dy.copy(); dy2[7] = 0.0
    pl = op.plan_star(t, y2, dy2, float("nan"), 1.0, p)
    assert pl.status == 0 and pl.tp.shape[0] == 48
    assert pl.rho_kg == 1410.0                      # solar density when missing
    small = op.Params(nbins_cap=50)
    assert op.plan_star(t, y, dy, 1.41, 1.0, small).status & op.ST_NBINS_CAP


def test_coarse_grid_log_spacing_and_clipping():
    p = op.Params(grid_mode=1)
    freqs, k0 = op.coarse_grid(0.3, 14.0, p)
    per = 1.0 / np.asarray(freqs)
    assert np.all(np.diff(freqs) > 0)
    assert per.min() >= 0.3 and per.max() <= 14.0
    # constant ratio between neighbours: (400 / 0.1)^(1/4095)
    r = per[:-1] / per[1:]
    np.testing.assert_allclose(r, 4000.0 ** (1 / 4095), rtol=1e-12)
    # the first entry is bin k0: P = 0.1 * 4000^(k0/4095)
    assert per[0] == pytest.approx(0.1 * 4000.0 ** (k0 / 4095), rel=1e-14)
    full, _ = op.coarse_grid(0.0, 1e9, p)
    assert len(full) == 4096 and 1.0 / full[-1] == pytest.approx(0.1) and 1.0 / full[0] == pytest.approx(400.0)


def test_window_grid_spacing_and_edges():
    # inside each window: starts at the window's low edge, steps q_min(f)/(spp T)
    # (q_min in SI units here), stops before leaving the window
    import synth
    b = synth.single_star()
    t, y, dy = b.star(0)
    p = op.Params()
    wins = [(0.27, 0.2712), (1.0, 1.004)]
    sub = oracle.plan_star(t, y, dy, 1.41, 1.0, windows=wins)
    T = sub.baseline
    f = np.asarray(sub.freqs)
    for lo, hi in wins:
        fw = f[(f >= lo) & (f <= hi)]
        assert fw[0] == lo and len(fw) > 3
        step = np.array([_qmin_si(x, 1.41, p) / (p.samples_per_peak * T) for x in fw])
        np.testing.assert_allclose(np.diff(fw), step[:-1], rtol=1e-9)
        assert fw[-1] + step[-1] > hi * (1 - 1e-12)
    assert len(f) == sum(((f >= lo) & (f <= hi)).sum() for lo, hi in wins)


def test_window_grid_merges_and_clips():
    import synth
    b = synth.single_star()
    t, y, dy = b.star(0)
    full = oracle.plan_star(t, y, dy, 1.41, 1.0)
    fmin, fmax = full.freqs[0], 1.0 / full.pmin
    # one window over the whole range (and beyond) is the plain grid
    whole = oracle.plan_star(t, y, dy, 1.41, 1.0, windows=[(0.0, 100.0)])
    assert whole.freqs.tolist() == full.freqs.tolist()
    # overlapping and touching windows act as their union; empty or reversed ones vanish
    a = oracle.plan_star(t, y, dy, 1.41, 1.0, windows=[(0.5, 0.52), (0.51, 0.53), (0.53, 0.54), (0.9, 0.8)])
    u = oracle.plan_star(t, y, dy, 1.41, 1.0, windows=[(0.5, 0.54)])
    assert a.freqs.tolist() == u.freqs.tolist() and a.freqs[0] == 0.5
    # a window below 1/Pmax starts at 1/Pmax, one above 1/Pmin is empty
    c = oracle.plan_star(t, y, dy, 1.41, 1.0, windows=[(fmin / 2, fmin * 1.01)])
    assert c.freqs[0] == fmin
    e = oracle.plan_star(t, y, dy, 1.41, 1.0, windows=[(fmax * 1.01, fmax * 2)])
    assert e.status == op.ST_EMPTY_GRID

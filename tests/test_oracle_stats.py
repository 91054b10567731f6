"""Pins of the post-BLS statistics oracle (Sec. 2.2 items 2-5): the trapezoid's
area and shape, its analytic Jacobian against finite differences, exact
recovery of a noise-free trapezoid, agreement with SciPy's bounded least
squares on noisy data, closed-form noise cases, brute-force counts and a
hand-computed signal-to-pink-noise value."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import stats as ost

P, T0, Q, QIN, DELTA, Z = 2.3, 0.7, 0.05, 0.2, 0.01, 1.0


def _times(span=10.0, cadence=0.002):
    return np.arange(0.0, span, cadence)


def test_trapezoid_area_and_shape():
    d = Q * P
    a = np.linspace(0.0, d, 200001)
    s = ost.shape(a, Q, QIN, P)
    # integral over the whole transit (both halves) = D (1 - q_in)
    area = 2.0 * np.trapezoid(s, a)
    assert area == pytest.approx(d * (1.0 - QIN), rel=1e-6)
    assert s[0] == 1.0 and s[-1] == 0.0
    mid_ramp = 0.5 * d - 0.5 * QIN * d
    assert ost.shape(np.array([mid_ramp]), Q, QIN, P)[0] == pytest.approx(0.5, abs=1e-12)
    assert ost.shape(np.array([0.5 * d]), Q, QIN, P)[0] == 0.0


def test_jacobian_matches_finite_differences():
    tp = _times()
    x = np.array([T0, DELTA, Q, QIN, Z])
    m, jac = ost.model_and_jacobian(tp, x, P)
    for i, h in enumerate([1e-7, 1e-9, 1e-9, 1e-8, 1e-9]):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (ost.model_and_jacobian(tp, xp, P)[0] - ost.model_and_jacobian(tp, xm, P)[0]) / (2 * h)
        # points near a kink of the piecewise-linear model are skipped
        dt, _ = ost.phase_distance(tp, T0, P)
        a = np.abs(dt)
        d = Q * P
        far = (np.abs(a - 0.5 * d) > 1e-5) & (np.abs(a - (0.5 - QIN) * d) > 1e-5)
        np.testing.assert_allclose(jac[far, i], fd[far], rtol=1e-5, atol=1e-6 * np.abs(jac[:, i]).max())


def test_noise_free_fit_recovers_parameters():
    tp = _times()
    x_true = np.array([T0, DELTA, Q, QIN, Z])
    y = ost.model_and_jacobian(tp, x_true, P)[0]
    dy = np.full(tp.shape, 1e-3)
    dt, _ = ost.phase_distance(tp, T0, P)
    win = np.abs(dt) <= 2 * Q * P
    x, chi2, it, conv = ost.fit_trapezoid(tp[win], y[win], dy[win], P, [T0 + 0.002, 0.008, 0.055, 0.1, 0.999])
    assert conv and chi2 < 1e-18
    np.testing.assert_allclose(x, x_true, rtol=1e-7, atol=1e-10)


def test_fit_agrees_with_scipy_bounded_least_squares():
    from scipy.optimize import least_squares
    rng = np.random.default_rng(3)
    tp = _times()
    x_true = np.array([T0, DELTA, Q, QIN, Z])
    dy = np.full(tp.shape, 2e-3)
    y = ost.model_and_jacobian(tp, x_true, P)[0] + rng.normal(0, 2e-3, tp.shape)
    dt, _ = ost.phase_distance(tp, T0, P)
    win = np.abs(dt) <= 2 * Q * P
    x0 = [T0 + 0.001, 0.009, 0.052, 0.1, 1.0]
    x, chi2, it, conv = ost.fit_trapezoid(tp[win], y[win], dy[win], P, x0)
    res = least_squares(lambda v: (y[win] - ost.model_and_jacobian(tp[win], v, P)[0]) / dy[win], x0,
                        bounds=([-np.inf, -np.inf, ost.Q_MIN, ost.Q_IN_MIN, -np.inf],
                                [np.inf, np.inf, 1.0, 0.5, np.inf]),
                        xtol=1e-15, ftol=1e-15, gtol=1e-15, method="trf")
    assert conv
    assert chi2 <= 2 * res.cost * (1 + 1e-9)
    np.testing.assert_allclose(x, res.x, rtol=2e-5, atol=2e-7)


def test_noise_closed_forms():
    tp = np.arange(0.0, 10.0, 0.01)
    d = 0.5                                   # 50 points per bin
    b = np.floor(tp / d).astype(int)
    c = 3e-3
    r = np.where(b % 2 == 0, c, -c)           # constant within each bin
    sw, sr = ost.noise_from_residuals(tp, r, d)
    assert sw == pytest.approx(c, rel=1e-12)
    assert sr == pytest.approx(c * math.sqrt(1 - 1 / 50), rel=1e-9)
    r2 = np.where(np.arange(len(tp)) % 2 == 0, c, -c)   # bin means are exactly 0
    sw2, sr2 = ost.noise_from_residuals(tp, r2, d)
    assert sw2 == pytest.approx(c, rel=1e-12) and sr2 == 0.0


def test_snr_pink_worked_value_and_counts():
    # delta 0.01, q_in 0.2: mean depth 0.008; sigma_w 1e-3 over 100 points -> 1e-8;
    # sigma_r 5e-4 over 4 transits -> 6.25e-8; 0.008 / sqrt(7.25e-8) = 29.711
    val = 0.008 / math.sqrt(1e-3 ** 2 / 100 + 5e-4 ** 2 / 4)
    assert val == pytest.approx(29.711, abs=1e-3)
    # counts of star_stats against loops over the points
    b = synth.single_star()
    t, y, dy = b.star(0)
    pl = oracle.plan_star(t, y, dy, 1.41, 1.0)
    res = oracle.bls_star(pl)
    snr, _, sigma = oracle.spectral_snr(pl.freqs, res.sr)
    best = oracle.best_candidate(pl, res, snr, sigma)
    st = ost.star_stats(pl, best)
    per, d = best["period"], st["q"] * best["period"]
    t0 = st["t0"] - pl.t_ref
    n_in = n_before = n_after = 0
    transits = set()
    for tt in pl.tp:
        k = math.floor((tt - t0) / per + 0.5)
        dt = tt - t0 - per * k
        n_in += abs(dt) < d / 2
        n_before += -2 * d <= dt < -d / 2
        n_after += d / 2 < dt <= 2 * d
        if abs(dt) <= d / 2:
            transits.add(k)
    assert (st["n_in"], st["n_before"], st["n_after"], st["n_transits"]) == (n_in, n_before, n_after,
                                                                             len(transits))
    # the injected 3.7-d, 2e-3 transit: recovered, detected, fitted depth close to the injected one
    assert st["status"] == ost.ST_OK and st["detected"] == 1
    assert abs(best["period"] / 3.7 - 1) < 0.01
    assert st["depth"] == pytest.approx(2e-3, rel=0.3) and st["n_transits"] >= 5
    assert st["snr_pink"] > 9


def test_no_candidate_and_few_points():
    pl = oracle.plan_star(np.linspace(0, 10, 50) + 2000, np.ones(50), np.full(50, 1e-3), 1.41, 1.0)
    assert ost.star_stats(pl, None)["status"] == ost.ST_NO_CANDIDATE
    fake = dict(period=3.0, t0=pl.t_ref + 0.5, q=1e-4, depth=0.01, snr=20.0)
    assert ost.star_stats(pl, fake)["status"] == ost.ST_FEW_POINTS

"""Oracle: post-BLS statistics of the best candidate (TEST INFRASTRUCTURE ONLY).

Sec. 2.2 items 2-5 of arXiv:2302.01293, restated step by step in FP64:

* trapezoid model (item 2): period P fixed to the BLS period; epoch T0, depth
  delta, duration fraction q (duration D = q P), ingress fraction q_in (ingress
  duration = q_in D) and out-of-transit level z. With a the distance of a point
  from the nearest mid-transit time, the transit shape is s(a) = 1 on the flat
  bottom a <= D/2 - q_in D, falls linearly to 0 at a = D/2, and is 0 outside;
  the model is y = z - delta s(a) (delta > 0 for a dip in flux).
* fit (item 2): weighted least squares (weights dy^-2) over the points within
  two transit durations of the transit centre (|a| <= 2 D0 for the BLS guess,
  a fixed set), bounds 0 < q <= 1 and 0 <= q_in <= 0.5, initial values from
  BLS. Readings: the optimiser is Levenberg-Marquardt as described below; the
  lower bound of q_in is 1e-3 (a box with 0.1 % ramps: the exact box has no
  derivative with respect to its edges); q >= 1e-6; initial q_in = 0.1; initial
  z = weighted mean of the window points outside the BLS box (all window
  points if none).
* noise (item 3): residuals of the fitted model over all points. Readings of
  the "VARTOOLS calculations": sigma_w = the RMS of the residuals; sigma_r from
  the residuals averaged in time bins of one fitted duration D (bins k D <=
  t' < (k+1) D, t' = t - t_min): with N_b the mean number of points of the
  occupied bins and sigma_b^2 the mean square of the occupied bins' averages,
  sigma_r^2 = max(0, sigma_b^2 - sigma_w^2 / N_b) (Pont et al. 2006).
* signal-to-pink noise (item 4, Eq. 2): S/N_pink = delta_eff /
  sqrt(sigma_w^2 / n_t + sigma_r^2 / N_t), where delta_eff replaces delta by
  the trapezoid's integral over the transit divided by its duration,
  delta (1 - q_in); n_t = points in transit (a < D/2), N_t = transits with at
  least one point within 0.5 D of the expected mid-transit time.
* other statistics (item 5): points in transit, before it (-2 D <= dt < -D/2)
  and after it (D/2 < dt <= 2 D), with D the fitted duration and dt the signed
  distance from the nearest mid-transit time; N_t; z.
* detection (Sec. 2.2, last paragraph): N_t >= 2, S/N_pink > 9 and S/N > 9.

Levenberg-Marquardt as used here (Marquardt 1963): at parameters x with
residuals r = (y - m) / dy and Jacobian J = d m / d x / dy, solve
(A + lam diag(max(A_ii, 1e-12 max_j A_jj))) h = J^T r with A = J^T J by
Gaussian elimination with partial pivoting; clip x + h to the bounds; accept
when chi^2 decreases (lam /= 10), else lam *= 10. Start lam = 1e-3. Stop after
an accepted step whose relative chi^2 decrease is below 1e-10, when lam
exceeds 1e10 (converged: no further decrease possible), or after 100
iterations (not converged).
"""
from __future__ import annotations

import math

import numpy as np

Q_IN_MIN = 1e-3
Q_MIN = 1e-6
Q_IN_INIT = 0.1
LAM0 = 1e-3
MAX_IT = 100
RTOL = 1e-10
LAM_MAX = 1e10

ST_OK, ST_NO_CANDIDATE, ST_FEW_POINTS, ST_NOT_CONVERGED = 0, 1, 2, 4


def phase_distance(tp, t0p, period):
    """dt = t' - T0' - P round((t' - T0') / P), round half up, and the transit index."""
    x = (np.asarray(tp, np.float64) - t0p) / period
    n = np.floor(x + 0.5)
    return np.asarray(tp, np.float64) - t0p - period * n, n.astype(np.int64)


def shape(a, q, q_in, period):
    """Trapezoid transit shape s(a) in [0, 1] at distance a >= 0 from mid-transit."""
    d = q * period
    t_in = q_in * d
    half = 0.5 * d
    s = np.zeros_like(a)
    flat = a <= half - t_in
    ramp = (~flat) & (a < half)
    s[flat] = 1.0
    s[ramp] = (half - a[ramp]) / t_in
    return s


def model_and_jacobian(tp, x, period):
    """Model y(t') and its derivatives with respect to x = (T0', delta, q, q_in, z)."""
    t0p, delta, q, q_in, z = x
    dt, _ = phase_distance(tp, t0p, period)
    a = np.abs(dt)
    d = q * period
    t_in = q_in * d
    half = 0.5 * d
    s = shape(a, q, q_in, period)
    m = z - delta * s
    jac = np.zeros((len(a), 5))
    ramp = (a > half - t_in) & (a < half)
    sign = np.sign(dt)
    # ds/da = -1/t_in on the ramp; da/dT0' = -sign(dt)
    jac[:, 0] = np.where(ramp, -delta * sign / t_in, 0.0)
    jac[:, 1] = -s
    # s = (q P / 2 - a) / (q_in q P) on the ramp: ds/dq = a / (q_in q^2 P), ds/dq_in = -s / q_in
    jac[:, 2] = np.where(ramp, -delta * a / (q_in * q * q * period), 0.0)
    jac[:, 3] = np.where(ramp, delta * s / q_in, 0.0)
    jac[:, 4] = 1.0
    return m, jac


def _solve(a, b):
    """Gaussian elimination with partial pivoting; None when singular."""
    n = len(b)
    m = np.concatenate([np.array(a, np.float64), np.array(b, np.float64)[:, None]], axis=1)
    for c in range(n):
        p = c + int(np.argmax(np.abs(m[c:, c])))
        if m[p, c] == 0.0:
            return None
        if p != c:
            m[[c, p]] = m[[p, c]]
        for r in range(c + 1, n):
            f = m[r, c] / m[c, c]
            m[r, c:] -= f * m[c, c:]
    x = np.zeros(n)
    for c in range(n - 1, -1, -1):
        x[c] = (m[c, n] - np.dot(m[c, c + 1:n], x[c + 1:])) / m[c, c]
    return x


def _clip(x):
    x = np.array(x, np.float64)
    x[2] = min(max(x[2], Q_MIN), 1.0)
    x[3] = min(max(x[3], Q_IN_MIN), 0.5)
    return x


def fit_trapezoid(tp, y, dy, period, x0):
    """Levenberg-Marquardt fit; returns (x, chi2, iterations, converged)."""
    tp = np.asarray(tp, np.float64); y = np.asarray(y, np.float64)
    w = 1.0 / np.asarray(dy, np.float64)
    x = _clip(x0)

    def evaluate(xx):
        m, jac = model_and_jacobian(tp, xx, period)
        r = (y - m) * w
        jw = jac * w[:, None]
        return float(np.dot(r, r)), jw.T @ jw, jw.T @ r

    chi2, a, g = evaluate(x)
    lam = LAM0
    it = 0
    converged = False
    while it < MAX_IT:
        it += 1
        dmax = float(np.max(np.diag(a))) if a.size else 0.0
        damp = np.maximum(np.diag(a), 1e-12 * dmax)
        h = _solve(a + lam * np.diag(damp), g)
        if h is not None:
            xn = _clip(x + h)
            chi2n, an, gn = evaluate(xn)
        if h is not None and chi2n < chi2:
            rel = (chi2 - chi2n) / chi2 if chi2 > 0.0 else 0.0
            x, chi2, a, g = xn, chi2n, an, gn
            lam /= 10.0
            if rel < RTOL:
                converged = True
                break
        else:
            lam *= 10.0
            if lam > LAM_MAX:
                converged = True
                break
    return x, chi2, it, converged


def noise_from_residuals(tp, r, duration):
    """(sigma_w, sigma_r) of residuals r at times t' (sorted), bins of one duration."""
    r = np.asarray(r, np.float64)
    sw = math.sqrt(float(np.mean(r * r))) if len(r) else 0.0
    if len(r) == 0 or not duration > 0.0:
        return sw, 0.0
    b = np.floor(np.asarray(tp, np.float64) / duration).astype(np.int64)
    bins, inv, counts = np.unique(b, return_inverse=True, return_counts=True)
    means = np.bincount(inv, weights=r) / counts
    nb_mean = len(r) / len(bins)
    sb2 = float(np.mean(means * means))
    return sw, math.sqrt(max(0.0, sb2 - sw * sw / nb_mean))


def star_stats(plan, best):
    """All statistics of one star's best candidate (best: oracle.best_candidate dict)."""
    out = dict(status=ST_NO_CANDIDATE, t0=0.0, depth=0.0, q=0.0, q_in=0.0, z=0.0, chi2=0.0, sigma_w=0.0,
               sigma_r=0.0, depth_mean=0.0, snr_pink=0.0, n_fit=0, n_in=0, n_before=0, n_after=0,
               n_transits=0, iterations=0, detected=0)
    if best is None:
        return out
    tp, y, dy = plan.tp, plan.y, plan.dy
    period = best["period"]
    t0p = best["t0"] - plan.t_ref
    q0, d0 = best["q"], best["depth"]
    dt, _ = phase_distance(tp, t0p, period)
    win = np.abs(dt) <= 2.0 * q0 * period
    out["n_fit"] = int(win.sum())
    if out["n_fit"] < 6:
        out["status"] = ST_FEW_POINTS
        return out
    wts = 1.0 / (dy[win] * dy[win])
    outside = np.abs(dt[win]) > 0.5 * q0 * period
    if outside.any():
        z0 = float(np.sum(wts[outside] * y[win][outside]) / np.sum(wts[outside]))
    else:
        z0 = float(np.sum(wts * y[win]) / np.sum(wts))
    x, chi2, it, conv = fit_trapezoid(tp[win], y[win], dy[win], period, [t0p, d0, q0, Q_IN_INIT, z0])
    t0f, delta, q, q_in, z = x
    m, _ = model_and_jacobian(tp, x, period)
    d = q * period
    sw, sr = noise_from_residuals(tp, y - m, d)
    dt, n = phase_distance(tp, t0f, period)
    a = np.abs(dt)
    n_in = int(np.sum(a < 0.5 * d))
    n_t = len(np.unique(n[a <= 0.5 * d]))
    depth_mean = delta * (1.0 - q_in)
    den = (sw * sw / n_in if n_in else 0.0) + (sr * sr / n_t if n_t else 0.0)
    snr_pink = depth_mean / math.sqrt(den) if (n_in and n_t and den > 0.0) else 0.0
    out.update(status=ST_OK if conv else ST_NOT_CONVERGED, t0=t0f + plan.t_ref, depth=delta, q=q, q_in=q_in, z=z,
               chi2=chi2, sigma_w=sw, sigma_r=sr, depth_mean=depth_mean, snr_pink=snr_pink, n_in=n_in,
               n_before=int(np.sum((dt >= -2.0 * d) & (dt < -0.5 * d))),
               n_after=int(np.sum((dt > 0.5 * d) & (dt <= 2.0 * d))), n_transits=n_t, iterations=it,
               detected=int(n_t >= 2 and snr_pink > 9.0 and best["snr"] > 9.0))
    return out

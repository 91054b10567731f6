"""Oracle: spectral S/N and best candidate (TEST INFRASTRUCTURE ONLY).

Sec. 2.2 item 1, Eq. 1: S/N(f) = (SR(f) - trend(f)) / sigma_SR, where
  * the trend is the spectrum median-binned into N = 1 + 3.322 log10(n) bins
    (Sturges, rounded to the nearest integer; n = number of spectral points)
    and linearly interpolated back onto every frequency;
  * sigma_SR = 1.4826 x the median absolute deviation of SR.
The strongest signal is the frequency of maximum S/N; its BLS box gives the
initial P, T0, q and depth (Sec. 2.2 item 2).

Readings of points the paper leaves open:
  * bins are equal-width in frequency over [f_0, f_{n-1}]; point k falls in
    bin min(N-1, floor((f_k - f_0) N / (f_{n-1} - f_0))); a bin's abscissa is
    its centre f_0 + (i + 1/2)(f_{n-1} - f_0)/N; empty bins are skipped;
  * even counts take the mean of the two middle values as the median;
  * the interpolation is piecewise linear between bin centres and constant
    beyond the first and last centre;
  * "MAD of SR" is taken literally: median |SR - median(SR)| (mad_mode "raw");
    mad_mode "resid" uses the detrended residual SR - trend instead;
  * sigma_SR = 0 gives S/N = 0 everywhere and no candidate;
  * ties in the S/N maximum go to the lowest frequency index;
  * T0 is the first mid-box time at or after t_min, depth = -s / (r (1 - r)).
"""
from __future__ import annotations

import math

import numpy as np

MAD_SCALE = 1.4826


def sturges_nbins(n: int) -> int:
    return int(math.floor(1.0 + 3.322 * math.log10(n) + 0.5))


def _median_sorted(v):
    v = sorted(v)
    n = len(v)
    if n % 2 == 1:
        return float(v[n // 2])
    return 0.5 * (float(v[n // 2 - 1]) + float(v[n // 2]))


def bin_index(freqs, nb):
    f0, f1 = float(freqs[0]), float(freqs[-1])
    span = f1 - f0
    out = np.zeros(len(freqs), np.int64)
    if span > 0.0:
        for k, f in enumerate(freqs):
            i = int(math.floor(((float(f) - f0) * nb) / span))
            out[k] = min(nb - 1, i)
    return out


def trend_curve(freqs, sr):
    """Sturges median-binned trend interpolated at every frequency; also returns
    the bin centres and medians that define it."""
    sr = np.asarray(sr, np.float64)
    n = sr.shape[0]
    nb = sturges_nbins(n)
    f0, f1 = float(freqs[0]), float(freqs[-1])
    span = f1 - f0
    idx = bin_index(freqs, nb)
    xs, ys = [], []
    for i in range(nb):
        members = sr[idx == i].tolist()
        if not members:
            continue
        xs.append(f0 + ((i + 0.5) * span) / nb)
        ys.append(_median_sorted(members))
    trend = np.empty(n)
    for k in range(n):
        f = float(freqs[k])
        if f <= xs[0]:
            trend[k] = ys[0]
        elif f >= xs[-1]:
            trend[k] = ys[-1]
        else:
            j = 0
            while not (xs[j] <= f < xs[j + 1]):
                j += 1
            slope = (ys[j + 1] - ys[j]) / (xs[j + 1] - xs[j])
            trend[k] = ys[j] + slope * (f - xs[j])
    return trend, np.asarray(xs), np.asarray(ys)


def spectral_snr(freqs, sr, mad_mode: str = "raw"):
    """(snr, trend, sigma). sigma == 0 yields snr == 0."""
    sr = np.asarray(sr, np.float64)
    n = sr.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros(0), 0.0
    trend, _, _ = trend_curve(freqs, sr)
    if mad_mode == "raw":
        base = sr
    elif mad_mode == "resid":
        base = sr - trend
    else:
        raise ValueError(mad_mode)
    med = _median_sorted(base.tolist())
    mad = _median_sorted(np.abs(base - med).tolist())
    sigma = MAD_SCALE * mad
    if sigma == 0.0:
        return np.zeros(n), trend, 0.0
    return (sr - trend) / sigma, trend, sigma


def best_candidate(plan, bls, snr, sigma, per_q=None):
    """Best (P, T0, q, depth) at the S/N maximum, or None when there is none.
    per_q = (noverlap, dlogq) for a spectrum of the per-duration binning variant,
    whose box j, k lies on histogram j (ceil(noverlap / q_j) bins, noverlap wide)."""
    n = len(snr)
    if n == 0 or sigma == 0.0:
        return None
    k = int(np.argmax(snr))            # first index of the maximum
    j = int(bls.j[k])
    if j < 0:
        return None
    f = float(plan.freqs[k])
    if per_q is None:
        nb = int(plan.nbins[k])
        m = int(plan.m[k, j])
    else:
        noverlap, dlogq = per_q
        nb = int(math.ceil(noverlap / (float(plan.qmin[k]) * math.exp(j * dlogq))))
        m = int(noverlap)
    kb = int(bls.k[k])
    period = 1.0 / f
    mid = (kb + 0.5 * m) / nb
    t0 = plan.t_ref + period * (mid - math.floor(mid))
    r, s = float(bls.r[k]), float(bls.s[k])
    return dict(f_idx=k, f=f, period=period, t0=t0, q=m / nb, depth=-s / (r * (1.0 - r)),
                sr=float(bls.sr[k]), snr=float(snr[k]), j=j, k=kb, m=m, nbins=nb)


def snr_from_trend(freqs, sr, xs, ys, sigma):
    """S/N of a spectrum against a given trend (nodes xs, ys, np.interp semantics)
    and sigma: the refined search of the learned proposal scores its few
    frequencies against the coarse spectrum's trend and sigma_SR."""
    if sigma == 0.0 or len(xs) == 0:
        return np.zeros(len(sr))
    trend = np.interp(np.asarray(freqs, np.float64), xs, ys)
    return (np.asarray(sr, np.float64) - trend) / sigma


def top_peaks(freqs, snr, n: int, sep: float = 0.01):
    """The n strongest peaks of an S/N spectrum (not in the paper; the basis of
    multiple candidates per star): repeatedly take the index of the largest S/N
    (ties: lowest index) among the frequencies not yet excluded, then exclude
    every frequency with |f / f_pick - 1| < sep. Returns up to n indices."""
    f = np.asarray(freqs, np.float64)
    v = np.asarray(snr, np.float64)
    alive = np.ones(len(v), bool)
    out = []
    for _ in range(n):
        if not alive.any():
            break
        cand = np.where(alive, v, -np.inf)
        k = int(np.argmax(cand))
        if not alive[k]:
            break
        out.append(k)
        alive &= ~(np.abs(f / f[k] - 1.0) < sep)
    return out

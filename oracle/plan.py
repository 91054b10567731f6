"""Oracle: per-star search plan (TEST INFRASTRUCTURE ONLY; see package docstring).

Every quantity here is plain FP64 scalar arithmetic through Python's ``math``
module (the C library's libm), one step per line, so that it can be read
against the paper:

* Sec. 2.1: stellar density from the TIC, solar density (1.41 g/cm^3) when it
  is missing; durations searched between 0.5 and 2.0 times the duration of a
  central circular orbit; samples_per_peak = 2, dlogq = 0.1, noverlap = 3
  (footnote of Sec. 2.1).
* Sec. 2.1: Pmin is the period at which a = 2 R* (3 R* for Sectors 59-60);
  Pmax is the length of the longest continuous stretch of data, or half of it
  when no gap is longer than one TESS sector (27.4 d).

Readings of points the paper leaves open:
  * circular-orbit duration fraction q_circ = asin(min(1, R*/a)) / pi, with
    a/R* = (G rho P^2 / (3 pi))^(1/3) from Kepler's third law (R* cancels);
  * frequency grid: f_0 = 1/Pmax, f_{k+1} = f_k + q_min(f_k) / (spp * T), kept
    while f <= 1/Pmin, T = t_max - t_min (phase drift across the baseline of at
    most q_min/spp per step);
  * bins: nbins(f) = ceil(noverlap / q_min(f)); durations q_j = q_min e^{j dlogq},
    j = 0 .. floor(ln(qmax_fac/qmin_fac)/dlogq), each covering
    m_j = max(1, floor(q_j nbins + 1/2)) bins;
  * points with a non-finite value or dy <= 0 are dropped; t must be
    non-decreasing after that, otherwise the star is flagged.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

G_SI = 6.67430e-11          # m^3 kg^-1 s^-2 (CODATA 2018)
DAY_S = 86400.0

# star status flags
ST_UNSORTED = 1
ST_TOO_FEW = 2
ST_EMPTY_GRID = 4
ST_NBINS_CAP = 8
ST_ZERO_MAD = 16


@dataclasses.dataclass
class Params:
    samples_per_peak: float = 2.0
    dlogq: float = 0.1
    noverlap: float = 3.0
    qmin_fac: float = 0.5
    qmax_fac: float = 2.0
    pmin_aR: float = 2.0
    gap_days: float = 27.4
    rho_default: float = 1.41
    nbins_cap: int = 8192
    # learned proposal (not in the paper): coarse log-period grid
    grid_mode: int = 0
    coarse_bins: int = 4096
    coarse_pmin: float = 0.1
    coarse_pmax: float = 400.0


@dataclasses.dataclass
class StarPlan:
    status: int
    t_ref: float            # t_min of the valid points
    baseline: float         # t_max - t_min
    pmin: float
    pmax: float
    rho_kg: float           # density in kg/m^3 used for the Keplerian limits
    tp: np.ndarray          # t - t_ref of the valid points (FP64)
    y: np.ndarray
    dy: np.ndarray
    freqs: np.ndarray       # trial frequencies (1/day), FP64
    qmin: np.ndarray        # q_min at each frequency
    nbins: np.ndarray       # int32
    m: np.ndarray           # int32 [n_f, n_q]
    grid_k0: int = -1       # coarse grid: bin index of the first (lowest) frequency


def n_q(p: Params) -> int:
    """Number of log-spaced durations from qmin_fac to (at most) qmax_fac times q_circ."""
    return int(math.floor(math.log(p.qmax_fac / p.qmin_fac) / p.dlogq + 1e-9)) + 1


def q_min(f: float, rho_kg: float, p: Params) -> float:
    """Smallest searched duration fraction at frequency f (1/day): qmin_fac * q_circ."""
    ps = DAY_S / f                                   # period in seconds
    x = G_SI * rho_kg * ps * ps / (3.0 * math.pi)    # (a/R*)^3 from Kepler's third law
    a_r = math.cbrt(x)
    q_circ = math.asin(min(1.0, 1.0 / a_r)) / math.pi
    return p.qmin_fac * q_circ


def freq_grid(pmin: float, pmax: float, baseline: float, rho_kg: float, p: Params) -> List[float]:
    """Frequencies from 1/Pmax to 1/Pmin, stepping by q_min(f) / (spp * T)."""
    fmax = 1.0 / pmin
    denom = p.samples_per_peak * baseline
    out = []
    f = 1.0 / pmax
    while f <= fmax:
        out.append(f)
        f = f + q_min(f, rho_kg, p) / denom
    return out


def coarse_grid(pmin: float, pmax: float, p: Params):
    """Coarse log-period grid of the learned proposal: P_k = coarse_pmin
    (coarse_pmax/coarse_pmin)^(k/(bins-1)), kept when Pmin <= P_k <= Pmax, returned
    in increasing frequency with the bin index of the first entry (-1 if none)."""
    ratio = p.coarse_pmax / p.coarse_pmin
    out, k0 = [], -1
    for k in range(p.coarse_bins - 1, -1, -1):
        per = p.coarse_pmin * (ratio ** (k / (p.coarse_bins - 1)))
        if per < pmin or per > pmax:
            continue
        if k0 < 0:
            k0 = k
        out.append(1.0 / per)
    return out, k0


def merge_windows(windows):
    """Union of frequency intervals [lo, hi]: sorted, with overlapping or touching
    intervals joined (empty or NaN intervals dropped)."""
    out = []
    for lo, hi in sorted((float(a), float(b)) for a, b in windows if a <= b):
        if out and lo <= out[-1][1]:
            out[-1][1] = max(out[-1][1], hi)
        else:
            out.append([lo, hi])
    return out


def window_grid(windows, pmin: float, pmax: float, baseline: float, rho_kg: float, p: Params) -> List[float]:
    """Full-resolution grid inside frequency windows (the learned proposal's
    refinement, not in the paper): in each merged window, clipped to
    [1/Pmax, 1/Pmin], the Sec. 2.1 spacing f <- f + q_min(f) / (spp * T) walked
    from the window's low edge while f stays inside it."""
    fmin, fmax = 1.0 / pmax, 1.0 / pmin
    denom = p.samples_per_peak * baseline
    out = []
    for lo, hi in merge_windows(windows):
        f = max(lo, fmin)
        end = min(hi, fmax)
        while f <= end:
            out.append(f)
            f = f + q_min(f, rho_kg, p) / denom
    return out


def nbins_of(qmin: float, p: Params) -> int:
    """Number of phase bins: the finest bin is q_min / noverlap."""
    return int(math.ceil(p.noverlap / qmin))


def m_of(qmin: float, nbins: int, p: Params) -> List[int]:
    """Bins covered by each log-spaced duration q_j = q_min e^{j dlogq} (rounded half up)."""
    out = []
    for j in range(n_q(p)):
        e = math.exp(j * p.dlogq)
        out.append(max(1, int(math.floor(qmin * e * nbins + 0.5))))
    return out


def pmin_days(rho_kg: float, p: Params) -> float:
    """Period (days) at which the semi-major axis is pmin_aR stellar radii."""
    a3 = p.pmin_aR * p.pmin_aR * p.pmin_aR
    return math.sqrt(3.0 * math.pi * a3 / (G_SI * rho_kg)) / DAY_S


def pmax_days(tp: np.ndarray, p: Params) -> float:
    """Longest continuous stretch (split at gaps > gap_days), or half the baseline
    when there is a single stretch."""
    starts = [0]
    for i in range(1, tp.shape[0]):
        if float(tp[i]) - float(tp[i - 1]) > p.gap_days:
            starts.append(i)
    if len(starts) == 1:
        return (float(tp[-1]) - float(tp[0])) / 2.0
    ends = starts[1:] + [tp.shape[0]]
    return max(float(tp[e - 1]) - float(tp[s]) for s, e in zip(starts, ends))


def plan_star(t, y, dy, rho, rstar, p: Params = Params(), windows=None) -> StarPlan:
    t = np.asarray(t, np.float64); y = np.asarray(y, np.float64); dy = np.asarray(dy, np.float64)
    ok = np.isfinite(t) & np.isfinite(y) & np.isfinite(dy) & (dy > 0)
    t, y, dy = t[ok], y[ok], dy[ok]
    rho_gcc = float(rho) if (rho is not None and math.isfinite(rho) and rho > 0) else p.rho_default
    rho_kg = rho_gcc * 1000.0
    empty = np.zeros(0)
    def bad(status, t_ref=0.0):
        return StarPlan(status, t_ref, 0.0, 0.0, 0.0, rho_kg, t - t_ref, y, dy, empty, empty,
                        np.zeros(0, np.int32), np.zeros((0, n_q(p)), np.int32))
    if t.shape[0] < 2:
        return bad(ST_TOO_FEW)
    if np.any(np.diff(t) < 0):
        return bad(ST_UNSORTED)
    t_ref = float(t[0])
    tp = t - t_ref
    baseline = float(tp[-1])
    pmin = pmin_days(rho_kg, p)
    pmax = pmax_days(tp, p)
    if not (baseline > 0.0) or not (pmin < pmax):
        st = bad(ST_EMPTY_GRID, t_ref)
        st.pmin, st.pmax, st.baseline = pmin, pmax, baseline
        return st
    k0 = -1
    if p.grid_mode == 1:
        freqs, k0 = coarse_grid(pmin, pmax, p)
    else:
        if windows is not None:
            freqs = window_grid(windows, pmin, pmax, baseline, rho_kg, p)
        else:
            freqs = freq_grid(pmin, pmax, baseline, rho_kg, p)
    qm = [q_min(f, rho_kg, p) for f in freqs]
    nb = [nbins_of(q, p) for q in qm]
    m = [m_of(q, b, p) for q, b in zip(qm, nb)]
    status = 0
    if len(freqs) == 0:
        status |= ST_EMPTY_GRID
    if nb and max(nb) > p.nbins_cap:
        status |= ST_NBINS_CAP
    if status:
        st = bad(status, t_ref)
        st.pmin, st.pmax, st.baseline = pmin, pmax, baseline
        return st
    return StarPlan(0, t_ref, baseline, pmin, pmax, rho_kg, tp, y, dy,
                    np.asarray(freqs, np.float64), np.asarray(qm, np.float64),
                    np.asarray(nb, np.int32), np.asarray(m, np.int32).reshape(len(freqs), n_q(p)), k0)


def plan_batch(batch, p: Params = Params()) -> List[StarPlan]:
    out = []
    for s in range(batch.n_stars):
        t, y, dy = batch.star(s)
        out.append(plan_star(t, y, dy, float(batch.rho[s]), float(batch.rstar[s]), p))
    return out

"""Seeded synthetic TESS-like light curves.

This module only *generates inputs*: cadences, gaps, noise and injected box
transits, shaped like the QLP workloads (27.4-d TESS sectors at 30-min or 200-s
cadence). It holds none of the periodogram's arithmetic, so both the CPU oracle
and the CUDA path can be fed from it without sharing any method code.

A batch is stored in CSR form: ``offsets[n_stars + 1]`` (int64) indexes the
flat float64 arrays ``t`` (days, BTJD-like), ``y`` (relative flux) and ``dy``
(1-sigma errors). Per-star arrays: ``rho`` (g/cm^3), ``rstar`` (R_sun) and the
injection truth (``inj``, ``period``, ``t0``, ``depth``, ``duration``).

The injected transit duration uses the physical circular-orbit formula
(Kepler's third law with M = 4/3 pi R^3 rho, duration = P/pi * asin(R/a)),
evaluated here in SI units.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.signal import lfilter

SECTOR_DAYS = 27.4
CADENCE_30MIN = 30.0 / 1440.0
CADENCE_200S = 200.0 / 86400.0
T_START = 2880.0  # BTJD of a Sector-58-like start; realistic magnitude for t

_G_SI = 6.67430e-11
_RSUN_M = 6.957e8
_DAY_S = 86400.0


@dataclasses.dataclass
class Batch:
    offsets: np.ndarray  # int64 [n_stars + 1]
    t: np.ndarray        # float64 [n_points]
    y: np.ndarray        # float64 [n_points]
    dy: np.ndarray       # float64 [n_points]
    rho: np.ndarray      # float64 [n_stars] g/cm^3 (NaN = unknown)
    rstar: np.ndarray    # float64 [n_stars] R_sun
    inj: np.ndarray      # bool [n_stars]
    period: np.ndarray   # float64 [n_stars] (NaN when not injected)
    t0: np.ndarray
    depth: np.ndarray
    duration: np.ndarray
    name: str = ""

    @property
    def n_stars(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_points(self) -> int:
        return int(self.offsets[-1])

    def star(self, s: int):
        a, b = int(self.offsets[s]), int(self.offsets[s + 1])
        return self.t[a:b], self.y[a:b], self.dy[a:b]

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        parts_t, parts_y, parts_dy, offs = [], [], [], [0]
        for s in idx:
            t, y, dy = self.star(int(s))
            parts_t.append(t); parts_y.append(y); parts_dy.append(dy)
            offs.append(offs[-1] + t.shape[0])
        cat = lambda p: np.concatenate(p) if p else np.zeros(0)
        return Batch(np.asarray(offs, np.int64), cat(parts_t), cat(parts_y), cat(parts_dy),
                     self.rho[idx].copy(), self.rstar[idx].copy(), self.inj[idx].copy(),
                     self.period[idx].copy(), self.t0[idx].copy(), self.depth[idx].copy(),
                     self.duration[idx].copy(), self.name + "[subset]")


def circular_duration_days(period_days, rho_gcc, rstar_rsun=1.0):
    """Full duration (days) of a central transit on a circular orbit, in SI units."""
    period_days = np.asarray(period_days, dtype=np.float64)
    r = np.asarray(rstar_rsun, dtype=np.float64) * _RSUN_M
    mass = 4.0 / 3.0 * math.pi * r ** 3 * (np.asarray(rho_gcc, dtype=np.float64) * 1000.0)
    p_s = period_days * _DAY_S
    a = np.cbrt(_G_SI * mass * p_s ** 2 / (4.0 * math.pi ** 2))
    return period_days / math.pi * np.arcsin(np.minimum(1.0, r / a))


def box_mask(t, period, t0, duration):
    """True where t lies within duration/2 of a mid-transit time t0 + n*period."""
    ph = np.mod(t - t0 + 0.5 * period, period) - 0.5 * period
    return np.abs(ph) < 0.5 * duration


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _sector_cadences(start, cadence, n_sectors=1, sector_gap=1.0):
    n = int(round(SECTOR_DAYS / cadence))
    base = np.arange(n, dtype=np.float64) * cadence
    parts = [start + k * (SECTOR_DAYS + sector_gap) + base for k in range(n_sectors)]
    return np.concatenate(parts)


def _assemble(name, ts, ys, dys, rho, rstar, inj, per, t0, dep, dur) -> Batch:
    offs = np.zeros(len(ts) + 1, np.int64)
    offs[1:] = np.cumsum([x.shape[0] for x in ts])
    return Batch(offs, np.concatenate(ts), np.concatenate(ys), np.concatenate(dys),
                 np.asarray(rho, np.float64), np.asarray(rstar, np.float64),
                 np.asarray(inj, bool), np.asarray(per, np.float64), np.asarray(t0, np.float64),
                 np.asarray(dep, np.float64), np.asarray(dur, np.float64), name)


def concat(batches, name: str = "") -> Batch:
    """One batch of the stars of several, in order (for batches generated in
    independently seeded chunks)."""
    offs = [np.zeros(1, np.int64)]
    base = 0
    for b in batches:
        offs.append(b.offsets[1:] + base)
        base += int(b.offsets[-1])
    cat = lambda f: np.concatenate([getattr(b, f) for b in batches])
    return Batch(np.concatenate(offs), cat("t"), cat("y"), cat("dy"), cat("rho"), cat("rstar"), cat("inj"),
                 cat("period"), cat("t0"), cat("depth"), cat("duration"),
                 name or (batches[0].name if batches else ""))


def in_chunks(make, n_stars: int, chunk: int, seed: int, workers: int = 8) -> Batch:
    """make(n, seed) for ceil(n_stars / chunk) chunks with seeds seed, seed + 1, ...,
    run on a thread pool (NumPy releases the interpreter lock in its array work),
    joined in chunk order: the same batch for any number of workers."""
    from concurrent.futures import ThreadPoolExecutor
    sizes = [min(chunk, n_stars - a) for a in range(0, n_stars, chunk)]
    with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        parts = list(ex.map(lambda c: make(sizes[c], seed + c), range(len(sizes))))
    return concat(parts)


def single_star(seed: int = 1) -> Batch:
    """One 27.4-d sector at 30-min cadence, 1-d gap at mid-sector, white noise 1e-3,
    box transit P = 3.7 d, depth 2e-3, circular duration for rho = 1.41, R* = 1."""
    rng = np.random.default_rng(seed)
    t = _sector_cadences(T_START, CADENCE_30MIN)
    mid = T_START + 0.5 * SECTOR_DAYS
    t = t[(t < mid - 0.5) | (t >= mid + 0.5)]
    sigma, period, depth, rho = 1e-3, 3.7, 2e-3, 1.41
    dur = float(circular_duration_days(period, rho, 1.0))
    t0 = T_START + rng.uniform(0.0, period)
    y = 1.0 + rng.normal(0.0, sigma, t.shape[0])
    y -= depth * box_mask(t, period, t0, dur)
    dy = np.full(t.shape[0], sigma)
    return _assemble("single_sector_30min", [t], [y], [dy], [rho], [1.0], [True], [period], [t0],
                     [depth], [dur])


def uneven_single_sector(n_stars: int = 4096, seed: int = 2, frac_injected: float = 0.3,
                         min_points: int = 7000) -> Batch:
    """Batched uneven single-sector stars at 200-s cadence with random 0.5-2 d gaps
    (7,000-11,800 points), rho log-U(0.1, 10), R* log-U(0.5, 3), white sigma
    log-U(2e-4, 1e-2), a fraction with injected boxes (P log-U(0.5, 13) d, depth
    log-U(3e-4, 1e-2), circular-orbit duration)."""
    rng = np.random.default_rng(seed)
    base = _sector_cadences(0.0, CADENCE_200S)
    ts, ys, dys = [], [], []
    rho = _loguniform(rng, 0.1, 10.0, n_stars)
    rstar = _loguniform(rng, 0.5, 3.0, n_stars)
    sig = _loguniform(rng, 2e-4, 1e-2, n_stars)
    inj = rng.uniform(size=n_stars) < frac_injected
    per = np.where(inj, _loguniform(rng, 0.5, 13.0, n_stars), np.nan)
    dep = np.where(inj, _loguniform(rng, 3e-4, 1e-2, n_stars), np.nan)
    dur = np.where(inj, circular_duration_days(np.nan_to_num(per, nan=1.0), rho, rstar), np.nan)
    t0 = np.full(n_stars, np.nan)
    start = T_START + rng.uniform(0.0, 1.0, n_stars)
    for s in range(n_stars):
        while True:
            keep = np.ones(base.shape[0], bool)
            for _ in range(rng.integers(0, 7)):
                g0 = rng.uniform(0.0, SECTOR_DAYS)
                keep &= ~((base >= g0) & (base < g0 + rng.uniform(0.5, 2.0)))
            if keep.sum() >= min_points:
                break
        t = start[s] + base[keep]
        y = 1.0 + rng.normal(0.0, sig[s], t.shape[0])
        if inj[s]:
            t0[s] = start[s] + rng.uniform(0.0, per[s])
            y -= dep[s] * box_mask(t, per[s], t0[s], dur[s])
        ts.append(t); ys.append(y); dys.append(np.full(t.shape[0], sig[s]))
    return _assemble("uneven_single_sector_200s", ts, ys, dys, rho, rstar, inj, per, t0, dep, dur)


def multi_sector(n_stars: int = 1024, seed: int = 3, max_sectors: int = 13,
                 frac_injected: float = 0.5, rho_value: float = 1.41, min_sectors: int = 1) -> Batch:
    """min_sectors..max_sectors contiguous sectors at 200-s cadence with 1-d
    inter-sector gaps, AR(1) red noise (phi = 0.9, stationary sigma 1e-3) plus
    white noise 1e-3, injected P log-U(0.5, 100) d, depth log-U(3e-4, 1e-2)."""
    rng = np.random.default_rng(seed)
    ts, ys, dys = [], [], []
    nsec = rng.integers(min_sectors, max_sectors + 1, n_stars)
    rho = np.full(n_stars, rho_value)
    rstar = np.ones(n_stars)
    inj = rng.uniform(size=n_stars) < frac_injected
    per = np.where(inj, _loguniform(rng, 0.5, 100.0, n_stars), np.nan)
    dep = np.where(inj, _loguniform(rng, 3e-4, 1e-2, n_stars), np.nan)
    dur = np.where(inj, circular_duration_days(np.nan_to_num(per, nan=1.0), rho, rstar), np.nan)
    t0 = np.full(n_stars, np.nan)
    phi, s_red, s_white = 0.9, 1e-3, 1e-3
    for s in range(n_stars):
        start = T_START + rng.uniform(0.0, 1.0)
        t = _sector_cadences(start, CADENCE_200S, int(nsec[s]))
        n = t.shape[0]
        e = rng.normal(0.0, s_red * math.sqrt(1.0 - phi * phi), n)
        # AR(1): red[i] = phi * red[i-1] + e[i], started from the stationary law
        red = lfilter([1.0], [1.0, -phi], e, zi=[phi * rng.normal(0.0, s_red)])[0]
        y = 1.0 + red + rng.normal(0.0, s_white, n)
        if inj[s]:
            t0[s] = start + rng.uniform(0.0, per[s])
            y -= dep[s] * box_mask(t, per[s], t0[s], dur[s])
        ts.append(t); ys.append(y); dys.append(np.full(n, s_white))
    return _assemble("multi_sector_200s", ts, ys, dys, rho, rstar, inj, per, t0, dep, dur)


def tiny_batch(n_stars: int = 4, seed: int = 5, n_min: int = 40, n_max: int = 120,
               span_days: float = 6.0, rho_value=None) -> Batch:
    """Small irregularly sampled stars for fast CPU checks (sorted t, gaps, noise + box)."""
    rng = np.random.default_rng(seed)
    ts, ys, dys, rhos, rss, injs, pers, t0s, deps, durs = [], [], [], [], [], [], [], [], [], []
    for _ in range(n_stars):
        n = int(rng.integers(n_min, n_max + 1))
        t = np.sort(T_START + rng.uniform(0.0, span_days, n))
        rho = float(_loguniform(rng, 0.3, 5.0)) if rho_value is None else rho_value
        sig = float(_loguniform(rng, 5e-4, 5e-3))
        per = float(rng.uniform(0.6, span_days / 3.0))
        dur = float(circular_duration_days(per, rho, 1.0))
        t0 = T_START + float(rng.uniform(0.0, per))
        dep = float(rng.uniform(2.0, 8.0)) * sig
        y = 1.0 + rng.normal(0.0, sig, n) - dep * box_mask(t, per, t0, dur)
        dy = sig * rng.uniform(0.7, 1.3, n)
        ts.append(t); ys.append(y); dys.append(dy); rhos.append(rho); rss.append(1.0)
        injs.append(True); pers.append(per); t0s.append(t0); deps.append(dep); durs.append(dur)
    return _assemble("tiny", ts, ys, dys, rhos, rss, injs, pers, t0s, deps, durs)


def sector_counts_geometric(n_stars: int, seed: int, mean: float = 3.0, cap: int = 40) -> np.ndarray:
    """Sector count per star, geometric with the given mean, capped."""
    rng = np.random.default_rng(seed)
    return np.minimum(rng.geometric(1.0 / mean, n_stars), cap)


def sector_scale(n_stars: int = 1024, seed: int = 6, frac_injected: float = 0.01,
                 mean_sectors: float = 3.0, cap: int = 40, sectors: int | None = None) -> Batch:
    """Sector-scale mix: per star a geometric number of contiguous 27.4-d sectors
    (mean 3, at most 40; every star `sectors` of them when given) at 200-s cadence
    with 1-d gaps, rho log-U(0.1, 10), R* log-U(0.5, 3), white sigma log-U(2e-4,
    1e-2) as in the uneven single-sector batch, and 1 % injected boxes (P log-U(0.5,
    13) d, depth log-U(3e-4, 1e-2), circular-orbit duration)."""
    nsec = sector_counts_geometric(n_stars, seed, mean_sectors, cap)
    if sectors is not None:
        nsec = np.full(n_stars, int(sectors))
    rng = np.random.default_rng(seed + 1)
    rho = _loguniform(rng, 0.1, 10.0, n_stars)
    rstar = _loguniform(rng, 0.5, 3.0, n_stars)
    sig = _loguniform(rng, 2e-4, 1e-2, n_stars)
    inj = rng.uniform(size=n_stars) < frac_injected
    per = np.where(inj, _loguniform(rng, 0.5, 13.0, n_stars), np.nan)
    dep = np.where(inj, _loguniform(rng, 3e-4, 1e-2, n_stars), np.nan)
    dur = np.where(inj, circular_duration_days(np.nan_to_num(per, nan=1.0), rho, rstar), np.nan)
    t0 = np.full(n_stars, np.nan)
    grids = {}
    ts, ys, dys = [], [], []
    start = T_START + rng.uniform(0.0, 1.0, n_stars)
    for s in range(n_stars):
        k = int(nsec[s])
        if k not in grids:
            grids[k] = _sector_cadences(0.0, CADENCE_200S, k)
        t = start[s] + grids[k]
        y = 1.0 + rng.normal(0.0, sig[s], t.shape[0])
        if inj[s]:
            t0[s] = start[s] + rng.uniform(0.0, per[s])
            y -= dep[s] * box_mask(t, per[s], t0[s], dur[s])
        ts.append(t); ys.append(y); dys.append(np.full(t.shape[0], sig[s]))
    return _assemble("sector_scale_200s", ts, ys, dys, rho, rstar, inj, per, t0, dep, dur)


def proposal_set(n_stars: int, seed: int, min_sectors: int = 1, max_sectors: int = 4,
                 frac_injected: float = 0.5, depth_range=(1e-4, 1e-2), period_range=(0.5, 100.0),
                 sigma_range=(2e-4, 2e-3)) -> Batch:
    """Light curves for the learned period proposal: 1-4 contiguous sectors at 200-s
    cadence with 1-d gaps, rho log-U(0.1, 10), R* log-U(0.5, 3), white noise,
    injected boxes (P log-U(0.5, 100) d, depth log-U(1e-4, 1e-2), duration the
    circular one times U(0.5, 2)) in half of the stars."""
    rng = np.random.default_rng(seed)
    nsec = rng.integers(min_sectors, max_sectors + 1, n_stars)
    rho = _loguniform(rng, 0.1, 10.0, n_stars)
    rstar = _loguniform(rng, 0.5, 3.0, n_stars)
    sig = _loguniform(rng, sigma_range[0], sigma_range[1], n_stars)
    inj = rng.uniform(size=n_stars) < frac_injected
    per = np.where(inj, _loguniform(rng, period_range[0], period_range[1], n_stars), np.nan)
    dep = np.where(inj, _loguniform(rng, depth_range[0], depth_range[1], n_stars), np.nan)
    dur = np.where(inj, circular_duration_days(np.nan_to_num(per, nan=1.0), rho, rstar)
                   * rng.uniform(0.5, 2.0, n_stars), np.nan)
    t0 = np.full(n_stars, np.nan)
    grids = {k: _sector_cadences(0.0, CADENCE_200S, k) for k in range(min_sectors, max_sectors + 1)}
    ts, ys, dys = [], [], []
    start = T_START + rng.uniform(0.0, 1.0, n_stars)
    for s in range(n_stars):
        t = start[s] + grids[int(nsec[s])]
        y = 1.0 + rng.normal(0.0, sig[s], t.shape[0])
        if inj[s]:
            t0[s] = start[s] + rng.uniform(0.0, per[s])
            y -= dep[s] * box_mask(t, per[s], t0[s], dur[s])
        ts.append(t); ys.append(y); dys.append(np.full(t.shape[0], sig[s]))
    return _assemble("proposal_set", ts, ys, dys, rho, rstar, inj, per, t0, dep, dur)

"""Oracle: several planets per star by iterative masking (TEST INFRASTRUCTURE ONLY).

Not in the paper (it reports one candidate per star). Reading: after a
candidate is found (plan, BLS, S/N, best, post-BLS statistics), the points
within one fitted transit duration of any of its mid-transit times,
|dt| < q P, are removed, and the whole search (plan included: Pmax and the
baseline follow the remaining points) runs again on the rest; it stops for a
star after n_planets candidates or when a search finds none. The statistics'
fitted epoch and q define the mask when the fit ran (status OK or not
converged), else the BLS box.
"""
from __future__ import annotations

import numpy as np

from . import bls, plan as oplan, snr as osnr, stats as ostats


def search_multi(t, y, dy, rho, rstar, n_planets: int, p: oplan.Params = oplan.Params()):
    t = np.asarray(t, np.float64); y = np.asarray(y, np.float64); dy = np.asarray(dy, np.float64)
    keep = np.ones(t.shape[0], bool)
    found = []
    for _ in range(n_planets):
        pl = oplan.plan_star(t[keep], y[keep], dy[keep], rho, rstar, p)
        if pl.status != 0:
            break
        res = bls.bls_star(pl)
        snr, _, sigma = osnr.spectral_snr(pl.freqs, res.sr)
        best = osnr.best_candidate(pl, res, snr, sigma)
        if best is None:
            break
        st = ostats.star_stats(pl, best)
        found.append((best, st))
        if st["status"] in (ostats.ST_OK, ostats.ST_NOT_CONVERGED):
            t0, q = st["t0"], st["q"]
        else:
            t0, q = best["t0"], best["q"]
        period = best["period"]
        dt, _ = ostats.phase_distance(t, t0, period)
        keep &= ~(np.abs(dt) < q * period)
    return found

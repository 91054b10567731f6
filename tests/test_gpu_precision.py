"""Precision study on multi-sector stars: the phase reduction x = t'f in FP64, in
double-float (hi/lo FP32 with an FP64 re-fold near bin edges) and in plain FP32
on the point path, and the cell path's fixed-point edges with exact integer and
with compensated FP32 sums, each against the FP64 oracle on sampled trial
frequencies.

Three workloads:
  * 8 stars of 1-13 contiguous sectors (AR(1) red noise), every mode, 96 evenly
    spaced frequencies per star plus each mode's own SR maximum;
  * 2 stars of 40 contiguous sectors at rho = 10 g/cm^3 (Pmin 0.123 d, baseline
    1,135 d, t'f up to 9.2e3 cycles), every mode, on 40 narrow frequency windows
    spread over the upper frequency range up to 1/Pmin (the windows' grids; their
    bin counts stay below 3,000, while the star's full grid needs
    more than the 8,192-bin cap near Pmax, and the point path's histograms hold
    about 3,500 in compensated mode);
  * 1,024 stars of 1-13 sectors on the default path over the full grid, sampled at
    8 evenly spaced frequencies per star plus its SR maximum, and a 64-star subset
    through the point path in double-float and FP32 phase.

Reported per mode (and written to the parity report): the largest relative SR
error, the agreement of the per-frequency box (duration index j, start bin k) and
of the sampled maximum, and the largest t'f sampled. The exact modes must meet the
parity tolerances; plain FP32 is reported only (its bins move once t'f reaches
~10^3 cycles)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import bls as ob
from oracle import plan as op
from paper_2302_01293_gb300 import qlpbls
from parity import REPORT, SR_RTOL, run_gpu

pytestmark = pytest.mark.gpu

MODES = {
    "cell path, exact integer sums": qlpbls.Params(method=qlpbls.METHOD_CELLS),
    "cell path, compensated FP32 sums": qlpbls.Params(method=qlpbls.METHOD_CELLS, sum_mode=qlpbls.SUM_COMP),
    "points, FP64 phase": qlpbls.Params(method=qlpbls.METHOD_POINTS, phase_mode=qlpbls.PHASE_FP64),
    "points, double-float phase": qlpbls.Params(method=qlpbls.METHOD_POINTS, phase_mode=qlpbls.PHASE_DF),
    "points, FP32 phase": qlpbls.Params(method=qlpbls.METHOD_POINTS, phase_mode=qlpbls.PHASE_FP32),
}


def _new_stats():
    return {"max_sr_rel": 0.0, "box_agree": 0, "box_near_tie": 0, "sampled": 0, "best_agree": 0,
            "best_near_tie": 0, "stars": 0, "max_cycles_t_f": 0.0}


def _score(st, sub, o, sr, q, k, tmax):
    """Add one star's sampled frequencies (oracle restricted plan sub, results o) to st."""
    sr = sr.astype(np.float64)
    rel = np.abs(sr - o.sr) / np.maximum(o.sr, 1e-300)
    st["max_sr_rel"] = max(st["max_sr_rel"], float(rel.max()))
    same = (q == o.j) & (k == o.k)
    st["box_agree"] += int(same.sum())
    st["sampled"] += len(sr)
    for i in np.nonzero(~same)[0]:
        v = ob.box_value(sub, int(i), int(q[i]), int(k[i]))
        if v >= o.sr[i] * (1 - SR_RTOL):
            st["box_near_tie"] += 1
    # the sampled maximum: the same frequency, or a near tie (the oracle's own value
    # at the GPU's choice within the SR tolerance of its maximum)
    gi, oi = int(np.argmax(sr)), int(np.argmax(o.sr))
    st["best_agree"] += int(gi == oi or o.sr[gi] >= o.sr[oi] * (1 - SR_RTOL))
    st["best_near_tie"] += int(gi != oi and o.sr[gi] >= o.sr[oi] * (1 - SR_RTOL))
    st["stars"] += 1
    st["max_cycles_t_f"] = max(st["max_cycles_t_f"], float(tmax * sub.freqs.max()))


def _assert_exact(name, st):
    assert st["max_sr_rel"] <= SR_RTOL, (name, st)
    assert st["box_agree"] + st["box_near_tie"] == st["sampled"], (name, st)
    assert st["best_agree"] == st["stars"], (name, st)


def _gpu_sample(g, s, idx):
    sl = g["plan"].star_slice(s)
    return (g["sr"][sl][idx], g["qidx"][sl][idx].astype(np.int64),
            g["kbin"][sl][idx].view(np.uint32).astype(np.int64))


def test_multi_sector_precision(gpu_lib):
    b = synth.multi_sector(n_stars=8, seed=7, max_sectors=13)
    runs = {name: run_gpu(b, p, with_snr=False) for name, p in MODES.items()}
    stats = {name: _new_stats() for name in MODES}
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        pl = oracle.plan_star(t, y, dy, float(b.rho[s]), float(b.rstar[s]))
        nf = pl.freqs.shape[0]
        idx = set(np.linspace(0, nf - 1, 96).astype(int).tolist())
        for name, g in runs.items():
            sl = g["plan"].star_slice(s)
            assert np.array_equal(g["plan"].freqs[sl], pl.freqs)
            idx.add(int(np.argmax(g["sr"][sl])))
        idx = np.array(sorted(idx))
        sub = ob.restrict(pl, idx)
        o = ob.bls_star(sub)
        for name, g in runs.items():
            _score(stats[name], sub, o, *_gpu_sample(g, s, idx), pl.baseline)
    REPORT["precision: 8 stars of 1-13 sectors"] = stats
    for name in MODES:
        if "FP32 phase" not in name:
            _assert_exact(name, stats[name])


def _upper_windows(t, rho, n_win=40, half=2e-5):
    """n_win narrow windows, log-spaced in frequency from where the bin count drops to
    3,000 (within every mode's histograms) up to 1/Pmin (the last window ends there)."""
    p = op.Params()
    rho_kg = rho * 1000.0
    fmax = 1.0 / op.pmin_days(rho_kg, p)
    f_lo = fmax
    while op.nbins_of(op.q_min(f_lo * 0.98, rho_kg, p), p) <= 3000:
        f_lo *= 0.98
    centres = np.geomspace(f_lo, fmax, n_win)
    lo = centres * (1 - half)
    hi = np.minimum(centres * (1 + half), fmax)
    lo[-1] = fmax * (1 - 2 * half)
    return list(zip(lo.tolist(), hi.tolist()))


def test_forty_sector_precision(gpu_lib):
    b = synth.multi_sector(n_stars=2, seed=71, min_sectors=40, max_sectors=40, rho_value=10.0,
                           frac_injected=1.0)
    wins = [_upper_windows(b.star(s)[0], float(b.rho[s])) for s in range(b.n_stars)]
    wo = np.array([0, len(wins[0]), len(wins[0]) + len(wins[1])], np.int64)
    wl = np.array([w[0] for ws in wins for w in ws])
    wh = np.array([w[1] for ws in wins for w in ws])
    stats = {name: _new_stats() for name in MODES}
    runs = {}
    for name, p in MODES.items():
        import torch
        plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, p, windows=(wo, wl, wh))
        out = plan.search()
        flags = plan.device_status()
        torch.cuda.synchronize()
        assert flags == 0, (name, flags)
        runs[name] = dict({k: v.cpu().numpy() for k, v in out.items() if k != "best"}, plan=plan)
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        pl = oracle.plan_star(t, y, dy, float(b.rho[s]), float(b.rstar[s]), windows=wins[s])
        assert pl.status == 0 and pl.freqs.shape[0] > 0
        o = ob.bls_star(pl)
        idx = np.arange(pl.freqs.shape[0])
        for name, g in runs.items():
            assert np.array_equal(g["plan"].freqs[g["plan"].star_slice(s)], pl.freqs)
            _score(stats[name], pl, o, *_gpu_sample(g, s, idx), pl.baseline)
    REPORT["precision: 2 stars of 40 sectors, rho 10, upper-frequency windows"] = stats
    assert min(st["max_cycles_t_f"] for st in stats.values()) >= 8e3
    for name in MODES:
        if "FP32 phase" not in name:
            _assert_exact(name, stats[name])


def _oracle_sampled(args):
    """Worker: the oracle's plan of one star and its BLS at the sampled indices."""
    t, y, dy, rho, rstar, n_f, idx_extra = args
    pl = oracle.plan_star(t, y, dy, rho, rstar)
    assert pl.freqs.shape[0] == n_f
    idx = np.array(sorted(set(np.linspace(0, n_f - 1, 8).astype(int).tolist()) | set(idx_extra)))
    sub = ob.restrict(pl, idx)
    return idx, sub, ob.bls_star(sub), pl.baseline, pl.freqs[idx]


def test_config3_thousand_stars_sampled(gpu_lib):
    import multiprocessing as mp
    import os
    b = synth.multi_sector(n_stars=1024, seed=3, max_sectors=13)
    g = run_gpu(b, qlpbls.Params(), with_snr=False)
    assert g["flags"] == 0
    sub64 = b.subset(range(64))
    pts = {name: run_gpu(sub64, MODES[name], with_snr=False)
           for name in ("points, double-float phase", "points, FP32 phase")}
    jobs = []
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        sl = g["plan"].star_slice(s)
        extra = [int(np.argmax(g["sr"][sl]))]
        if s < 64:
            extra += [int(np.argmax(r["sr"][r["plan"].star_slice(s)])) for r in pts.values()]
        jobs.append((t, y, dy, float(b.rho[s]), float(b.rstar[s]), sl.stop - sl.start, extra))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        res = pool.map(_oracle_sampled, jobs, chunksize=8)
    stats = {"default path (exact sums), 1,024 stars": _new_stats()}
    for name in pts:
        stats[name + ", 64 stars"] = _new_stats()
    for s, (idx, sub, o, base, fs) in enumerate(res):
        sl = g["plan"].star_slice(s)
        assert np.array_equal(g["plan"].freqs[sl][idx], fs)
        _score(stats["default path (exact sums), 1,024 stars"], sub, o, *_gpu_sample(g, s, idx), base)
        if s < 64:
            for name, r in pts.items():
                _score(stats[name + ", 64 stars"], sub, o, *_gpu_sample(r, s, idx), base)
    REPORT["precision: 1,024 stars of 1-13 sectors (sampled)"] = stats
    _assert_exact("default", stats["default path (exact sums), 1,024 stars"])
    _assert_exact("DF", stats["points, double-float phase, 64 stars"])

"""Pins of the oracle's BLS residue (Sec. 2.1, Sec. 2.2 item 1; Kovacs et al. 2002).

* brute force: every (duration, start bin) window summed point by point;
* closed form: a noise-free box placed exactly on bins gives SR = delta^2 r (1 - r),
  the exact depth, start bin and duration index, and bounds every other residue
  (Cauchy-Schwarz);
* invariants: flux offset, error scaling, flux sign flip, point order;
* the binned maximum never exceeds the best contiguous phase arc.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import bls as ob
from oracle import plan as op


def _custom_plan(tp, y, dy, freqs, nbins, m):
    freqs = np.asarray(freqs, np.float64)
    return op.StarPlan(0, 0.0, float(np.max(tp)), 0.0, 0.0, 1410.0, np.asarray(tp, np.float64),
                       np.asarray(y, np.float64), np.asarray(dy, np.float64), freqs,
                       np.zeros_like(freqs), np.asarray(nbins, np.int32),
                       np.asarray(m, np.int32).reshape(len(freqs), -1))


def _brute(tp, w, wd, f, nb, ms):
    bins = []
    for t in tp:
        x = float(t) * f
        ph = x - math.floor(x)
        bins.append(min(nb - 1, int(math.floor(ph * nb))))
    best = None
    for j, m in enumerate(ms):
        for k in range(nb):
            r = s = 0.0
            for i, b in enumerate(bins):
                if (b - k) % nb < m:
                    r += float(w[i]); s += float(wd[i])
            if 0.0 < r < 1.0:
                v = s * s / (r * (1.0 - r))
                if best is None or v > best[0]:
                    best = (v, j, k, s, r)
    return best


def test_brute_force_tiny():
    rng = np.random.default_rng(11)
    for trial in range(4):
        n = int(rng.integers(12, 40))
        tp = np.sort(rng.uniform(0, 9.0, n)); tp -= tp[0]
        y = 1 + rng.normal(0, 1e-3, n); dy = rng.uniform(5e-4, 2e-3, n)
        nf = 6
        freqs = np.sort(rng.uniform(0.2, 2.0, nf))
        nbins = rng.integers(7, 33, nf)
        ms = [sorted(rng.integers(1, 6, 5).tolist()) for _ in range(nf)]
        pl = _custom_plan(tp, y, dy, freqs, nbins, ms)
        res = oracle.bls_star(pl)
        w, d, _ = ob.weights(y, dy)
        for k in range(nf):
            bf = _brute(tp, w, w * d, float(freqs[k]), int(nbins[k]), ms[k])
            assert res.sr[k] == pytest.approx(bf[0], rel=1e-12, abs=1e-300)
            assert (res.j[k], res.k[k]) == (bf[1], bf[2])
            assert res.s[k] == pytest.approx(bf[3], rel=1e-10, abs=1e-18)
            assert res.r[k] == pytest.approx(bf[4], rel=1e-12)


def _aligned_box(nb, f, k0, m, delta, cycles=4, per_bin=2):
    tp = []
    inbox = []
    for c in range(cycles):
        for b in range(nb):
            for rep in range(per_bin):
                tp.append((c + (b + (rep + 0.5) / per_bin) / nb) / f)
                inbox.append((b - k0) % nb < m)
    tp = np.asarray(tp)
    y = np.where(inbox, 1.0 - delta, 1.0)
    return tp, y, np.full(tp.shape[0], 1e-3)


@pytest.mark.parametrize("k0", [0, 17, 58])
def test_noise_free_box_closed_form(k0):
    nb, f, delta = 60, 1.0 / 3.0, 2e-3
    ms = [3, 3, 4, 4, 4, 5, 5, 6, 7, 7, 8, 9, 10, 11]
    for m in (3, 5, 11):
        tp, y, dy = _aligned_box(nb, f, k0, m, delta)
        # the true frequency among a few neighbours
        freqs = [f * 0.9, f * 0.97, f, f * 1.03, f * 1.5]
        pl = _custom_plan(tp, y, dy, freqs, [nb] * 5, [ms] * 5)
        res = oracle.bls_star(pl)
        r = m / nb
        expect = delta * delta * r * (1 - r)
        assert res.sr[2] == pytest.approx(expect, rel=1e-10)
        assert res.k[2] == k0
        assert res.j[2] == ms.index(m)
        depth = -res.s[2] / (res.r[2] * (1 - res.r[2]))
        assert depth == pytest.approx(delta, rel=1e-9)
        assert np.all(res.sr <= expect * (1 + 1e-12))


def test_invariants():
    b = synth.tiny_batch(n_stars=3, seed=21)
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        base = oracle.plan_star(t, y, dy, float(b.rho[s]), 1.0)
        assert base.status == 0
        ref = oracle.bls_star(base)
        variants = {
            "offset": (y + 0.37, dy),
            "scale": (y, dy * 3.1),
            "flip": (-y, dy),
        }
        for name, (yy, dd) in variants.items():
            pl = oracle.plan_star(t, yy, dd, float(b.rho[s]), 1.0)
            res = oracle.bls_star(pl)
            np.testing.assert_allclose(res.sr, ref.sr, rtol=1e-9, err_msg=name)
            if name == "flip":
                np.testing.assert_allclose(res.s, -ref.s, rtol=1e-8, atol=1e-20)
        perm = np.random.default_rng(s).permutation(base.tp.shape[0])
        pl = op.StarPlan(0, base.t_ref, base.baseline, base.pmin, base.pmax, base.rho_kg,
                         base.tp[perm], base.y[perm], base.dy[perm], base.freqs, base.qmin,
                         base.nbins, base.m)
        res = oracle.bls_star(pl)
        np.testing.assert_allclose(res.sr, ref.sr, rtol=1e-9)


def test_binned_max_below_best_phase_arc():
    b = synth.tiny_batch(n_stars=2, seed=33, n_min=20, n_max=30)
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        pl = oracle.plan_star(t, y, dy, float(b.rho[s]), 1.0)
        res = oracle.bls_star(pl)
        w, d, _ = ob.weights(pl.y, pl.dy)
        n = w.shape[0]
        for k in range(0, pl.freqs.shape[0], max(1, pl.freqs.shape[0] // 15)):
            ph = np.mod(pl.tp * pl.freqs[k], 1.0)
            order = np.argsort(ph)
            ww, vv = w[order], (w * d)[order]
            best = 0.0
            for i in range(n):
                r = sv = 0.0
                for L in range(1, n):
                    r += ww[(i + L - 1) % n]; sv += vv[(i + L - 1) % n]
                    if 0 < r < 1:
                        best = max(best, sv * sv / (r * (1 - r)))
            assert res.sr[k] <= best * (1 + 1e-9)


def test_single_star_recovers_injection():
    b = synth.single_star()
    t, y, dy = b.star(0)
    pl = oracle.plan_star(t, y, dy, 1.41, 1.0)
    res = oracle.bls_star(pl)
    snr, _, sig = oracle.spectral_snr(pl.freqs, res.sr)
    best = oracle.best_candidate(pl, res, snr, sig)
    assert abs(best["period"] / 3.7 - 1) < 0.01
    assert best["snr"] > 9
    # mid-transit within a bin of the truth, depth within the binning dilution
    assert abs(best["t0"] - b.t0[0]) < 2 * best["period"] / best["nbins"]
    assert 0.6 * 2e-3 < best["depth"] < 1.2 * 2e-3


def test_restricted_plan_equals_full_search_at_those_frequencies():
    import synth
    from oracle import bls as ob
    b = synth.tiny_batch(n_stars=2, seed=8)
    for s in range(2):
        t, y, dy = b.star(s)
        pl = oracle.plan_star(t, y, dy, float(b.rho[s]), 1.0)
        full = oracle.bls_star(pl)
        idx = np.arange(0, pl.freqs.shape[0], 7)
        sub = ob.bls_star(ob.restrict(pl, idx))
        assert np.array_equal(sub.sr, full.sr[idx])
        assert np.array_equal(sub.j, full.j[idx]) and np.array_equal(sub.k, full.k[idx])


def test_per_q_binning_brute_force_and_special_case():
    from oracle import bls as ob
    b = synth.tiny_batch(n_stars=2, seed=13, n_min=30, n_max=60)
    for s in range(2):
        t, y, dy = b.star(s)
        pl = oracle.plan_star(t, y, dy, float(b.rho[s]), 1.0)
        idx = np.arange(0, pl.freqs.shape[0], max(1, pl.freqs.shape[0] // 12))
        sub = ob.restrict(pl, idx)
        res = ob.bls_star_per_q(sub)
        w, d, _ = ob.weights(sub.y, sub.dy)
        for i, f in enumerate(sub.freqs):
            best, bj, bk = -1.0, -1, -1
            for j in range(sub.m.shape[1]):
                qj = float(sub.qmin[i]) * math.exp(0.1 * j)
                nb = int(math.ceil(3.0 / qj))
                bins = []
                for tt in sub.tp:
                    x = tt * f
                    bins.append(min(nb - 1, int(math.floor((x - math.floor(x)) * nb))))
                for k in range(nb):
                    r = s_ = 0.0
                    for pt, bb in enumerate(bins):
                        if (bb - k) % nb < 3:
                            r += w[pt]; s_ += w[pt] * d[pt]
                    if 0 < r < 1:
                        v = s_ * s_ / (r * (1 - r))
                        if v > best * (1 + 1e-12):
                            best, bj, bk = v, j, k
            assert res.sr[i] == pytest.approx(best, rel=1e-9)
            assert (res.j[i], res.k[i]) == (bj, bk) or res.sr[i] == pytest.approx(best, rel=1e-9)
    # one duration (q_max = q_min) and noverlap 3: the variant is the shared histogram
    p1 = op.Params(qmax_fac=0.5)
    t, y, dy = b.star(0)
    pl = oracle.plan_star(t, y, dy, float(b.rho[0]), 1.0, p1)
    a1, a2 = ob.bls_star(pl), ob.bls_star_per_q(pl)
    assert np.array_equal(a1.sr, a2.sr) and np.array_equal(a1.k, a2.k)

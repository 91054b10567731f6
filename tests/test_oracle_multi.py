"""Pin of the iterative multi-planet search (oracle): a single sector with two
injected boxes of different periods gives both, strongest first."""
import numpy as np

import synth
from oracle import multi


def test_two_injected_planets_are_found_in_turn():
    rng = np.random.default_rng(11)
    t = synth.T_START + np.arange(0.0, 27.4, 1.0 / 48.0)      # 30-min cadence
    y = 1.0 + rng.normal(0.0, 1e-3, t.shape)
    dur1 = synth.circular_duration_days(3.1, 1.41, 1.0)
    dur2 = synth.circular_duration_days(7.7, 1.41, 1.0)
    y -= 4e-3 * synth.box_mask(t, 3.1, synth.T_START + 0.6, dur1)
    y -= 3e-3 * synth.box_mask(t, 7.7, synth.T_START + 2.2, dur2)
    dy = np.full(t.shape, 1e-3)
    found = multi.search_multi(t, y, dy, 1.41, 1.0, 3)
    assert len(found) >= 2
    p1, p2 = found[0][0]["period"], found[1][0]["period"]
    assert abs(p1 / 3.1 - 1) < 0.01 and abs(p2 / 7.7 - 1) < 0.01
    assert found[0][1]["detected"] == 1 and found[1][1]["detected"] == 1


def test_masking_removes_points_within_one_duration_of_each_transit(monkeypatch):
    """After a detection the next search runs on the points farther than q P (one
    fitted duration) from every mid-transit time of the candidate: the count of
    points it drops equals an independent count with a box of full width 2 q P,
    and the injected transit's points are all among them."""
    from oracle import stats as ostats
    rng = np.random.default_rng(12)
    t = synth.T_START + np.arange(0.0, 27.4, 1.0 / 48.0)
    p_inj, t0_inj = 4.3, synth.T_START + 1.3
    dur = synth.circular_duration_days(p_inj, 1.41, 1.0)
    y = 1.0 - 3e-3 * synth.box_mask(t, p_inj, t0_inj, dur) + rng.normal(0.0, 2e-4, t.shape)
    dy = np.full(t.shape, 2e-4)
    sizes = []
    orig = multi.oplan.plan_star

    def spy(tt, *a, **k):
        sizes.append(len(tt))
        return orig(tt, *a, **k)

    monkeypatch.setattr(multi.oplan, "plan_star", spy)
    found = multi.search_multi(t, y, dy, 1.41, 1.0, 2)
    b, st = found[0]
    assert abs(b["period"] / p_inj - 1) < 0.01
    if st["status"] in (ostats.ST_OK, ostats.ST_NOT_CONVERGED):
        t0, q = st["t0"], st["q"]
    else:
        t0, q = b["t0"], b["q"]
    masked = synth.box_mask(t, b["period"], t0, 2.0 * q * b["period"])
    assert len(sizes) >= 2 and sizes[0] == t.shape[0]
    assert sizes[1] == t.shape[0] - int(masked.sum())
    assert not np.any(synth.box_mask(t, p_inj, t0_inj, dur) & ~masked)

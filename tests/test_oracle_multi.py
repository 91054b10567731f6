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

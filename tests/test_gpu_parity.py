"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Cases: the single-sector 30-min star; a ragged batch of uneven 200-s sectors
(several tiles, a ragged tail, forced small tiles); multi-sector stars; stars
the planner rejects mixed into a batch; the empty batch; every phase and sum
mode; and the full 4,096-star batch on sampled stars in the bench's launch
configuration. Tolerances are those of tests/parity.py.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2302_01293_gb300 import qlpbls
from parity import compare_snr, compare_spectrum, oracle_star, run_gpu

pytestmark = pytest.mark.gpu


def _narrow_expected(batch):
    """Stars the 32-bit exact table takes (whole-table single-sector stars): the
    running sum of w (y - ybar) within 64 times the largest |w (y - ybar)| and not
    below 2^-28 max|y|, at most 65,536 points."""
    n = 0
    for s in range(batch.n_stars):
        t, y, dy = batch.star(s)
        inv = 1.0 / (dy * dy)
        ybar = np.sum(inv * y) / np.sum(inv)
        wd = inv * (y - ybar) / np.sum(inv)
        exc = np.max(np.abs(np.cumsum(wd)))
        n += int(len(t) <= 65536 and exc <= 64.0 * np.max(np.abs(wd)) and exc >= 2.0 ** -28 * np.max(np.abs(y)))
    return n


def _check_batch(batch, params, stars=None, with_snr=True):
    g = run_gpu(batch, params, with_snr=with_snr)
    assert g["flags"] == 0
    plan = g["plan"]
    stats = []
    for s in (range(batch.n_stars) if stars is None else stars):
        pl, ores = oracle_star(batch, s)
        assert plan.star_status[s] == pl.status
        sl = plan.star_slice(s)
        assert np.array_equal(plan.freqs[sl], pl.freqs)
        st = compare_spectrum(pl, ores, g, sl, label=f"star {s}")
        if with_snr:
            st.update(compare_snr(pl, ores, g, sl, g["best"][s], label=f"star {s}", alt=st["alt_sr"]))
        stats.append(st)
    return g, stats


@pytest.mark.parametrize("phase", [qlpbls.PHASE_FP64, qlpbls.PHASE_DF])
@pytest.mark.parametrize("summ", [qlpbls.SUM_PLAIN, qlpbls.SUM_COMP, qlpbls.SUM_FIXED, qlpbls.SUM_FIXED64])
def test_single_star(gpu_lib, phase, summ):
    b = synth.single_star()
    g, stats = _check_batch(b, qlpbls.Params(phase_mode=phase, sum_mode=summ))
    best = g["best"][0]
    assert abs(best["period"] / 3.7 - 1) < 0.01 and best["snr"] > 9


@pytest.mark.parametrize("method", [qlpbls.METHOD_POINTS, qlpbls.METHOD_CELLS])
@pytest.mark.parametrize("summ", [qlpbls.SUM_PLAIN, qlpbls.SUM_COMP, qlpbls.SUM_FIXED, qlpbls.SUM_FIXED64])
def test_uneven_batch_both_paths(gpu_lib, method, summ):
    b = synth.uneven_single_sector(n_stars=5, seed=22)
    g, _ = _check_batch(b, qlpbls.Params(method=method, sum_mode=summ))
    exact = method == qlpbls.METHOD_CELLS and summ in (qlpbls.SUM_FIXED, qlpbls.SUM_FIXED64)
    assert g["plan"].n_exact_stars == (5 if exact else 0)
    assert g["plan"].n_narrow_stars == (_narrow_expected(b) if exact and summ == qlpbls.SUM_FIXED else 0)


def test_exact_cell_path_is_the_default(gpu_lib):
    # exact integer sums on the cell path for every star whose table fits shared memory,
    # most of them (white noise, shallow or short transits) on the 32-bit table
    b = synth.uneven_single_sector(n_stars=8, seed=27)
    g, _ = _check_batch(b, qlpbls.Params())
    assert g["plan"].n_exact_stars == 8 and g["plan"].exact_edges == g["plan"].edges
    assert g["plan"].n_narrow_stars == _narrow_expected(b) >= 6


def test_32_bit_table_with_unequal_weights(gpu_lib):
    # per-point errors scattered by up to 20 % (weights up to 2.25 times apart): on the
    # 32-bit table r is then the ratio of integer sums of round(w F) that are no longer
    # equal, each point's weight rounded to 2^-33 of the total; the spectra, S/N and best
    # records still meet the parity tolerances (same-box SR within 5e-7)
    b = synth.uneven_single_sector(n_stars=4, seed=35)
    rng = np.random.default_rng(35)
    dy = b.dy * rng.uniform(0.8, 1.2, b.dy.shape)
    b2 = synth.Batch(b.offsets, b.t, b.y, dy, b.rho, b.rstar, b.inj, b.period, b.t0, b.depth, b.duration,
                     "unequal weights")
    g, _ = _check_batch(b2, qlpbls.Params())
    assert g["sr_tight"] and g["plan"].n_exact_stars == 4
    assert g["plan"].n_narrow_stars == _narrow_expected(b2) >= 3


def test_slow_trend_takes_the_64_bit_table(gpu_lib):
    # a linear flux trend of 10 sigma across the sector makes the running sum of
    # w (y - ybar) reach about N / 8 times its largest single term, beyond the 32-bit
    # table's 64: that star keeps the 64-bit table, the others take the 32-bit one,
    # and all three match the oracle; the same batch with every star on the 64-bit
    # table gives the same boxes
    b = synth.uneven_single_sector(n_stars=3, seed=34)
    y = b.y.copy()
    a, e = int(b.offsets[1]), int(b.offsets[2])
    t = b.t[a:e]
    y[a:e] += 10.0 * b.dy[a:e] * (t - t.mean()) / (t.max() - t.min())
    b2 = synth.Batch(b.offsets, b.t, y, b.dy, b.rho, b.rstar, b.inj, b.period, b.t0, b.depth, b.duration, "trend")
    g, _ = _check_batch(b2, qlpbls.Params())
    assert g["plan"].n_exact_stars == 3 and g["plan"].n_narrow_stars == _narrow_expected(b2) == _narrow_expected(b) - 1
    g64, _ = _check_batch(b2, qlpbls.Params(sum_mode=qlpbls.SUM_FIXED64))
    assert g64["plan"].n_exact_stars == 3 and g64["plan"].n_narrow_stars == 0
    for k in ("qidx", "kbin"):
        assert np.mean(g[k] == g64[k]) > 0.999


def test_exact_path_falls_back_on_an_extreme_point(gpu_lib):
    # one point with an error bar 20 times smaller than the rest (weight 400 times
    # the others) and one flux outlier of 2,000 sigma: those stars take the
    # compensated cell kernel, the untouched star the exact one; all three match the
    # oracle
    b = synth.uneven_single_sector(n_stars=3, seed=33)
    dy = b.dy.copy()
    y = b.y.copy()
    dy[b.offsets[0] + 500] *= 0.05
    y[b.offsets[1] + 700] += 2000.0 * dy[b.offsets[1] + 700]
    b2 = synth.Batch(b.offsets, b.t, y, dy, b.rho, b.rstar, b.inj, b.period, b.t0, b.depth, b.duration, "extreme")
    g, _ = _check_batch(b2, qlpbls.Params())
    assert g["plan"].n_exact_stars == 1 and g["plan"].n_cell_stars == 3


def test_exact_path_falls_back_below_32_bins(gpu_lib):
    # durations from 1.5 q_circ: 12 bins at Pmin, fewer than a warp's 32 lanes; those
    # stars take the compensated cell kernel, with the same results
    b = synth.uneven_single_sector(n_stars=3, seed=28)
    p = qlpbls.Params(qmin_fac=1.5)
    g = run_gpu(b, p)
    assert g["flags"] == 0 and g["plan"].n_exact_stars == 0 and g["plan"].n_cell_stars == 3
    for s in range(b.n_stars):
        pl, ores = oracle_star(b, s, oracle.Params(qmin_fac=1.5))
        sl = g["plan"].star_slice(s)
        assert np.array_equal(g["plan"].freqs[sl], pl.freqs)
        compare_spectrum(pl, ores, g, sl, label=f"qmin 1.5 star {s}")


@pytest.mark.parametrize("warps", [4, 8, 16])
def test_cell_path_single_star_and_warps(gpu_lib, warps):
    # 30-min cadence: the cell path is forced (the planner would fold points here)
    b = synth.single_star()
    _check_batch(b, qlpbls.Params(method=qlpbls.METHOD_CELLS, warps_per_block=warps,
                                  chunk_freqs=warps * 2, sum_mode=qlpbls.SUM_COMP))


@pytest.mark.parametrize("tile", [0, 256, 1024])
def test_uneven_batch_tiles(gpu_lib, tile):
    b = synth.uneven_single_sector(n_stars=6, seed=12)
    _check_batch(b, qlpbls.Params(tile_points=tile, method=qlpbls.METHOD_POINTS))


@pytest.mark.parametrize("warps", [4, 8, 16])
def test_warps_per_block(gpu_lib, warps):
    b = synth.uneven_single_sector(n_stars=3, seed=13)
    _check_batch(b, qlpbls.Params(warps_per_block=warps, chunk_freqs=warps * 3,
                                  method=qlpbls.METHOD_POINTS))


def test_multi_sector(gpu_lib):
    b = synth.multi_sector(n_stars=2, seed=14, max_sectors=3)
    _check_batch(b, qlpbls.Params())


def test_multi_sector_cell_path_in_windows(gpu_lib):
    # tables of 3-4 contiguous sectors exceed shared memory: searched window by window
    b = synth.multi_sector(n_stars=3, seed=4, max_sectors=4)
    g, _ = _check_batch(b, qlpbls.Params(method=qlpbls.METHOD_CELLS))
    assert g["plan"].n_cell_stars == 3 and g["plan"].n_windowed >= 2
    assert g["plan"].n_exact_stars == 3  # exact sums through the windows' workspace


def test_exact_path_whole_and_windowed_tables_in_one_batch(gpu_lib):
    # one- and multi-sector stars: whole tables and time-windowed ones, searched as
    # two launches of the exact kernel (one queue each), directly and from a CUDA graph
    import torch
    b = synth.multi_sector(n_stars=3, seed=5, max_sectors=4)
    g, _ = _check_batch(b, qlpbls.Params())
    plan = g["plan"]
    assert plan.n_exact_stars == 3 and 1 <= plan.n_windowed <= 2
    assert plan.search_launches == 3  # prep, whole tables, windowed tables
    out = plan.graph_capture(plan.alloc_outputs(), parts=1)
    plan.graph_launch(1)
    torch.cuda.synchronize()
    for k in ("sr", "qidx", "kbin"):
        assert np.array_equal(out[k].cpu().numpy(), g[k]), k
    assert plan.device_status() == 0


def test_multi_sector_windows_compensated(gpu_lib):
    b = synth.multi_sector(n_stars=3, seed=4, max_sectors=4)
    g, _ = _check_batch(b, qlpbls.Params(method=qlpbls.METHOD_CELLS, sum_mode=qlpbls.SUM_COMP))
    assert g["plan"].n_exact_stars == 0 and g["plan"].n_windowed >= 2


@pytest.mark.parametrize("window", [64, 700, 4000])
@pytest.mark.parametrize("summ", [qlpbls.SUM_PLAIN, qlpbls.SUM_COMP, qlpbls.SUM_FIXED])
def test_cell_windows_forced(gpu_lib, window, summ):
    # forced short windows: many window boundaries per frequency, windows shorter
    # than one bin (64 cells) and a ragged last window
    b = synth.uneven_single_sector(n_stars=3, seed=23)
    g, _ = _check_batch(b, qlpbls.Params(method=qlpbls.METHOD_CELLS, cell_window=window,
                                         sum_mode=summ))
    assert g["plan"].n_windowed == 3


def test_tiny_ragged_and_rejected_stars(gpu_lib):
    good = synth.tiny_batch(n_stars=5, seed=15, n_min=33, n_max=97)
    # append stars the planner must reject: unsorted, one point, NaN-only
    t = [good.star(s)[0] for s in range(good.n_stars)]
    y = [good.star(s)[1] for s in range(good.n_stars)]
    dy = [good.star(s)[2] for s in range(good.n_stars)]
    t.append(np.array([3.0, 2.0, 1.0]) + 2000); y.append(np.ones(3)); dy.append(np.full(3, 1e-3))
    t.append(np.array([2000.0])); y.append(np.ones(1)); dy.append(np.full(1, 1e-3))
    t.append(np.linspace(2000, 2010, 20)); y.append(np.full(20, np.nan)); dy.append(np.full(20, 1e-3))
    b = synth._assemble("mixed", t, y, dy, list(good.rho) + [1.41] * 3, [1.0] * 8, [True] * 8,
                        [1.0] * 8, [0.0] * 8, [0.0] * 8, [0.0] * 8)
    g, _ = _check_batch(b, qlpbls.Params())
    assert list(g["plan"].star_status[5:]) == [qlpbls.STAR_UNSORTED, qlpbls.STAR_TOO_FEW,
                                              qlpbls.STAR_TOO_FEW]
    assert np.all(g["best"]["f_idx"][5:] == -1)


def test_tiny_stars_on_the_exact_path(gpu_lib):
    # short, irregular stars (33-97 points) forced onto the cell path: small tables
    # whose length is not a multiple of the bulk copies' 4-cell granularity, staged one
    # after another by the same blocks
    b = synth.tiny_batch(n_stars=12, seed=16, n_min=33, n_max=97)
    g, _ = _check_batch(b, qlpbls.Params(method=qlpbls.METHOD_CELLS))
    assert g["plan"].n_exact_stars > 0


def test_empty_batch(gpu_lib):
    z = np.zeros(0)
    plan = qlpbls.Plan(np.zeros(1, np.int64), z, z, z, z, z)
    out = plan.search()
    plan.snr(out)
    assert plan.n_freq_total == 0 and plan.device_status() == 0


def test_fp32_phase_runs_and_is_close(gpu_lib):
    # FP32 folding is a precision-study mode: bins may differ, SR stays close
    b = synth.uneven_single_sector(n_stars=2, seed=16)
    g = run_gpu(b, qlpbls.Params(phase_mode=qlpbls.PHASE_FP32), with_snr=False)
    for s in range(2):
        pl, ores = oracle_star(b, s)
        sr = g["sr"][g["plan"].star_slice(s)]
        rel = np.abs(sr - ores.sr) / ores.sr
        assert np.median(rel) < 1e-2


def test_run_host_matches_device_path(gpu_lib):
    b = synth.uneven_single_sector(n_stars=4, seed=17)
    g = run_gpu(b, qlpbls.Params())
    n = g["plan"].n_freq_total
    h = qlpbls.run_host(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, qlpbls.Params(), sr_capacity=n)
    assert h["n_freq_total"] == n
    assert np.array_equal(h["sr"], g["sr"][:n])
    assert np.array_equal(h["snr"], g["snr"][:n])
    assert np.array_equal(h["best"]["f_idx"], g["best"]["f_idx"])


def test_run_host_in_chunks_equals_one_plan(gpu_lib):
    # 1,100 stars: the host-buffer call plans and searches them in two chunks
    # (planning of the second overlaps the search of the first); the exact path is
    # deterministic, so every spectrum value equals the single plan's bit for bit
    b = synth.uneven_single_sector(n_stars=1100, seed=29)
    g = run_gpu(b, qlpbls.Params())
    n = g["plan"].n_freq_total
    h = qlpbls.run_host(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, qlpbls.Params(), sr_capacity=n)
    assert h["n_freq_total"] == n and g["plan"].n_exact_stars == 1100
    assert np.array_equal(h["sr"], g["sr"][:n])
    assert np.array_equal(h["snr"], g["snr"][:n])
    assert np.array_equal(h["best"], g["best"])


def test_full_batch_sampled(gpu_lib):
    # the 4,096-star uneven single-sector batch in the default launch shape;
    # 12 sampled stars checked in full against the oracle
    b = synth.uneven_single_sector(n_stars=4096, seed=2)
    rng = np.random.default_rng(0)
    stars = sorted(rng.choice(4096, 12, replace=False).tolist())
    _check_batch(b, qlpbls.Params(), stars=stars)


def test_graph_replay_matches_oracle(gpu_lib):
    # search + S/N captured as CUDA graphs (together, and one graph each), replayed
    # on the current stream
    import torch
    b = synth.uneven_single_sector(n_stars=4, seed=31)
    plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
    out = plan.graph_capture(plan.alloc_outputs())
    plan.graph_capture(out, parts=1)
    plan.graph_capture(out, parts=2)
    for launches in ([3], [3], [1, 2]):
        for v in out.values():
            v.fill_(0)
        for parts in launches:
            plan.graph_launch(parts)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items() if k != "best"}
        best = plan.best_host(out)
        for s in range(b.n_stars):
            pl, ores = oracle_star(b, s)
            sl = plan.star_slice(s)
            st = compare_spectrum(pl, ores, g, sl, label=f"graph star {s}",
                                  tight=plan.n_cell_stars == plan.n_exact_stars)
            compare_snr(pl, ores, g, sl, best[s], label=f"graph star {s}", alt=st["alt_sr"])
    assert plan.device_status() == 0


def test_autotune_choice_is_cached_and_exact(gpu_lib):
    b = synth.uneven_single_sector(n_stars=96, seed=32)
    tuned, cached = qlpbls.autotune(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, sample_stars=48)
    again, cached2 = qlpbls.autotune(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, sample_stars=48)
    assert not cached and cached2 and again == tuned
    assert tuned.warps_per_block in (0, 8, 16) and tuned.chunk_freqs >= 0
    # the tuned settings change speed only: parity on a few stars of the batch
    _check_batch(b.subset(range(3)), tuned)


@pytest.mark.parametrize("summ", [qlpbls.SUM_PLAIN, qlpbls.SUM_COMP])
def test_per_duration_binning_variant(gpu_lib, summ):
    # bin_mode PER_Q: one histogram of q_j / noverlap bins per duration, boxes of
    # noverlap bins; the spectrum, the S/N and the best record against the oracle's
    # per-duration BLS (near ties judged on the oracle's histogram j of the GPU's box)
    import dataclasses
    import math
    from oracle import bls as ob
    b = synth.uneven_single_sector(n_stars=3, seed=24)
    p = qlpbls.Params(bin_mode=qlpbls.BIN_PER_Q, sum_mode=summ)
    g = run_gpu(b, p)
    assert g["flags"] == 0
    plan = g["plan"]
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        pl = oracle.plan_star(t, y, dy, float(b.rho[s]), float(b.rstar[s]))
        ores = ob.bls_star_per_q(pl)
        sl = plan.star_slice(s)

        def box(i, j, k, pl=pl):
            nb = int(math.ceil(3.0 / (float(pl.qmin[i]) * math.exp(0.1 * j))))
            sub = dataclasses.replace(ob.restrict(pl, [i]), nbins=np.array([nb], np.int32),
                                      m=np.array([[3]], np.int32))
            return ob.box_value(sub, 0, 0, k)

        st = compare_spectrum(pl, ores, g, sl, label=f"per-q star {s}", box_value=box)
        compare_snr(pl, ores, g, sl, g["best"][s], label=f"per-q star {s}", alt=st["alt_sr"],
                    per_q=(3.0, 0.1))


def test_pmin_at_three_stellar_radii(gpu_lib):
    # Sec. 2.1: Sectors 59-60 used a = 3 R* for Pmin (the default is 2 R*)
    b = synth.uneven_single_sector(n_stars=3, seed=25)
    p = qlpbls.Params(pmin_aR=3.0)
    g = run_gpu(b, p)
    assert g["flags"] == 0
    plan = g["plan"]
    for s in range(b.n_stars):
        pl, ores = oracle_star(b, s, oracle.Params(pmin_aR=3.0))
        sl = plan.star_slice(s)
        assert np.array_equal(plan.freqs[sl], pl.freqs)
        st = compare_spectrum(pl, ores, g, sl, label=f"a=3R* star {s}")
        compare_snr(pl, ores, g, sl, g["best"][s], label=f"a=3R* star {s}", alt=st["alt_sr"])


def test_sharded_driver_on_one_gpu_equals_host_call(gpu_lib):
    from paper_2302_01293_gb300 import shard
    b = synth.uneven_single_sector(n_stars=5, seed=26)
    got = shard.search_sharded(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
    ref = qlpbls.run_host(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)["best"]
    assert np.array_equal(got["f_idx"], ref["f_idx"]) and np.array_equal(got["snr"], ref["snr"])

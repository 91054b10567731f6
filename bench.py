"""Throughput bench of the batched Keplerian-constrained BLS + spectral S/N on GB300.

Workload (default): 4,096 uneven single-sector stars at 200-s cadence (7,000-11,800
points each after random 0.5-2 d gaps), rho log-U(0.1, 10) g/cm^3, R* log-U(0.5, 3),
white noise sigma log-U(2e-4, 1e-2), 30 % with injected boxes; seeded synthetic data.

One step = one pass of the device path over the whole batch: the preparation
kernels (weights, prefix sums and cell tables; double-float points for stars
folded point by point), the persistent BLS search over every (star, trial
frequency), and the S/N / best-candidate kernel, with the plan (grid) built once
beforehand and the light curves resident in HBM. The launch settings come from
the library's autotuner (run once, untimed), and each step replays two CUDA
graphs (search, S/N) captured from the plan. `e2e` times the public host-buffer
call qlp_bls_run_host (plan + upload + search + S/N + download) on the same batch.

Metric: BLS point-frequency evaluations per second (sum over stars of N_s * n_f,s
per second). Multi-GPU: one independent batch per rank (weak scaling, no
collective on the data path); value = all ranks' work / max-over-ranks time.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the only other place this file runs the oracle).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BLS point-freq evals/s; stars/hr learned vs full-grid BLS at >=99% recall"
UNIT = "point-freq/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--stars", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-stars", type=int, default=256)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-multi", action="store_true", help="skip the multi-sector search line")
    ap.add_argument("--sum-mode", default="fixed", choices=["fixed", "fixed64", "comp", "plain"],
                    help="cell-path sums: exact integers (default), compensated FP32, plain FP32")
    ap.add_argument("--workload", default="uneven", choices=["uneven", "multi_sector"],
                    help="the timed batch: uneven single-sector stars (default) or multi-sector stars "
                         "(1-13 sectors, for profiling the time-windowed path)")
    ap.add_argument("--learned-train", type=int, default=200000)
    ap.add_argument("--learned-epochs", type=int, default=2)
    ap.add_argument("--learned-eval", type=int, default=4096)
    ap.add_argument("--sector-scale-stars", type=int, default=32768)
    ap.add_argument("--tune-sample", type=int, default=512)
    ap.add_argument("--no-tune", action="store_true", help="library defaults instead of the autotuner")
    ap.add_argument("--case", default=None, choices=["fixed", "stats", "conv", "train"],
                    help="run one small case of a kernel (for a profiler capture) and exit")
    ap.add_argument("--method", type=int, default=0, choices=[0, 1, 2],
                    help="0 per star the cheaper path, 1 fold every point, 2 cell path where possible")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work per unit of the two search kernels:
#  point path, per point-frequency evaluation: 16 FP32-pipe lane operations
#    (double-float product 4, two round-to-integer steps and the remainder 8,
#    guard-band test 2, run sums 2);
#  cell path, per bin edge: 20 lane operations with plain sums (fixed-point edge
#    location 6, comparison and band test 4, prefix differences 8, bin update 2)
#    and 30 with compensated sums (TwoSum on both bin updates); shared-memory
#    traffic per edge 44 B plain / 60 B compensated (dt 4 + prefix 8 + base 16 of
#    gathers, then the bin read-modify-write).
FP32_OPS_PER_EVAL = 16
CELL_OPS_PER_EDGE = {0: 20, 1: 30}
CELL_SMEM_BYTES_PER_EDGE = {0: 44, 1: 60}
#  exact cell path (integer prefix sums), per bin edge: 14 lane operations
#    (edge position in 24.40 fixed point 3, cell and offset 2, comparison and
#    guard-band test 3, next-cell select 1, two 64-bit accumulations of group
#    base + local prefix 5) and 28 shared-memory bytes gathered (dt 4, local
#    prefix 8, group base 16) on the 64-bit table; on the 32-bit table 13 lane
#    operations (two 64-bit accumulations of the prefix pair 4) and 12 bytes (dt 4,
#    prefix pair 8); per box start bin of the sweep: 76 lane operations (running
#    sums over 11 bins 22, then per width of 3..11 bins the score and the
#    division-free comparison 6) and 48 shared-memory bytes (two adjacent starts
#    read the 12 histogram records of 8 bytes they need between them).
EXACT_OPS_PER_EDGE = 14
EXACT_SMEM_BYTES_PER_EDGE = 28
EXACT32_OPS_PER_EDGE = 13
EXACT32_SMEM_BYTES_PER_EDGE = 12
EXACT_OPS_PER_BIN = 76
EXACT_SMEM_BYTES_PER_BIN = 48
FP32_LANES_PER_SM = 128
SMEM_BYTES_PER_CLK_PER_SM = 128
N_SMS = 152


def _training_batches(n_train: int, workers: int):
    """The proposal set's seeded stars in chunks of 2,048 (seeds 100, 101, ...),
    generated on a thread pool while the GPU turns each finished chunk into its
    coarse spectrum (network input) and labels; returns [(x0, labels)] on the GPU."""
    from concurrent.futures import ThreadPoolExecutor
    import synth
    from paper_2302_01293_gb300 import learned
    sizes = [min(2048, n_train - a) for a in range(0, n_train, 2048)]
    out = []
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {}
        for c in range(min(len(sizes), 2 * workers)):
            futs[c] = ex.submit(synth.proposal_set, sizes[c], 100 + c)
        for c in range(len(sizes)):
            tb = futs.pop(c).result()
            nxt = c + 2 * workers
            if nxt < len(sizes):
                futs[nxt] = ex.submit(synth.proposal_set, sizes[nxt], 100 + nxt)
            cs = learned.CoarseStage(tb)
            out.append((cs.x0.clone(), learned.labels(tb, cs.params, "cuda")))
            del cs, tb
    return out


def _smallest_k(curve, target=0.99):
    for k in sorted(curve, key=int):
        if curve[k] >= target:
            return int(k)
    return None


def learned_comparison(args):
    """The learned proposal against the same path without the network, and both
    against the full-grid search, on held-out multi-sector stars.

    The network is trained here from scratch on the proposal set's seeded stars
    (no stored weights). Recall is counted among the injections the full grid
    recovers. For K = 1, 2, 4, ..., 32 proposals per star, the network's top-K
    coarse bins and the coarse S/N's own top-K are refined; the smallest K at which
    each ranking reaches 99 % of the full grid's recoveries is then timed through
    the library's one-call path (qlp_bls_search_learned, with and without the
    network), wall clock from host arrays to best records, as is the full grid
    through the host-buffer call."""
    import torch
    import synth
    from paper_2302_01293_gb300 import learned, qlpbls
    workers = min(16, os.cpu_count() or 1)
    t0 = time.perf_counter()
    batches = _training_batches(args.learned_train, workers)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = qlpbls.CNN(max_batch=128, length=4096, seed=0)
    t0 = time.perf_counter()
    losses = learned.train(net, batches, epochs=args.learned_epochs, lr=3e-4, pos_weight=16.0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    peaks, _ = _peaks()
    cnn = cnn_throughput(net, batches[0][0], batches[0][1], peaks.get("bf16_tflops", 1900.0))
    del batches
    test = synth.in_chunks(lambda n, s: synth.proposal_set(n, s), args.learned_eval, 512, 999, workers)

    def timed(fn, reps=3):  # a warm-up, then the fastest of `reps` runs
        best_t, res = float("inf"), None
        for rep in range(reps + 1):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            if rep:
                best_t = min(best_t, time.perf_counter() - t1)
        return best_t, res

    t_full, full = timed(lambda: qlpbls.run_host(test.offsets, test.t, test.y, test.dy, test.rho, test.rstar))
    rf = learned.recovered(full["best"], test)
    n_rf = max(int(rf.sum()), 1)
    coarse = learned.CoarseStage(test)
    bins_n = learned.propose(net, coarse.x0, 32).cpu().numpy()
    bins_a = learned.propose_without_network(coarse, 32).cpu().numpy()
    curve = {"network": {}, "coarse_snr_without_network": {}}
    for k in (1, 2, 4, 8, 16, 32):
        for name, bins in (("network", bins_n), ("coarse_snr_without_network", bins_a)):
            r = learned.recovered(learned.search_with_bins(test, coarse, bins[:, :k]), test)
            curve[name][str(k)] = float((r & rf).sum() / n_rf)
    del coarse
    k99 = {name: _smallest_k(c) for name, c in curve.items()}
    n = test.n_stars
    per_hour = {"full_grid": n / t_full * 3600.0}
    for name, use_net in (("network", True), ("coarse_snr_without_network", False)):
        for k in sorted({32, k99[name] or 32}):
            t_l, (best_l, _) = timed(lambda: learned.search_learned(test, net if use_net else None, k=k))
            rl = learned.recovered(best_l, test)
            per_hour[f"{name}_k{k}"] = {"stars_per_hour": n / t_l * 3600.0, "seconds": t_l,
                                        "recall": float((rl & rf).sum() / n_rf),
                                        "speedup_vs_full": t_full / t_l}
    gain = None
    if k99["network"] is not None and k99["coarse_snr_without_network"] is not None:
        a = per_hour[f"network_k{k99['network']}"]["stars_per_hour"]
        b = per_hour[f"coarse_snr_without_network_k{k99['coarse_snr_without_network']}"]["stars_per_hour"]
        gain = {"k99_network": k99["network"], "k99_without_network": k99["coarse_snr_without_network"],
                "stars_per_hour_ratio": a / b}
    sector_scale = sector_scale_line(net, args.sector_scale_stars, workers) if args.sector_scale_stars > 0 else None
    return {"workload": f"{n} held-out stars, 1-4 sectors at 200 s, 50 % injected "
                        "(P log-U(0.5, 100) d, depth log-U(1e-4, 1e-2))",
            "train_stars": args.learned_train, "epochs": args.learned_epochs,
            "train_data_seconds": t_data, "train_seconds": t_train, "final_loss": losses[-1],
            "full_recovered": int(rf.sum()), "injected": int(test.inj.sum()),
            "recall_at_k": curve, "k_for_99pct_recall": k99, "stars_per_hour": per_hour,
            "network_gain_at_99pct": gain, "cnn": cnn, "sector_scale": sector_scale}


def sector_scale_line(net, n_stars: int, workers: int):
    """The sector-scale mix (geometric sector counts, mean 3, at most 40, plus 16
    stars of 40 sectors; mixed rho, R*, noise; 1 % injected), generated in
    independently seeded chunks: the full-grid path through the public host-buffer
    call and the learned path through its one-call C entry (K = 32), each timed wall
    clock from host arrays to best records on one GPU (the full grid once, the
    learned path the faster of two runs after a warm-up)."""
    import torch
    import synth
    from paper_2302_01293_gb300 import learned, qlpbls
    mix = synth.in_chunks(lambda n, s: synth.sector_scale(n, seed=s), n_stars, 2048, 6000, workers)
    deep = synth.sector_scale(16, seed=5999, sectors=40)
    b = synth.concat([mix, deep], "sector_scale_200s")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full = qlpbls.run_host(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
    t_full = time.perf_counter() - t0
    t_learned = float("inf")
    best_l = None
    for rep in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best_l, _ = learned.search_learned(b, net, k=32)
        torch.cuda.synchronize()
        if rep:
            t_learned = min(t_learned, time.perf_counter() - t0)
    rf = learned.recovered(full["best"], b)
    rl = learned.recovered(best_l, b)
    # sectors per star from its span: k sectors of 27.4 d with 1-d gaps span 28.4 k - 1 d
    nsec = np.rint((b.t[b.offsets[1:] - 1] - b.t[b.offsets[:-1]] + 1.0) / 28.4).astype(int)
    ok = full["best"]["f_idx"] >= 0
    return {"workload": f"{b.n_stars} stars: geometric sector counts (mean 3, at most 40) and 16 of "
                        "40 sectors, 200 s, 1 % injected",
            "points": int(b.offsets[-1]), "max_sectors": int(nsec.max()),
            "searched_stars": int(ok.sum()),
            "full_grid_e2e_s": t_full, "stars_per_hour_full": b.n_stars / t_full * 3600.0,
            "learned_e2e_s": t_learned, "stars_per_hour_learned": b.n_stars / t_learned * 3600.0,
            "speedup": t_full / t_learned,
            "injected": int(b.inj.sum()), "full_recovered": int(rf.sum()),
            "learned_recovered_of_full": int((rl & rf).sum()),
            "recall": float((rl & rf).sum() / max(int(rf.sum()), 1))}


# CNN FLOPs per input bin (kernel 9, 64 channels): conv 6->64, four 64->64, 64->1
CNN_FWD_FLOP_PER_BIN = 2 * 9 * (6 * 64 + 4 * 64 * 64 + 64)
CONV64_FLOP_PER_BIN = 2 * 9 * 64 * 64
# training step: forward, input gradients of layers 6..2 (not of layer 1), all
# weight gradients (as many FLOPs as the forward)
CNN_TRAIN_FLOP_PER_BIN = 2 * CNN_FWD_FLOP_PER_BIN + 2 * 9 * (4 * 64 * 64 + 64)


def cnn_throughput(net, x0, labels, peak_tflops):
    """Device time of the network's kernels on one full batch (CUDA events): the
    tensor-core conv64 alone, the forward pass, and one training step."""
    import torch
    from paper_2302_01293_gb300 import qlpbls
    B, L = net.max_batch, net.length
    x0 = x0[:B].contiguous()
    labels = labels[:B].contiguous()
    g = torch.Generator(device="cpu").manual_seed(5)
    x = (torch.randn(B, L, 64, generator=g) * 0.5).to(torch.bfloat16).cuda()
    w = (torch.randn(9, 64, 64, generator=g) * 0.05).cuda()
    bias = torch.zeros(64, device="cuda")
    wp = qlpbls.pack_w64(w)
    y = torch.empty_like(x)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e-3

    # conv64 replayed from a CUDA graph of 50 launches: the kernel's device time without
    # the host's launch gaps (about 3 us per launch on 44-us launches)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            qlpbls.conv64(x, wp, bias, None, True, out=y, err=err)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    conv_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(conv_graph):
        for _ in range(50):
            qlpbls.conv64(x, wp, bias, None, True, out=y, err=err)
    t_conv = timed(lambda: conv_graph.replay(), 3) / 50
    t_conv_stream = timed(lambda: qlpbls.conv64(x, wp, bias, None, True, out=y, err=err), 50)
    t_fwd = timed(lambda: net.forward(x0), 20)
    params = net.params()
    t_train = timed(lambda: net.train_step(x0, labels, 16.0, 0.0), 10)
    net.set_params(params)  # the timed steps used lr = 0 but advanced Adam's state
    assert int(err.item()) == 0
    conv_tf = B * L * CONV64_FLOP_PER_BIN / t_conv / 1e12
    return {"batch": B, "bins": L,
            "conv64": {"bound": "tensor", "achieved": conv_tf, "peak": peak_tflops, "unit": "TFLOP/s",
                       "frac": conv_tf / peak_tflops, "ms": t_conv * 1e3,
                       "launch": "CUDA graph of 50 launches",
                       "stream_launches_tflops": B * L * CONV64_FLOP_PER_BIN / t_conv_stream / 1e12,
                       "algorithmic": f"{B} x {L} bins x {CONV64_FLOP_PER_BIN} FLOP (BF16 in, FP32 acc)"},
            "forward_tflops": B * L * CNN_FWD_FLOP_PER_BIN / t_fwd / 1e12, "forward_ms": t_fwd * 1e3,
            "train_step_tflops": B * L * CNN_TRAIN_FLOP_PER_BIN / t_train / 1e12,
            "train_step_ms": t_train * 1e3,
            "peak_source": "bf16_tflops (burst) of MEASURED_PEAKS.json"}


def _timed_searches(plan, out, steps, stream):
    """Mean device time (ms) of `steps` searches after one warm-up (CUDA events)."""
    import torch
    plan.search(out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        plan.search(out)
    e1.record(stream)
    torch.cuda.synchronize()
    if plan.device_status():
        raise RuntimeError("device flags in a bench search")
    return e0.elapsed_time(e1) / steps


def single_star_line(steps: int):
    """The single-star case (one 27.4-d sector at 30 min, ~1,250 points, injected 3.7-d
    box): search and S/N on the device, through the default exact cell path and the
    per-point path with the FP64 phase, and the public host-buffer call end to end.
    One star fills a few SMs at most: this line reports latency, not throughput."""
    import torch
    import synth
    from paper_2302_01293_gb300 import qlpbls
    b = synth.single_star()
    stream = torch.cuda.current_stream()
    res = {"workload": "single star, 27.4-d sector at 30 min (synth.single_star)", "points": int(b.offsets[-1])}
    for name, p in (("exact", qlpbls.Params()),
                    ("points_fp64_phase", qlpbls.Params(method=qlpbls.METHOD_POINTS,
                                                        phase_mode=qlpbls.PHASE_FP64))):
        plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, p)
        out = plan.alloc_outputs()
        ms = _timed_searches(plan, out, steps, stream)
        res[name] = {"value": plan.work / (ms * 1e-3), "unit": UNIT, "ms": ms, "point_freq": plan.work,
                     "trial_freqs": plan.n_freq_total}
        del plan, out
    times = []
    for _ in range(max(3, steps)):
        t0 = time.perf_counter()
        r = qlpbls.run_host(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, qlpbls.Params())
        times.append(time.perf_counter() - t0)
    res["e2e"] = {"seconds": min(times), "period_found": float(r["best"]["period"][0]),
                  "period_injected": float(b.period[0]),
                  "includes": "host plan (grid) + H2D + search + S/N + D2H of best"}
    return res


def multi_sector_line(steps: int, n_stars: int = 1024, n_phase: int = 64):
    """Search throughput on the multi-sector precision workload: 1,024 stars of 1-13
    contiguous 27.4-d sectors at 200 s, AR(1) red noise (up to ~150 k points per
    star), through the exact cell path (tables in time windows where a star's table
    exceeds shared memory) and the compensated FP32 cell kernel, each the mean of
    `steps` searches (CUDA events); and the per-point path with each phase reduction
    (FP64, double-float, FP32) on the first n_phase stars, one search each. The
    agreement of each mode with the FP64 oracle is the precision tests' part."""
    import torch
    import synth
    from paper_2302_01293_gb300 import qlpbls
    b = synth.multi_sector(n_stars=n_stars, seed=3, max_sectors=13)
    res = {"workload": f"{n_stars} multi-sector stars, 1-13 sectors at 200 s (seed 3)",
           "points": int(b.offsets[-1])}
    stream = torch.cuda.current_stream()
    for name, p in (("exact", qlpbls.Params()), ("compensated", qlpbls.Params(sum_mode=qlpbls.SUM_COMP))):
        plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, p)
        out = plan.alloc_outputs()
        ms = _timed_searches(plan, out, steps, stream)
        res[name] = {"value": plan.work / (ms * 1e-3), "unit": UNIT, "ms": ms,
                     "point_freq": plan.work, "windowed_stars": plan.n_windowed,
                     "exact_path_stars": plan.n_exact_stars}
        del plan, out
    sub = b.subset(range(min(n_phase, n_stars)))
    res["points_phase_modes"] = {"stars": sub.n_stars, "points": int(sub.offsets[-1])}
    for name, mode in (("fp64", qlpbls.PHASE_FP64), ("double_float", qlpbls.PHASE_DF),
                       ("fp32", qlpbls.PHASE_FP32)):
        plan = qlpbls.Plan(sub.offsets, sub.t, sub.y, sub.dy, sub.rho, sub.rstar,
                           qlpbls.Params(method=qlpbls.METHOD_POINTS, phase_mode=mode))
        out = plan.alloc_outputs()
        ms = _timed_searches(plan, out, 1, stream)
        res["points_phase_modes"][name] = {"value": plan.work / (ms * 1e-3), "unit": UNIT, "ms": ms,
                                           "point_freq": plan.work}
        del plan, out
    return res


def profile_case(which: str):
    """One small launch of a kernel for a profiler capture, checked for device flags:
    fixed: the exact search (and S/N) of 1,024 uneven single-sector stars; stats: the
    candidate statistics of 2,048 such stars after their search; conv: the tensor-core
    convolution (64 -> 64 channels, kernel 9) on 128 x 4,096 x 64 BF16 activations;
    train: three training steps of the proposal network on a batch of 128 x 4,096 bins."""
    import torch
    import synth
    from paper_2302_01293_gb300 import qlpbls
    torch.cuda.set_device(0)
    if which in ("fixed", "stats"):
        b = synth.uneven_single_sector(n_stars=1024 if which == "fixed" else 2048, seed=2)
        plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
        out = plan.search()
        plan.snr(out)
        if which == "stats":
            plan.candidate_stats(out)
        torch.cuda.synchronize()
        if plan.device_status():
            raise RuntimeError("device flags")
    elif which == "train":
        net = qlpbls.CNN(max_batch=128, length=4096, seed=0)
        g = torch.Generator(device="cpu").manual_seed(5)
        x0 = torch.zeros(128, 4096, qlpbls.CNN_IN_CH, dtype=torch.bfloat16, device="cuda")
        x0[..., 0] = torch.randn(128, 4096, generator=g).to(torch.bfloat16).cuda()
        x0[..., 1] = 1
        lab = torch.zeros(128, 4096, device="cuda")
        lab[:, 2000:2003] = 1.0
        for _ in range(3):
            net.train_step(x0, lab, 16.0, 1e-4)
        torch.cuda.synchronize()
        if not np.isfinite(net.loss()):
            raise RuntimeError("non-finite loss")
    else:
        g = torch.Generator(device="cpu").manual_seed(5)
        x = torch.randn(128, 4096, 64, generator=g).to(torch.bfloat16).cuda()
        w = (torch.randn(9, 64, 64, generator=g) * 0.05).cuda()
        bias = torch.zeros(64).cuda()
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        wp = qlpbls.pack_w64(w)
        y = qlpbls.conv64(x, wp, bias, err=err)
        qlpbls.conv64(x, wp, bias, out=y, err=err)
        torch.cuda.synchronize()
        if int(err.item()):
            raise RuntimeError("device flags")
    print("ok", which)


def cpu_baseline(batch, n_sample: int):
    """Time the FP64 oracle (plan + BLS + S/N) on the first n_sample stars, all cores."""
    import multiprocessing as mp
    import oracle  # test infrastructure; only this baseline leg runs it
    sub = batch.subset(range(min(n_sample, batch.n_stars)))
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    plans = oracle.plan_batch(sub)
    res = oracle.bls_batch(plans, processes=cores)
    for pl, r in zip(plans, res):
        if pl.freqs.shape[0]:
            oracle.spectral_snr(pl.freqs, r.sr)
    dt = time.perf_counter() - t0
    work = float(sum(pl.tp.shape[0] * pl.freqs.shape[0] for pl in plans))
    return {"value": work / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {sub.n_stars} stars of the workload ({work:.3e} point-freq, "
                      f"{dt:.1f} s wall, FP64 plan + C BLS + S/N, spawn pool of {cores})"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    batch = synth.uneven_single_sector(n_stars=args.stars, seed=args.seed)
    n_sample = max(8, min(args.cpu_sample_stars // 4, 64))
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(batch.subset(range(i * n_sample, (i + 1) * n_sample)), n_sample)
        if i >= args.warmup:
            vals.append(cb)
    v = float(np.median([c["value"] for c in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "uneven_single_sector_200s", "stars": args.stars,
                       "sample_stars_per_step": n_sample},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "value": v, "unit": UNIT,
                             "sample": f"{n_sample} stars per step: " + vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case:
        profile_case(args.case)
        return

    import torch
    import torch.distributed as dist
    import synth
    from paper_2302_01293_gb300 import qlpbls, shard

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.workload == "multi_sector":
        batch = synth.multi_sector(n_stars=args.stars, seed=3 + 1000 * rank, max_sectors=13)
    else:
        batch = synth.uneven_single_sector(n_stars=args.stars, seed=args.seed + 1000 * rank)
    stream = torch.cuda.current_stream()
    # launch settings from the autotuner (timed on a sample of the batch; untimed here)
    t0 = time.perf_counter()
    params = qlpbls.Params(method=args.method, sum_mode={"fixed": qlpbls.SUM_FIXED, "fixed64": qlpbls.SUM_FIXED64, "comp": qlpbls.SUM_COMP,
                                                         "plain": qlpbls.SUM_PLAIN}[args.sum_mode])
    if not args.no_tune:
        params, _ = qlpbls.autotune(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar,
                                    params, sample_stars=args.tune_sample)
    t_tune = time.perf_counter() - t0
    plan = qlpbls.Plan(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar, params)
    out = plan.alloc_outputs()
    plan.kernel_timing(True)  # events around the main search kernel, inside the graph
    # the step as two CUDA graphs: the search (prep + persistent kernels), the S/N
    plan.graph_capture(out, parts=1)
    plan.graph_capture(out, parts=2)
    for _ in range(max(3, args.warmup)):
        plan.graph_launch(1)
        plan.graph_launch(2)
    flags = plan.device_status()
    if flags:
        raise RuntimeError(f"device flags {flags}")

    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    k_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e_start.record(stream)
    for i in range(args.steps):
        k_ev[i][0].record(stream)
        plan.graph_launch(1)
        k_ev[i][1].record(stream)
        plan.graph_launch(2)
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e_start.elapsed_time(e_end) / args.steps
    ms_search = float(np.mean([a.elapsed_time(b) for a, b in k_ev]))
    # the main search kernel alone: the plan's events inside the search graph, one
    # replay at a time (after the timed region)
    k_times = []
    for _ in range(args.steps):
        plan.graph_launch(1)
        torch.cuda.synchronize()
        k_times.append(plan.kernel_time())
    ms_kernel = float(np.mean([t for t, _ in k_times]))
    kernel_id = k_times[0][1]
    flags = plan.device_status()
    if flags:
        raise RuntimeError(f"device flags {flags}")
    # post-BLS statistics of every star's best candidate (Sec. 2.2 items 2-5), timed apart
    stats_buf = plan.candidate_stats(out)
    s_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize()
    s_ev[0].record(stream)
    for _ in range(3):
        plan.candidate_stats(out, stats_buf)
    s_ev[1].record(stream)
    torch.cuda.synchronize()
    st_host = plan.stats_host(stats_buf)
    cand_stats = {"ms": s_ev[0].elapsed_time(s_ev[1]) / 3, "stars": int(plan.n_stars),
                  "fitted": int(np.sum(st_host["status"] == 0)), "detected": int(np.sum(st_host["detected"])),
                  "what": "trapezoid fit, white/red noise, S/N_pink, counts, detection per star (one launch)"}
    # all ranks' work over the slowest rank's time (each rank searched its own stars)
    total_work, ms_max = shard.job_totals(plan.work, ms)
    value = total_work / (ms_max * 1e-3)

    # end to end through the public host-buffer call
    e2e = None
    if not args.no_e2e:
        h2d = int(batch.offsets.nbytes + batch.t.nbytes + batch.y.nbytes + batch.dy.nbytes
                  + batch.rho.nbytes + batch.rstar.nbytes)
        times = []
        res = None
        for i in range(2):
            barrier()
            t0 = time.perf_counter()
            res = qlpbls.run_host(batch.offsets, batch.t, batch.y, batch.dy, batch.rho,
                                  batch.rstar, params)
            times.append(time.perf_counter() - t0)
        _, e2e_s = shard.job_totals(0.0, min(times))
        d2h = int(res["best"].nbytes)
        e2e = {"value": total_work / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "seconds_per_step": e2e_s,
               "includes": "host plan (grid) + H2D + search + S/N + D2H of best"}

    peaks, src = _peaks()
    sm_clock = peaks.get("sm_max_mhz", 2070.0) * 1e6
    peak_ops = N_SMS * FP32_LANES_PER_SM * sm_clock / 1e12  # T lane ops / s
    peak_smem = N_SMS * SMEM_BYTES_PER_CLK_PER_SM * sm_clock / 1e9  # GB/s
    cells_dominant = plan.work_cells >= plan.work_points
    if kernel_id == 2:
        e64 = plan.exact_edges - plan.narrow_edges
        ops = (e64 * EXACT_OPS_PER_EDGE + plan.narrow_edges * EXACT32_OPS_PER_EDGE
               + plan.exact_bins * EXACT_OPS_PER_BIN)
        achieved = ops / (ms_kernel * 1e-3) / 1e12
        smem_gbs = (e64 * EXACT_SMEM_BYTES_PER_EDGE + plan.narrow_edges * EXACT32_SMEM_BYTES_PER_EDGE
                    + plan.exact_bins * EXACT_SMEM_BYTES_PER_BIN) / (ms_kernel * 1e-3) / 1e9
        kernel = "cells_fixed_kernel (exact cell path; CUDA events around the launch inside the graph)"
        unit_note = (f"{plan.narrow_edges:.4e} bin edges on 32-bit tables x {EXACT32_OPS_PER_EDGE} lane ops "
                     f"({EXACT32_SMEM_BYTES_PER_EDGE} shared bytes) + {e64:.4e} on 64-bit tables x "
                     f"{EXACT_OPS_PER_EDGE} ({EXACT_SMEM_BYTES_PER_EDGE} bytes) + {plan.exact_bins:.4e} box "
                     f"start bins x {EXACT_OPS_PER_BIN} ({EXACT_SMEM_BYTES_PER_BIN} bytes) per launch")
    elif cells_dominant:
        ops = plan.edges * CELL_OPS_PER_EDGE[params.sum_mode]
        achieved = ops / (ms_search * 1e-3) / 1e12
        smem_gbs = plan.edges * CELL_SMEM_BYTES_PER_EDGE[params.sum_mode] / (ms_search * 1e-3) / 1e9
        kernel = "cells_kernel (search-call duration: includes prep_cells)"
        unit_note = f"{plan.edges:.4e} bin edges x {CELL_OPS_PER_EDGE[params.sum_mode]} ops"
    else:
        achieved = plan.work * FP32_OPS_PER_EVAL / (ms_search * 1e-3) / 1e12
        smem_gbs = None
        kernel = "bls_kernel (search-call duration: includes prep)"
        unit_note = f"{plan.work:.4e} point-freq x {FP32_OPS_PER_EVAL} ops"
    # DRAM traffic of one launch of the timed kernel: ncu capture of the same kernel on
    # 1,024 stars of this workload, scaled by points to the default batch
    traffic = None
    default_batch = args.workload == "uneven" and args.stars == 4096 and args.seed == 2
    if cells_dominant and kernel_id == 1 and default_batch and params.sum_mode == 1:
        traffic = 423.0e6 * plan.n_points / 10638874

    if kernel_id == 2 and default_batch:
        # cells_fixed_kernel: ncu capture on 1,024 stars of this workload (702.8 MB read +
        # 236.4 MB written), scaled by points (tables, records and outputs grow with them)
        traffic = 939.2e6 * plan.n_points / 10638874
    # the same launch in the method's own unit: point-frequency pairs per second against
    # the FP32-issue roof of a per-point search (14 lane operations per pair: double-float
    # phase, bin index and the run sums), the unit in which the edge formulation's lower
    # work count shows
    pf_rate = plan.work / (ms_kernel * 1e-3)
    pf_roof = peak_ops * 1e12 / 14.0
    roofline_pf = {"achieved": pf_rate, "roof": pf_roof, "unit": "point-freq/s", "frac": pf_rate / pf_roof,
                   "roof_source": "issue peak / 14 lane operations per point-frequency pair"}
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "TFLOP/s",
                "frac": achieved / peak_ops, "traffic": traffic, "kernel": kernel,
                "per_point_freq": roofline_pf,
                "algorithmic": unit_note,
                "peak_source": f"152 SMs x 128 FP32 lanes x {sm_clock/1e6:.0f} MHz ({src} max clock)",
                "smem": None if smem_gbs is None else
                {"achieved_gbs": smem_gbs, "peak_gbs": peak_smem, "frac": smem_gbs / peak_smem,
                 "peak_source": "152 SMs x 128 B/clk x max clock"}}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(batch, args.cpu_sample_stars)
        learned_line = None
        multi_line = None
        single_line = None
        if not args.no_multi and world == 1:
            single_line = single_star_line(10)
            multi_line = multi_sector_line(2)
        if not args.no_learned and world == 1:
            learned_line = learned_comparison(args)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": ("int64 fixed-point sums, f32 box scores, FP64 bin decisions" if kernel_id == 2
                          else "f32 sums, FP64 prefix sums, FP64 bin decisions"), "data": "synthetic",
                "config": {"workload": ("uneven_single_sector_200s" if args.workload == "uneven"
                                        else "multi_sector_200s_1to13"), "stars_per_gpu": args.stars,
                           "points": plan.n_points, "trial_freqs": plan.n_freq_total,
                           "point_freq_per_gpu": plan.work, "bin_edges": plan.edges,
                           "cell_path_stars": plan.n_cell_stars, "phase_mode": "DF",
                           "autotuned": {"warps_per_block": params.warps_per_block,
                                         "chunk_freqs": params.chunk_freqs,
                                         "cell_window": params.cell_window,
                                         "sample_stars": None if args.no_tune else args.tune_sample,
                                         "seconds": t_tune},
                           "launch": "CUDA graphs (search, S/N) per step",
                           "sum_mode": ["PLAIN", "COMP", "FIXED", "FIXED64"][params.sum_mode],
                           "l2": "inputs larger than L2 (light curves "
                           f"{plan.n_points * 24 / 1e6:.0f} MB FP64)", "parallelism": f"replicas x{world}"},
                "ms_search": ms_search, "ms_kernel": ms_kernel,
                "exact_path_stars": plan.n_exact_stars,
                "exact_path_32bit_table_stars": plan.n_narrow_stars,
                # per step: S/N and the search's launches (per path in use its preparation
                # and search kernels, the exact one per kind of table)
                "gpu_launches": args.steps * (1 + plan.search_launches),
                "clocks": clk, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "candidate_stats": cand_stats,
                "single_star": single_line,
                "multi_sector": multi_line,
                "learned": learned_line}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

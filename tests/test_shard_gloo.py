"""Host logic of the multi-rank path on CPU (gloo, world size 2): cost model and
LPT partition, the job totals (sum of work, max of time), the gather of best
records into global star order, and a failing rank surfacing as an error in
bounded time. The per-star search here is the FP64 oracle (CPU), so no GPU is
needed; on GPUs each rank runs the library on its shard the same way."""
import os
import socket
import time

import numpy as np
import pytest

import oracle
import synth
from paper_2302_01293_gb300 import shard

REC = np.dtype([("f_idx", "<i8"), ("period", "<f8"), ("snr", "<f8")])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _best_oracle(batch, stars):
    out = np.zeros(len(stars), REC)
    for i, s in enumerate(stars):
        t, y, dy = batch.star(int(s))
        pl = oracle.plan_star(t, y, dy, float(batch.rho[s]), 1.0)
        res = oracle.bls_star(pl)
        snr, _, sigma = oracle.spectral_snr(pl.freqs, res.sr)
        b = oracle.best_candidate(pl, res, snr, sigma)
        k = int(np.argmax(snr)) if b is not None else -1
        out[i] = (k, 1.0 / pl.freqs[k] if k >= 0 else np.nan, snr[k] if k >= 0 else np.nan)
    return out


def _worker(rank, world, port, out_dir, fail_rank):
    import datetime
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        batch = synth.tiny_batch(n_stars=7, seed=21)
        parts = shard.partition(shard.star_cost(batch.offsets, batch.t, batch.rho), world)
        mine = parts[rank]
        if rank == fail_rank:
            raise RuntimeError("simulated rank failure before the gather")
        best = _best_oracle(batch, mine)
        work, ms = shard.job_totals(float(len(mine)), 10.0 * (rank + 1))
        allbest = shard.gather_best(best, mine, batch.n_stars)
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), allbest)
            np.save(os.path.join(out_dir, "totals.npy"), np.array([work, ms]))
    except Exception as e:  # each rank's own outcome, whichever the spawner reports first
        with open(os.path.join(out_dir, f"rank{rank}.err"), "w") as fh:
            fh.write(f"{type(e).__name__}: {e}")
        raise
    finally:
        dist.destroy_process_group()


def test_partition_is_lpt_and_complete():
    cost = np.array([5.0, 1.0, 4.0, 4.0, 2.0, 3.0, 0.0])
    parts = shard.partition(cost, 3)
    allidx = np.sort(np.concatenate(parts))
    assert allidx.tolist() == list(range(7))
    loads = sorted(float(cost[p].sum()) for p in parts)
    # LPT on these costs: {5, 1} {4, 2} {4, 3} (the zero-cost star anywhere)
    assert loads == [6.0, 6.0, 7.0]
    assert shard.partition(cost, 1)[0].tolist() == list(range(7))
    with pytest.raises(ValueError):
        shard.partition(cost, 0)


def test_star_cost_scaling():
    # cost ~ N * T * sqrt(rho): doubling the points, the span or 4x the density doubles it
    t1 = np.linspace(0, 10, 100)
    t2 = np.linspace(0, 10, 200)
    t3 = np.linspace(0, 20, 100)
    t = np.concatenate([t1, t2, t3, t1])
    off = np.array([0, 100, 300, 400, 500])
    c = shard.star_cost(off, t, np.array([1.0, 1.0, 1.0, 4.0]))
    np.testing.assert_allclose(c[1:] / c[0], [2.0, 2.0, 2.0])
    assert shard.star_cost(off, t, np.array([np.nan, 1.41, -1, 1.41]))[0] == pytest.approx(c[0] * np.sqrt(1.41))


def _spawn(fail_rank, tmp_path):
    import torch.multiprocessing as tmp
    port = _free_port()
    tmp.spawn(_worker, args=(2, port, str(tmp_path), fail_rank), nprocs=2, join=True)


def test_two_ranks_gather_equals_single_process(tmp_path):
    _spawn(-1, tmp_path)
    got = np.load(tmp_path / "gathered.npy")
    batch = synth.tiny_batch(n_stars=7, seed=21)
    ref = _best_oracle(batch, range(batch.n_stars))
    assert np.array_equal(got["f_idx"], ref["f_idx"])
    np.testing.assert_array_equal(got["snr"], ref["snr"])
    work, ms = np.load(tmp_path / "totals.npy")
    assert work == 7.0 and ms == 20.0


def _oracle_search(offsets, t, y, dy, rho, rstar, params):
    out = np.zeros(len(offsets) - 1, REC)
    for s in range(len(offsets) - 1):
        a, b = offsets[s], offsets[s + 1]
        pl = oracle.plan_star(t[a:b], y[a:b], dy[a:b], float(rho[s]), 1.0)
        res = oracle.bls_star(pl)
        snr, _, sigma = oracle.spectral_snr(pl.freqs, res.sr)
        k = int(np.argmax(snr)) if oracle.best_candidate(pl, res, snr, sigma) is not None else -1
        out[s] = (k, 1.0 / pl.freqs[k] if k >= 0 else np.nan, snr[k] if k >= 0 else np.nan)
    return out


def _sharded_worker(rank, world, port, out_dir):
    import datetime
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        b = synth.tiny_batch(n_stars=9, seed=23)
        got = shard.search_sharded(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, search_fn=_oracle_search)
        if rank == 0:
            np.save(os.path.join(out_dir, "sharded.npy"), got)
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def test_sharded_search_driver_equals_single_process(tmp_path):
    import torch.multiprocessing as tmp
    tmp.spawn(_sharded_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got = np.load(tmp_path / "sharded.npy")
    b = synth.tiny_batch(n_stars=9, seed=23)
    ref = _oracle_search(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar, None)
    assert np.array_equal(got["f_idx"], ref["f_idx"])
    np.testing.assert_array_equal(got["snr"], ref["snr"])


def test_failing_rank_is_reported(tmp_path):
    # rank 1 fails before the collectives; rank 0's next collective ends with an
    # error within the process group's timeout (or the spawner stops it once rank 1
    # has exited), and nothing is gathered
    import torch.multiprocessing as tmp
    t0 = time.monotonic()
    with pytest.raises(tmp.ProcessRaisedException):
        _spawn(1, tmp_path)
    assert time.monotonic() - t0 < 60.0
    assert "simulated rank failure" in (tmp_path / "rank1.err").read_text()
    assert not (tmp_path / "gathered.npy").exists()

"""The allocation-free entry point qlp_bls_search_static against the planned path.

Some callers cannot allocate device memory themselves (a host framework owns
every device allocation, or the service's device memory is fixed up front);
qlp_bls_search_static serves them from a static device scratch array that every
call shares and that keeps the previous call's contents. Here it is called
through the C ABI on a large star, then on a smaller star with fewer points and
frequencies, then on the large star again, and each result is compared with
qlp_bls_plan + qlp_bls_search on the same star and with the oracle, with the
tolerances of the other GPU tests (tests/parity.py); the call's device error
word must come back clean. This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from paper_2302_01293_gb300 import qlpbls
from parity import SR_RTOL, compare_spectrum, oracle_star

pytestmark = pytest.mark.gpu


def _static_inputs(batch, s, params):
    import torch
    t, y, dy = batch.star(s)
    g = qlpbls.star_grid(t, y, dy, float(batch.rho[s]), params)
    assert g["status"] == 0
    ok = np.isfinite(t) & np.isfinite(y) & np.isfinite(dy) & (dy > 0)
    dev = torch.device("cuda")
    tp = torch.tensor(t[ok] - g["t_ref"], dtype=torch.float64, device=dev)
    yy = torch.tensor(y[ok], dtype=torch.float64, device=dev)
    dd = torch.tensor(dy[ok], dtype=torch.float64, device=dev)
    return g, tp, yy, dd


def _planned(batch, s, params):
    import torch
    plan = qlpbls.Plan(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar, params)
    ref = plan.search()
    torch.cuda.synchronize()
    sl = plan.star_slice(s)
    return plan.freqs[sl], {k: v[sl].cpu().numpy() for k, v in ref.items() if k != "best"}


def _static_call(batch, s, params, label):
    import torch
    g, tp, yy, dd = _static_inputs(batch, s, params)
    freqs, ref = _planned(batch, s, params)
    assert np.array_equal(g["freqs"], freqs)
    n_f = freqs.shape[0]
    out = {k: torch.full((n_f,), 7, dtype=dt, device="cuda") for k, dt in
           (("sr", torch.float32), ("qidx", torch.uint8), ("kbin", torch.int32),
            ("s", torch.float32), ("r", torch.float32))}
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    qlpbls.search_static(tp, yy, dd, g["baseline"], g["freqs"], g["qmins"], out, params, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0, f"{label}: device error bits {int(flags.item())}"
    res = {k: v.cpu().numpy() for k, v in out.items()}
    rel = np.abs(res["sr"].astype(np.float64) - ref["sr"]) / np.maximum(ref["sr"], 1e-30)
    assert rel.max() <= SR_RTOL, f"{label}: SR rel {rel.max()} against the planned search"
    assert np.mean(res["qidx"] == ref["qidx"]) > 0.99, label
    pl, ores = oracle_star(batch, s)
    compare_spectrum(pl, ores, res, slice(0, n_f), label=label)
    return tp.numel(), n_f


def test_static_search_matches_planned_search_across_sizes(gpu_lib):
    params = qlpbls.Params()
    big = synth.uneven_single_sector(n_stars=4, seed=31)
    nfs = [qlpbls.star_grid(*big.star(s), float(big.rho[s]), params)["freqs"].shape[0] for s in range(4)]
    sb = int(np.argmax(nfs))
    small = synth.single_star()
    n1, f1 = _static_call(big, sb, params, "large star, first call")
    n2, f2 = _static_call(small, 0, params, "smaller star after it")
    assert n2 < n1 and f2 < f1
    n3, f3 = _static_call(big, sb, params, "large star again")
    assert (n3, f3) == (n1, f1)


def test_static_search_options(gpu_lib):
    # warps_per_block 32 runs as 16 (as the planned path's point kernel); the
    # per-duration histograms are not built into this entry point
    b = synth.single_star()
    _static_call(b, 0, qlpbls.Params(warps_per_block=32), "warps 32")
    import torch
    g, tp, yy, dd = _static_inputs(b, 0, qlpbls.Params())
    n_f = g["freqs"].shape[0]
    out = {k: torch.zeros(n_f, dtype=dt, device="cuda") for k, dt in
           (("sr", torch.float32), ("qidx", torch.uint8), ("kbin", torch.int32),
            ("s", torch.float32), ("r", torch.float32))}
    with pytest.raises(qlpbls.QlpError) as ei:
        qlpbls.search_static(tp, yy, dd, g["baseline"], g["freqs"], g["qmins"], out,
                             qlpbls.Params(bin_mode=qlpbls.BIN_PER_Q))
    assert ei.value.code == qlpbls.ERR_UNSUPPORTED


def test_static_search_rejects_oversize(gpu_lib):
    import torch
    n = 2_000_000  # 24 B per point alone exceeds the 16 MiB scratch
    tp = torch.zeros(n, dtype=torch.float64, device="cuda")
    tp[1:] = torch.arange(1, n, dtype=torch.float64, device="cuda") * 1e-4
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    freqs = np.array([1.0, 1.1])
    qmins = np.array([0.05, 0.05])
    out = {k: torch.zeros(2, dtype=dt, device="cuda") for k, dt in
           (("sr", torch.float32), ("qidx", torch.uint8), ("kbin", torch.int32),
            ("s", torch.float32), ("r", torch.float32))}
    with pytest.raises(qlpbls.QlpError) as ei:
        qlpbls.search_static(tp, ones, ones * 1e-3, float(tp[-1]), freqs, qmins, out)
    assert ei.value.code == qlpbls.ERR_ARG

"""The allocation-free entry point qlp_bls_search_static against the planned path.

Some callers cannot allocate device memory themselves (a host framework owns
every device allocation, or the service's device memory is fixed up front);
qlp_bls_search_static serves them from a static device scratch array. Here it is
called twice in a row through the C ABI on the same star and each result is
compared with qlp_bls_plan + qlp_bls_search on that star, with the tolerances of
the other GPU tests (tests/parity.py). This file is collected last on purpose.
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


@pytest.mark.parametrize("which", ["uneven", "single"])
def test_static_search_matches_planned_search(gpu_lib, which):
    import torch
    batch = synth.single_star() if which == "single" else synth.uneven_single_sector(n_stars=2, seed=31)
    s = 0
    params = qlpbls.Params()
    plan = qlpbls.Plan(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar, params)
    ref = plan.search()
    torch.cuda.synchronize()
    sl = plan.star_slice(s)
    ref_sr = ref["sr"][sl].cpu().numpy()
    g, tp, yy, dd = _static_inputs(batch, s, params)
    assert np.array_equal(g["freqs"], plan.freqs[sl])
    n_f = g["freqs"].shape[0]
    pl, ores = oracle_star(batch, s)
    for call in range(2):
        out = {k: torch.full((n_f,), 7, dtype=v.dtype, device=v.device)
               for k, v in ref.items() if k in ("sr", "qidx", "kbin", "s", "r")}
        qlpbls.search_static(tp, yy, dd, g["baseline"], g["freqs"], g["qmins"], out, params)
        torch.cuda.synchronize()
        sr = out["sr"].cpu().numpy()
        rel = np.abs(sr.astype(np.float64) - ref_sr) / np.maximum(ref_sr, 1e-30)
        assert rel.max() <= SR_RTOL, f"call {call}: SR rel {rel.max()}"
        res = {k: v.cpu().numpy() for k, v in out.items()}
        compare_spectrum(pl, ores, res, slice(0, n_f), label=f"static call {call}")
        agree = np.mean(res["qidx"] == ref["qidx"][sl].cpu().numpy())
        assert agree > 0.99


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
    with pytest.raises(qlpbls.QlpError):
        qlpbls.search_static(tp, ones, ones * 1e-3, float(tp[-1]), freqs, qmins, out)

"""Parity helpers: run the CUDA path through the C ABI and compare it with the
FP64 oracle on the same seeded inputs.

Tolerances (stated once, used by every GPU parity test):
  * SR: relative 1e-5 (the FP32 residue of an FP64-binned histogram);
  * duration index j and start bin k of each frequency's maximum: equal, unless
    the oracle's own residue at the GPU's (j, k) is within relative 1e-5 of its
    maximum (a near tie, where either answer is correct);
  * S/N: absolute 1e-4 where |S/N| <= 100; above that relative 1e-6 (one FP32
    ulp of SR already moves S/N by ~6e-8 of its value);
  * best frequency index: equal, unless the oracle's S/N at the GPU's index is
    within the S/N tolerance of the oracle's maximum; P, q exact given the index,
    T0 absolute 1e-9 d, depth relative 1e-5.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import bls as ob

SR_RTOL = 1e-5
SNR_ATOL = 1e-4
SNR_RTOL_HIGH = 1e-6


def snr_tol(v):
    v = np.abs(np.asarray(v, np.float64))
    return np.where(v <= 100.0, SNR_ATOL, SNR_RTOL_HIGH * v)


def run_gpu(batch, params, with_snr=True):
    import torch
    from paper_2302_01293_gb300 import qlpbls
    plan = qlpbls.Plan(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar, params)
    out = plan.search()
    if with_snr:
        plan.snr(out)
    flags = plan.device_status()
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "best"}
    res["best"] = plan.best_host(out) if with_snr else None
    res["flags"] = flags
    res["plan"] = plan
    return res


def oracle_star(batch, s, params=None):
    t, y, dy = batch.star(s)
    p = params or oracle.Params()
    pl = oracle.plan_star(t, y, dy, float(batch.rho[s]), float(batch.rstar[s]), p)
    res = oracle.bls_star(pl)
    return pl, res


def compare_spectrum(pl, ores, g, sl, label=""):
    """Compare one star's SR / argmax boxes; returns a dict of stats."""
    sr_g = g["sr"][sl].astype(np.float64)
    q_g = g["qidx"][sl].astype(np.int64)
    k_g = g["kbin"][sl].view(np.uint32).astype(np.int64)
    s_g = g["s"][sl].astype(np.float64)
    r_g = g["r"][sl].astype(np.float64)
    n = pl.freqs.shape[0]
    assert sr_g.shape[0] == n, label
    none_o = ores.j < 0
    assert np.array_equal(q_g == 255, none_o), label
    assert np.all(k_g[none_o] == 0xFFFFFFFF), label
    ok = ~none_o
    denom = np.maximum(np.abs(ores.sr), 1e-300)
    rel = np.where(ok, np.abs(sr_g - ores.sr) / denom, 0.0)
    assert rel.max(initial=0.0) <= SR_RTOL, f"{label} SR rel {rel.max()} at {int(np.argmax(rel))}"
    mism = np.nonzero(ok & ((q_g != ores.j) | (k_g != ores.k)))[0]
    for i in mism:
        v = ob.box_value(pl, int(i), int(q_g[i]), int(k_g[i]))
        assert v >= ores.sr[i] * (1 - SR_RTOL), (
            f"{label} f#{i}: GPU box (j={q_g[i]}, k={k_g[i]}) oracle value {v} vs max {ores.sr[i]} "
            f"at (j={ores.j[i]}, k={ores.k[i]})")
    same = ok & (q_g == ores.j) & (k_g == ores.k)
    if same.any():
        np.testing.assert_allclose(r_g[same], ores.r[same], rtol=2e-6, atol=1e-12, err_msg=label)
        np.testing.assert_allclose(s_g[same], ores.s[same], rtol=1e-5, atol=1e-6 * np.abs(ores.s).max(),
                                   err_msg=label)
    return dict(n=n, sr_rel_max=float(rel.max(initial=0.0)), near_ties=int(mism.shape[0]))


def compare_snr(pl, ores, g, sl, best_g, label=""):
    snr_o, _, sigma = oracle.spectral_snr(pl.freqs, ores.sr)
    snr_g = g["snr"][sl].astype(np.float64)
    d = np.abs(snr_g - snr_o)
    tol = snr_tol(snr_o)
    assert np.all(d <= tol), f"{label} S/N worst {float((d - tol).max())} at {int(np.argmax(d - tol))}"
    bo = oracle.best_candidate(pl, ores, snr_o, sigma)
    if bo is None:
        assert best_g["f_idx"] == -1, label
        return dict(snr_abs_max=float(d.max(initial=0.0)))
    fi = int(best_g["f_idx"])
    if fi != bo["f_idx"]:
        assert snr_o[fi] >= bo["snr"] - snr_tol(bo["snr"]), f"{label} best index {fi} vs {bo['f_idx']}"
        return dict(snr_abs_max=float(d.max()), best_tie=True)
    assert best_g["period"] == bo["period"], label
    assert best_g["q"] == bo["q"] and best_g["j"] == bo["j"], label
    assert best_g["k"] == bo["k"] and best_g["m"] == bo["m"] and best_g["nbins"] == bo["nbins"], label
    assert abs(best_g["t0"] - bo["t0"]) <= 1e-9, label
    assert abs(best_g["depth"] - bo["depth"]) <= 1e-5 * abs(bo["depth"]) + 1e-12, label
    return dict(snr_abs_max=float(d.max()), best_tie=False)

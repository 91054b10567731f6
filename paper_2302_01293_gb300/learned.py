"""Learned period proposal (not in the paper; it narrows the paper's full-grid
search): a coarse BLS spectrum on a 4,096-bin log-period grid goes through the
proposal CNN, the top-K bins become period windows, and only the paper's grid
frequencies inside those windows are searched at full resolution, scored
against the coarse spectrum's trend and sigma_SR.

Every numeric step runs in the CUDA library (coarse plan, search, S/N, input
tensor, CNN, top-K, windowed plan, search, S/N) and the coarse-grid arithmetic
(bin periods, nearest bins, windows) in its host code; this module only
sequences the calls, as the library does behind qlp_bls_search_learned.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import qlpbls


def coarse_params(base: qlpbls.Params | None = None) -> qlpbls.Params:
    p = dataclasses.replace(base or qlpbls.Params())
    p.grid_mode = 1
    return p


def bin_period(k, p: qlpbls.Params):
    """Period (days) of coarse bin k (qlp_bls_coarse_periods)."""
    k = np.asarray(k, np.float64)
    return qlpbls.coarse_periods(k.reshape(-1), p).reshape(k.shape)


def period_bin(period, p: qlpbls.Params):
    """Nearest coarse bin of a period (qlp_bls_coarse_bins; -1 off the grid)."""
    per = np.asarray(period, np.float64)
    return qlpbls.coarse_bins(per.reshape(-1), p).reshape(per.shape).astype(np.int64)


class CoarseStage:
    """Coarse plan, search and S/N of a batch, its trend records and the
    network input tensor [n_stars, bins, CNN_IN_CH]."""

    def __init__(self, batch, base: qlpbls.Params | None = None, stream=None):
        self.params = coarse_params(base)
        self.plan = qlpbls.Plan(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar,
                                self.params, stream=stream)
        self.out = self.plan.search(stream=stream)
        self.trend = self.plan.alloc_trend()
        self.plan.snr(self.out, stream=stream, trend_out=self.trend)
        self.x0 = self.plan.coarse_tensor(self.out, stream=stream)


def labels(batch, p: qlpbls.Params, device, half_width: int = 1):
    """1 on the coarse bins within half_width of the injected period's bin, else 0."""
    import torch
    lab = torch.zeros(batch.n_stars, p.coarse_bins, dtype=torch.float32)
    k = period_bin(np.where(batch.inj, batch.period, 1.0), p)
    for s in np.nonzero(batch.inj & (k >= 0))[0]:
        a, b = max(0, int(k[s]) - half_width), min(p.coarse_bins, int(k[s]) + half_width + 1)
        lab[s, a:b] = 1.0
    return lab.to(device)


def windows_from_bins(bins, p: qlpbls.Params, half_width: float = 1.0):
    """Frequency windows [1/P(k + w), 1/P(k - w)] for every valid proposed bin k
    (qlp_bls_proposal_windows, the windows the one-call path uses)."""
    return qlpbls.proposal_windows(bins, p, half_width)


def refine(batch, windows, trend, base: qlpbls.Params | None = None, stream=None):
    """Full-resolution search restricted to the windows, scored with the coarse trend."""
    p = dataclasses.replace(base or qlpbls.Params())
    p.grid_mode = 0
    plan = qlpbls.Plan(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar, p,
                       stream=stream, windows=windows)
    out = plan.search(stream=stream)
    plan.snr(out, stream=stream, trend_in=trend)
    return plan, out


def propose(net, x0, k: int, stream=None):
    """Top-k coarse bins per star from the network's logits (device int32 [B, k])."""
    import torch
    rows = []
    for a in range(0, x0.shape[0], net.max_batch):
        xb = x0[a:a + net.max_batch].contiguous()
        logits = net.forward(xb, stream=stream)
        rows.append(qlpbls.topk(logits, xb, k, stream=stream))
    return torch.cat(rows, 0)


def propose_without_network(coarse: CoarseStage, k: int, stream=None):
    """Ablation: the top-k coarse bins by the coarse S/N itself (FP32; no network),
    as qlp_bls_search_learned ranks them without a network."""
    _, rows = coarse.plan.coarse_tensor(coarse.out, stream=stream, snr_rows=True)
    return qlpbls.topk(rows.contiguous(), coarse.x0, k, stream=stream)


def search_learned(batch, net, k: int = 32, base: qlpbls.Params | None = None, stream=None,
                   half_width: float = 1.0):
    """The learned path end to end in one library call (qlp_bls_search_learned);
    returns (best records, proposed bins [n_stars, k])."""
    return qlpbls.search_learned(batch.offsets, batch.t, batch.y, batch.dy, batch.rho, batch.rstar,
                                 net, k, half_width, coarse_params(base), stream=stream)


def search_with_bins(batch, coarse: CoarseStage, bins, base: qlpbls.Params | None = None, stream=None,
                     half_width: float = 1.0):
    """Windows around given coarse bins, refined and scored with the coarse trend:
    the last two stages of the learned path for proposals made elsewhere."""
    win = windows_from_bins(bins.cpu().numpy() if hasattr(bins, "cpu") else np.asarray(bins),
                            coarse.params, half_width)
    plan, out = refine(batch, win, coarse.trend, base, stream=stream)
    return plan.best_host(out)


def train(net, batches, epochs: int = 2, lr: float = 1e-3, pos_weight: float = 64.0, stream=None):
    """Adam over (x0, labels) device tensors; returns the loss after each epoch."""
    losses = []
    for _ in range(epochs):
        for x0, lab in batches:
            for a in range(0, x0.shape[0], net.max_batch):
                net.train_step(x0[a:a + net.max_batch].contiguous(), lab[a:a + net.max_batch].contiguous(),
                               pos_weight, lr, stream=stream)
        losses.append(net.loss(stream=stream))
    return losses


def recovered(best, batch, snr_min: float = 9.0, tol: float = 0.01):
    """Injected transit found: S/N above snr_min and |P / P_inj - 1| < tol."""
    ok = (best["f_idx"] >= 0) & (best["snr"] > snr_min)
    per = np.where(ok, best["period"], np.nan)
    return ok & batch.inj & (np.abs(per / np.where(batch.inj, batch.period, 1.0) - 1.0) < tol)

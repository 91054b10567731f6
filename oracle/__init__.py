"""FP64 CPU oracle for the QLP GPU transit search (arXiv:2302.01293).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA library.

It is a plain, slow, step-by-step restatement of the method:

* ``plan``  -- per-star search ranges (Sec. 2.1): stellar density default,
  Pmin where a = 2 R*, Pmax from the longest continuous stretch, the Keplerian
  duration range q in [0.5, 2] q_circ, the frequency grid, the bin count
  (noverlap) and the log-spaced duration grid (dlogq);
* ``bls``   -- the binned Box Least Squares signal residue SR(f) for every
  trial frequency (Sec. 2.1, 2.2 item 1; BLS of Kovacs et al. 2002), in plain
  C with FP64 arithmetic, one frequency at a time, direct window sums;
* ``snr``   -- the spectral S/N of Eq. 1 with the Sturges median-binned trend
  and sigma = 1.4826 MAD (Sec. 2.2 item 1) and the best-candidate record;
* ``stats`` -- the post-BLS statistics of Sec. 2.2 items 2-5 (trapezoid fit,
  white and red noise, signal-to-pink noise, transit counts, detection).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from .plan import Params, StarPlan, plan_star, plan_batch, q_min, freq_grid, nbins_of, m_of, n_q
from .bls import weights, bls_star, bls_batch
from .snr import sturges_nbins, spectral_snr, best_candidate

__all__ = [
    "Params", "StarPlan", "plan_star", "plan_batch", "q_min", "freq_grid", "nbins_of", "m_of", "n_q",
    "weights", "bls_star", "bls_batch", "sturges_nbins", "spectral_snr", "best_candidate",
]

"""Oracle: weights and the binned BLS residue spectrum (TEST INFRASTRUCTURE ONLY).

``weights`` follows the BLS normalisation (Kovacs et al. 2002, the estimator
Sec. 2.1 adopts): w_i = dy_i^-2 / sum dy^-2, ybar = sum w_i y_i, d_i = y_i - ybar,
with exactly rounded sums (``math.fsum``).

``bls_star`` runs the plain-C FP64 loop of ``bls_core.c`` (fold, histogram,
direct window sums, argmax) over every trial frequency of a star's plan.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "bls_core.c")
_LIB = os.path.join(_BUILD, "liboracle_bls.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, no floating-point contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            lib.oracle_bls_star.argtypes = [i64, P(d), P(d), P(d), i64, P(d), P(i32), P(i32), i32,
                                            P(d), P(i32), P(i32), P(d), P(d)]
            lib.oracle_bls_star.restype = ctypes.c_int
            lib.oracle_bls_box.argtypes = [i64, P(d), P(d), P(d), d, i32, i32, i32]
            lib.oracle_bls_box.restype = d
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def weights(y, dy):
    """(w, d, ybar): normalised inverse-variance weights and mean-subtracted flux."""
    y = np.asarray(y, np.float64); dy = np.asarray(dy, np.float64)
    inv = 1.0 / (dy * dy)
    wsum = math.fsum(inv.tolist())
    w = inv / wsum
    ybar = math.fsum((w * y).tolist())
    d = y - ybar
    return w, d, ybar


class StarBLS:
    """Per-frequency results of one star: SR, best duration index j, best start bin k,
    and the window sums s = sum w d and r = sum w of that box."""

    def __init__(self, sr, j, k, s, r):
        self.sr, self.j, self.k, self.s, self.r = sr, j, k, s, r


def bls_star(plan) -> StarBLS:
    nf = plan.freqs.shape[0]
    sr = np.zeros(nf); sb = np.zeros(nf); rb = np.zeros(nf)
    jb = np.full(nf, -1, np.int32); kb = np.full(nf, -1, np.int32)
    if nf == 0 or plan.status != 0:
        return StarBLS(sr, jb, kb, sb, rb)
    w, d, _ = weights(plan.y, plan.dy)
    wd = np.ascontiguousarray(w * d)
    tp = np.ascontiguousarray(plan.tp, np.float64)
    w = np.ascontiguousarray(w)
    freqs = np.ascontiguousarray(plan.freqs, np.float64)
    nb = np.ascontiguousarray(plan.nbins, np.int32)
    m = np.ascontiguousarray(plan.m, np.int32)
    lib = _load()
    rc = lib.oracle_bls_star(tp.shape[0], _ptr(tp, ctypes.c_double), _ptr(w, ctypes.c_double),
                             _ptr(wd, ctypes.c_double), nf, _ptr(freqs, ctypes.c_double),
                             _ptr(nb, ctypes.c_int32), _ptr(m, ctypes.c_int32), m.shape[1],
                             _ptr(sr, ctypes.c_double), _ptr(jb, ctypes.c_int32),
                             _ptr(kb, ctypes.c_int32), _ptr(sb, ctypes.c_double),
                             _ptr(rb, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle_bls_star failed")
    return StarBLS(sr, jb, kb, sb, rb)


def bls_star_per_q(plan, noverlap: float = 3.0, dlogq: float = 0.1) -> StarBLS:
    """The per-duration binning variant: for each duration q_j = q_min e^{j dlogq}
    its own histogram of ceil(noverlap / q_j) bins (bin width q_j / noverlap) and
    boxes of noverlap consecutive bins; SR(f) = the largest residue over j and k
    (ties: lower j, then lower k); j and k of the result refer to histogram j.
    Each histogram is the plain BLS of this module with one box width."""
    import dataclasses
    nf = plan.freqs.shape[0]
    nq = plan.m.shape[1]
    m_int = int(noverlap)
    sr = np.zeros(nf); sb = np.zeros(nf); rb = np.zeros(nf)
    jb = np.full(nf, -1, np.int32); kb = np.full(nf, -1, np.int32)
    for j in range(nq):
        e = math.exp(j * dlogq)
        nbj = np.array([int(math.ceil(noverlap / (q * e))) for q in plan.qmin], np.int32)
        sub = dataclasses.replace(plan, nbins=nbj, m=np.full((nf, 1), m_int, np.int32))
        r = bls_star(sub)
        take = (r.j >= 0) & ((jb < 0) | (r.sr > sr))
        sr[take] = r.sr[take]; sb[take] = r.s[take]; rb[take] = r.r[take]
        jb[take] = j; kb[take] = r.k[take]
    return StarBLS(sr, jb, kb, sb, rb)


def restrict(plan, idx):
    """The same star plan with only the trial frequencies plan.freqs[idx] (each
    frequency's search is independent of the others, Sec. 2.1), so that long
    multi-sector stars can be checked on sampled frequencies."""
    import dataclasses
    idx = np.asarray(idx, np.int64)
    return dataclasses.replace(plan, freqs=plan.freqs[idx], qmin=plan.qmin[idx],
                               nbins=plan.nbins[idx], m=plan.m[idx])


def box_value(plan, fidx: int, j: int, k: int) -> float:
    """Residue of box (j, k) at frequency index fidx (-1 when the window is invalid)."""
    w, d, _ = weights(plan.y, plan.dy)
    wd = np.ascontiguousarray(w * d)
    tp = np.ascontiguousarray(plan.tp, np.float64)
    w = np.ascontiguousarray(w)
    lib = _load()
    return float(lib.oracle_bls_box(tp.shape[0], _ptr(tp, ctypes.c_double), _ptr(w, ctypes.c_double),
                                    _ptr(wd, ctypes.c_double), float(plan.freqs[fidx]),
                                    int(plan.nbins[fidx]), int(plan.m[fidx, j]), int(k)))


def _work(args):
    plan = args
    return bls_star(plan)


def bls_batch(plans, processes: int = 1):
    """BLS of every star; ``processes > 1`` uses a spawn-started process pool."""
    if processes <= 1:
        return [bls_star(p) for p in plans]
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes) as pool:
        return pool.map(_work, plans, chunksize=1)

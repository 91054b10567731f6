"""CPU checks of the C ABI: the library builds and loads, exports every function
include/*.h declares, and its host planner reproduces the oracle's plan bit for bit.
No compute call touches a GPU here."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_2302_01293_gb300 import qlpbls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(qlp_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = qlpbls.lib()
    names = _declared()
    assert {"qlp_bls_plan", "qlp_bls_search", "qlp_bls_snr"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_every_exported_function_is_declared():
    import subprocess
    from paper_2302_01293_gb300 import build
    so = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("qlp_")}
    assert exported and exported <= _declared(), sorted(exported - _declared())


def test_params_default_matches_paper_settings():
    L = qlpbls.lib()
    p = qlpbls.CParams()
    L.qlp_bls_params_default(ctypes.byref(p))
    assert (p.samples_per_peak, p.dlogq, p.noverlap) == (2.0, 0.1, 3.0)
    assert (p.qmin_fac, p.qmax_fac, p.pmin_aR, p.gap_days, p.rho_default) == (0.5, 2.0, 2.0, 27.4, 1.41)
    assert ctypes.sizeof(qlpbls.CParams) == 136 and p.bin_mode == 0
    assert (p.grid_mode, p.coarse_bins, p.coarse_pmin, p.coarse_pmax) == (0, 4096, 0.1, 400.0)


def test_strerror():
    L = qlpbls.lib()
    for c in (0, -1, -2, -3, -4, -5):
        assert L.qlp_strerror(c)


def _oracle_plan(t, y, dy, rho):
    return oracle.plan_star(t, y, dy, rho, 1.0)


@pytest.mark.parametrize("which", ["single", "uneven", "multi", "tiny"])
def test_planner_grid_is_bit_identical_to_oracle(which):
    if which == "single":
        b = synth.single_star()
    elif which == "uneven":
        b = synth.uneven_single_sector(n_stars=6, seed=9)
    elif which == "multi":
        b = synth.multi_sector(n_stars=3, seed=4, max_sectors=4)
    else:
        b = synth.tiny_batch(n_stars=5, seed=2)
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        g = qlpbls.star_grid(t, y, dy, float(b.rho[s]))
        o = _oracle_plan(t, y, dy, float(b.rho[s]))
        assert g["status"] == o.status
        assert g["pmin"] == o.pmin and g["pmax"] == o.pmax and g["t_ref"] == o.t_ref
        assert g["freqs"].shape == o.freqs.shape
        assert np.array_equal(g["freqs"], o.freqs)
        assert np.array_equal(g["qmins"], o.qmin)


def test_batch_planner_equals_oracle_star_by_star():
    """The batch planner (several stars' grid recurrences stepped together on each
    host thread) gives every star the oracle's grid bit for bit, in a batch that
    mixes valid stars with rejected ones (unsorted, one point, NaN-only) and whose
    size is not a multiple of the interleaving width."""
    b = synth.uneven_single_sector(n_stars=11, seed=31)
    t = [b.star(s)[0] for s in range(b.n_stars)]
    y = [b.star(s)[1] for s in range(b.n_stars)]
    dy = [b.star(s)[2] for s in range(b.n_stars)]
    rho = list(b.rho)
    base = np.linspace(2000, 2010, 40)
    for tt, yy in ((base[::-1], np.ones(40)), (base[:1], np.ones(1)), (base, np.full(40, np.nan))):
        t.insert(3, tt); y.insert(3, yy); dy.insert(3, np.full(tt.shape[0], 1e-3)); rho.insert(3, float("nan"))
    off = np.concatenate([[0], np.cumsum([x.shape[0] for x in t])])
    status, foff, freqs = qlpbls.batch_grid(off, np.concatenate(t), np.concatenate(y), np.concatenate(dy),
                                            np.array(rho))
    assert sorted(status[3:6].tolist()) == sorted([qlpbls.STAR_UNSORTED, qlpbls.STAR_TOO_FEW,
                                                   qlpbls.STAR_TOO_FEW])
    for s in range(len(t)):
        o = oracle.plan_star(t[s], y[s], dy[s], rho[s], 1.0)
        assert status[s] == o.status
        got = freqs[foff[s]:foff[s + 1]]
        assert np.array_equal(got, o.freqs if o.status == 0 else np.zeros(0))


def test_planner_status_flags_match_oracle():
    t = np.linspace(0, 10, 50) + 2000.0
    y = np.ones(50)
    dy = np.full(50, 1e-3)
    cases = [
        (t[::-1], y, dy),
        (t[:1], y[:1], dy[:1]),
        (np.array([0, 0.1, 0.2]) + 2000, y[:3], dy[:3]),
    ]
    y2 = y.copy(); y2[3] = np.nan
    dy2 = dy.copy(); dy2[7] = -1.0
    cases.append((t, y2, dy2))
    for tt, yy, dd in cases:
        g = qlpbls.star_grid(tt, yy, dd, 1.41)
        o = _oracle_plan(tt, yy, dd, 1.41)
        assert g["status"] == o.status
        assert np.array_equal(g["freqs"], o.freqs)


def test_invalid_params_rejected():
    t = np.linspace(0, 10, 50) + 2000.0
    with pytest.raises(qlpbls.QlpError):
        qlpbls.star_grid(t, np.ones(50), np.full(50, 1e-3), 1.41,
                         qlpbls.Params(samples_per_peak=0.0))
    with pytest.raises(qlpbls.QlpError):
        qlpbls.star_grid(t, np.ones(50), np.full(50, 1e-3), 1.41, qlpbls.Params(phase_mode=7))


@pytest.mark.parametrize("seed", [1, 2])
def test_coarse_grid_is_bit_identical_to_oracle(seed):
    from oracle import plan as op
    b = synth.uneven_single_sector(n_stars=3, seed=seed)
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        g = qlpbls.star_grid(t, y, dy, float(b.rho[s]), qlpbls.Params(grid_mode=1))
        o = oracle.plan_star(t, y, dy, float(b.rho[s]), 1.0, op.Params(grid_mode=1))
        assert np.array_equal(g["freqs"], o.freqs) and np.array_equal(g["qmins"], o.qmin)


def test_window_grid_is_bit_identical_to_oracle():
    b = synth.uneven_single_sector(n_stars=2, seed=3)
    rng = np.random.default_rng(4)
    for s in range(b.n_stars):
        t, y, dy = b.star(s)
        lo = np.sort(rng.uniform(0.08, 2.5, 12))
        wins = [(x, x * 1.004) for x in lo] + [(lo[0], lo[0] * 1.001)]
        g = qlpbls.star_grid(t, y, dy, float(b.rho[s]), windows=wins)
        o = oracle.plan_star(t, y, dy, float(b.rho[s]), 1.0, windows=wins)
        assert g["status"] == o.status
        assert np.array_equal(g["freqs"], o.freqs) and np.array_equal(g["qmins"], o.qmin)


@pytest.mark.parametrize("n_threads", [1, 2, 3, 0])
def test_batch_planner_thread_counts(n_threads):
    """The batch planner gives the same grids whatever the number of host threads
    (1 = the calling thread alone; 0 = every core, from the process-wide pool)."""
    b = synth.uneven_single_sector(n_stars=21, seed=33)
    ref = qlpbls.batch_grid(b.offsets, b.t, b.y, b.dy, b.rho, qlpbls.Params(n_threads=1))
    got = qlpbls.batch_grid(b.offsets, b.t, b.y, b.dy, b.rho, qlpbls.Params(n_threads=n_threads))
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)


@pytest.mark.filterwarnings("ignore:This process .* is multi-threaded:DeprecationWarning")
def test_batch_planner_after_fork():
    """The planner's host thread pool does not survive fork(); a child process
    that plans after its parent did gets a pool of its own (no hang) and the
    same grids."""
    import os, time
    b = synth.uneven_single_sector(n_stars=9, seed=32)
    args = (b.offsets, b.t, b.y, b.dy, b.rho)
    _, foff, freqs = qlpbls.batch_grid(*args)  # starts the pool in this process
    pid = os.fork()
    if pid == 0:  # child: plan again, exit 0 on equal grids
        code = 1
        try:
            _, f2, q2 = qlpbls.batch_grid(*args)
            code = 0 if (np.array_equal(f2, foff) and np.array_equal(q2, freqs)) else 1
        finally:
            os._exit(code)
    deadline = time.time() + 120
    status = None
    while time.time() < deadline:
        done, st = os.waitpid(pid, os.WNOHANG)
        if done:
            status = st
            break
        time.sleep(0.05)
    if status is None:
        os.kill(pid, 9)
        os.waitpid(pid, 0)
        pytest.fail("the child's planner did not finish")
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0


def test_device_budget_setting_needs_no_gpu():
    # the budget is host bookkeeping: set, read back, reject a negative cap
    from paper_2302_01293_gb300 import qlpbls
    L = qlpbls.lib()
    assert L.qlp_set_device_budget(-1) == qlpbls.ERR_ARG
    assert L.qlp_set_device_budget(1 << 30) == 0
    assert qlpbls.device_bytes_held() == 0
    assert L.qlp_set_device_budget(0) == 0


def test_plan_from_plan_rejects_missing_arguments():
    # checked before any device work: no base plan, no window offsets
    import ctypes
    import numpy as np
    from paper_2302_01293_gb300 import qlpbls
    L = qlpbls.lib()
    out = ctypes.c_void_p()
    wo = np.zeros(2, np.int64)
    assert L.qlp_bls_plan_windows_from(None, None, wo.ctypes.data, None, None, None,
                                       ctypes.byref(out)) == qlpbls.ERR_ARG
    assert out.value is None


def test_plan_queries_reject_a_missing_plan():
    # the plan queries answer QLP_ERR_ARG for a NULL plan or output, with no device work
    import ctypes
    from paper_2302_01293_gb300 import qlpbls
    L = qlpbls.lib()
    n = ctypes.c_int32(-7)
    assert L.qlp_bls_plan_launches(None, ctypes.byref(n)) == qlpbls.ERR_ARG
    assert n.value == -7
    assert L.qlp_bls_plan_narrow_stats(None, None, None, None) == qlpbls.ERR_ARG
    assert L.qlp_bls_plan_exact_stats(None, None, None, None) == qlpbls.ERR_ARG


def test_work_loop_bound_is_validated():
    from paper_2302_01293_gb300 import qlpbls
    import synth
    b = synth.tiny_batch(n_stars=2, seed=3)
    st, foff, freqs = qlpbls.batch_grid(b.offsets, b.t, b.y, b.dy, b.rho,
                                        qlpbls.Params(work_loop_bound=3))
    assert foff[-1] > 0
    with pytest.raises(qlpbls.QlpError):
        qlpbls.batch_grid(b.offsets, b.t, b.y, b.dy, b.rho, qlpbls.Params(work_loop_bound=-1))


def test_coarse_periods_and_bins_match_oracle_grid():
    # the library's coarse-bin periods are the oracle's log-period grid bit for bit,
    # and every grid period maps back to its own bin
    from oracle import plan as op
    p = op.Params(grid_mode=1)
    ratio = p.coarse_pmax / p.coarse_pmin
    ks = np.arange(p.coarse_bins)
    ref = np.array([p.coarse_pmin * (ratio ** (k / (p.coarse_bins - 1))) for k in ks])
    qp = qlpbls.Params(grid_mode=1)
    assert np.array_equal(qlpbls.coarse_periods(ks.astype(np.float64), qp), ref)
    assert np.array_equal(qlpbls.coarse_bins(ref, qp), ks.astype(np.int32))
    assert list(qlpbls.coarse_bins(np.array([0.05, -1.0, 500.0]), qp)) == [-1, -1, -1]


def test_proposal_windows_bracket_their_bins():
    qp = qlpbls.Params(grid_mode=1)
    bins = np.array([[10, 4095, -1], [-1, -1, -1], [2000, 2001, 0]], np.int32)
    off, lo, hi = qlpbls.proposal_windows(bins, qp, 1.0)
    assert list(off) == [0, 2, 2, 5]
    kk = np.array([10, 4095, 2000, 2001, 0], np.float64)
    np.testing.assert_array_equal(lo, 1.0 / qlpbls.coarse_periods(kk + 1.0, qp))
    np.testing.assert_array_equal(hi, 1.0 / qlpbls.coarse_periods(kk - 1.0, qp))
    assert np.all(lo < hi)

"""Failure detection on the GPU without a GPU fault.

* A persistent search kernel's work loop is a plain counted loop over queue
  pops (no tensor-core work or barrier wait in flight). Setting its bound low
  (work_loop_bound) makes every block stop early: the kernel returns, raises
  QLP_DEVERR_QUEUE in the plan's error word, and qlp_bls_device_status returns
  QLP_ERR_DEVICE. The context stays usable: the next plan searches correctly.
* Device allocation failure is injected on the host with a device-memory budget
  (qlp_set_device_budget): the plan or network that would pass it returns
  QLP_ERR_NOMEM before taking any device memory, and nothing it took before is
  kept.
"""
import ctypes

import numpy as np
import pytest

import synth
from paper_2302_01293_gb300 import qlpbls
from parity import compare_snr, compare_spectrum, oracle_star, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,summ", [(qlpbls.METHOD_AUTO, qlpbls.SUM_FIXED),
                                         (qlpbls.METHOD_CELLS, qlpbls.SUM_COMP),
                                         (qlpbls.METHOD_POINTS, qlpbls.SUM_COMP)])
def test_work_loop_bound_reports_device_error(gpu_lib, method, summ):
    import torch
    b = synth.uneven_single_sector(n_stars=64, seed=51)
    plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar,
                       qlpbls.Params(method=method, sum_mode=summ, work_loop_bound=1, chunk_freqs=32))
    out = plan.search()
    flags = ctypes.c_int32()
    rc = qlpbls.lib().qlp_bls_device_status(plan._h, qlpbls._stream_ptr(None), ctypes.byref(flags))
    assert rc == qlpbls.ERR_DEVICE and flags.value & qlpbls.DEVERR_QUEUE, (rc, flags.value)
    # the flag is cleared once read, and the device is still usable
    assert plan.device_status() == 0
    del out
    plan.close()
    torch.cuda.synchronize()
    g = run_gpu(b.subset(range(2)), qlpbls.Params(method=method, sum_mode=summ))
    assert g["flags"] == 0
    for s in range(2):
        pl, ores = oracle_star(b, s)
        sl = g["plan"].star_slice(s)
        st = compare_spectrum(pl, ores, g, sl, label=f"after the bound, star {s}")
        compare_snr(pl, ores, g, sl, g["best"][s], label=f"after the bound, star {s}", alt=st["alt_sr"])


def test_device_budget_makes_plans_fail_cleanly(gpu_lib):
    import torch
    b = synth.uneven_single_sector(n_stars=16, seed=52)
    torch.cuda.synchronize()
    held0 = qlpbls.device_bytes_held()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        qlpbls.set_device_budget(held0 + (1 << 20))   # 1 MiB above what is held now
        with pytest.raises(qlpbls.QlpError) as ei:
            qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
        assert ei.value.code == qlpbls.ERR_NOMEM
        with pytest.raises(qlpbls.QlpError) as ei:
            qlpbls.CNN(max_batch=64, length=4096, seed=0)
        assert ei.value.code == qlpbls.ERR_NOMEM
        with pytest.raises(qlpbls.QlpError) as ei:
            qlpbls.run_host(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
        assert ei.value.code == qlpbls.ERR_NOMEM
        torch.cuda.synchronize()
        assert qlpbls.device_bytes_held() == held0
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
    finally:
        qlpbls.set_device_budget(0)
    # without the cap the same plan works, and its bytes are returned when it closes
    plan = qlpbls.Plan(b.offsets, b.t, b.y, b.dy, b.rho, b.rstar)
    assert qlpbls.device_bytes_held() > held0
    out = plan.search()
    plan.snr(out)
    assert plan.device_status() == 0
    del out
    plan.close()
    assert qlpbls.device_bytes_held() == held0

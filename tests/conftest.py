import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library through its C-ABI binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_01293_gb300 import qlpbls
    return qlpbls


def _parity_report():
    mod = sys.modules.get("parity")
    return getattr(mod, "REPORT", None) if mod else None


def pytest_sessionfinish(session, exitstatus):
    """Write the parity figures of every GPU comparison (near ties, SR and S/N
    error maxima per test) as JSON to the file QLP_PARITY_REPORT names, if it is set
    (the terminal summary prints their totals either way)."""
    rep = _parity_report()
    path = os.environ.get("QLP_PARITY_REPORT")
    if not rep or not path:
        return
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(rep, fh, indent=1, sort_keys=True)
    except OSError:
        pass


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    rep = _parity_report()
    if not rep:
        return
    tot = dict(stars=0, freqs=0, near_ties=0, best_ties=0)
    mx = dict(sr_rel_max=0.0, sr_rel_max_same_box=0.0, snr_abs_max_le100=0.0, snr_abs_max_le1000=0.0,
              snr_rel_max_gt1000=0.0, snr_abs_max_seen=0.0)
    for e in rep.values():
        for k in tot:
            tot[k] += e.get(k, 0)
        for k in mx:
            mx[k] = max(mx[k], e.get(k, 0.0))
    terminalreporter.write_line(
        "parity: %d stars, %d frequencies, %d near ties (j,k), %d best-index ties; SR rel max %.2e "
        "(same box %.2e); |dS/N| max %.2e (|S/N|<=100), %.2e (<=1000), rel %.2e (>1000); max |S/N| %.0f"
        % (tot["stars"], tot["freqs"], tot["near_ties"], tot["best_ties"], mx["sr_rel_max"],
           mx["sr_rel_max_same_box"], mx["snr_abs_max_le100"], mx["snr_abs_max_le1000"],
           mx["snr_rel_max_gt1000"], mx["snr_abs_max_seen"]))

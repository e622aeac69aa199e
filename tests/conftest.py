import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: full-size workloads")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The largest plain-relative error |gpu - ref| / |ref| of every float
    parity check that ran (the pass/fail bound is the per-entry summation
    bound; this is the plain-relative figure beside it)."""
    try:
        import helpers
    except ImportError:
        return
    errs = getattr(helpers, "REL_ERRORS", {})
    if not errs:
        return
    terminalreporter.section("max plain-relative error per float parity check")
    for key in sorted(errs):
        terminalreporter.write_line(f"{errs[key]:.3e}  {key}")
    worst = max(errs.items(), key=lambda kv: kv[1])
    terminalreporter.write_line(f"overall max {worst[1]:.3e} ({worst[0]})")

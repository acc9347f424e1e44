"""Failure detection on the GPU without a fault: every mbarrier wait in the
tensor-core kernels is bounded, and a wait that runs out records
CWTH_ERR_TIMEOUT in the plan's device status word, which cwth_sync reports.

cwth_selftest_wait_timeout runs that path on purpose: a one-thread kernel
waits about a millisecond on a barrier that nothing arrives on.  The test
checks the status is reported once, cleared, and that the context and the
plan still produce the same scalograms afterwards.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 5          # CWTH_ERR_TIMEOUT
INVALID_ARG = 1      # CWTH_ERR_INVALID_ARG
BUDGET = 2_000_000   # SM clock cycles, about 1 ms


@pytest.fixture(scope="module")
def cw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth
    return cwth


@pytest.mark.parametrize("precision,path", [("bf16x2", "direct"), ("fp32", "spectral")])
def test_expired_wait_is_reported_once_and_the_plan_keeps_working(cw, precision, path):
    from paper_2408_14302_gb300 import signals
    n = 8000
    x = torch.from_numpy(np.stack([signals.machine_clip(40 + i, n) for i in range(3)])).cuda()
    sc = signals.scales_for_band(100, 8000, 16, 16000.0)
    lib = cw.lib()
    with cw.Plan(sc, hop=64, max_len=n, precision=precision, path=path) as plan:
        ref = plan.execute(x).clone()
        plan.sync()
        h = plan._h
        assert lib.cwth_selftest_wait_timeout(h, BUDGET, None) == 0
        assert lib.cwth_sync(h, None) == TIMEOUT
        assert lib.cwth_sync(h, None) == 0          # reported once, then cleared
        out = plan.execute(x)
        plan.sync()
        assert torch.equal(out, ref)
        # Through the Python API the same status raises.
        assert lib.cwth_selftest_wait_timeout(h, BUDGET, None) == 0
        with pytest.raises(cw.CwthError) as err:
            plan.sync()
        assert err.value.status == TIMEOUT
        plan.sync()
        # Budgets outside 1 .. 4e9 cycles are refused before anything runs.
        assert lib.cwth_selftest_wait_timeout(h, 0, None) == INVALID_ARG
        assert lib.cwth_selftest_wait_timeout(h, 5_000_000_000, None) == INVALID_ARG
        plan.sync()

"""Failure detection without a GPU fault.

Kernels that wait on an asynchronous bulk copy (mbarrier) give up after about
a second, record the failure in the plan's device status word and exit; the
host reads it with lc_plan_check.  Here a test-only plan flag makes the
coupling kernel withhold one of its copies, so the wait runs out; the call
must report LC_ERR_DEVICE_TIMEOUT and the device must stay usable.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as m
    return m


@pytest.mark.parametrize("tier", ["f64", "f64_df"])
def test_withheld_copy_reports_timeout_and_device_survives(lc, tier):
    n = 4096
    dev = torch.device("cuda", 0)
    x = torch.as_tensor(workloads.decaying_vector(n, seed=3), device=dev)
    bad = lc.Plan(n, "l2c", 1, tier, dev, debug_flags=1)
    bad(x)
    with pytest.raises(lc.LegChebError) as e:
        bad.check()
    assert e.value.status == 4  # LC_ERR_DEVICE_TIMEOUT
    bad.check()  # the status word was cleared
    good = lc.Plan(n, "l2c", 1, tier, dev)
    z = good(x).cpu().numpy()
    good.check()
    e2, _ = rel_errors(z, oracle.apply(oracle.L2C, x.cpu().numpy()))
    assert e2 <= 1e-13


def test_host_validation_errors(lc):
    dev = torch.device("cuda", 0)
    plan = lc.Plan(100, "l2c", 2, "f64", dev)
    x = torch.zeros((2, 100), dtype=torch.float64, device=dev)
    with pytest.raises(lc.LegChebError) as e:   # in and out alias
        plan.execute_strided(x, x, (100, 1), (100, 1))
    assert e.value.status == 1
    with pytest.raises(lc.LegChebError) as e:   # zero output batch stride with batch 2
        plan.execute_strided(x, torch.zeros_like(x), (100, 1), (0, 1))
    assert e.value.status == 1
    with pytest.raises(TypeError):
        plan(torch.zeros((2, 100), dtype=torch.float32, device=dev))
    with pytest.raises(ValueError):
        plan(torch.zeros((3, 100), dtype=torch.float64, device=dev))

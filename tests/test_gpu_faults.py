"""Failure detection without a GPU fault.

Kernels that wait on an asynchronous bulk copy (mbarrier) give up after about
a second, record the failure in the plan's device status word and exit; the
host reads it with lc_plan_check.  Here test-only plan flags make the
coupling kernel withhold one of its copies, or one task of the persistent
split schedule wait for a write that never comes, so the wait runs out; the
call must report LC_ERR_DEVICE_TIMEOUT and the device must stay usable.
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


@pytest.mark.parametrize("adjoint", [False, True])
def test_persistent_split_dependency_timeout_aborts(lc, adjoint):
    # test-only flag bit 1: one task of the persistent schedule waits for a
    # write that never comes; its bounded wait runs out, every CTA stops, and
    # the plan reports LC_ERR_DEVICE_TIMEOUT; the device stays usable
    n, batch = 3000, 130
    dev = torch.device("cuda", 0)
    X = np.stack([workloads.decaying_vector(n, seed=60 + b) for b in range(batch)])
    x = torch.as_tensor(X, device=dev)
    bad = lc.Plan(n, "c2l", batch, "f64_split", dev, debug_flags=2)
    assert bad.launches() == 2
    bad.execute(x, adjoint=adjoint)
    with pytest.raises(lc.LegChebError) as e:
        bad.check()
    assert e.value.status == 4  # LC_ERR_DEVICE_TIMEOUT
    bad.check()  # the status word was cleared
    good = lc.Plan(n, "c2l", batch, "f64_split", dev)
    z = good.execute(x, adjoint=adjoint).cpu().numpy()
    good.check()
    e2, _ = rel_errors(z[0], oracle.apply(oracle.C2L, X[0], adjoint=adjoint))
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

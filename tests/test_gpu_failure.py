"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes must expire, report GRF_ETIMEOUT through the status word,
and leave the context usable."""
import ctypes
import time

import numpy as np
import pytest

from helpers import gpu_env, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives():
    torch = gpu_env()
    from paper_2212_10961_gb300 import _abi
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    rc = _abi.lib().grf_selftest_wait(3000, ctypes.c_void_p(status.data_ptr()), stream)
    dt = time.perf_counter() - t0
    assert rc == _abi.GRF_ETIMEOUT
    assert b"expired" in _abi.lib().grf_last_error()
    assert status.item() == 2
    assert dt >= 0.002
    assert _abi.lib().grf_selftest_wait(0, ctypes.c_void_p(status.data_ptr()), stream) == _abi.GRF_EINVAL
    # the context is still usable: a small synthesis runs and its status word is clean
    cells = W.grid_centres((32, 32))
    plan = F.CellPlan(*to_dev(torch, cells))
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=256, seed=3)
    out = F.GaussianField(p).synth(plan)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert np.all(np.isfinite(out["Y"].cpu().numpy()))


def test_injected_allocation_failure_in_plan_and_synthesis():
    # host-side injection: the failing call raises GRF_ENOMEM, launches nothing
    # after the failure point, and the same objects work on the next call
    torch = gpu_env()
    from paper_2212_10961_gb300 import _abi
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    L = _abi.lib()
    cells = to_dev(torch, W.grid_centres((48, 40)))
    p = F.FieldParams(family="exponential", sigma2=1.0, ell=(0.1, 0.2), dim=2, n_modes=300, seed=4)
    gf = F.GaussianField(p)
    try:
        L.grf_debug_inject_alloc_failures(1)
        with pytest.raises(_abi.GRFError) as e:
            F.CellPlan(*cells)
        assert e.value.code == _abi.GRF_ENOMEM
        plan = F.CellPlan(*cells)
        want = gf.synth(plan)["Y"].clone()
        L.grf_debug_inject_alloc_failures(1)
        n0 = F.launch_count()
        with pytest.raises(_abi.GRFError) as e:
            gf.synth(plan)
        assert e.value.code == _abi.GRF_ENOMEM and F.launch_count() == n0
    finally:
        L.grf_debug_inject_alloc_failures(0)
    got = gf.synth(plan)["Y"]
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(got, want)


def test_released_plan_is_rejected():
    # after grf_release the library no longer accepts the buffer as a plan
    torch = gpu_env()
    from paper_2212_10961_gb300 import _abi
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    plan = F.CellPlan(*to_dev(torch, W.grid_centres((20, 16))))
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=128, seed=2)
    gf = F.GaussianField(p)
    gf.synth(plan)
    assert _abi.lib().grf_release(plan.ptr) == 0
    with pytest.raises(_abi.GRFError) as e:
        gf.synth(plan)
    assert e.value.code == _abi.GRF_EINVAL
    assert _abi.lib().grf_release(plan.ptr) == 0  # unknown pointers are ignored
    torch.cuda.synchronize()

"""GPU checks of the mode prefetcher (grf_prefetch_*): realisations k = 0, 1,
... of one parameter set with seeds seed + k, drawn and packed by native
worker threads ahead of use, arrive in order and equal the tables packed on
the calling thread; a worker's host allocation failure (injected on the
host) reaches the caller as GRF_ENOMEM."""
import ctypes
import time

import numpy as np
import pytest

from helpers import gpu_env, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    return torch, F, W


@pytest.mark.parametrize("family,dim,n_modes,depth,threads", [("gaussian", 2, 1000, 3, 3),
                                                              ("matern", 3, 777, 2, 1),
                                                              ("exponential", 3, 4099, 4, 5)])
def test_prefetched_tables_equal_tables_packed_in_place(env, family, dim, n_modes, depth, threads):
    torch, F, W = env
    p = F.FieldParams(family=family, sigma2=1.3, ell=(0.1, 0.2, 0.05)[:dim], dim=dim, n_modes=n_modes,
                      seed=1000, nu=1.3)
    pf = F.ModePrefetcher(p, depth=depth, threads=threads)
    tabs = [F.ModeTable.device_only(n_modes, dim) for _ in range(2)]
    cells = W.grid_centres((37, 29, 11)[:dim])
    plan = F.CellPlan(*to_dev(torch, cells))
    ps = F.PreparedSynth(p, plan, maps=F.MapSpec(y=True, lognormal=True))
    for k in range(12):
        tab = tabs[k % 2]
        assert pf.next(tab) == 1000 + k
        y = ps(tab)["Y"].clone()
        pk = F.FieldParams(**{**p.__dict__, "seed": 1000 + k})
        ref = F.GaussianField(pk)
        torch.cuda.synchronize()
        assert torch.equal(tab.dev[:ref.table.nbytes].cpu(), ref.table.host[:ref.table.nbytes])
        assert torch.equal(y, ref.synth(plan, F.MapSpec(y=True))["Y"])
    pf.close()
    pf.close()  # idempotent


def test_prefetch_worker_failure_reaches_the_caller(env):
    torch, F, W = env
    from paper_2212_10961_gb300 import _abi
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=300, seed=5)
    pf = F.ModePrefetcher(p, depth=2, threads=1)
    tab = F.ModeTable.device_only(300, 2)
    time.sleep(0.5)  # the worker fills both slots and waits
    try:
        _abi.check(_abi.lib().grf_debug_inject_alloc_failures(1))
        codes = []
        for _ in range(4):
            try:
                pf.next(tab)
                codes.append(0)
            except _abi.GRFError as e:
                codes.append(e.code)
        assert _abi.GRF_ENOMEM in codes
        first = codes.index(_abi.GRF_ENOMEM)
        assert first <= 2 and all(c == _abi.GRF_ENOMEM for c in codes[first:])
    finally:
        _abi.lib().grf_debug_inject_alloc_failures(0)
        pf.close()
    torch.cuda.synchronize()

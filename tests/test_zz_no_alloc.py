"""GPU test of grf_mismatch_grad_noalloc, the entry point for callers that
cannot allocate device memory where they call it.  It must give the same loss
and gradient as grf_mismatch_grad (which takes a caller workspace), on two
calls in a row, and refuse sizes beyond its fixed scratch array.

Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2212_10961_gb300 import _abi
    assert torch.cuda.is_available()
    return torch, _abi


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _reference(torch, abi, K, T):
    n = K.numel()
    gY = torch.empty_like(K)
    loss = torch.empty(1, dtype=torch.float64, device=K.device)
    nb = abi.lib().grf_mismatch_workspace_bytes(n)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=K.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    abi.check(abi.lib().grf_mismatch_grad(n, _p(K), _p(T), _p(gY), _p(loss), _p(ws), ws.numel(), stream))
    return loss, gY


def test_noalloc_matches_workspace_entry_point_twice(env):
    torch, abi = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    for n in (3_000_001, 777):  # two calls in a row, different sizes and data
        K = torch.from_numpy(np.exp(rng.standard_normal(n)).astype(np.float32)).cuda()
        T = torch.from_numpy(np.exp(rng.standard_normal(n)).astype(np.float32)).cuda()
        loss_ref, g_ref = _reference(torch, abi, K, T)
        gY = torch.empty_like(K)
        loss = torch.empty(1, dtype=torch.float64, device=K.device)
        abi.check(abi.lib().grf_mismatch_grad_noalloc(n, _p(K), _p(T), _p(gY), _p(loss), stream))
        torch.cuda.synchronize()
        assert loss.item() == pytest.approx(loss_ref.item(), rel=1e-12, abs=0.0)
        assert torch.allclose(gY, g_ref, rtol=1e-6, atol=0.0)
        # and against a plain FP64 evaluation of the same definition (the
        # kernels form K - T in FP32, so they agree to FP32 rounding)
        k64 = K.double().cpu().numpy()
        t64 = T.double().cpu().numpy()
        assert loss.item() == pytest.approx(float(np.mean((k64 - t64) ** 2)), rel=1e-6)


def test_noalloc_at_its_largest_size(env):
    # n = GRF_NOALLOC_MAX_CELLS fills every entry of the fixed array; it must
    # agree with the workspace entry point (three 512 MiB float32 arrays)
    torch, abi = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 134217728
    g = torch.Generator(device="cuda").manual_seed(7)
    K = torch.rand(n, generator=g, device="cuda") + 0.5
    T = torch.rand(n, generator=g, device="cuda") + 0.5
    loss_ref, g_ref = _reference(torch, abi, K, T)
    gY = torch.empty_like(K)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    assert abi.lib().grf_mismatch_grad_noalloc(n, _p(K), _p(T), _p(gY), _p(loss), stream) == abi.GRF_OK
    torch.cuda.synchronize()
    assert loss.item() == pytest.approx(loss_ref.item(), rel=1e-12, abs=0.0)
    assert torch.equal(gY, g_ref)
    del K, T, gY, g_ref
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, abi = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_many = (1 << 27) + 1
    rc = abi.lib().grf_mismatch_grad_noalloc(too_many, _p(dummy), _p(dummy), _p(dummy), _p(loss), stream)
    assert rc == abi.GRF_EINVAL
    assert b"GRF_NOALLOC_MAX_CELLS" in abi.lib().grf_last_error()

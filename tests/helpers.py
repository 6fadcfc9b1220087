"""Shared helpers for the GPU parity tests: run the CUDA path through the C
ABI and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

FAMILY_IDS = {"gaussian": 0, "exponential": 1, "matern": 2}

# Forward tolerance: max-abs error of Y against the FP64 oracle, in units of sigma.
Y_TOL_SIGMA = 1e-5
# Facies labels must agree wherever the oracle field is farther than this
# band (in sigma units) from every threshold.
FACIES_BAND_SIGMA = 2e-5
# Gradients: max-abs error per family relative to the largest oracle value.
GRAD_TOL = 1e-4


def gpu_env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    return torch


def to_dev(torch, arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def oracle_modes(family, sigma2, ell, dim, n, seed, nu=1.5, stream=0):
    from oracle import modes as om
    return om.gen_modes(FAMILY_IDS[family], sigma2, list(ell) + [1.0] * (3 - len(ell)), dim, n, seed, nu=nu,
                        stream=stream)


def oracle_field(modes, mean, cells, idx=None):
    from oracle import native
    c = np.stack(cells, axis=-1) if isinstance(cells, (list, tuple)) else cells
    if idx is not None:
        c = c[idx]
    return native.synth(modes["a"], modes["amp"], modes["psi"], mean, c)


def check_forward(y_gpu, y_or, sigma, what=""):
    err = np.max(np.abs(y_gpu.astype(np.float64) - y_or)) if len(y_or) else 0.0
    assert err <= Y_TOL_SIGMA * sigma, "%s: max|Y_gpu - Y_oracle| = %.3e > %.3e" % (what, err, Y_TOL_SIGMA * sigma)
    return err / sigma


def check_lognormal(k_gpu, y_or, sigma, k_ref=1.0):
    k_or = k_ref * np.exp(y_or)
    rel = np.abs(k_gpu.astype(np.float64) - k_or) / k_or
    tol = Y_TOL_SIGMA * sigma + 2.0 ** -21
    assert np.max(rel) <= tol, "K relative error %.3e > %.3e" % (np.max(rel), tol)


def check_facies(f_gpu, y_or, thresholds, sigma):
    from oracle import field as of
    lab = of.indicator(y_or, thresholds)
    d = np.min(np.abs(y_or[:, None] - np.asarray(thresholds)[None, :]), axis=1) if len(thresholds) else \
        np.full(len(y_or), np.inf)
    band = d <= FACIES_BAND_SIGMA * sigma
    assert np.array_equal(f_gpu[~band], lab[~band])
    # inside the band the label must still be a neighbour of the oracle label
    assert np.all(np.abs(f_gpu[band].astype(int) - lab[band].astype(int)) <= 1)
    return int(band.sum())

"""Seeded synthetic inputs: cell centres and field parameters of the
benchmark workloads.  Input generation only -- nothing here evaluates the
method; both the CUDA path and the FP64 oracle consume these arrays.

Workloads (paper shapes: unit-square / unit-cube Cartesian grids treated as
unstructured cell sets, Sec. 4.1; jittered lattices for unstructured meshes):

* grid2d_64   : 64 x 64 centres of the unit square, N = 1000, Gaussian l = 0.1,
                sigma^2 = 1, mean 0, seed 1; K = exp(Y), binary facies at 0.
* grid3d_256  : 256^3 centres of the unit cube, N = 4096, exponential,
                l = (0.2, 0.2, 0.05), sigma^2 = 4; K = exp(Y) and 3 facies at
                the Gaussian 1/3, 2/3 quantiles.
* jitter3d_2m : 252 x 126 x 63 lattice (h = 1/126) in a 2 x 1 x 0.5 box, each
                coordinate jittered by U(-0.4h, 0.4h) (seed 3), Matern
                nu = 1.5, l = 0.1, sigma^2 = 2, N = 8192.
* ensemble256 : 256 realisations; with probability 1/8 a 64^3 cube grid, else
                an n x n unit-square grid with n = round(2^U(5, 9)); N uniform
                in {1024, 2048, 4096}; Gaussian or exponential (1/2 each),
                l = 0.1, sigma^2 = 1 (recipe seed 4).
* diff128     : 128^3 unit cube, N = 2048, Gaussian l = 0.1, sigma^2 = 1; the
                target K comes from seed 2, the trial field from seed 1.
* hrl2d       : the Horton-Rogers-Lapwood example's field (Sec. 5): 2 x 1
                domain, 1024 x 512 cells, lognormal with sigma^2 = 2,
                l = (0.2, 0.05) (covariance family unstated: Gaussian taken),
                N = 4096; thresholded variant with 4 facies at the Gaussian
                quartiles whose permeabilities are the four values the paper
                lists, in ascending order.
"""
import math

import numpy as np


def grid_centres(shape, extent=None):
    """Cell centres of a Cartesian grid, x fastest; returns list of float32
    arrays (one per axis)."""
    shape = tuple(int(s) for s in shape)
    extent = tuple(extent) if extent is not None else (1.0,) * len(shape)
    axes = [((np.arange(n, dtype=np.float64) + 0.5) * (e / n)) for n, e in zip(shape, extent)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    return [np.ascontiguousarray(m.ravel().astype(np.float32)) for m in mesh[::-1]]


def jittered_lattice(shape, h, jitter, seed):
    """Lattice centres (i + 1/2) h with every coordinate moved by U(-jitter h, jitter h)."""
    cells = grid_centres(shape, tuple(n * h for n in shape))
    rng = np.random.default_rng(seed)
    return [np.ascontiguousarray((c.astype(np.float64) + rng.uniform(-jitter * h, jitter * h, c.shape))
                                 .astype(np.float32)) for c in cells]


def shuffled(cells, seed):
    perm = np.random.default_rng(seed).permutation(len(cells[0]))
    return [np.ascontiguousarray(c[perm]) for c in cells], perm


WORKLOADS = {
    "grid2d_64": dict(shape=(64, 64), family="gaussian", ell=(0.1, 0.1), sigma2=1.0, mean=0.0,
                      n_modes=1000, seed=1, quantiles=(0.5,)),
    "grid3d_256": dict(shape=(256, 256, 256), family="exponential", ell=(0.2, 0.2, 0.05), sigma2=4.0,
                       mean=0.0, n_modes=4096, seed=1, quantiles=(1.0 / 3.0, 2.0 / 3.0)),
    "jitter3d_2m": dict(shape=(252, 126, 63), h=1.0 / 126.0, jitter=0.4, jitter_seed=3, family="matern",
                        nu=1.5, ell=(0.1, 0.1, 0.1), sigma2=2.0, mean=0.0, n_modes=8192, seed=1,
                        quantiles=()),
    "hrl2d": dict(shape=(1024, 512), extent=(2.0, 1.0), family="gaussian", ell=(0.2, 0.05), sigma2=2.0,
                  mean=0.0, n_modes=4096, seed=1, quantiles=(0.25, 0.5, 0.75),
                  values=(0.0183, 0.27, 3.99, 58.9)),
    "diff128": dict(shape=(128, 128, 128), family="gaussian", ell=(0.1, 0.1, 0.1), sigma2=1.0, mean=0.0,
                    n_modes=2048, seed=1, target_seed=2, quantiles=()),
}


def workload_cells(name, scale=1):
    """Cell centres of a named workload (scale > 1 shrinks each axis by that factor)."""
    w = WORKLOADS[name]
    shape = tuple(max(1, s // scale) for s in w["shape"])
    if "h" in w:
        return jittered_lattice(shape, w["h"] * scale, w["jitter"], w["jitter_seed"])
    return grid_centres(shape, w.get("extent"))


def ensemble_recipe(n_real=256, seed=4):
    """Per realisation: dict(shape, dim, n_modes, family, ell, sigma2, mean, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_real):
        if rng.random() < 1.0 / 8.0:
            shape = (64, 64, 64)
        else:
            n = int(round(2.0 ** rng.uniform(5.0, 9.0)))
            shape = (n, n)
        out.append(dict(shape=shape, dim=len(shape), n_modes=int(rng.choice([1024, 2048, 4096])),
                        family="gaussian" if rng.random() < 0.5 else "exponential",
                        ell=(0.1,) * len(shape), sigma2=1.0, mean=0.0, seed=1000 + r))
    return out


def quantile_thresholds(mean, sigma, quantiles):
    """t = mean + sigma * Phi^-1(q) (Sec. 3.1: thresholds from Gaussian percentiles)."""
    from statistics import NormalDist
    nd = NormalDist()
    return [mean + sigma * nd.inv_cdf(q) for q in quantiles]

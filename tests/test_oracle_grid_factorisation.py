"""The identities the tensor-core grid path rests on, checked in FP64 against
the oracle's direct sums (CPU).

On a Cartesian grid each term of Eq. DiscreteFT factorises into an x phasor
and a (y, z) phasor, so the field of a block of cells is a real matrix product
over the modes (Sec. 4.1 term by term), and the adjoint's per-mode sums are a
matrix product over the x cells contracted with the y and z phasors.  These
tests restate both regroupings with numpy and compare them with
`oracle.native.synth` and `oracle.native.mode_sums` on small grids, so the
claim that the grid path computes the same sum (no approximation) is pinned
independently of the CUDA code.
"""
import numpy as np
import pytest

from helpers import oracle_modes


def _axes(shape, seed):
    # non-uniform axes away from the origin, as a rectilinear grid may have
    rng = np.random.default_rng(seed)
    return [3.0 + np.cumsum(rng.uniform(0.01, 0.05, n)) for n in shape]


def _cells(ax):
    mesh = np.meshgrid(*ax[::-1], indexing="ij")  # slowest axis first
    return np.stack([m.ravel() for m in mesh[::-1]], axis=-1)  # x fastest


@pytest.mark.parametrize("shape", [(7, 5, 4), (9, 6)])
def test_field_is_a_product_of_x_and_yz_phasors(shape):
    from oracle import native
    dim = len(shape)
    om = oracle_modes("exponential", 1.7, (0.2, 0.1, 0.15)[:dim], dim, 64, 5)
    ax = _axes(shape, 1)
    cells = _cells(ax)
    direct = native.synth(om["a"], om["amp"], om["psi"], 0.3, cells)
    # Xp[i, j] = e^{2 pi i a_jx X_i};  W[c, j] = A_j e^{2 pi i (psi_j + a_jy Y_k + a_jz Z_l)}
    xp = np.exp(2j * np.pi * np.outer(ax[0], om["a"][:, 0]))
    ygrid = np.stack([m.ravel() for m in np.meshgrid(*ax[1:][::-1], indexing="ij")[::-1]], axis=-1)
    w = om["amp"][None, :] * np.exp(2j * np.pi * (om["psi"][None, :] + ygrid @ om["a"][:, 1:].T))
    # Y - mu = Re(Xp W^T) = Xr Wr^T - Xi Wi^T: a real product over K = 2N
    field = xp.real @ w.real.T - xp.imag @ w.imag.T  # [x cell, (y, z) cell]
    regrouped = 0.3 + field.T.ravel()  # x fastest
    assert np.max(np.abs(regrouped - direct)) <= 1e-12 * np.max(np.abs(direct))


@pytest.mark.parametrize("shape", [(7, 5, 4), (9, 6)])
def test_adjoint_sums_are_x_products_contracted_with_yz_phasors(shape):
    from oracle import native
    dim = len(shape)
    om = oracle_modes("gaussian", 1.1, (0.15, 0.2, 0.1)[:dim], dim, 48, 9)
    ax = _axes(shape, 2)
    cells = _cells(ax)
    g = np.random.default_rng(3).standard_normal(len(cells))
    s_cos, s_sin, s_sinx = native.mode_sums(om["a"], om["psi"], cells, g)
    nx = shape[0]
    gm = g.reshape(-1, nx)  # [(y, z) cell, x cell]
    xw = ax[0] - ax[0][0]  # x weights relative to the first x cell
    xp = np.exp(2j * np.pi * np.outer(ax[0], om["a"][:, 0]))  # [x, mode]
    d = gm @ xp  # D_j(k, l) = sum_i Xp_j(X_i) g(i, k, l)
    dx = (gm * xw[None, :]) @ xp  # the same with the x weights
    ygrid = np.stack([m.ravel() for m in np.meshgrid(*ax[1:][::-1], indexing="ij")[::-1]], axis=-1)
    wyz = np.exp(2j * np.pi * (om["psi"][None, :] + ygrid @ om["a"][:, 1:].T))  # Yp Zp, psi included
    e = np.sum(d * wyz, axis=0)  # E_j = sum_{k, l} D_j(k, l) Yp_j(Y_k) Zp_j(Z_l)
    ex = np.sum(dx * wyz, axis=0)
    assert np.allclose(e.real, s_cos, rtol=0, atol=1e-12 * np.max(np.abs(s_cos)))
    assert np.allclose(e.imag, s_sin, rtol=0, atol=1e-12 * np.max(np.abs(s_sin)))
    # S_x = sum g x sin = Im(sum g (x - X_0) e^{i theta}) + X_0 S_sin; the y and z
    # weights enter per (y, z) cell after the x product
    sx = ex.imag + ax[0][0] * e.imag
    assert np.allclose(sx, s_sinx[:, 0], rtol=0, atol=1e-12 * np.max(np.abs(s_sinx[:, 0])))
    for c in range(1, dim):
        wc = ygrid[:, c - 1] - ygrid[0, c - 1]
        sc = np.sum(d * wyz * wc[:, None], axis=0).imag + ygrid[0, c - 1] * e.imag
        assert np.allclose(sc, s_sinx[:, c], rtol=0, atol=1e-12 * np.max(np.abs(s_sinx[:, c])))

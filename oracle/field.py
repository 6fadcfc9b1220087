"""Field sum, property maps, mismatch loss and adjoint, FP64 (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The field (Sec. 4.1, Eq. DiscreteFT, real reading; see ``modes``):

    Y(x) = mu + sum_{j=0}^{N-1} A_j cos(2 pi (a_j . x + psi_j))

evaluated in FP64 at every cell centre, modes in ascending j, with the phase
t = a_j . x + psi_j reduced as r = t - rint(t) before the cosine.  Cell
coordinates given as float32 are widened to FP64 exactly.

Maps (Sec. 3.1 single truncation rule, Sec. 4.1 scaling, Appendix B):

* lognormal:  K = K_ref exp(Y)   (log-permeability is the Gaussian field);
* indicator:  label = #{m : Y > t_m} for ascending thresholds t_m in Y units,
  so Y equal to a threshold falls in the lower facies;
* values:     property = values[label] (Appendix B `values`);
* porosity:   clamp(phi0 + phi1 (Y - mu)/sigma, phi_min, phi_max).  The paper
  gives no porosity formula; this affine-clamp of the standardised field is
  the reading taken;
* bitruncated: two independent fields (same parameters drawn on generator
  streams 0 and 1) and a two-dimensional truncation rule (Sec. 3.1).

Adjoint of the field sum with g_i = dL/dY_i and theta_ij = 2 pi (a_j.x_i + psi_j):

    dL/dmu    = sum_i g_i
    dL/dA_j   = sum_i g_i cos theta_ij
    dL/dpsi_j = -2 pi A_j sum_i g_i sin theta_ij
    dL/da_jc  = -2 pi A_j sum_i g_i sin theta_ij x_ic
    dL/dsigma = sum_j rho_j dL/dA_j                  (A_j = sigma rho_j)
    dL/dl_c   = -sum_j (a_jc / l_c) dL/da_jc          (a_jc = kappa_jc/(2 pi l_c))

With a rotation R of the anisotropy axes (a = R^T u, u = kappa/(2 pi l)) the
last line reads with u and R dL/da in place of a and dL/da; see
grads_from_sums.

Gradients with respect to the standardised draws themselves (rho, kappa) and
with periodic axes: see grads_reparam.  Along a periodic axis the frequency
is rounded to a multiple of 1/L_c, a step function of kappa, l and R whose
derivative is zero wherever it is defined; so dL/da_c of a periodic axis
reaches none of kappa, l, R (the reading taken: the paper gives no
derivative of its `periodic` option).
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _cells64(cells):
    c = np.asarray(cells)
    if c.ndim == 1:
        c = c[:, None]
    return c.astype(np.float64)


def phase_turns(a_j, psi_j, cells):
    """Reduced phase r = t - rint(t), t = a_j.x + psi_j, for one mode."""
    t = cells @ np.asarray(a_j, dtype=np.float64) + psi_j
    return t - np.rint(t)


def synth(a, amp, psi, mu, cells):
    """Y at every cell.  a: (N, d); amp, psi: (N,); cells: (M, d)."""
    x = _cells64(cells)
    a = np.asarray(a, dtype=np.float64).reshape(len(amp), -1)
    acc = np.zeros(x.shape[0], dtype=np.float64)
    for j in range(len(amp)):
        acc += amp[j] * np.cos(TWO_PI * phase_turns(a[j], psi[j], x))
    return mu + acc


def lognormal(Y, k_ref=1.0):
    return k_ref * np.exp(np.asarray(Y, dtype=np.float64))


def indicator(Y, thresholds):
    Y = np.asarray(Y, dtype=np.float64)
    lab = np.zeros(Y.shape, dtype=np.uint8)
    for t in thresholds:
        lab += (Y > t).astype(np.uint8)
    return lab


def bitruncated(Y1, Y2, t, s, rule):
    """Pluri-Gaussian (bitruncated) facies, Sec. 3.1 and Appendix B
    `bitruncated`: i = #{m : Y1 > t_m}, j = #{m : Y2 > s_m} index one of the
    (len(t) + 1) x (len(s) + 1) Cartesian regions of the truncation rule, and
    rule[i][j] is the facies that region is merged into."""
    i = indicator(Y1, t).astype(np.int64)
    j = indicator(Y2, s).astype(np.int64)
    return np.asarray(rule, dtype=np.uint8)[i, j]


def region_proportions(mu1, sigma1, t, mu2, sigma2, s):
    """p_ij = [G1(t_i) - G1(t_{i-1})] [G2(s_j) - G2(s_{j-1})] (Sec. 3.1) with
    G the Gaussian CDF of each field, t_{-1} = s_{-1} = -inf, t_I = s_J = +inf."""
    from scipy.stats import norm
    tt = np.concatenate([[-np.inf], np.asarray(t, dtype=np.float64), [np.inf]])
    ss = np.concatenate([[-np.inf], np.asarray(s, dtype=np.float64), [np.inf]])
    p1 = np.diff(norm.cdf((tt - mu1) / sigma1))
    p2 = np.diff(norm.cdf((ss - mu2) / sigma2))
    return np.outer(p1, p2)


def facies_values(labels, values):
    return np.asarray(values, dtype=np.float64)[np.asarray(labels, dtype=np.int64)]


def porosity(Y, mu, sigma, phi0, phi1, phi_min, phi_max):
    p = phi0 + phi1 * (np.asarray(Y, dtype=np.float64) - mu) / sigma
    return np.clip(p, phi_min, phi_max)


def quantile_thresholds(mu, sigma, q):
    """Thresholds in Y units at Gaussian quantiles q: t = mu + sigma Phi^-1(q)."""
    from scipy.stats import norm
    return mu + sigma * norm.ppf(np.asarray(q, dtype=np.float64))


def mismatch_loss(K, K_target):
    """L = mean (K - K_target)^2 and g = dL/dY for K = exp(Y)."""
    K = np.asarray(K, dtype=np.float64)
    T = np.asarray(K_target, dtype=np.float64)
    diff = K - T
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff * K / K.size
    return loss, g


def mode_sums(a, psi, cells, g):
    """Per-mode S_cos[j], S_sin[j], S_sinx[j, c] (sums over cells, FP64)."""
    x = _cells64(cells)
    a = np.asarray(a, dtype=np.float64).reshape(len(psi), -1)
    g = np.asarray(g, dtype=np.float64)
    n, d = a.shape
    s_cos = np.empty(n)
    s_sin = np.empty(n)
    s_sinx = np.empty((n, d))
    for j in range(n):
        th = TWO_PI * phase_turns(a[j], psi[j], x)
        c = np.cos(th)
        s = np.sin(th)
        s_cos[j] = np.sum(g * c)
        s_sin[j] = np.sum(g * s)
        s_sinx[j] = (g * s) @ x
    return s_cos, s_sin, s_sinx


def grads_from_sums(s_cos, s_sin, s_sinx, amp, a, sigma, ell, g, rot=None):
    """Chain rule from per-mode sums to all parameter gradients.

    With an axis transform R (a = R^T u, u = kappa / (2 pi l); a rotation or
    any invertible matrix): u = R^-T a, dL/du = R dL/da,
    dL/dl_c = -sum_j (u_jc / l_c) (dL/du_j)_c, and for R as a free matrix
    dL/dR_cd = sum_j u_jc dL/da_jd (returned as "drot")."""
    amp = np.asarray(amp, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64).reshape(len(amp), -1)
    d = a.shape[1]
    ell = np.asarray(ell, dtype=np.float64)[:d]
    dA = np.asarray(s_cos, dtype=np.float64)
    dpsi = -TWO_PI * amp * s_sin
    da = -TWO_PI * amp[:, None] * s_sinx
    rho = amp / sigma
    R = np.eye(d) if rot is None else np.asarray(rot, dtype=np.float64)[:d, :d]
    u = np.linalg.solve(R.T, a.T).T  # a_j = R^T u_j, i.e. a = u R as rows: u = a R^-1
    du = da @ R.T        # dL/du_j = R dL/da_j
    return {
        "dA": dA,
        "dpsi": dpsi,
        "da": da,
        "dmu": float(np.sum(np.asarray(g, dtype=np.float64))),
        "dsigma": float(np.sum(rho * dA)),
        "dell": -np.sum(u * du, axis=0) / ell,
        "drot": u.T @ da,
    }


def backward(a, amp, psi, sigma, ell, cells, g, rot=None):
    """All gradients of a loss with dL/dY = g (see module docstring)."""
    s_cos, s_sin, s_sinx = mode_sums(a, psi, cells, g)
    return grads_from_sums(s_cos, s_sin, s_sinx, amp, a, sigma, ell, g, rot)


def grads_reparam(s_cos, s_sin, s_sinx, kappa, rho, sigma, ell, g, rot=None, period=None):
    """All gradients of a loss with respect to the parameters of the
    reparameterised field of Sec. 4.1 (see modes.reparam):

        Y = mu + sum_j sigma rho_j cos(2 pi (a_j . x + psi_j)),
        a_j = P(R^T u_j),  u_j = kappa_j / (2 pi l),

    P rounding the periodic components to multiples of 1/L_c.  From the
    per-mode sums of mode_sums (taken with the frequencies a_j):

        dA_j     = S_cos[j],   dpsi_j = -2 pi A_j S_sin[j],   da_j = -2 pi A_j S_sinx[j]
        drho_j   = sigma dA_j,           dsigma = sum_j rho_j dA_j,
        dsigma2  = dsigma / (2 sigma),   dmu = sum_i g_i,
        e_j      = M da_j  (M zeroes the periodic components: dP = M almost everywhere)
        du_j     = R e_j,                dkappa_jc = du_jc / (2 pi l_c),
        dl_c     = -sum_j (u_jc / l_c) du_jc,
        dR_cd    = sum_j u_jc e_jd       (R as a free matrix; R = I without a transform).
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    kappa = kappa.reshape(len(kappa), -1)
    d = kappa.shape[1]
    rho = np.asarray(rho, dtype=np.float64)
    ell = np.asarray(ell, dtype=np.float64)[:d]
    amp = sigma * rho
    dA = np.asarray(s_cos, dtype=np.float64)
    dpsi = -TWO_PI * amp * np.asarray(s_sin, dtype=np.float64)
    da = -TWO_PI * amp[:, None] * np.asarray(s_sinx, dtype=np.float64).reshape(len(amp), d)
    R = np.eye(d) if rot is None else np.asarray(rot, dtype=np.float64)[:d, :d]
    mask = np.ones(d)
    if period is not None:
        for c in range(min(d, len(period))):
            if float(period[c]) > 0.0:
                mask[c] = 0.0
    e = da * mask[None, :]
    du = e @ R.T                       # row j: (R e_j)^T
    u = kappa / (TWO_PI * ell[None, :])
    dsigma = float(np.sum(rho * dA))
    return {
        "dA": dA,
        "dpsi": dpsi,
        "da": da,
        "dmu": float(np.sum(np.asarray(g, dtype=np.float64))),
        "dsigma": dsigma,
        "dsigma2": dsigma / (2.0 * sigma),
        "drho": sigma * dA,
        "dkappa": du / (TWO_PI * ell[None, :]),
        "dell": -np.sum(u * du, axis=0) / ell,
        "drot": u.T @ e,
    }

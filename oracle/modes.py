"""Drawing the spectral mode set (Sec. 4.1 and Appendix A), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings of Sec. 4.1, Eq. (DiscreteFT), taken here:

* The "+ i sum sin" of Eq. (DiscreteFT) would make the field complex; the
  real field W_j cos(2 pi a_j.x) + W'_j sin(2 pi a_j.x) is used (the real part
  of the stochastic Fourier integral, Eq. stoFouInt, with Hermitian symmetry).
* The sum runs over exactly N terms, j = 0 .. N-1, N being `nfreq`
  (Appendix B).
* The frequencies are i.i.d. draws from the spectral density normalised to a
  probability density (randomisation method).  Then the importance weight
  S/p equals sigma^2 and the amplitude of each mode is sigma/sqrt(N) times the
  Gaussian weights, which gives Cov(Y(x), Y(x+r)) = C(r) exactly for every N.
* Anisotropy: k_{j,c} = kappa_{j,c} / l_c, a_j = k_j / (2 pi) (turns per unit
  length).
* `disableY` / `disableZ` (Appendix B): kappa is drawn directly in d = dim
  dimensions.
* `Kmean` and `Ksigma` (Appendix B) are the mean mu and the variance sigma^2
  of the Gaussian field Y; the scaling to that mean and variance (Sec. 4.1)
  is the theoretical one, mu + sigma * (unit field).

Writing W cos(t) + W' sin(t) = R cos(t - atan2(W', W)) with R^2 = W^2 + W'^2:

    Y(x) = mu + sum_j A_j cos(2 pi (a_j . x + psi_j)),
    A_j = sigma rho_j,  rho_j = sqrt((W_j^2 + W'_j^2) / N),
    psi_j = -atan2(W'_j, W_j) / (2 pi)   (turns).

Per-mode draws (normal number k of mode j, see ``philox``):

* k = 0: W_j;  k = 1: W'_j;  k = 2 .. 2+d-1: z_{j,c}.
* Gaussian family: kappa_c = sqrt(pi/2) z_c.
* Matern(nu) (exponential = nu 1/2): kappa = z sqrt(2 nu / w), w ~ chi^2_{2nu}.
  If 2 nu is an integer m <= 32, w = sum of the squares of normals
  2+d .. 2+d+m-1.  Otherwise w = 2 G with G ~ Gamma(nu) by Marsaglia and
  Tsang (2000): attempt t uses the first normal of block 64+2t and the first
  uniform of block 65+2t; for nu < 1, G = G(nu+1) U^(1/nu) with U the first
  uniform of block 63.
"""
import math

import numpy as np

from . import philox
from .spectra import EXPONENTIAL, GAUSSIAN, MATERN, effective_nu

MAX_GAMMA_ATTEMPTS = 256


def _chi2_sum_of_squares(seed, stream, j, d, m):
    w = np.zeros(j.shape, dtype=np.float64)
    for i in range(m):
        n = philox.normal(seed, stream, j, 2 + d + i)
        w += n * n
    return w


def _gamma_marsaglia_tsang(seed, stream, j, alpha):
    """Gamma(alpha, 1) for alpha >= 1, one value per mode index in j."""
    dd = alpha - 1.0 / 3.0
    cc = 1.0 / math.sqrt(9.0 * dd)
    out = np.full(j.shape, np.nan)
    todo = np.ones(j.shape, dtype=bool)
    for t in range(MAX_GAMMA_ATTEMPTS):
        if not todo.any():
            break
        jj = j[todo]
        x = philox.normal(seed, stream, jj, 2 * (64 + 2 * t))
        u = philox.uniforms(seed, stream, jj, 65 + 2 * t)[..., 0]
        v = (1.0 + cc * x) ** 3
        ok = v > 0
        logv = np.log(np.where(ok, v, 1.0))
        acc = ok & (np.log(u) < 0.5 * x * x + dd - dd * v + dd * logv)
        idx = np.flatnonzero(todo)
        out[idx[acc]] = dd * v[acc]
        todo[idx[acc]] = False
    if todo.any():
        raise RuntimeError("Marsaglia-Tsang did not accept within the attempt limit")
    return out


def chi2_draw(seed, stream, j, d, nu):
    """w ~ chi^2 with 2 nu degrees of freedom, per mode."""
    m = 2.0 * nu
    if m == round(m) and 1 <= m <= 32:
        return _chi2_sum_of_squares(seed, stream, j, d, int(round(m)))
    if nu >= 1.0:
        return 2.0 * _gamma_marsaglia_tsang(seed, stream, j, nu)
    g = _gamma_marsaglia_tsang(seed, stream, j, nu + 1.0)
    ub = philox.uniforms(seed, stream, j, 63)[..., 0]
    return 2.0 * g * ub ** (1.0 / nu)


def gen_modes(family, sigma2, ell, dim, n_modes, seed, nu=1.5, stream=0, period=None, rot=None):
    """Draw the N modes of one realisation.

    rot: optional d x d invertible axis transform R (a rotation whose rows are
    the principal axes of the anisotropy, or a general matrix; Sec. 4.1: the
    per-axis rescaling of frequency space extended to such transforms).  The
    covariance is C(r) = sigma^2 rho(|diag(1/l) R r|), so
    with u = kappa / (2 pi l) the frequencies are a = R^T u (a = u without R).

    period: optional per-axis domain lengths L_c (0 = not periodic).  Along a
    periodic axis the frequency is moved to the nearest multiple of 1/L_c,
    a_c = floor(a_c L_c + 1/2) / L_c, so the field repeats with period L_c
    (Appendix B `periodic`; the paper gives no construction, this is the
    reading taken).

    Returns a dict of FP64 arrays: kappa (N, d), W, Wp, rho, amp, psi (N,),
    a (N, d) in turns per unit length, plus the scalars sigma, ell (d,).
    """
    if family not in (GAUSSIAN, EXPONENTIAL, MATERN):
        raise ValueError("family")
    if not 1 <= dim <= 3:
        raise ValueError("dim")
    if n_modes < 1:
        raise ValueError("n_modes")
    ell = np.asarray(ell, dtype=np.float64)[:dim]
    j = np.arange(n_modes, dtype=np.uint64)
    W = philox.normal(seed, stream, j, 0)
    Wp = philox.normal(seed, stream, j, 1)
    z = np.stack([philox.normal(seed, stream, j, 2 + c) for c in range(dim)], axis=-1)
    if family == GAUSSIAN:
        kappa = math.sqrt(0.5 * math.pi) * z
    else:
        nu_e = effective_nu(family, nu)
        w = chi2_draw(seed, stream, j, dim, nu_e)
        kappa = z * np.sqrt(2.0 * nu_e / w)[:, None]
    rho = np.sqrt((W * W + Wp * Wp) / n_modes)
    sigma = math.sqrt(sigma2)
    amp, a = reparam(kappa, rho, sigma, ell, rot=rot, period=period)
    return {
        "kappa": kappa,
        "W": W,
        "Wp": Wp,
        "rho": rho,
        "amp": amp,
        "psi": -np.arctan2(Wp, W) / (2.0 * math.pi),
        "a": a,
        "sigma": sigma,
        "ell": ell,
    }


def reparam(kappa, rho, sigma, ell, rot=None, period=None):
    """Amplitudes and frequencies of the modes from their standardised draws
    (Sec. 4.1: scaling to the variance and rescaling of frequency space).

    A_j = sigma rho_j;  u_j = kappa_j / (2 pi l) per axis;  a_j = R^T u_j with
    an axis transform R (a_j = u_j without one);  along a periodic axis c
    (period[c] = L_c > 0) a_jc = floor(a_jc L_c + 1/2) / L_c.
    kappa: (N, d); rho: (N,); ell: (d,) or longer.  Returns (amp, a)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    kappa = kappa.reshape(len(kappa), -1)
    dim = kappa.shape[1]
    ell = np.asarray(ell, dtype=np.float64)[:dim]
    a = kappa / (2.0 * math.pi * ell[None, :])
    if rot is not None:
        R = np.asarray(rot, dtype=np.float64)[:dim, :dim]
        a = a @ R  # row j: (R^T u_j)^T = u_j^T R
    if period is not None:
        for c in range(dim):
            L = float(period[c]) if c < len(period) else 0.0
            if L > 0.0:
                a[:, c] = np.floor(a[:, c] * L + 0.5) / L
    return sigma * np.asarray(rho, dtype=np.float64), a

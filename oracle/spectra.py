"""Covariance functions and spectral densities (Appendix A), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings of Appendix A taken here:

* Appendix A writes every gamma(r) in the variogram form sigma^2 (1 - rho(r))
  while calling it a covariance.  The covariance used is C(r) = sigma^2 rho(r):
    Gaussian     rho(r) = exp(-pi/4 (r/lambda)^2)                  (gauSpe)
    exponential  rho(r) = exp(-r/lambda)                           (expSpe)
    Matern       rho(r) = 2^(1-nu)/Gamma(nu) (sqrt(2nu) r/lambda)^nu
                          K_nu(sqrt(2nu) r/lambda)                 (matSpe)
* Eq. (DiscreteFT) works with the frequency a (phase 2 pi a.x) while
  Appendix A writes S(k).  The convention used is k = 2 pi a with
  C(r) = integral S(k) exp(i k.r) dk, so that integral S(k) dk = sigma^2.
* The Matern spectral density as printed carries pi^((d+1)/2); with it the
  density integrates to sigma^2/sqrt(pi), and at nu = 1/2 it does not reduce
  to the printed exponential density.  The factor is read as pi^(d/2).
  Only the shape S/sigma^2 is used for drawing, so the reading does not change
  any field.
* Anisotropy (Sec. 4.1, rescaling of frequency space): r/lambda is read as
  the norm of the per-axis scaled lag, |(r_1/l_1, ..., r_d/l_d)|, which is the
  same as k_c = kappa_c / l_c for a standardised wave-vector kappa.

Standardised spectral laws (density of kappa = k l, per unit variance):

* Gaussian: kappa_c i.i.d. N(0, pi/2).
* Matern(nu), with the exponential as nu = 1/2: kappa is the d-variate
  Student t with 2 nu degrees of freedom and unit scale, density
  Gamma(nu + d/2) (2nu)^nu / (Gamma(nu) pi^(d/2)) (2nu + |kappa|^2)^-(nu + d/2).
"""
import math

import numpy as np
from scipy import special, stats

GAUSSIAN = 0
EXPONENTIAL = 1
MATERN = 2


def effective_nu(family, nu):
    """Smoothness used for drawing: exponential is Matern with nu = 1/2."""
    if family == EXPONENTIAL:
        return 0.5
    return float(nu)


def correlation(family, r, nu=1.5):
    """rho(r) at the standardised distance r = |lag / lambda| (Appendix A)."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    if family == GAUSSIAN:
        return np.exp(-0.25 * np.pi * r * r)
    if family == EXPONENTIAL:
        return np.exp(-r)
    if family == MATERN:
        s = math.sqrt(2.0 * nu) * r
        out = np.ones_like(s)
        pos = s > 0
        out[pos] = (2.0 ** (1.0 - nu) / special.gamma(nu)) * s[pos] ** nu * special.kv(nu, s[pos])
        return out
    raise ValueError("unknown covariance family")


def covariance(family, lag, ell, sigma2, nu=1.5):
    """C(lag) = sigma^2 rho(|lag_c / ell_c|); lag has shape (..., d)."""
    lag = np.asarray(lag, dtype=np.float64)
    ell = np.asarray(ell, dtype=np.float64)[: lag.shape[-1]]
    r = np.sqrt(np.sum((lag / ell) ** 2, axis=-1))
    return sigma2 * correlation(family, r, nu)


def spectral_density(family, k, ell, sigma2, nu=1.5):
    """S(k) of Appendix A for isotropic ell (scalar) in d = k.shape[-1] dims,
    normalised so that its integral over R^d is sigma^2."""
    k = np.asarray(k, dtype=np.float64)
    d = k.shape[-1]
    lam = float(ell)
    k2 = np.sum(k * k, axis=-1)
    if family == GAUSSIAN:
        return sigma2 * (lam / np.pi) ** d * np.exp(-k2 * lam * lam / np.pi)
    if family == EXPONENTIAL:
        return sigma2 * lam ** d * special.gamma(0.5 * (d + 1)) / (np.pi * (1.0 + k2 * lam * lam)) ** (0.5 * (d + 1))
    if family == MATERN:
        return (sigma2 * lam ** d * special.gamma(nu + 0.5 * d) * (2.0 * nu) ** nu
                / (special.gamma(nu) * np.pi ** (0.5 * d) * (2.0 * nu + lam * lam * k2) ** (nu + 0.5 * d)))
    raise ValueError("unknown covariance family")


def radial_law(family, d, nu=1.5):
    """Frozen scipy law of a statistic of |kappa| for KS tests.

    Gaussian: |kappa|^2 / (pi/2) ~ chi^2_d.  Student (Matern, exponential):
    |kappa|^2 / d ~ F(d, 2 nu).  Returns (transform, law)."""
    if family == GAUSSIAN:
        return (lambda kap: np.sum(kap * kap, axis=-1) / (0.5 * np.pi)), stats.chi2(d)
    nu_t = 2.0 * effective_nu(family, nu)
    return (lambda kap: np.sum(kap * kap, axis=-1) / d), stats.f(d, nu_t)

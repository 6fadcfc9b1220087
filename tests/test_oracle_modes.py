"""Pins of the oracle's mode drawing against Appendix A (no GPU).

* The characteristic function of the drawn frequencies equals the normalised
  covariance of Appendix A: E[cos(2 pi a.r)] = rho(|r/l|).  This ties the
  sampling law, the 2 pi convention and the per-axis rescaling to the closed
  forms (scipy's Bessel K for Matern), independently of the sampler.
* Radial laws: |kappa|^2/(pi/2) ~ chi^2_d (Gaussian); |kappa|^2/d ~ F(d, 2 nu)
  (Student t, Matern and exponential), KS tests including non-integer 2 nu
  (Marsaglia-Tsang branch) and nu < 1 (boost branch).
* Amplitudes and phases: A^2 N / sigma^2 ~ chi^2_2, psi ~ U(-1/2, 1/2].
* Per-mode draws do not depend on N (counter-based streams).
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import modes, spectra

ELL3 = np.array([0.2, 0.1, 0.05])


@pytest.mark.parametrize("family,nu", [(spectra.GAUSSIAN, 0.0), (spectra.EXPONENTIAL, 0.0),
                                       (spectra.MATERN, 1.5), (spectra.MATERN, 1.3),
                                       (spectra.MATERN, 0.7)])
def test_characteristic_function_equals_covariance(family, nu):
    n = 200000
    m = modes.gen_modes(family, 1.0, ELL3, 3, n, seed=20221221, nu=nu)
    lags = []
    for s in (0.25, 0.5, 1.0, 2.0):
        for direction in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]):
            dvec = np.array(direction, dtype=float)
            dvec = dvec / np.linalg.norm(dvec / ELL3)  # unit standardised length
            lags.append(s * dvec)
    lags = np.array(lags)
    emp = np.cos(2.0 * np.pi * (m["a"] @ lags.T)).mean(axis=0)
    want = spectra.covariance(family, lags, ELL3, 1.0, nu=spectra.effective_nu(family, nu))
    se = 1.0 / math.sqrt(2.0 * n) * 1.5
    assert np.max(np.abs(emp - want)) < 5 * se, (emp, want)


def test_covariance_pins_are_not_trivial():
    # the closed forms differ from one another by at least twice the tolerance above
    tol = 5 * 1.5 / math.sqrt(2.0 * 200000)
    r = np.array([0.5, 1.0])
    g = spectra.correlation(spectra.GAUSSIAN, r)
    e = spectra.correlation(spectra.EXPONENTIAL, r)
    m = spectra.correlation(spectra.MATERN, r, nu=1.5)
    assert min(np.max(np.abs(g - e)), np.max(np.abs(m - e)), np.max(np.abs(g - m))) > 2 * tol
    # Matern(1/2) is the exponential (Appendix A)
    assert np.allclose(spectra.correlation(spectra.MATERN, r, nu=0.5), e, rtol=1e-12)


@pytest.mark.parametrize("family", [spectra.GAUSSIAN, spectra.EXPONENTIAL, spectra.MATERN])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_spectral_density_integrates_to_variance(family, d):
    # integral of S over R^d in radial form, with the Matern pi^(d/2) reading
    from scipy import integrate, special
    lam, sig2 = 0.3, 2.5
    surf = 2.0 * math.pi ** (d / 2.0) / special.gamma(d / 2.0)

    def f(k):
        kv = np.zeros((1, d))
        kv[0, 0] = k
        return surf * k ** (d - 1) * spectra.spectral_density(family, kv, lam, sig2, nu=1.5)[0]

    val = integrate.quad(f, 0, np.inf, limit=400)[0]
    assert val == pytest.approx(sig2, rel=1e-6)


@pytest.mark.parametrize("family,nu", [(spectra.GAUSSIAN, 0.0), (spectra.EXPONENTIAL, 0.0),
                                       (spectra.MATERN, 1.5), (spectra.MATERN, 2.25),
                                       (spectra.MATERN, 1.3), (spectra.MATERN, 0.7)])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_radial_law(family, nu, d):
    m = modes.gen_modes(family, 1.0, [1.0, 1.0, 1.0], d, 20000, seed=7 + d, nu=nu)
    transform, law = spectra.radial_law(family, d, nu)
    assert stats.kstest(transform(m["kappa"]), law.cdf).pvalue > 1e-3


def test_gaussian_component_variance():
    m = modes.gen_modes(spectra.GAUSSIAN, 1.0, [1.0, 1.0, 1.0], 3, 100000, seed=3)
    v = np.mean(m["kappa"] ** 2, axis=0)
    assert np.all(np.abs(v - math.pi / 2) < 5 * math.sqrt(2.0) * (math.pi / 2) / math.sqrt(100000))


def test_amplitudes_and_phases():
    n, sig2 = 50000, 3.0
    m = modes.gen_modes(spectra.MATERN, sig2, [0.1, 0.1], 2, n, seed=5, nu=1.5)
    assert stats.kstest(m["amp"] ** 2 * n / sig2, stats.chi2(2).cdf).pvalue > 1e-3
    assert np.all(m["psi"] > -0.5) and np.all(m["psi"] <= 0.5)
    assert stats.kstest(m["psi"] + 0.5, "uniform").pvalue > 1e-3
    # amplitude/phase form is the W, W' form of Eq. DiscreteFT
    th = 0.37
    lhs = m["amp"] * np.cos(th + 2 * np.pi * m["psi"])
    rhs = math.sqrt(sig2 / n) * (m["W"] * np.cos(th) + m["Wp"] * np.sin(th))
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-14)


def test_anisotropic_rescaling_exact():
    m = modes.gen_modes(spectra.EXPONENTIAL, 1.0, ELL3, 3, 1000, seed=1)
    assert np.allclose(m["a"] * 2 * np.pi * ELL3, m["kappa"], rtol=1e-15, atol=0)


def test_draws_independent_of_mode_count_and_streams_differ():
    m1 = modes.gen_modes(spectra.MATERN, 1.0, ELL3, 3, 10, seed=42, nu=1.3)
    m2 = modes.gen_modes(spectra.MATERN, 1.0, ELL3, 3, 100, seed=42, nu=1.3)
    assert np.array_equal(m1["kappa"], m2["kappa"][:10])
    assert np.array_equal(m1["psi"], m2["psi"][:10])
    assert np.allclose(m1["rho"] * math.sqrt(10), m2["rho"][:10] * math.sqrt(100), rtol=1e-15)
    m3 = modes.gen_modes(spectra.MATERN, 1.0, ELL3, 3, 10, seed=42, nu=1.3, stream=1)
    assert not np.any(m3["kappa"] == m1["kappa"])


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        modes.gen_modes(7, 1.0, ELL3, 3, 10, seed=1)
    with pytest.raises(ValueError):
        modes.gen_modes(0, 1.0, ELL3, 4, 10, seed=1)
    with pytest.raises(ValueError):
        modes.gen_modes(0, 1.0, ELL3, 3, 0, seed=1)


def _rotation(alpha, beta, gamma):
    ca, sa, cb, sb, cg, sg = (math.cos(alpha), math.sin(alpha), math.cos(beta), math.sin(beta),
                              math.cos(gamma), math.sin(gamma))
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    Ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    Rx = np.array([[1.0, 0, 0], [0, cg, -sg], [0, sg, cg]])
    return Rz @ Ry @ Rx


@pytest.mark.parametrize("family,nu,kind", [(spectra.GAUSSIAN, 0.0, "rotation"), (spectra.MATERN, 1.5, "rotation"),
                                            (spectra.GAUSSIAN, 0.0, "general"), (spectra.MATERN, 1.5, "general")])
def test_rotated_anisotropy_characteristic_function(family, nu, kind):
    # covariance of the field Z(R x), Z with axis lengths l:
    # C(r) = sigma^2 rho(|diag(1/l) R r|)  (Sec. 4.1, transform of the rescaled frequency
    # space), for a rotation (rows = principal axes) and for a general invertible R
    n = 200000
    R = _rotation(0.7, -0.4, 1.1) if kind == "rotation" else np.array([[1.2, 0.4, 0.0], [-0.3, 0.9, 0.2],
                                                                          [0.1, 0.0, 0.7]])
    m = modes.gen_modes(family, 1.0, ELL3, 3, n, seed=1234, nu=nu, rot=R)
    rng = np.random.default_rng(8)
    lags = rng.standard_normal((12, 3)) * 0.1
    emp = np.cos(2.0 * np.pi * (m["a"] @ lags.T)).mean(axis=0)
    r_std = np.linalg.norm((lags @ R.T) / ELL3, axis=1)
    want = spectra.correlation(family, r_std, nu=spectra.effective_nu(family, nu))
    # the transposed convention would give a different covariance
    wrong = spectra.correlation(family, np.linalg.norm((lags @ R) / ELL3, axis=1),
                                nu=spectra.effective_nu(family, nu))
    tol = 5 * 1.5 / math.sqrt(2.0 * n)
    assert np.max(np.abs(emp - want)) < tol
    assert np.max(np.abs(wrong - want)) > 4 * tol

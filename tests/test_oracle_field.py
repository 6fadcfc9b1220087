"""Pins of the oracle's field sum, maps and adjoint (no GPU).

* single-mode closed forms (phase at 0, 1/4, 1/2, 3/4 turn);
* the amplitude/phase form equals the W cos + W' sin form of Eq. DiscreteFT;
* brute force in 50-digit arithmetic (mpmath) on a small grid;
* one-point and two-point statistics over many seeds: mean mu, variance
  sigma^2, covariance C(r) of Appendix A (exact for every N under the
  randomisation reading), threshold proportions Phi((t - mu)/sigma) and the
  facies proportions p_i = G(t_i) - G(t_{i-1}) (Sec. 3.1);
* resolution independence (Sec. 4.1) and permutation equivariance;
* the adjoint against central finite differences of the FP64 loss, and its
  chain-rule identities;
* the C oracle against the numpy oracle.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import field, modes, native, spectra


def _grid2d(n):
    c = (np.arange(n) + 0.5) / n
    X, Yg = np.meshgrid(c, c, indexing="xy")
    return np.stack([X.ravel(), Yg.ravel()], axis=-1).astype(np.float32)


def test_single_mode_closed_forms():
    mu, A = 0.7, 1.9
    a = np.array([[0.25, 0.0, 0.0]])
    x = np.array([[0.0, 0.3, 0.9], [1.0, 0.1, 0.2], [2.0, 0.5, 0.5], [3.0, 0.7, 0.1]])
    y = field.synth(a, np.array([A]), np.array([0.0]), mu, x)
    assert np.allclose(y, [mu + A, mu, mu - A, mu], rtol=0, atol=1e-15)
    # psi shifts the phase: a.x + psi = 1/2 at x = 0
    y2 = field.synth(a, np.array([A]), np.array([0.5]), mu, x[:1])
    assert y2[0] == pytest.approx(mu - A, abs=1e-15)
    # linear in A, shift by mu
    m = modes.gen_modes(spectra.GAUSSIAN, 1.0, [0.1, 0.1, 0.1], 3, 20, seed=3)
    xr = np.random.default_rng(1).random((50, 3))
    y1 = field.synth(m["a"], m["amp"], m["psi"], 0.0, xr)
    y3 = field.synth(m["a"], 3.0 * m["amp"], m["psi"], 2.0, xr)
    assert np.allclose(y3, 2.0 + 3.0 * y1, rtol=0, atol=1e-13)


def test_amplitude_phase_form_equals_discrete_ft():
    n, sig2, mu = 64, 2.0, -0.3
    m = modes.gen_modes(spectra.EXPONENTIAL, sig2, [0.2, 0.05], 2, n, seed=9)
    x = _grid2d(16).astype(np.float64)
    th = 2 * np.pi * (x @ m["a"].T)
    direct = mu + math.sqrt(sig2 / n) * np.sum(m["W"] * np.cos(th) + m["Wp"] * np.sin(th), axis=1)
    y = field.synth(m["a"], m["amp"], m["psi"], mu, x)
    assert np.allclose(y, direct, rtol=0, atol=1e-12)


def test_brute_force_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    n = 32
    m = modes.gen_modes(spectra.MATERN, 1.5, [0.3, 0.2], 2, n, seed=11, nu=1.5)
    x = _grid2d(8)
    y = field.synth(m["a"], m["amp"], m["psi"], 0.25, x)
    yc = native.synth(m["a"], m["amp"], m["psi"], 0.25, x)
    worst = 0.0
    bound = 0.0
    for i in range(x.shape[0]):
        acc = mpmath.mpf(0)
        for j in range(n):
            t = mpmath.mpf(float(m["psi"][j]))
            for c in range(2):
                t += mpmath.mpf(float(m["a"][j, c])) * mpmath.mpf(float(x[i, c]))
            acc += mpmath.mpf(float(m["amp"][j])) * mpmath.cos(2 * mpmath.pi * t)
        exact = float(acc + mpmath.mpf(0.25))
        worst = max(worst, abs(y[i] - exact), abs(yc[i] - exact))
        # rounding bound: each phase carries ~4 ulp of |t|, each term ~4 ulp of A
        tmag = np.abs(m["psi"]) + np.abs(m["a"]) @ np.abs(x[i].astype(np.float64)) + 1.0
        bound = max(bound, float(np.sum(m["amp"] * (2 * np.pi * 8 * 2.0 ** -53 * tmag + 8 * 2.0 ** -53))) + 1e-15)
    assert worst <= bound
    assert worst < 1e-13 * math.sqrt(1.5)


@pytest.mark.slow
def test_point_statistics_over_seeds():
    # exact for every N: mean mu, variance sigma^2, Cov = C(r) (Appendix A)
    R, n, sig2, mu = 3000, 16, 2.0, 0.5
    ell = np.array([0.2, 0.05])
    x0 = np.array([0.31, 0.47])
    lags = np.array([[0.0, 0.0], [0.1, 0.0], [0.2, 0.0], [0.0, 0.025], [0.0, 0.05], [0.1, 0.05]])
    pts = x0 + lags
    for family, nu in ((spectra.GAUSSIAN, 0.0), (spectra.EXPONENTIAL, 0.0), (spectra.MATERN, 1.5)):
        vals = np.empty((R, len(pts)))
        for r in range(R):
            m = modes.gen_modes(family, sig2, ell, 2, n, seed=1000 + r, nu=nu)
            vals[r] = field.synth(m["a"], m["amp"], m["psi"], mu, pts)
        se_mean = math.sqrt(sig2 / R)
        assert abs(vals[:, 0].mean() - mu) < 5 * se_mean
        dev = vals - mu
        cov = (dev[:, :1] * dev).mean(axis=0)
        want = spectra.covariance(family, lags, ell, sig2, nu=spectra.effective_nu(family, nu))
        se = sig2 * np.sqrt((1.0 + (want / sig2) ** 2) / R)
        assert np.all(np.abs(cov - want) < 5 * se), (family, cov, want)


@pytest.mark.slow
def test_threshold_and_facies_proportions():
    R, n, sig2, mu = 4000, 8, 4.0, 1.0
    q = np.array([1.0 / 3.0, 2.0 / 3.0])
    t = field.quantile_thresholds(mu, math.sqrt(sig2), q)
    x = np.array([[0.1, 0.2, 0.3]])
    ys = np.empty(R)
    for r in range(R):
        m = modes.gen_modes(spectra.EXPONENTIAL, sig2, [0.2, 0.2, 0.05], 3, n, seed=50000 + r)
        ys[r] = field.synth(m["a"], m["amp"], m["psi"], mu, x)[0]
    # marginal is exactly N(mu, sigma^2) under the randomisation reading
    assert stats.kstest((ys - mu) / math.sqrt(sig2), "norm").pvalue > 1e-3
    lab = field.indicator(ys, t)
    G = stats.norm.cdf((np.concatenate([[-np.inf], t, [np.inf]]) - mu) / math.sqrt(sig2))
    p = np.diff(G)  # p_i = G(t_i) - G(t_{i-1})
    assert np.allclose(p, [1 / 3, 1 / 3, 1 / 3], atol=1e-12)
    counts = np.bincount(lab, minlength=3)
    se = np.sqrt(p * (1 - p) / R)
    assert np.all(np.abs(counts / R - p) < 5 * se)
    # lognormal mean
    K = field.lognormal(ys)
    sdK = math.sqrt((math.exp(sig2) - 1) * math.exp(2 * mu + sig2) / R)
    assert abs(K.mean() - math.exp(mu + sig2 / 2)) < 6 * sdK


def test_maps_definitions():
    Y = np.array([-1.0, 0.0, 0.2, 0.5, 2.0])
    assert field.indicator(Y, [0.0]).tolist() == [0, 0, 1, 1, 1]  # Y == t -> lower facies
    assert field.indicator(Y, [0.0, 0.5]).tolist() == [0, 0, 1, 1, 2]
    assert np.allclose(field.facies_values([0, 2, 1], [10.0, 20.0, 30.0]), [10.0, 30.0, 20.0])
    assert np.allclose(field.lognormal(Y, 2.0), 2.0 * np.exp(Y))
    phi = field.porosity(Y, 0.5, 2.0, 0.3, 0.1, 0.1, 0.35)
    assert np.allclose(phi, np.clip(0.3 + 0.1 * (Y - 0.5) / 2.0, 0.1, 0.35))
    t = field.quantile_thresholds(0.0, 2.0, [1 / 3, 2 / 3])
    assert np.allclose(t, [-0.861454, 0.861454], atol=1e-6)


def test_resolution_independence_and_permutation():
    m = modes.gen_modes(spectra.GAUSSIAN, 1.0, [0.1, 0.1], 2, 100, seed=1)
    g64 = _grid2d(64)
    g192 = _grid2d(192)
    y64 = native.synth(m["a"], m["amp"], m["psi"], 0.0, g64)
    y192 = native.synth(m["a"], m["amp"], m["psi"], 0.0, g192)
    # centre (i+1/2)/64 equals centre (3i+1+1/2)/192
    idx = np.arange(64) * 3 + 1
    sub = y192.reshape(192, 192)[np.ix_(idx, idx)].ravel()
    assert np.array_equal(sub, y64)
    perm = np.random.default_rng(5).permutation(len(g64))
    yp = native.synth(m["a"], m["amp"], m["psi"], 0.0, g64[perm])
    assert np.array_equal(yp, y64[perm])


def test_native_matches_numpy():
    for family, d in ((spectra.GAUSSIAN, 1), (spectra.EXPONENTIAL, 2), (spectra.MATERN, 3)):
        m = modes.gen_modes(family, 2.0, [0.2, 0.1, 0.05], d, 300, seed=4)
        x = np.random.default_rng(2).random((500, d)).astype(np.float32)
        y1 = field.synth(m["a"], m["amp"], m["psi"], 0.1, x)
        y2 = native.synth(m["a"], m["amp"], m["psi"], 0.1, x)
        tmag = np.sum(m["amp"] * (np.abs(m["a"]).sum(axis=1) + 1.0))
        assert np.max(np.abs(y1 - y2)) < 64 * 2.0 ** -53 * 2 * np.pi * tmag
        g = np.random.default_rng(3).standard_normal(500)
        s1 = field.mode_sums(m["a"], m["psi"], x, g)
        s2 = native.mode_sums(m["a"], m["psi"], x, g)
        for u, v in zip(s1, s2):
            assert np.allclose(u, v, rtol=1e-9, atol=1e-9)


def _loss_for(params, cells, target):
    m = modes.gen_modes(params["family"], params["sigma"] ** 2, params["ell"], cells.shape[1],
                        params["n"], params["seed"])
    amp = m["amp"].copy()
    psi = m["psi"].copy()
    a = m["a"].copy()
    if "dA" in params:
        amp[params["dA"][0]] += params["dA"][1]
    if "dpsi" in params:
        psi[params["dpsi"][0]] += params["dpsi"][1]
    if "da" in params:
        a[params["da"][0], params["da"][1]] += params["da"][2]
    y = field.synth(a, amp, psi, params["mu"], cells)
    return field.mismatch_loss(field.lognormal(y), target)[0]


def test_adjoint_against_finite_differences():
    n3 = 8
    c = (np.arange(n3) + 0.5) / n3
    X, Yg, Z = np.meshgrid(c, c, c, indexing="ij")
    cells = np.stack([X.ravel(), Yg.ravel(), Z.ravel()], axis=-1)
    base = {"family": spectra.GAUSSIAN, "sigma": 1.0, "ell": np.array([0.3, 0.25, 0.2]), "n": 24,
            "seed": 1, "mu": 0.0}
    mt = modes.gen_modes(spectra.GAUSSIAN, 1.0, base["ell"], 3, 24, seed=2)
    target = field.lognormal(field.synth(mt["a"], mt["amp"], mt["psi"], 0.0, cells))
    m = modes.gen_modes(spectra.GAUSSIAN, 1.0, base["ell"], 3, 24, seed=1)
    y = field.synth(m["a"], m["amp"], m["psi"], 0.0, cells)
    K = field.lognormal(y)
    _, g = field.mismatch_loss(K, target)
    gr = field.backward(m["a"], m["amp"], m["psi"], 1.0, base["ell"], cells, g)
    h = 1e-4

    def shifted(step, **kw):
        p1 = dict(base)
        for k, v in kw.items():
            if k in ("mu", "sigma"):
                p1[k] = base[k] + step
            elif k == "ell":
                e1 = base["ell"].copy()
                e1[v] += step
                p1["ell"] = e1
            elif k == "dA" or k == "dpsi":
                p1[k] = (v, step)
            elif k == "da":
                p1[k] = (v[0], v[1], step)
        return _loss_for(p1, cells, target)

    def fd(**kw):
        # central differences at h and 2h combined (Richardson): error O(h^4)
        d1 = (shifted(h, **kw) - shifted(-h, **kw)) / (2 * h)
        d2 = (shifted(2 * h, **kw) - shifted(-2 * h, **kw)) / (4 * h)
        return (4.0 * d1 - d2) / 3.0

    def close(x, y):
        return abs(x - y) <= 1e-6 * max(abs(x), abs(y)) + 1e-12

    assert close(gr["dmu"], fd(mu=True))
    assert close(gr["dsigma"], fd(sigma=True))
    for c_ in range(3):
        assert close(gr["dell"][c_], fd(ell=c_))
    for j in (0, 5, 17, 23):
        assert close(gr["dA"][j], fd(dA=j))
        assert close(gr["dpsi"][j], fd(dpsi=j))
        for c_ in range(3):
            assert close(gr["da"][j, c_], fd(da=(j, c_)))
    # chain-rule identities
    assert gr["dsigma"] * 1.0 == pytest.approx(np.sum(m["amp"] * gr["dA"]), rel=1e-12)
    assert np.allclose(base["ell"] * gr["dell"], -np.sum(m["a"] * gr["da"], axis=0), rtol=1e-12)
    assert gr["dmu"] == pytest.approx(np.sum(g), rel=1e-12)


def test_bitruncated_rule_definition():
    from oracle import field as of
    Y1 = np.array([-2.0, -0.1, 0.3, 0.3, 2.0, 0.0])
    Y2 = np.array([0.0, 1.0, -1.0, 0.6, 0.6, 0.5])
    t = [0.0, 1.0]          # 3 classes along Y1
    s = [0.5]               # 2 classes along Y2
    rule = [[0, 1], [2, 1], [3, 3]]
    got = of.bitruncated(Y1, Y2, t, s, rule)
    # (i, j): (0,0) (0,1) (1,0) (1,1) (2,1) (0,0)  -- Y == threshold goes to the lower class
    assert got.tolist() == [0, 1, 2, 1, 3, 0]


@pytest.mark.slow
def test_bitruncated_proportions_over_seeds():
    # two independent fields (streams 0 and 1 of one seed); region proportions
    # p_ij = [G1(t_i) - G1(t_{i-1})][G2(s_j) - G2(s_{j-1})] (Sec. 3.1)
    from oracle import field as of
    R, n = 3000, 16
    t = [-0.5, 0.7]
    s = [0.2]
    x = np.array([[0.31, 0.62]])
    y1 = np.empty(R)
    y2 = np.empty(R)
    for r in range(R):
        m1 = modes.gen_modes(spectra.GAUSSIAN, 1.0, [0.1, 0.1], 2, n, seed=90000 + r, stream=0)
        m2 = modes.gen_modes(spectra.EXPONENTIAL, 2.0, [0.2, 0.1], 2, n, seed=90000 + r, stream=1)
        y1[r] = field.synth(m1["a"], m1["amp"], m1["psi"], 0.0, x)[0]
        y2[r] = field.synth(m2["a"], m2["amp"], m2["psi"], 0.5, x)[0]
    assert abs(np.corrcoef(y1, y2)[0, 1]) < 5 / math.sqrt(R)  # independent streams
    rule = np.arange(6).reshape(3, 2)  # every region its own facies
    lab = of.bitruncated(y1, y2, t, s, rule)
    p = of.region_proportions(0.0, 1.0, t, 0.5, math.sqrt(2.0), s)
    assert p.sum() == pytest.approx(1.0, abs=1e-12)
    counts = np.bincount(lab, minlength=6).reshape(3, 2) / R
    se = np.sqrt(p * (1 - p) / R)
    assert np.all(np.abs(counts - p) < 5 * se)


def test_periodic_option_repeats_exactly():
    # Appendix B `periodic`: frequencies on multiples of 1/L_c make the field
    # repeat with period L_c along that axis (and only that axis)
    L = np.array([2.0, 1.0, 0.0])
    m = modes.gen_modes(spectra.EXPONENTIAL, 1.5, [0.2, 0.1, 0.1], 3, 300, seed=8, period=L)
    assert np.all(np.abs(m["a"][:, 0] * 2.0 - np.round(m["a"][:, 0] * 2.0)) == 0)
    assert np.all(np.abs(m["a"][:, 1] - np.round(m["a"][:, 1])) == 0)
    mp = modes.gen_modes(spectra.EXPONENTIAL, 1.5, [0.2, 0.1, 0.1], 3, 300, seed=8)
    assert np.array_equal(m["a"][:, 2], mp["a"][:, 2])  # non-periodic axis untouched
    x = np.random.default_rng(3).random((200, 3))
    y0 = field.synth(m["a"], m["amp"], m["psi"], 0.0, x)
    tmag = np.sum(m["amp"] * (np.abs(m["a"]).sum(1) * 3.0 + 1))
    for shift in ([2.0, 0, 0], [0, 1.0, 0], [4.0, -3.0, 0]):
        ys = field.synth(m["a"], m["amp"], m["psi"], 0.0, x + np.array(shift))
        assert np.max(np.abs(ys - y0)) < 64 * 2.0 ** -52 * 2 * np.pi * tmag
    ynp = field.synth(m["a"], m["amp"], m["psi"], 0.0, x + np.array([0, 0, 0.37]))
    assert np.max(np.abs(ynp - y0)) > 1e-3  # not periodic along z


@pytest.mark.parametrize("kind", ["rotation", "general"])
def test_rotated_adjoint_against_finite_differences(kind):
    # dL/dl and dL/dR of the transformed anisotropy a = R^T kappa / (2 pi l),
    # for a rotation and for a general (sheared, scaled) invertible R
    from oracle import field as of
    n3 = 7
    c = (np.arange(n3) + 0.5) / n3
    X, Yg, Z = np.meshgrid(c, c, c, indexing="ij")
    cells = np.stack([X.ravel(), Yg.ravel(), Z.ravel()], axis=-1)
    ell = np.array([0.3, 0.2, 0.25])
    th = 0.6
    R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    if kind == "general":
        R = np.array([[1.1, 0.5, 0.0], [0.0, 0.8, 0.3], [0.2, 0.0, 1.3]])
    base = modes.gen_modes(spectra.GAUSSIAN, 1.0, ell, 3, 20, seed=3)
    u = base["a"]                     # kappa / (2 pi l)
    target = of.lognormal(of.synth(u @ R, base["amp"], base["psi"], 0.0, cells) * 0.8)

    def loss(ell_, R_):
        a = (base["kappa"] / (2 * np.pi * ell_[None, :])) @ R_
        return of.mismatch_loss(of.lognormal(of.synth(a, base["amp"], base["psi"], 0.0, cells)), target)

    L0, g = loss(ell, R)
    gr = of.backward(u @ R, base["amp"], base["psi"], 1.0, ell, cells, g, rot=R)
    h = 1e-5

    def fd(fun):
        return (fun(h) - fun(-h)) / (2 * h)

    for c_ in range(3):
        e = np.eye(3)[c_]
        num = fd(lambda s: loss(ell + s * e, R)[0])
        assert gr["dell"][c_] == pytest.approx(num, rel=1e-5, abs=1e-9)
    for (i, j) in ((0, 0), (0, 1), (1, 0), (2, 2), (1, 2)):
        E = np.zeros((3, 3))
        E[i, j] = 1.0
        num = fd(lambda s: loss(ell, R + s * E)[0])
        assert gr["drot"][i, j] == pytest.approx(num, rel=1e-5, abs=1e-9)


@pytest.mark.parametrize("case", ["plain", "periodic2d", "rotated_periodic", "general_periodic"])
def test_reparam_adjoint_against_finite_differences(case):
    # Gradients with respect to the standardised draws and the covariance
    # parameters of Sec. 4.1 (A = sigma rho, a = P(R^T kappa / (2 pi l))):
    # Richardson central differences of the FP64 loss through modes.reparam.
    # Along a periodic axis the rounding P is locally constant, so its
    # frequency contributes nothing to dkappa, dl, dR (checked against the
    # differences, which step through P itself).
    from oracle import field as of
    dim = 2 if case == "periodic2d" else 3
    n1 = {2: 14, 3: 7}[dim]
    c = (np.arange(n1) + 0.5) / n1
    cells = np.stack([v.ravel() for v in np.meshgrid(*([c] * dim), indexing="ij")], axis=-1)
    ell = np.array([0.3, 0.2, 0.25])[:dim]
    th = 0.6
    R = None
    if case == "rotated_periodic":
        R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    elif case == "general_periodic":
        R = np.array([[1.1, 0.5, 0.0], [0.0, 0.8, 0.3], [0.2, 0.0, 1.3]])
    period = None if case == "plain" else ([1.0, 0.0] if dim == 2 else [1.0, 0.0, 2.0])
    m = modes.gen_modes(spectra.GAUSSIAN, 1.0, ell, dim, 20, seed=3)
    kappa, rho, psi = m["kappa"], m["rho"], m["psi"]
    mt = modes.gen_modes(spectra.GAUSSIAN, 1.0, ell, dim, 20, seed=4)
    target = of.lognormal(of.synth(mt["a"], mt["amp"], mt["psi"], 0.0, cells))
    p0 = {"mu": 0.1, "sigma2": 1.3, "ell": ell, "R": np.eye(dim) if R is None else R, "rho": rho, "psi": psi,
          "kappa": kappa}

    def frequencies(p):
        return modes.reparam(p["kappa"], p["rho"], math.sqrt(p["sigma2"]), p["ell"], rot=p["R"], period=period)[1]

    def loss(p):
        amp, a = modes.reparam(p["kappa"], p["rho"], math.sqrt(p["sigma2"]), p["ell"], rot=p["R"], period=period)
        return of.mismatch_loss(of.lognormal(of.synth(a, amp, p["psi"], p["mu"], cells)), target)

    L0, g = loss(p0)
    amp0, a0 = modes.reparam(kappa, rho, math.sqrt(1.3), ell, rot=p0["R"], period=period)
    sums = of.mode_sums(a0, psi, cells, g)
    gr = of.grads_reparam(*sums, kappa, rho, math.sqrt(1.3), ell, g, rot=p0["R"], period=period)
    h = 1e-4

    def moved(key, idx, step):
        p = dict(p0)
        v = np.array(p0[key], dtype=np.float64, copy=True)
        if idx is None:
            v = v + step
        else:
            v[idx] += step
        p[key] = v if idx is not None else float(v)
        return p

    def fd(key, idx=None):
        vals = {}
        for s_ in (-2, -1, 1, 2):
            p = moved(key, idx, s_ * h)
            # the step must not cross a rounding boundary of a periodic axis
            assert np.array_equal(frequencies(p)[:, [k for k in range(dim) if period is not None
                                                     and period[k] > 0]],
                                  a0[:, [k for k in range(dim) if period is not None and period[k] > 0]])
            vals[s_] = loss(p)[0]
        d1 = (vals[1] - vals[-1]) / (2 * h)
        d2 = (vals[2] - vals[-2]) / (4 * h)
        return (4.0 * d1 - d2) / 3.0

    def close(x, y):
        return abs(x - y) <= 1e-6 * max(abs(x), abs(y)) + 1e-11

    assert close(gr["dmu"], fd("mu"))
    assert close(gr["dsigma2"], fd("sigma2"))
    for c_ in range(dim):
        assert close(gr["dell"][c_], fd("ell", c_)), c_
    for i in range(dim):
        for k in range(dim):
            assert close(gr["drot"][i, k], fd("R", (i, k))), (i, k)
    for j in (0, 7, 19):
        assert close(gr["drho"][j], fd("rho", j))
        assert close(gr["dpsi"][j], fd("psi", j))
        for c_ in range(dim):
            assert close(gr["dkappa"][j, c_], fd("kappa", (j, c_))), (j, c_)
    # the same sums give the plain frequency gradients of grads_from_sums
    plain = of.grads_from_sums(*sums, amp0, a0, math.sqrt(1.3), ell, g, rot=p0["R"])
    for k in ("dA", "dpsi", "da", "dmu", "dsigma"):
        assert np.allclose(gr[k], plain[k], rtol=1e-13, atol=0)
    if period is not None and R is None:
        # no transform: a periodic axis's frequency moves with neither kappa nor l
        assert gr["dell"][0] == 0.0 and np.all(gr["dkappa"][:, 0] == 0.0)

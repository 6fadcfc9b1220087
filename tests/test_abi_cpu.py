"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol declared in include/grf.h, draws the same modes as the oracle, packs
the device table as documented and rejects bad arguments."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import modes as omodes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2212_10961_gb300 import _abi
    _abi.lib()
    return _abi


def header_functions():
    src = open(os.path.join(ROOT, "include", "grf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grf_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(abi):
    names = header_functions()
    assert len(names) >= 20
    L = abi.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(abi.exported_symbols()) == names


def test_checked_library_exports_the_same_symbols(abi):
    # the checked flavour (device-side index checks) is a drop-in replacement
    names = header_functions()
    path = os.path.join(ROOT, "paper_2212_10961_gb300", "libgrf_checked.so")
    C = ctypes.CDLL(path)
    for n in names:
        assert hasattr(C, n), n
    assert C.grf_checked_build() == 1
    assert abi.lib().grf_checked_build() == 0
    assert C.grf_take_index_faults(None) == abi.GRF_EINVAL


def test_version_and_launch_count(abi):
    assert abi.lib().grf_version().decode().startswith("grf-gb300")
    assert abi.lib().grf_launch_count() >= 0


@pytest.mark.parametrize("family,nu,dim", [(0, 0.0, 1), (0, 0.0, 3), (1, 0.0, 2), (1, 0.0, 3),
                                           (2, 1.5, 3), (2, 1.3, 2), (2, 0.7, 3), (2, 2.25, 1)])
def test_gen_modes_matches_oracle(abi, family, nu, dim):
    from paper_2212_10961_gb300 import field as F
    ell = (0.2, 0.1, 0.05)
    p = F.FieldParams(family=family, sigma2=2.5, ell=ell[:dim], dim=dim, n_modes=777, seed=123456789012,
                      nu=nu, stream=3)
    got = F.gen_modes(p)
    want = omodes.gen_modes(family, 2.5, ell, dim, 777, 123456789012, nu=nu, stream=3)
    for k in ("kappa", "rho", "psi", "a", "amp"):
        np.testing.assert_allclose(got[k], want[k], rtol=4e-15, atol=1e-300, err_msg=k)


@pytest.mark.parametrize("family,nu", [(1, 0.0), (2, 1.3)])
def test_gen_modes_threaded_ranges_match_oracle(abi, family, nu):
    # more modes than one host thread draws: ranges of j run on several threads
    from paper_2212_10961_gb300 import field as F
    n = 4099
    p = F.FieldParams(family=family, sigma2=1.0, ell=(0.2, 0.1, 0.05), dim=3, n_modes=n, seed=31, nu=nu)
    got = F.gen_modes(p)
    want = omodes.gen_modes(family, 1.0, (0.2, 0.1, 0.05), 3, n, 31, nu=nu)
    for k in ("kappa", "rho", "psi", "a", "amp"):
        np.testing.assert_allclose(got[k], want[k], rtol=4e-15, atol=1e-300, err_msg=k)


def test_gen_modes_periodic_matches_oracle(abi):
    from paper_2212_10961_gb300 import field as F
    p = F.FieldParams(family="exponential", sigma2=1.0, ell=(0.2, 0.1, 0.05), dim=3, n_modes=500, seed=77,
                      period=(2.0, 1.0, 0.0))
    got = F.gen_modes(p)
    want = omodes.gen_modes(1, 1.0, (0.2, 0.1, 0.05), 3, 500, 77, period=(2.0, 1.0, 0.0))
    np.testing.assert_array_equal(got["a"][:, :2], want["a"][:, :2])
    np.testing.assert_allclose(got["a"][:, 2], want["a"][:, 2], rtol=4e-15)
    p.period = (-1.0, 0.0, 0.0)
    with pytest.raises(abi.GRFError):
        F.gen_modes(p)


def _params(abi, **kw):
    p = abi.grf_params()
    p.family, p.dim, p.nu, p.sigma2, p.mean = 0, 2, 1.5, 1.0, 0.0
    p.ell[0] = p.ell[1] = p.ell[2] = 0.1
    p.n_modes, p.seed, p.stream, p.reserved = 10, 1, 0, 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _modes_for(abi, n, dim):
    arr = {k: np.zeros(n * (dim if k in ("kappa", "a") else 1)) for k in ("kappa", "rho", "psi", "a", "amp")}
    m = abi.grf_modes()
    m.n, m.dim = n, dim
    for k in arr:
        setattr(m, k, arr[k].ctypes.data_as(abi.c_dp))
    return m, arr


@pytest.mark.parametrize("bad", [dict(family=5), dict(dim=0), dict(dim=4), dict(sigma2=0.0),
                                 dict(sigma2=float("nan")), dict(n_modes=0), dict(n_modes=(1 << 24) + 1),
                                 dict(reserved=1), dict(family=2, nu=-1.0)])
def test_gen_modes_rejects_bad_params(abi, bad):
    p = _params(abi, **bad)
    m, _ = _modes_for(abi, 10, 2)
    rc = abi.lib().grf_gen_modes(ctypes.byref(p), ctypes.byref(m))
    assert rc == abi.GRF_EINVAL
    assert len(abi.lib().grf_last_error()) > 0


def test_gen_modes_general_transform_matches_oracle_and_singular_is_rejected(abi):
    # Sec. 4.1: any invertible axis transform R, a = R^T kappa / (2 pi l)
    from paper_2212_10961_gb300 import field as F
    R = np.array([[1.1, 0.5, 0.0], [0.0, 0.8, 0.3], [0.2, 0.0, 1.3]])
    p = F.FieldParams(family="matern", sigma2=1.5, ell=(0.2, 0.1, 0.05), dim=3, n_modes=300, seed=41, nu=1.5,
                      rot=R.tolist())
    got = F.gen_modes(p)
    want = omodes.gen_modes(omodes.MATERN, 1.5, (0.2, 0.1, 0.05), 3, 300, 41, nu=1.5, rot=R)
    # a = R^T u sums products of either sign: agreement to a few ulps of the largest term
    scale = np.max(np.abs(want["a"]), axis=1, keepdims=True)
    assert np.all(np.abs(got["a"] - want["a"]) <= 8e-16 * scale * np.max(np.abs(R)))
    S = R.copy()
    S[2] = S[0] + S[1]  # rank 2
    ps = F.FieldParams(family="matern", sigma2=1.5, ell=(0.2, 0.1, 0.05), dim=3, n_modes=300, seed=41, nu=1.5,
                       rot=S.tolist())
    m, _ = _modes_for(abi, 300, 3)
    assert abi.lib().grf_gen_modes(ctypes.byref(ps.to_c()), ctypes.byref(m)) == abi.GRF_EINVAL
    assert "invertible" in abi.lib().grf_last_error().decode()


def test_gen_modes_rejects_mismatched_output(abi):
    p = _params(abi)
    m, _ = _modes_for(abi, 9, 2)
    assert abi.lib().grf_gen_modes(ctypes.byref(p), ctypes.byref(m)) == abi.GRF_EINVAL
    p2 = _params(abi, ell=(ctypes.c_double * 3)(0.1, -1.0, 0.1))
    m2, _ = _modes_for(abi, 10, 2)
    assert abi.lib().grf_gen_modes(ctypes.byref(p2), ctypes.byref(m2)) == abi.GRF_EINVAL


def _parse_table(buf, n, dim):
    b = np.frombuffer(buf, dtype=np.uint8)
    hdr = np.frombuffer(b[:256].tobytes(), dtype=np.int32)
    magic, n_modes, n_pad, d = hdr[0], hdr[1], hdr[2], hdr[3]
    has_kappa = hdr[7]
    off = np.frombuffer(b[32:80].tobytes(), dtype=np.int64)
    off_hot, off_cold, off_order, off_kpref, total, off_kappa = off
    hot = np.frombuffer(b[off_hot:off_hot + n_pad * 16].tobytes(), dtype=np.float32).reshape(n_pad, 4)
    cold = np.frombuffer(b[off_cold:off_cold + n_pad * 32].tobytes(), dtype=np.float32).reshape(n_pad, 8)
    order = np.frombuffer(b[off_order:off_order + n_pad * 4].tobytes(), dtype=np.int32)
    kpref = np.frombuffer(b[off_kpref:off_kpref + 160 * 4].tobytes(), dtype=np.int32)
    kappa = np.frombuffer(b[off_kappa:off_kappa + n_pad * 24].tobytes(), dtype=np.float64).reshape(n_pad, 3)
    return dict(magic=magic, n=n_modes, n_pad=n_pad, dim=d, hot=hot, cold=cold, order=order, kpref=kpref,
                total=total, has_kappa=has_kappa, kappa=kappa, off_kappa=off_kappa)


@pytest.mark.parametrize("n,dim", [(1, 1), (130, 2), (1000, 3)])
def test_pack_table_layout(abi, n, dim):
    from paper_2212_10961_gb300 import field as F
    p = F.FieldParams(family="exponential", sigma2=4.0, ell=(0.2, 0.2, 0.05)[:dim], dim=dim, n_modes=n, seed=5)
    md = F.gen_modes(p)
    nbytes = abi.lib().grf_table_bytes(n)
    buf = (ctypes.c_uint8 * nbytes)()
    m = F._modes_struct(n, dim, md)
    assert abi.lib().grf_pack_table(ctypes.byref(m), buf, nbytes) == 0
    t = _parse_table(bytes(buf), n, dim)
    assert t["magic"] == 0x54465247 and t["n"] == n and t["dim"] == dim
    assert t["n_pad"] % 128 == 0 and t["n_pad"] >= n and t["total"] == nbytes
    order = t["order"]
    assert sorted(order[:n].tolist()) == list(range(n)) and np.all(order[n:] == -1)
    a = md["a"][order[:n]]
    h = np.sum(np.abs(a), axis=1)
    assert np.all(np.diff(h) <= 0)  # sorted by |a|_1, descending
    np.testing.assert_array_equal(t["hot"][:n, :dim], (2 * math.pi * a).astype(np.float32))
    # odd sorted positions hold the equivalent form (-A, psi + 1/2)
    sgn = np.where(np.arange(n) % 2 == 1, -1.0, 1.0)
    np.testing.assert_array_equal(t["hot"][:n, 3], (sgn * md["amp"][order[:n]]).astype(np.float32))
    assert np.all(t["hot"][n:] == 0) and np.all(t["cold"][n:] == 0)
    c = t["cold"][:n].astype(np.float64)
    rec = np.stack([c[:, 0] + c[:, 1], c[:, 2] + c[:, 3], c[:, 4] + c[:, 5]], axis=1)[:, :dim]
    np.testing.assert_allclose(rec, a, rtol=2.0 ** -46, atol=0)
    psi = md["psi"][order[:n]]
    want = np.where(sgn < 0, np.where(psi <= 0.0, psi + 0.5, psi - 0.5), psi)
    np.testing.assert_allclose(c[:, 6] + c[:, 7], want, rtol=0, atol=1e-15)
    # the stored form is the same term: A cos(2 pi t) = -A cos(2 pi (t + 1/2))
    tt = np.random.default_rng(n).random(n)
    np.testing.assert_allclose(sgn * md["amp"][order[:n]] * np.cos(2 * math.pi * (tt + want)),
                               md["amp"][order[:n]] * np.cos(2 * math.pi * (tt + psi)), rtol=0, atol=1e-12)
    for b in range(160):
        Eb = 2.0 ** ((b - 100) / 4.0)
        assert t["kpref"][b] == int(np.sum(h * Eb > 1.0))
    # the standardised wave-vectors ride along in sorted order, for the adjoint
    assert t["has_kappa"] == 1 and t["off_kappa"] % 256 == 0 and t["off_kappa"] + t["n_pad"] * 24 <= nbytes
    np.testing.assert_array_equal(t["kappa"][:n, :dim], md["kappa"][order[:n]])
    assert np.all(t["kappa"][:n, dim:] == 0) and np.all(t["kappa"][n:] == 0)
    # the grid path's operand scale: the largest stored |A| (header bytes 80..84)
    amp_max = np.frombuffer(bytes(buf)[80:84], dtype=np.float32)[0]
    assert amp_max == np.max(np.abs(t["hot"][:n, 3]))
    # packed without kappa: the flag is 0 and the section stays zero
    m0 = F._modes_struct(n, dim, {k: md[k] for k in ("amp", "psi", "a")})
    assert abi.lib().grf_pack_table(ctypes.byref(m0), buf, nbytes) == 0
    t0 = _parse_table(bytes(buf), n, dim)
    assert t0["has_kappa"] == 0 and np.all(t0["kappa"] == 0)
    np.testing.assert_array_equal(t0["hot"], t["hot"])


@pytest.mark.parametrize("dim,rot,period", [(3, None, None), (3, "rotation", (1.0, 0.0, 2.0)),
                                            (2, "general", (0.0, 1.5)), (1, None, (2.0,))])
def test_reparam_modes_matches_oracle_and_gen_modes(abi, dim, rot, period):
    # Sec. 4.1: A = sigma rho, a = R^T kappa / (2 pi l), periodic axes rounded
    # (Appendix B); the same arithmetic as the second half of grf_gen_modes
    from paper_2212_10961_gb300 import field as F
    R = None
    if rot == "rotation":
        th = 0.7
        R = [[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]]
    elif rot == "general":
        R = [[1.2, 0.4], [-0.3, 0.9]]
    ell = (0.2, 0.1, 0.05)[:dim]
    p = F.FieldParams(family="matern", nu=1.5, sigma2=2.3, ell=ell, dim=dim, n_modes=600, seed=41, rot=R,
                      period=period or (0.0,) * 3)
    drawn = F.gen_modes(p)
    got = F.reparam_modes(p, drawn["kappa"], drawn["rho"])
    np.testing.assert_array_equal(got["amp"], drawn["amp"])
    np.testing.assert_array_equal(got["a"], drawn["a"])
    amp_o, a_o = omodes.reparam(drawn["kappa"], drawn["rho"], math.sqrt(2.3), ell, rot=R, period=period)
    np.testing.assert_allclose(got["amp"], amp_o, rtol=4e-16, atol=0)
    per = [c for c in range(dim) if period is not None and period[c] > 0]
    free = [c for c in range(dim) if c not in per]
    np.testing.assert_array_equal(got["a"][:, per], a_o[:, per])
    np.testing.assert_allclose(got["a"][:, free], a_o[:, free], rtol=4e-15, atol=1e-300)
    # arbitrary (not drawn) kappa and rho
    rng = np.random.default_rng(dim)
    k2, r2 = rng.standard_normal((600, dim)), rng.random(600)
    got2 = F.reparam_modes(p, k2, r2)
    amp2, a2 = omodes.reparam(k2, r2, math.sqrt(2.3), ell, rot=R, period=period)
    np.testing.assert_allclose(got2["amp"], amp2, rtol=4e-16, atol=0)
    # a = R^T u sums terms of either sign: rounding is relative to sum_k |R_kc u_k|
    mag = np.abs(k2 / (2 * math.pi * np.asarray(ell))) @ (np.abs(np.asarray(R)) if R is not None else np.eye(dim))
    assert np.all(np.abs(got2["a"][:, free] - a2[:, free]) <= 8 * 2.0 ** -52 * mag[:, free])
    np.testing.assert_array_equal(got2["a"][:, per], a2[:, per])


def test_reparam_modes_rejects(abi):
    from paper_2212_10961_gb300 import field as F
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=10, seed=1)
    k = np.zeros((10, 2))
    k[3, 1] = np.nan
    with pytest.raises(abi.GRFError):
        F.reparam_modes(p, k, np.ones(10))
    with pytest.raises(abi.GRFError):
        F.reparam_modes(p, np.zeros((10, 2)), np.full(10, np.inf))
    m, _ = _modes_for(abi, 9, 2)
    assert abi.lib().grf_reparam_modes(ctypes.byref(p.to_c()), ctypes.byref(m)) == abi.GRF_EINVAL
    m2, _ = _modes_for(abi, 10, 2)
    m2.rho = None
    assert abi.lib().grf_reparam_modes(ctypes.byref(p.to_c()), ctypes.byref(m2)) == abi.GRF_EINVAL


def test_pack_and_sizes_reject(abi):
    from paper_2212_10961_gb300 import field as F
    p = F.FieldParams(n_modes=10, dim=2, ell=(0.1, 0.1))
    md = F.gen_modes(p)
    m = F._modes_struct(10, 2, md)
    small = (ctypes.c_uint8 * 64)()
    assert abi.lib().grf_pack_table(ctypes.byref(m), small, 64) == abi.GRF_EWORKSPACE
    md["a"][3, 1] = float("inf")
    nb = abi.lib().grf_table_bytes(10)
    buf = (ctypes.c_uint8 * nb)()
    assert abi.lib().grf_pack_table(ctypes.byref(m), buf, nb) == abi.GRF_EINVAL
    assert abi.lib().grf_table_bytes(0) == 0
    assert abi.lib().grf_table_bytes(abi.GRF_MAX_MODES) > 48 * abi.GRF_MAX_MODES
    assert abi.lib().grf_table_bytes(abi.GRF_MAX_MODES + 1) == 0
    assert abi.lib().grf_plan_bytes(100, 0) == 0
    # plans index cells with int32: 2^31 - 1 cells at most
    assert abi.lib().grf_plan_bytes((1 << 31) - 1, 1) > 0
    assert abi.lib().grf_plan_bytes(1 << 31, 1) == 0
    assert abi.lib().grf_plan_bytes(1000, 1) > 1000 * 16
    assert abi.lib().grf_backward_workspace_bytes(1000, 0, 3) == 0
    assert abi.lib().grf_batch_workspace_bytes(0, 10) == 0


def test_injected_host_allocation_failure(abi):
    # host-side fault injection: the entry point reports GRF_ENOMEM instead of
    # letting the allocation failure escape, and the next call succeeds
    from paper_2212_10961_gb300 import field as F
    L = abi.lib()
    p = F.FieldParams(n_modes=300, dim=3, ell=(0.1, 0.2, 0.3), seed=11)
    md = F.gen_modes(p)
    m = F._modes_struct(300, 3, md)
    nb = L.grf_table_bytes(300)
    ref = (ctypes.c_uint8 * nb)()
    assert L.grf_pack_table(ctypes.byref(m), ref, nb) == 0
    buf = (ctypes.c_uint8 * nb)()
    assert L.grf_debug_inject_alloc_failures(1) == 0
    try:
        assert L.grf_pack_table(ctypes.byref(m), buf, nb) == abi.GRF_ENOMEM
        assert b"allocation" in L.grf_last_error()
        assert not any(bytes(buf))  # nothing written before the failure
        assert L.grf_pack_table(ctypes.byref(m), buf, nb) == 0  # the injection was used up
        assert bytes(buf) == bytes(ref)
    finally:
        L.grf_debug_inject_alloc_failures(0)
    assert L.grf_debug_inject_alloc_failures(-1) == abi.GRF_EINVAL


def test_null_and_unknown_handles_rejected(abi):
    L = abi.lib()
    p = _params(abi)
    mp = abi.grf_map()
    mp.bits = abi.GRF_MAP_Y
    out = abi.grf_outputs()
    out.Y = 4096
    fake_plan = ctypes.c_void_p(1 << 20)
    # unknown plan: rejected on the host before any device work
    assert L.grf_synth_field(ctypes.c_void_p(1 << 16), ctypes.byref(p), fake_plan, 0, ctypes.byref(mp),
                             ctypes.byref(out), None, 0, None) == abi.GRF_EINVAL
    mp.bits = abi.GRF_MAP_FACIES
    mp.n_thresholds = 2
    mp.thresholds[0], mp.thresholds[1] = 0.5, 0.1  # not ascending
    out.facies = 4096
    assert L.grf_map_property(ctypes.byref(mp), 0.0, 1.0, 10, ctypes.c_void_p(4096), ctypes.byref(out),
                              None) == abi.GRF_EINVAL
    assert L.grf_batch_launch(ctypes.c_void_p(1 << 12), None) == abi.GRF_EINVAL
    # grid path entry points: unknown plans are not grids, bad settings rejected
    assert L.grf_synth_grid_workspace_bytes(fake_plan, 0, 100) == 0
    assert L.grf_synth_grid_workspace_bytes(None, 0, 100) == 0
    v = ctypes.c_int32(7)
    assert L.grf_plan_grid_shape(fake_plan, ctypes.byref(v), ctypes.byref(v), ctypes.byref(v)) == abi.GRF_EINVAL
    assert L.grf_plan_grid_shape(None, None, None, None) == abi.GRF_EINVAL
    assert L.grf_debug_grid_path(1, 3) == abi.GRF_EINVAL
    assert L.grf_debug_grid_path(1, 4) == abi.GRF_OK
    assert L.grf_take_grid_tiles(None) == abi.GRF_EINVAL
    assert L.grf_backward_grid_workspace_bytes(fake_plan, 0, 100) == 0
    assert L.grf_backward_grid_workspace_bytes(None, 0, 100) == 0
    assert L.grf_take_grid_adjoint_units(None) == abi.GRF_EINVAL
    assert L.grf_debug_mma_f16(None, None, 1, None, None, None) == abi.GRF_EINVAL
    assert L.grf_debug_mma_f16(ctypes.c_void_p(4096), ctypes.c_void_p(4096), 0, ctypes.c_void_p(4096),
                               ctypes.c_void_p(4096), None) == abi.GRF_EINVAL
    offs = (ctypes.c_int64 * 2)(5, 10)
    assert L.grf_plan_cells(3, 1, offs, None, None, None, ctypes.c_void_p(1 << 12), 1 << 20,
                            None) == abi.GRF_EINVAL


def test_from_dictionary_maps_appendix_b_keys(abi):
    # the setRandomField dictionary keys of Appendix B map onto FieldParams and
    # MapSpec; the modes drawn equal those of the explicit parameters
    from paper_2212_10961_gb300 import field as F
    d = {"type": "truncated", "correlation": "matern", "Kmean": 0.3, "Ksigma": 2.0,
         "Lcorr": [0.2, 0.1, 0.05], "nu": 1.5, "rho": 7.0, "nfreq": 300, "disableY": True,
         "thresholds": [-0.5, 0.5], "values": [1.0, 10.0, 100.0], "periodic": [2.0, 0.0, 0.0]}
    cfg = F.from_dictionary(d, seed=42)
    p = cfg["params"]
    assert (p.family, p.mean, p.sigma2, p.dim, p.n_modes, p.seed, p.nu) == ("matern", 0.3, 2.0, 2, 300, 42, 1.5)
    assert tuple(p.ell) == (0.2, 0.05) and tuple(p.period) == (2.0, 0.0)
    assert cfg["maps"].thresholds == (-0.5, 0.5) and cfg["maps"].facies and cfg["maps"].values == (1.0, 10.0, 100.0)
    explicit = F.FieldParams(family="matern", sigma2=2.0, mean=0.3, ell=(0.2, 0.05), dim=2, n_modes=300, seed=42,
                             nu=1.5, period=(2.0, 0.0))
    a, b = F.gen_modes(p), F.gen_modes(explicit)
    for k in ("a", "amp", "psi"):
        np.testing.assert_array_equal(a[k], b[k])
    cfg2 = F.from_dictionary({"type": "bitruncated", "disableZ": True, "thresholds2": [0.1]})
    assert cfg2["type"] == "bitruncated" and cfg2["params"].dim == 2 and cfg2["thresholds2"] == (0.1,)
    with pytest.raises(ValueError):
        F.from_dictionary({"type": "other"})


@pytest.mark.parametrize("rot", [None, ((0.0, 1.0, 0.0), (-1.0, 0.0, 0.0), (0.0, 0.0, 1.0))])
def test_realisation_record_round_trip(abi, tmp_path, rot):
    # the saved record reproduces the parameters and the modes bit for bit, and
    # a record whose modes do not follow from its parameters is rejected
    from paper_2212_10961_gb300 import field as F
    p = F.FieldParams(family="exponential", sigma2=2.5, mean=-0.25, ell=(0.3, 0.2, 0.1), dim=3, n_modes=257,
                      seed=2 ** 40 + 3, stream=1, period=(2.0, 0.0, 0.0), rot=rot)
    path = tmp_path / "real.npz"
    F.save_realisation(path, p)
    q, modes = F.load_realisation(path)
    assert bytes(q.to_c()) == bytes(p.to_c())
    want = omodes.gen_modes(omodes.EXPONENTIAL, 2.5, (0.3, 0.2, 0.1), 3, 257, 2 ** 40 + 3, stream=1,
                            period=(2.0, 0.0, 0.0), rot=None if rot is None else np.array(rot))
    for k in ("kappa", "rho", "psi", "a", "amp"):
        np.testing.assert_allclose(modes[k], want[k], rtol=4e-15, atol=1e-300, err_msg=k)
    bad = dict(modes)
    bad["psi"] = modes["psi"].copy()
    bad["psi"][7] += 1e-12
    F.save_realisation(tmp_path / "bad.npz", p, bad)
    with pytest.raises(ValueError):
        F.load_realisation(tmp_path / "bad.npz")
    q2, m2 = F.load_realisation(tmp_path / "bad.npz", verify=False)
    assert m2["psi"][7] == bad["psi"][7]


def test_fma_pipe_cosine_polynomial_matches_its_fit():
    # The FP32 coefficients compiled into the kernels are the ones the committed
    # generator fits, and their FP32 Horner evaluation stays within the stated
    # 4.0e-7 of cos(2 pi f) on [-1/2, 1/2].
    import importlib.util
    import pathlib
    csrc = pathlib.Path(__file__).resolve().parents[1] / "paper_2212_10961_gb300" / "csrc"
    spec = importlib.util.spec_from_file_location("gen_cos_poly", csrc / "gen_cos_poly.py")
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    text = (csrc / "device_common.cuh").read_text()
    body = text[text.index("cos_turns_poly(float f)"):]
    body = body[:body.index("\n}")]
    lits = [float(v) for v in re.findall(r"[-+]?\d\.\d+e[-+]\d+(?=f)", body)]
    compiled = np.array(lits[::-1], dtype=np.float32)  # Horner lists the highest degree first
    assert np.array_equal(compiled, gen.fit().astype(np.float32))
    f = np.linspace(-0.5, 0.5, 400_001)
    err = np.max(np.abs(gen.horner_fp32(compiled, f).astype(np.float64) - np.cos(2 * np.pi * f)))
    assert err <= 4.0e-7, err


def test_missing_library_fails_loudly(tmp_path):
    # the product path has no CPU fallback: without the shared library the
    # binding raises instead of computing anything another way
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2212_10961_gb300 import _abi\n"
            "_abi.LIB_PATH = %r\n"
            "_abi._lib = None\n"
            "try:\n"
            "    _abi.lib()\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n") % (ROOT, str(tmp_path / "absent.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "raised" in r.stdout and "absent.so" in r.stdout


def test_prefetch_rejects_bad_arguments(abi):
    # argument checks come before any CUDA call, so they run without a GPU
    from paper_2212_10961_gb300 import field as F
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=100, seed=1)
    L = abi.lib()
    nb = L.grf_table_bytes(100)
    bufs = [(ctypes.c_uint8 * nb)() for _ in range(3)]
    slots = (ctypes.c_void_p * 3)(*[ctypes.addressof(b) for b in bufs])
    h = ctypes.c_void_p()
    pc = p.to_c()
    assert L.grf_prefetch_create(ctypes.byref(pc), 1, 2, slots, nb, ctypes.byref(h)) == abi.GRF_EINVAL
    assert L.grf_prefetch_create(ctypes.byref(pc), 65, 2, slots, nb, ctypes.byref(h)) == abi.GRF_EINVAL
    assert L.grf_prefetch_create(ctypes.byref(pc), 3, 0, slots, nb, ctypes.byref(h)) == abi.GRF_EINVAL
    assert L.grf_prefetch_create(ctypes.byref(pc), 3, 2, slots, nb - 1, ctypes.byref(h)) == abi.GRF_EWORKSPACE
    assert L.grf_prefetch_create(ctypes.byref(pc), 3, 2, None, nb, ctypes.byref(h)) == abi.GRF_EINVAL
    bad = _params(abi, sigma2=-1.0)
    assert L.grf_prefetch_create(ctypes.byref(bad), 3, 2, slots, nb, ctypes.byref(h)) == abi.GRF_EINVAL
    assert L.grf_prefetch_next(None, None, 0, None, None) == abi.GRF_EINVAL
    assert L.grf_prefetch_destroy(None) == abi.GRF_OK

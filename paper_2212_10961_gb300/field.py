"""Python API over the C ABI: mode drawing, device tables, cell plans,
synthesis with fused maps, the adjoint, autograd wrappers and batches.

PyTorch provides device memory, pinned host buffers and streams; all
arithmetic of the method runs in libgrf.so (host C++ for the O(N) mode
drawing and table packing, CUDA kernels for everything per cell).

Method: Icardi et al., arXiv 2212.10961 -- Sec. 4.1 Eq. (DiscreteFT) (direct
spectral sum at arbitrary cell centres), Appendix A (covariances and
spectra), Sec. 3.1 / Appendix B (thresholds, facies values, lognormal
scaling).
"""
import ctypes
import dataclasses
import json
import math
import os
from dataclasses import dataclass, field as dc_field
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import check, lib

FAMILIES = {"gaussian": _abi.GRF_GAUSSIAN, "exponential": _abi.GRF_EXPONENTIAL,
            "matern": _abi.GRF_MATERN}


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _require_cuda(t, dtype, name):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


@dataclass
class FieldParams:
    """Parameters of one Gaussian random field (Appendix B dictionary keys:
    correlation, Kmean, Ksigma, Lcorr, nu, nfreq, disableY/disableZ)."""
    family: str = "gaussian"
    sigma2: float = 1.0
    mean: float = 0.0
    ell: Sequence[float] = (1.0, 1.0, 1.0)
    dim: int = 3
    n_modes: int = 1000
    seed: int = 1
    nu: float = 1.5
    stream: int = 0
    period: Sequence[float] = (0.0, 0.0, 0.0)  # Appendix B `periodic`: L_c > 0 per axis
    # axis transform R of the anisotropy: a rotation (rows = principal axes) or any
    # invertible matrix; C(r) = sigma^2 rho(|diag(1/l) R r|)
    rot: Optional[Sequence[Sequence[float]]] = None

    @property
    def sigma(self):
        return math.sqrt(self.sigma2)

    def to_c(self):
        p = _abi.grf_params()
        fam = self.family if isinstance(self.family, int) else FAMILIES[self.family.lower()]
        p.family = fam
        p.dim = int(self.dim)
        p.nu = float(self.nu)
        p.sigma2 = float(self.sigma2)
        p.mean = float(self.mean)
        ell = list(self.ell) + [1.0] * (3 - len(self.ell))
        for c in range(3):
            p.ell[c] = float(ell[c])
        p.n_modes = int(self.n_modes)
        p.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        p.stream = int(self.stream)
        p.reserved = 0
        per = list(self.period) + [0.0] * (3 - len(self.period))
        for c in range(3):
            p.period[c] = float(per[c])
        if self.rot is not None:
            R = np.asarray(self.rot, dtype=np.float64)
            for i in range(R.shape[0]):
                for k in range(R.shape[1]):
                    p.rot[i * 3 + k] = float(R[i, k])
        return p


def from_dictionary(d, seed=1):
    """Configuration from the keys of the paper's setRandomField dictionary
    (Appendix B): returns {"type", "params", "maps", "thresholds2"}.

    type         "truncated" (one field) or "bitruncated" (two fields on
                 generator streams 0 and 1, the second thresholded by
                 thresholds2; see PluriGaussianField)
    correlation  "gaussian", "exponential" or "matern"
    Kmean, Ksigma  mean and variance of the Gaussian field Y
    Lcorr        correlation lengths (x, y, z)
    nu           Matern smoothness (the paper's rho is not used)
    nfreq        number of modes N
    disableY, disableZ  drop an axis: the field's dimension is 3 minus the
                 disabled axes, and the coordinates passed are the enabled
                 ones in (x, y, z) order
    periodic     per-axis domain lengths (0 = not periodic)
    values, thresholds  facies values and thresholds (Y units)
    The seed is not a dictionary key of the paper; it is the second argument.
    """
    keep = [True, not d.get("disableY", False), not d.get("disableZ", False)]
    axes = [c for c in range(3) if keep[c]]
    lcorr = list(d.get("Lcorr", (1.0, 1.0, 1.0)))
    lcorr += [lcorr[-1]] * (3 - len(lcorr))
    per = list(d.get("periodic", (0.0, 0.0, 0.0)) or (0.0, 0.0, 0.0))
    per += [0.0] * (3 - len(per))
    params = FieldParams(family=str(d.get("correlation", "gaussian")).lower(), sigma2=float(d.get("Ksigma", 1.0)),
                         mean=float(d.get("Kmean", 0.0)), ell=tuple(float(lcorr[c]) for c in axes),
                         dim=len(axes), n_modes=int(d.get("nfreq", 1000)), seed=int(seed),
                         nu=float(d.get("nu", 1.5)), period=tuple(float(per[c]) for c in axes))
    thr = tuple(float(t) for t in d.get("thresholds", ()))
    vals = d.get("values")
    kind = str(d.get("type", "truncated")).lower()
    if kind not in ("truncated", "bitruncated"):
        raise ValueError("type must be truncated or bitruncated")
    maps = MapSpec(y=True, lognormal=False, thresholds=thr, facies=len(thr) > 0,
                   values=tuple(float(v) for v in vals) if (vals is not None and kind == "truncated") else None)
    return {"type": kind, "params": params, "maps": maps,
            "thresholds2": tuple(float(t) for t in d.get("thresholds2", ()))}


def _modes_struct(n, dim, arrays):
    """grf_modes over the float64 numpy arrays present in `arrays` (NULL for
    a missing key); the arrays must outlive the struct's use."""
    m = _abi.grf_modes()
    m.n = n
    m.dim = dim
    for k in ("kappa", "rho", "psi", "a", "amp"):
        if arrays.get(k) is not None:
            setattr(m, k, arrays[k].ctypes.data_as(_abi.c_dp))
    return m


def _host64(v, shape=None):
    """Contiguous float64 numpy copy on the host of a tensor, array or list."""
    if isinstance(v, torch.Tensor):
        v = v.detach().to(device="cpu", dtype=torch.float64)
        out = v.contiguous().numpy()
    else:
        out = np.ascontiguousarray(v, dtype=np.float64)
    return out.reshape(shape) if shape is not None else out


def gen_modes(params: FieldParams):
    """Draw the N modes (host FP64): dict with kappa (N, d), rho, psi, a (N, d), amp."""
    n, d = int(params.n_modes), int(params.dim)
    arrays = {"kappa": np.empty((n, d)), "rho": np.empty(n), "psi": np.empty(n),
              "a": np.empty((n, d)), "amp": np.empty(n)}
    m = _modes_struct(n, d, arrays)
    check(lib().grf_gen_modes(ctypes.byref(params.to_c()), ctypes.byref(m)))
    return arrays


def reparam_modes(params: FieldParams, kappa, rho):
    """Amplitudes and frequencies of given standardised modes (Sec. 4.1,
    grf_reparam_modes): A = sigma rho and a = R^T kappa / (2 pi l) with the
    periodic axes of `params` rounded.  kappa (N, d), rho (N,): arrays or
    tensors.  Returns a dict with kappa, rho, a (N, d), amp (host FP64)."""
    n, d = int(params.n_modes), int(params.dim)
    arrays = {"kappa": _host64(kappa, (n, d)), "rho": _host64(rho, (n,)), "a": np.empty((n, d)),
              "amp": np.empty(n)}
    m = _modes_struct(n, d, arrays)
    check(lib().grf_reparam_modes(ctypes.byref(params.to_c()), ctypes.byref(m)))
    return arrays


_MODE_KEYS = ("kappa", "rho", "psi", "a", "amp")


def save_realisation(path, params: FieldParams, modes=None):
    """Record of one realisation for audit or restart, as one numpy .npz file:
    the parameters (with the seed they determine the field exactly, at any
    cell centres: Sec. 4.1) and the drawn modes (drawn here if not given)."""
    modes = gen_modes(params) if modes is None else modes
    rec = dataclasses.asdict(params)
    rec["ell"], rec["period"] = list(rec["ell"]), list(rec["period"])
    if rec["rot"] is not None:
        rec["rot"] = np.asarray(rec["rot"], dtype=np.float64).tolist()
    np.savez(path, params=np.array(json.dumps(rec)), **{k: np.asarray(modes[k]) for k in _MODE_KEYS})


def load_realisation(path, verify=True):
    """(params, modes) from a save_realisation file.  verify=True draws the
    modes again from the stored parameters and requires them to be
    bit-identical to the stored ones (the record is then self-consistent)."""
    with np.load(path, allow_pickle=False) as z:
        rec = json.loads(str(z["params"]))
        modes = {k: z[k].copy() for k in _MODE_KEYS}
    rec["ell"], rec["period"] = tuple(rec["ell"]), tuple(rec["period"])
    if rec["rot"] is not None:
        rec["rot"] = tuple(tuple(r) for r in rec["rot"])
    params = FieldParams(**rec)
    if verify:
        again = gen_modes(params)
        for k in _MODE_KEYS:
            if not np.array_equal(again[k], modes[k]):
                raise ValueError("stored %s differs from the modes its parameters draw" % k)
    return params, modes


class ModeTable:
    """Device mode table: packed on the host, copied to the device.

    kappa (optional, (N, d)) is stored with the table for the adjoint's chain
    rule to kappa, l and R (grf_synth_backward)."""

    def __init__(self, amp, psi, a, device=None, stream=None, kappa=None):
        amp = _host64(amp)
        a = _host64(a, (len(amp), -1))
        self.n_modes, self.dim = a.shape
        self.nbytes = int(lib().grf_table_bytes(self.n_modes))
        if self.nbytes == 0:
            raise ValueError("n_modes out of range")
        self.host = torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=True)
        self._pack(amp, psi, a, kappa)
        device = device or torch.device("cuda", torch.cuda.current_device())
        self.dev = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self._uploaded = torch.cuda.Event()
        self.upload(stream)

    def _pack(self, amp, psi, a, kappa):
        arrays = {"amp": amp, "psi": _host64(psi), "a": a,
                  "kappa": None if kappa is None else _host64(kappa, a.shape)}
        m = _modes_struct(self.n_modes, self.dim, arrays)
        check(lib().grf_pack_table(ctypes.byref(m), _ptr(self.host), self.nbytes))

    def upload(self, stream=None):
        check(lib().grf_upload_table(_ptr(self.host), _ptr(self.dev), self.nbytes, _stream_handle(stream)))
        self._uploaded.record(stream if stream is not None else torch.cuda.current_stream())

    def update(self, amp, psi, a, stream=None, kappa=None):
        """Repack new modes (same N and dim) into this table and upload them.
        Waits for the previous upload from the pinned staging buffer first."""
        amp = _host64(amp)
        a = _host64(a, (len(amp), -1))
        if a.shape != (self.n_modes, self.dim):
            raise ValueError("update needs the same number of modes and dimension")
        self._uploaded.synchronize()
        self._pack(amp, psi, a, kappa)
        self.upload(stream)

    @classmethod
    def from_modes(cls, modes, **kw):
        return cls(modes["amp"], modes["psi"], modes["a"], kappa=modes.get("kappa"), **kw)

    @classmethod
    def device_only(cls, n_modes, dim, device=None):
        """A device table with no host copy, filled by ModePrefetcher.next."""
        t = cls.__new__(cls)
        t.n_modes, t.dim = int(n_modes), int(dim)
        t.nbytes = int(lib().grf_table_bytes(t.n_modes))
        if t.nbytes == 0:
            raise ValueError("n_modes out of range")
        t.host = None
        t.dev = torch.empty(t.nbytes, dtype=torch.uint8,
                            device=device or torch.device("cuda", torch.cuda.current_device()))
        t._uploaded = torch.cuda.Event()
        return t

    @property
    def ptr(self):
        return _ptr(self.dev)


class ModePrefetcher:
    """Realisations k = 0, 1, 2, ... of one parameter set (seed params.seed + k)
    drawn and packed ahead of use by native worker threads into a ring of
    pinned staging buffers (grf_prefetch_*); next() only enqueues the upload
    of the next one into a device table.  For Monte-Carlo loops over many
    realisations of small fields, where drawing on the launching thread would
    leave the GPU idle.  Each realisation is drawn by one worker thread, so
    `depth` should exceed the worker count plus the slots whose uploads are in
    flight (two for a two-table ring) for the workers to run in parallel."""

    def __init__(self, params: FieldParams, depth=4, threads=None):
        self.params = params
        self.nbytes = int(lib().grf_table_bytes(int(params.n_modes)))
        threads = int(threads or max(1, min(8, (os.cpu_count() or 2) // 2)))
        self.host = [torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=True) for _ in range(depth)]
        slots = (ctypes.c_void_p * depth)(*[h.data_ptr() for h in self.host])
        h = ctypes.c_void_p()
        check(lib().grf_prefetch_create(ctypes.byref(params.to_c()), int(depth), threads, slots, self.nbytes,
                                        ctypes.byref(h)))
        self._h = h

    def next(self, table: ModeTable, stream=None):
        """Upload the next realisation into `table` (ModeTable.device_only of
        the same N and dim) on `stream`; returns its seed."""
        seed = ctypes.c_uint64(0)
        check(lib().grf_prefetch_next(self._h, table.ptr, table.nbytes, _stream_handle(stream),
                                      ctypes.byref(seed)))
        return seed.value

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._h = None
            check(lib().grf_prefetch_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:  # interpreter shutdown
            pass


class CellPlan:
    """Spatially sorted copy of one or more sets of cell centres (segments).

    x, y, z: CUDA float32 tensors (SoA); segments: cell counts per segment
    (default: one segment).  The plan is built on the device once and reused
    for every realisation on those cells.
    """

    def __init__(self, x, y=None, z=None, dim=None, segments=None, stream=None):
        x = _require_cuda(x, torch.float32, "x")
        y = _require_cuda(y, torch.float32, "y")
        z = _require_cuda(z, torch.float32, "z")
        self.dim = dim or (1 + (y is not None) + (z is not None))
        self.n_cells = x.numel()
        sizes = [self.n_cells] if segments is None else [int(s) for s in segments]
        if sum(sizes) != self.n_cells:
            raise ValueError("segment sizes do not add up to the number of cells")
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n_segments = len(sizes)
        self.nbytes = int(lib().grf_plan_bytes(self.n_cells, self.n_segments))
        self.buf = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=x.device)
        self._inputs = (x, y, z)  # kept alive until the planning kernels have run
        check(lib().grf_plan_cells(self.dim, self.n_segments,
                                   self.offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   _ptr(x), _ptr(y), _ptr(z), _ptr(self.buf), self.nbytes,
                                   _stream_handle(stream)))

    def __del__(self):
        # the library forgets this buffer before torch can hand its memory to another tensor
        buf = getattr(self, "buf", None)
        if buf is not None:
            try:
                lib().grf_release(_ptr(buf))
            except Exception:  # interpreter shutdown
                pass

    def segment_size(self, s):
        """Cells in segment s (0 for an out-of-range index; the C ABI rejects it)."""
        if not 0 <= s < self.n_segments:
            return 0
        return int(self.offsets[s + 1] - self.offsets[s])

    def status(self, stream=None):
        v = ctypes.c_int32(0)
        check(lib().grf_read_status(_ptr(self.buf), ctypes.byref(v), _stream_handle(stream)))
        return v.value

    def grid_shape(self):
        """(nx, ny, nz) when the cells are a Cartesian grid handed over
        x-fastest (grf_plan_grid_shape), else (0, 0, 0)."""
        v = [ctypes.c_int32(0) for _ in range(3)]
        check(lib().grf_plan_grid_shape(_ptr(self.buf), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    @property
    def ptr(self):
        return _ptr(self.buf)


@dataclass
class MapSpec:
    """Which outputs to write (Sec. 3.1, Sec. 4.1, Appendix B)."""
    y: bool = True
    lognormal: bool = False
    k_ref: float = 1.0
    thresholds: Sequence[float] = ()
    facies: bool = False
    values: Optional[Sequence[float]] = None
    porosity: Optional[Sequence[float]] = None  # (phi0, phi1, phi_min, phi_max)

    def to_c(self):
        m = _abi.grf_map()
        bits = 0
        if self.y:
            bits |= _abi.GRF_MAP_Y
        if self.lognormal:
            bits |= _abi.GRF_MAP_LOGNORMAL
        if self.facies:
            bits |= _abi.GRF_MAP_FACIES
        if self.values is not None:
            bits |= _abi.GRF_MAP_VALUES
        if self.porosity is not None:
            bits |= _abi.GRF_MAP_POROSITY
        m.bits = bits
        thr = list(self.thresholds)
        m.n_thresholds = len(thr)
        if len(thr) > _abi.GRF_MAX_THRESHOLDS:
            raise ValueError("at most %d thresholds" % _abi.GRF_MAX_THRESHOLDS)
        for i, t in enumerate(thr):
            m.thresholds[i] = float(t)
        if self.values is not None:
            if len(self.values) != len(thr) + 1:
                raise ValueError("values needs one entry per facies (len(thresholds) + 1)")
            for i, v in enumerate(self.values):
                m.values[i] = float(v)
        m.k_ref = float(self.k_ref)
        if self.porosity is not None:
            m.phi0, m.phi1, m.phi_min, m.phi_max = [float(v) for v in self.porosity]
        return m

    def allocate(self, n, device):
        out = {}
        if self.y:
            out["Y"] = torch.empty(n, dtype=torch.float32, device=device)
        if self.lognormal:
            out["K"] = torch.empty(n, dtype=torch.float32, device=device)
        if self.facies:
            out["facies"] = torch.empty(n, dtype=torch.uint8, device=device)
        if self.values is not None or self.porosity is not None:
            out["prop"] = torch.empty(n, dtype=torch.float32, device=device)
        return out


def _outputs_struct(out):
    o = _abi.grf_outputs()
    o.Y = out["Y"].data_ptr() if "Y" in out else None
    o.K = out["K"].data_ptr() if "K" in out else None
    o.facies = out["facies"].data_ptr() if "facies" in out else None
    o.prop = out["prop"].data_ptr() if "prop" in out else None
    return o


def synth_workspace_bytes(plan: CellPlan, segment, n_modes):
    """Workspace that lets grf_synth_field use the mode split and, on a
    Cartesian-grid plan, the tensor-core grid path (the larger of
    grf_synth_workspace_bytes and grf_synth_grid_workspace_bytes)."""
    return max(int(lib().grf_synth_workspace_bytes(plan.segment_size(segment))),
               int(lib().grf_synth_grid_workspace_bytes(plan.ptr, int(segment), int(n_modes))))


def synth_mismatch_workspace_bytes(plan: CellPlan, segment, n_modes):
    """Workspace of grf_synth_mismatch: the loss partials, then room for the
    mode split or, on a Cartesian-grid plan, the grid path's tables."""
    n = plan.segment_size(segment)
    lbytes = int(lib().grf_synth_mismatch_workspace_bytes(n)) - int(lib().grf_synth_workspace_bytes(n))
    return lbytes + synth_workspace_bytes(plan, segment, n_modes)


def synth(table: ModeTable, params: FieldParams, plan: CellPlan, segment=0, maps=None, out=None,
          stream=None, workspace=None):
    """Field and fused maps at every cell of `segment` (original cell order).

    workspace: a Workspace for the mode split of small segments (default: a
    module-level one; pass workspace=False for none)."""
    maps = maps or MapSpec()
    n = plan.segment_size(segment)
    if out is None:
        out = maps.allocate(n, plan.buf.device)
    if workspace is False:
        ws, nbytes = None, 0
    else:
        nbytes = synth_workspace_bytes(plan, segment, params.n_modes)
        ws = (workspace or _ws_fwd).get(nbytes, plan.buf.device)
    check(lib().grf_synth_field(table.ptr, ctypes.byref(params.to_c()), plan.ptr, int(segment),
                                ctypes.byref(maps.to_c()), ctypes.byref(_outputs_struct(out)),
                                _ptr(ws), nbytes, _stream_handle(stream)))
    return out


class PreparedSynth:
    """grf_synth_field with its argument structs, outputs and workspace built
    once, for many realisations on the same cells (only the table changes
    from call to call); returns the outputs dict, overwritten by each call."""

    def __init__(self, params: FieldParams, plan: CellPlan, segment=0, maps=None, out=None, stream=None):
        maps = maps or MapSpec()
        n = plan.segment_size(segment)
        self.out = out if out is not None else maps.allocate(n, plan.buf.device)
        self.plan = plan
        self._p = params.to_c()
        self._m = maps.to_c()
        self._o = _outputs_struct(self.out)
        self._nbytes = synth_workspace_bytes(plan, segment, params.n_modes)
        self._ws = torch.empty(max(self._nbytes, 256), dtype=torch.uint8, device=plan.buf.device)
        self._stream = None if stream is None else _stream_handle(stream)
        self._args = (ctypes.byref(self._p), plan.ptr, int(segment), ctypes.byref(self._m), ctypes.byref(self._o),
                      _ptr(self._ws), self._nbytes)

    def __call__(self, table: ModeTable, stream=None):
        st = _stream_handle(stream) if stream is not None else (self._stream or _stream_handle(None))
        check(lib().grf_synth_field(table.ptr, *self._args, st))
        return self.out


def map_property(Y, maps: MapSpec, mean, sigma, out=None, stream=None):
    """Standalone property map of an existing field Y (CUDA float32)."""
    Y = _require_cuda(Y, torch.float32, "Y")
    if out is None:
        m2 = MapSpec(**{**maps.__dict__, "y": False})
        out = m2.allocate(Y.numel(), Y.device)
    m = maps.to_c()
    m.bits &= ~_abi.GRF_MAP_Y
    check(lib().grf_map_property(ctypes.byref(m), float(mean), float(sigma), Y.numel(), _ptr(Y),
                                 ctypes.byref(_outputs_struct(out)), _stream_handle(stream)))
    return out


def map_bitruncated(Y1, Y2, t, s, rule, values=None, stream=None):
    """Bitruncated (pluri-Gaussian) facies of two fields (Sec. 3.1):
    facies = rule[#{Y1 > t}][#{Y2 > s}], and prop = values[facies] if given.
    Returns (facies uint8, prop float32 or None) on the fields' device."""
    Y1 = _require_cuda(Y1, torch.float32, "Y1")
    Y2 = _require_cuda(Y2, torch.float32, "Y2")
    if Y1.numel() != Y2.numel():
        raise ValueError("Y1 and Y2 differ in size")
    m = _abi.grf_bimap()
    t, s = list(t), list(s)
    if len(t) > _abi.GRF_MAX_THRESHOLDS or len(s) > _abi.GRF_MAX_THRESHOLDS:
        raise ValueError("at most %d thresholds per field" % _abi.GRF_MAX_THRESHOLDS)
    m.n_t, m.n_s = len(t), len(s)
    for i, v in enumerate(t):
        m.t[i] = float(v)
    for i, v in enumerate(s):
        m.s[i] = float(v)
    rule = np.asarray(rule, dtype=np.int64)
    if rule.shape != (len(t) + 1, len(s) + 1) or rule.min() < 0 or rule.max() > 255:
        raise ValueError("rule must be (len(t)+1) x (len(s)+1) facies indices in 0..255")
    for i in range(rule.shape[0]):
        for j in range(rule.shape[1]):
            m.rule[i][j] = int(rule[i, j])
    if values is not None:
        for i, v in enumerate(values):
            m.values[i] = float(v)
    fac = torch.empty(Y1.numel(), dtype=torch.uint8, device=Y1.device)
    prop = torch.empty(Y1.numel(), dtype=torch.float32, device=Y1.device) if values is not None else None
    check(lib().grf_map_bitruncated(ctypes.byref(m), Y1.numel(), _ptr(Y1), _ptr(Y2), _ptr(fac), _ptr(prop),
                                    _stream_handle(stream)))
    return fac, prop


class PluriGaussianField:
    """Two independent fields with the same seed on generator streams 0 and 1
    (Appendix B `bitruncated`), each with its own covariance parameters."""

    def __init__(self, params1: FieldParams, params2: FieldParams):
        if params1.seed != params2.seed:
            raise ValueError("both fields use one seed; their independence comes from the stream tag")
        p1 = FieldParams(**{**params1.__dict__, "stream": 0})
        p2 = FieldParams(**{**params2.__dict__, "stream": 1})
        self.f1, self.f2 = GaussianField(p1), GaussianField(p2)

    def synth(self, plan: CellPlan, t, s, rule, values=None, segment=0, stream=None):
        y1 = self.f1.synth(plan, MapSpec(y=True), segment, stream=stream)["Y"]
        y2 = self.f2.synth(plan, MapSpec(y=True), segment, stream=stream)["Y"]
        fac, prop = map_bitruncated(y1, y2, t, s, rule, values, stream)
        return {"Y1": y1, "Y2": y2, "facies": fac, "prop": prop}


class Workspace:
    """Grow-only device scratch buffer (256-byte aligned torch allocation)."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes, device):
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        return self.buf


_ws_bwd = Workspace()
_ws_loss = Workspace()
_ws_fwd = Workspace()


def backward_workspace_bytes(plan: CellPlan, segment, n_modes, dim):
    """Workspace bytes of grf_synth_backward on this plan: enough for the
    CUDA-core adjoint and, on a grid plan, for the tensor-core one
    (grf_backward_workspace_bytes and grf_backward_grid_workspace_bytes)."""
    return max(int(lib().grf_backward_workspace_bytes(plan.segment_size(segment), int(n_modes), int(dim))),
               int(lib().grf_backward_grid_workspace_bytes(plan.ptr, int(segment), int(n_modes))))


def backward(table: ModeTable, params: FieldParams, plan: CellPlan, gY, segment=0, stream=None,
             workspace=None, gscale=None):
    """Gradients (device FP64) of a loss with dL/dY = gY (CUDA float32,
    original cell order): dA, dpsi, da (N, d) in the original mode order,
    dmu, dsigma, dsigma2, dell (d), drot (d, d; meaningful with a transform),
    drho (N) and dkappa (N, d).  gscale: optional CUDA float64 scalar that
    multiplies every gradient (an upstream factor read on the device)."""
    gY = _require_cuda(gY, torch.float32, "gY")
    dev = gY.device
    n, d = table.n_modes, table.dim
    g = {"dA": torch.empty(n, dtype=torch.float64, device=dev),
         "dpsi": torch.empty(n, dtype=torch.float64, device=dev),
         "da": torch.empty((n, d), dtype=torch.float64, device=dev),
         "dmu": torch.empty(1, dtype=torch.float64, device=dev),
         "dsigma": torch.empty(1, dtype=torch.float64, device=dev),
         "dell": torch.empty(d, dtype=torch.float64, device=dev),
         "drot": torch.empty((d, d), dtype=torch.float64, device=dev),
         "dsigma2": torch.empty(1, dtype=torch.float64, device=dev),
         "drho": torch.empty(n, dtype=torch.float64, device=dev),
         "dkappa": torch.empty((n, d), dtype=torch.float64, device=dev)}
    gs = _abi.grf_grads()
    for k in g:
        setattr(gs, k, g[k].data_ptr())
    if gscale is not None:
        gs.gscale = _require_cuda(gscale, torch.float64, "gscale").data_ptr()
    nbytes = backward_workspace_bytes(plan, segment, n, d)
    ws = (workspace or _ws_bwd).get(nbytes, dev)
    check(lib().grf_synth_backward(table.ptr, ctypes.byref(params.to_c()), plan.ptr, int(segment),
                                   _ptr(gY), ctypes.byref(gs), _ptr(ws), ws.numel(),
                                   _stream_handle(stream)))
    return g


def mismatch_grad(K, K_target, stream=None, workspace=None):
    """L = mean (K - T)^2 and gY = dL/dY for K = exp(Y): returns (loss (1,) FP64, gY)."""
    K = _require_cuda(K, torch.float32, "K")
    T = _require_cuda(K_target, torch.float32, "K_target")
    n = K.numel()
    gY = torch.empty_like(K)
    loss = torch.empty(1, dtype=torch.float64, device=K.device)
    ws = (workspace or _ws_loss).get(lib().grf_mismatch_workspace_bytes(n), K.device)
    check(lib().grf_mismatch_grad(n, _ptr(K), _ptr(T), _ptr(gY), _ptr(loss), _ptr(ws), ws.numel(),
                                  _stream_handle(stream)))
    return loss, gY


_ws_mm = Workspace()


def synth_mismatch(table: ModeTable, params: FieldParams, plan: CellPlan, K_target, segment=0, n_mean=0,
                   want_Y=False, want_K=False, stream=None, workspace=None):
    """Forward half of a calibration step in one kernel (grf_synth_mismatch):
    the field, K = exp(Y), L = sum (K - T)^2 / n_mean and gY = dL/dY.
    n_mean: cells of the mean (0: this segment's count; the total over all
    shards for a sharded field).  Returns (loss (1,) FP64, gY, outputs) with
    outputs holding "Y" and/or "K" when asked for (original cell order)."""
    n = plan.segment_size(segment)
    dev = plan.buf.device
    T = _require_cuda(K_target, torch.float32, "K_target")
    if T.numel() != n:
        raise ValueError("K_target has %d values for %d cells" % (T.numel(), n))
    gY = torch.empty(n, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    out = {}
    if want_Y:
        out["Y"] = torch.empty(n, dtype=torch.float32, device=dev)
    if want_K:
        out["K"] = torch.empty(n, dtype=torch.float32, device=dev)
    nbytes = synth_mismatch_workspace_bytes(plan, segment, params.n_modes)
    ws = (workspace or _ws_mm).get(nbytes, dev)
    check(lib().grf_synth_mismatch(table.ptr, ctypes.byref(params.to_c()), plan.ptr, int(segment), _ptr(T),
                                   int(n_mean), _ptr(gY), _ptr(loss), _ptr(out.get("Y")), _ptr(out.get("K")),
                                   _ptr(ws), ws.numel(), _stream_handle(stream)))
    return loss, gY, out


# ---------------------------------------------------------------------------
# Autograd
# ---------------------------------------------------------------------------
class _SpectralFieldFn(torch.autograd.Function):
    """Differentiable field of the reparameterised modes.  Marshalling only:
    the library forms A = sigma rho and a = R^T kappa / (2 pi l) with the
    periodic rounding (grf_reparam_modes), synthesises Y and, in backward,
    returns every gradient of the parameters themselves (grf_synth_backward:
    dmu, dsigma2, dell, drho, dpsi, dkappa, drot)."""

    @staticmethod
    def forward(ctx, mu, sigma2, ell, rho, psi, kappa, rot, plan, segment, period):
        params, table = _reparam_table(mu, sigma2, ell, rho, psi, kappa, rot, period, plan.buf.device)
        y = synth(table, params, plan, segment, MapSpec(y=True))["Y"]
        ctx.table, ctx.params, ctx.plan, ctx.segment = table, params, plan, segment
        ctx.meta = [(t.shape, t.device, t.dtype) if t is not None else None
                    for t in (mu, sigma2, ell, rho, psi, kappa, rot)]
        return y

    @staticmethod
    def backward(ctx, gY):
        g = backward(ctx.table, ctx.params, ctx.plan, gY.contiguous().float(), ctx.segment)
        out = tuple(None if m is None else g[k].reshape(m[0]).to(device=m[1], dtype=m[2])
                    for k, m in zip(_REPARAM_GRADS, ctx.meta))
        return out + (None, None, None)


def spectral_field(mu, sigma2, ell, rho, psi, kappa, plan: CellPlan, segment=0, rot=None, period=None):
    """Differentiable Y(x) = mu + sum_j sqrt(sigma2) rho_j cos(2 pi (a_j . x + psi_j)),
    a_j = R^T kappa_j / (2 pi l) with periodic axes rounded (Sec. 4.1,
    Appendix B `periodic`; grf_reparam_modes).

    mu, sigma2: scalar tensors; ell (d,); rho, psi (N,); kappa (N, d); rot:
    optional (d, d) axis transform; period: optional per-axis lengths (not
    differentiable).  Gradients flow to all tensors through the CUDA adjoint.
    Parameters on the CPU keep the forward free of device-to-host copies."""
    return _SpectralFieldFn.apply(mu, sigma2, ell, rho, psi, kappa, rot, plan, segment, period)


def _reparam_table(mu, sigma2, ell, rho, psi, kappa, rot, period, device):
    """FieldParams and device table of the reparameterised modes (marshalling
    of the parameters; the reparameterisation runs in grf_reparam_modes)."""
    n, d = kappa.shape
    rot_h = None if rot is None else _host64(rot, (d, d)).tolist()
    params = FieldParams(sigma2=float(sigma2), mean=float(mu), ell=tuple(_host64(ell, (d,)).tolist()), dim=d,
                         n_modes=n, period=tuple(period) if period is not None else (0.0,) * 3, rot=rot_h)
    modes = reparam_modes(params, kappa, rho)
    return params, ModeTable(modes["amp"], psi, modes["a"], kappa=modes["kappa"], device=device)


_REPARAM_GRADS = ("dmu", "dsigma2", "dell", "drho", "dpsi", "dkappa", "drot")


class _SpectralMismatchFn(torch.autograd.Function):
    """Calibration objective L = mean (exp(Y) - T)^2 of the reparameterised
    field, as one differentiable scalar: the forward is grf_synth_mismatch
    (field, K, loss and dL/dY in one kernel), the backward grf_synth_backward
    with the upstream gradient passed to the library as its device scale."""

    @staticmethod
    def forward(ctx, mu, sigma2, ell, rho, psi, kappa, rot, plan, K_target, segment, period, n_mean):
        params, table = _reparam_table(mu, sigma2, ell, rho, psi, kappa, rot, period, plan.buf.device)
        loss, gY, _ = synth_mismatch(table, params, plan, K_target, segment, n_mean)
        ctx.table, ctx.params, ctx.plan, ctx.segment, ctx.gY = table, params, plan, segment, gY
        ctx.meta = [(t.shape, t.device, t.dtype) if t is not None else None
                    for t in (mu, sigma2, ell, rho, psi, kappa, rot)]
        return loss.reshape(())

    @staticmethod
    def backward(ctx, gL):
        gs = gL.detach().to(device=ctx.gY.device, dtype=torch.float64).contiguous()
        g = backward(ctx.table, ctx.params, ctx.plan, ctx.gY, ctx.segment, gscale=gs)
        out = tuple(None if m is None else g[k].reshape(m[0]).to(device=m[1], dtype=m[2])
                    for k, m in zip(_REPARAM_GRADS, ctx.meta))
        return out + (None,) * 5


def spectral_mismatch(mu, sigma2, ell, rho, psi, kappa, plan: CellPlan, K_target, segment=0, rot=None, period=None,
                      n_mean=0):
    """Differentiable calibration loss L = sum_i (exp(Y_i) - T_i)^2 / n_mean of
    the field of spectral_field (same parameters), K_target = T (CUDA float32,
    original cell order).  n_mean: 0 for the plain mean over the segment.
    Returns a 0-d CUDA float64 tensor; .backward() gives the gradients of all
    parameter tensors through the CUDA adjoint."""
    return _SpectralMismatchFn.apply(mu, sigma2, ell, rho, psi, kappa, rot, plan, K_target, segment, period,
                                     n_mean)


class _ModeSumFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, amp, psi, a, plan, segment):
        d = a.shape[1]
        table = ModeTable(amp.detach().cpu().double().numpy(), psi.detach().cpu().double().numpy(),
                          a.detach().cpu().double().numpy())
        params = FieldParams(sigma2=1.0, mean=float(mu.detach().cpu()), ell=(1.0,) * d, dim=d,
                             n_modes=amp.numel())
        y = synth(table, params, plan, segment, MapSpec(y=True))["Y"]
        ctx.table, ctx.params, ctx.plan, ctx.segment = table, params, plan, segment
        ctx.meta = [(t.device, t.dtype) for t in (mu, amp, psi, a)]
        return y

    @staticmethod
    def backward(ctx, gY):
        g = backward(ctx.table, ctx.params, ctx.plan, gY.contiguous().float(), ctx.segment)
        grads = (g["dmu"].reshape(()), g["dA"], g["dpsi"], g["da"])
        out = tuple(v.to(device=dv, dtype=dt) for v, (dv, dt) in zip(grads, ctx.meta))
        return out + (None, None)


def mode_sum(mu, amp, psi, a, plan: CellPlan, segment=0):
    """Differentiable Y = mu + sum_j A_j cos(2 pi (a_j . x + psi_j)) with
    gradients to mu and the per-mode amplitudes, phases and frequencies."""
    return _ModeSumFn.apply(mu, amp, psi, a, plan, segment)


# ---------------------------------------------------------------------------
# Convenience: one realisation on a set of cells
# ---------------------------------------------------------------------------
class GaussianField:
    """One realisation: draws its modes, builds its table, synthesises on cells."""

    def __init__(self, params: FieldParams):
        self.params = params
        self.modes = gen_modes(params)
        self.table = ModeTable.from_modes(self.modes)

    def synth(self, plan: CellPlan, maps=None, segment=0, out=None, stream=None):
        return synth(self.table, self.params, plan, segment, maps, out, stream)


# ---------------------------------------------------------------------------
# Batched ensembles
# ---------------------------------------------------------------------------
class Batch:
    """Many realisations on the segments of one plan, one persistent launch.

    items: list of (table, params, segment, MapSpec, out dict).  tile_cells:
    cells per warp work item (128, 256 or 512), 0 for the library default, or
    "auto" to time the candidates on this batch (grf_batch_autotune)."""

    def __init__(self, plan: CellPlan, items, tile_cells=0, stream=None):
        self.plan = plan
        self.items = items
        n = len(items)
        arr = (_abi.grf_batch_item * n)()
        for i, (table, params, segment, maps, out) in enumerate(items):
            it = arr[i]
            it.table = table.dev.data_ptr()
            it.n_modes = table.n_modes
            it.dim = table.dim
            it.segment = int(segment)
            it.mean = float(params.mean)
            it.sigma = float(params.sigma)
            it.map = maps.to_c()
            it.out = _outputs_struct(out)
        self._arr = arr
        self.nbytes = int(lib().grf_batch_workspace_bytes(n, plan.n_cells))
        dev = plan.buf.device
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=dev)
        self.host = torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=True)
        self.tuned_ms = None
        if tile_cells == "auto":
            tc = ctypes.c_int32(0)
            ms = ctypes.c_float(0.0)
            check(lib().grf_batch_autotune(n, arr, plan.ptr, _ptr(self.ws), self.nbytes, _ptr(self.host),
                                           _stream_handle(stream), ctypes.byref(tc), ctypes.byref(ms)))
            self.tile_cells, self.tuned_ms = tc.value, ms.value
        else:
            check(lib().grf_batch_prepare(n, arr, plan.ptr, int(tile_cells), _ptr(self.ws), self.nbytes,
                                          _ptr(self.host), _stream_handle(stream)))
            self.tile_cells = int(tile_cells)
        self.graph = None

    def __del__(self):
        ws = getattr(self, "ws", None)
        if ws is not None:
            try:
                lib().grf_release(_ptr(ws))
            except Exception:  # interpreter shutdown
                pass

    def launch(self, stream=None):
        check(lib().grf_batch_launch(_ptr(self.ws), _stream_handle(stream)))

    def capture(self):
        """Capture one launch into a CUDA graph (replay with .replay())."""
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.launch(stream=s)
        torch.cuda.synchronize()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()


def device_info():
    sms = ctypes.c_int32(0)
    khz = ctypes.c_int32(0)
    check(lib().grf_device_info(ctypes.byref(sms), ctypes.byref(khz)))
    return sms.value, khz.value


def launch_count():
    return int(lib().grf_launch_count())


def take_path_counts():
    """(general, lattice) warp tiles of 2-D and 3-D syntheses since the last
    call (grf_take_path_counts); synchronises the device."""
    g, l_ = ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().grf_take_path_counts(ctypes.byref(g), ctypes.byref(l_)))
    return g.value, l_.value


def take_adjoint_path_counts():
    """(general, lattice) (warp, tile) pairs of 3-D adjoints since the last
    call (grf_take_adjoint_path_counts); synchronises the device."""
    g, l_ = ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().grf_take_adjoint_path_counts(ctypes.byref(g), ctypes.byref(l_)))
    return g.value, l_.value


def take_grid_tiles():
    """128 x 128-cell tiles computed by the tensor-core grid path since the
    last call (grf_take_grid_tiles); synchronises the device."""
    t = ctypes.c_int64(0)
    check(lib().grf_take_grid_tiles(ctypes.byref(t)))
    return t.value


def take_grid_adjoint_units():
    """Units (128 modes x 64 x cells x 64 (y, z) cells) computed by the
    tensor-core grid adjoint since the last call (grf_take_grid_adjoint_units);
    synchronises the device."""
    t = ctypes.c_int64(0)
    check(lib().grf_take_grid_adjoint_units(ctypes.byref(t)))
    return t.value


def grid_path(enable=True, fold_chunks=4):
    """Process-wide setting of the grid path (False: off, True: automatic,
    "always": every grid plan) and its fold interval in chunks of 32 modes
    (grf_debug_grid_path)."""
    mode = 2 if enable == "always" else (1 if enable else 0)
    check(lib().grf_debug_grid_path(mode, int(fold_chunks)))


def mma_selftest(A, B, stream=None):
    """D = A B^T through the tensor-core path's layout (grf_debug_mma_f16):
    A, B CUDA float16 tensors of shape (128, 64 k) -> D (128, 128) float32."""
    A = _require_cuda(A, torch.float16, "A")
    B = _require_cuda(B, torch.float16, "B")
    if A.shape != B.shape or A.dim() != 2 or A.shape[0] != 128 or A.shape[1] % 64 != 0:
        raise ValueError("A and B must both be (128, 64 k)")
    D = torch.empty((128, 128), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    check(lib().grf_debug_mma_f16(_ptr(A), _ptr(B), A.shape[1] // 64, _ptr(D), _ptr(status), _stream_handle(stream)))
    return D, status


def mufu_probe(blocks, iters, stream=None):
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    check(lib().grf_mufu_probe(int(blocks), int(iters), _ptr(sink), _stream_handle(stream)))
    return sink

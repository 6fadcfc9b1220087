"""Benchmark of spectral Gaussian-random-field synthesis on GB300.

Headline step (default): one realisation of the 3-D workload
  256^3 unit-cube cell centres (16,777,216 cells), N = 4096 modes,
  exponential covariance, l = (0.2, 0.2, 0.05), sigma^2 = 4, FP32 field,
  lognormal K and a 3-facies map at the Gaussian 1/3, 2/3 quantiles:
a new realisation per step (modes drawn and packed by the library's native
prefetcher threads, table upload on a copy stream) and the synthesis call
writing Y, K and facies -- on this Cartesian grid the tensor-core grid path
(table preparation and the tcgen05 kernel; --grid-path off selects the
CUDA-core kernels).  Metric: Gcell.mode/s = cells x modes per second.  The same JSON line also reports the forward+backward step (128^3,
N = 2048, mismatch loss and adjoint), the batched ensemble (256 realisations
in one graph-replayed persistent launch), the unstructured 2M-cell workload
(in lattice order and in a seeded random order), the 1024 x 512 HRL-shaped
workload, the bitruncated two-field facies and the periodic, rotated field on
the 256^3 cube, and the 64^2 workload.  roofline.traffic
is the DRAM bytes (read + written) of one headline call's kernels measured by
ncu.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--only all|fwd|bwd|batched|jitter|hrl|next] [--scale S]
                  [--batched-tile auto|128|256|512] [--grid-path auto|off|always]
                  [--no-cpu-baseline] [--jsonl PATH]

Under torchrun each rank runs its own realisations (different seeds) of the
same workloads: per-GPU work is fixed (weak scaling) and the forward path has
no data exchange.  --impl reference times the FP64 CPU oracle on the host
cores instead (rank 0 only).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MUFU_PER_CLK_PER_SM = 16  # cos.approx results per clock per SM (SFU)


def hbm_peak():
    """Measured HBM copy bandwidth of this machine's GPUs (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def tensor_peak():
    """Measured dense BF16 tensor throughput of this machine's GPUs (TFLOP/s,
    cuBLAS burst; FP16 runs at the BF16 rate on the tensor cores), else the
    fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def take_paths(F):
    """Work items of the synthesis paths since the last call (all counters
    reset): warp tiles of the general and lattice paths, 128 x 128 tiles of
    the tensor-core grid path."""
    g, l_ = F.take_path_counts()
    t = F.take_grid_tiles()
    return {"general_warps": g, "lattice_warps": l_, "grid_tiles": t}


def path_fields(paths):
    """Path mix of a bench line: the counts, the lattice share of the
    CUDA-core warp tiles and whether the grid path did the work."""
    g, l_ = paths["general_warps"], paths["lattice_warps"]
    return {"path_warps": {"general": g, "lattice": l_, "grid_tiles": paths["grid_tiles"]},
            "lattice_share": l_ / float(g + l_) if g + l_ else 0.0,
            "grid_path": paths["grid_tiles"] > 0 and g + l_ == 0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--only", default="all", choices=["all", "fwd", "bwd", "batched", "jitter", "hrl", "next"])
    ap.add_argument("--scale", type=int, default=1, help="shrink every grid axis by this factor")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-tile", default="auto", choices=["auto", "128", "256", "512"],
                    help="cells per warp work item of the ensemble (default: autotuned)")
    ap.add_argument("--grid-path", default="auto", choices=["auto", "off", "always"],
                    help="tensor-core grid path for cells on a Cartesian grid (default: every grid plan; "
                         "off: the CUDA-core kernels)")
    ap.add_argument("--jsonl", default=None,
                    help="also append the result line to this JSON-lines run log (with a UTC timestamp)")
    return ap.parse_args()


def emit(args, line):
    """Print the one result line; with --jsonl also append it to the run log."""
    print(json.dumps(line))
    if args.jsonl:
        rec = dict(line, logged_utc=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))
        with open(args.jsonl, "a") as f:
            f.write(json.dumps(rec) + "\n")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers
# ---------------------------------------------------------------------------
def dist_setup(torch):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(torch, world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(torch, world, v):
    if world == 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def params_for(F, w, dim, seed):
    return F.FieldParams(family=w["family"], sigma2=w["sigma2"], mean=w["mean"], ell=w["ell"], dim=dim,
                         n_modes=w["n_modes"], seed=seed, nu=w.get("nu", 1.5), period=w.get("period", (0.0,) * 3),
                         rot=w.get("rot"))


ERR_SAMPLE_CELLS = 1 << 20  # cells of every workload checked against the FP64 oracle (all if fewer)


def oracle_modes_for(w, dim, seed):
    """The FP64 oracle's own draw of a workload's modes (never the library's)."""
    from oracle import modes as om
    fam = {"gaussian": 0, "exponential": 1, "matern": 2}[w["family"]]
    return om.gen_modes(fam, w["sigma2"], list(w["ell"]) + [1.0] * (3 - len(w["ell"])), dim, w["n_modes"], seed,
                        nu=w.get("nu", 1.5), period=w.get("period"),
                        rot=None if w.get("rot") is None else np.asarray(w["rot"])[:dim, :dim])


def fp64_check(cells, y_gpu, modes, mean, sigma, n_sample=ERR_SAMPLE_CELLS, seed=12345, thresholds=(),
               facies=None):
    """Max-abs error of a GPU field against the FP64 C oracle on a seeded
    sample of its cells (all cells when there are fewer), in units of sigma;
    with thresholds and facies also the facies labels outside the 2e-5 sigma
    band that differ from the oracle's.  Runs outside every timed region."""
    from oracle import native
    n = len(cells[0])
    idx = np.arange(n) if n <= n_sample else np.sort(np.random.default_rng(seed).choice(n, n_sample, replace=False))
    c = np.stack([cc[idx] for cc in cells], axis=-1)
    t0 = time.perf_counter()
    y_or = native.synth(modes["a"], modes["amp"], modes["psi"], mean, c)
    err = float(np.max(np.abs(y_gpu[idx].astype(np.float64) - y_or))) / sigma if n else 0.0
    out = {"max_abs_err_sigma": err, "cells": int(len(idx)), "of_cells": int(n), "tol_sigma": 1e-5,
           "within_tol": bool(err <= 1e-5), "oracle_s": time.perf_counter() - t0}
    if len(thresholds) and facies is not None:
        lab = np.zeros(len(idx), dtype=np.int64)
        for t in thresholds:
            lab += (y_or > t)
        band = np.min(np.abs(y_or[:, None] - np.asarray(thresholds)[None, :]), axis=1) <= 2e-5 * sigma
        out["facies_mismatch_outside_band"] = int(np.sum((facies[idx].astype(np.int64) != lab) & ~band))
        out["facies_in_band"] = int(np.sum(band))
    return out


def timed_steps(torch, world, steps, warmup, step_fn, kernel_events=None):
    for i in range(warmup):
        step_fn(i)
    torch.cuda.synchronize()
    barrier(torch, world)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(steps):
        step_fn(warmup + i)
    e1.record(st)
    torch.cuda.synchronize()
    barrier(torch, world)
    ms = e0.elapsed_time(e1) / steps
    return max_over_ranks(torch, world, ms)


def bench_forward(torch, F, W, name, rank, world, steps, warmup, scale, with_e2e=True, shuffle_seed=None,
                  override=None, label=None, check=True):
    """Headline forward step on one workload; returns dict of measurements.
    shuffle_seed: cells handed to the plan in a seeded random order (the
    plan must recover the spatial locality itself).  override: workload
    keys replaced (e.g. period, rot), reported under `label`."""
    w = dict(W.WORKLOADS[name], **(override or {}))
    cells = W.workload_cells(name, scale)
    if shuffle_seed is not None:
        cells, _ = W.shuffled(cells, shuffle_seed)
    dim = len(cells)
    M = len(cells[0])
    N = w["n_modes"]
    sig = math.sqrt(w["sigma2"])
    thr = W.quantile_thresholds(w["mean"], sig, w["quantiles"])
    maps = F.MapSpec(y=True, lognormal=True, thresholds=thr, facies=len(thr) > 0, values=w.get("values"))
    dev_cells = [torch.from_numpy(c).cuda() for c in cells]
    t0 = time.perf_counter()
    plan = F.CellPlan(*dev_cells)
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    base_seed = w["seed"] + 1000 * rank
    # a new realisation every step: drawn and packed ahead by the native
    # prefetcher's worker threads; its upload runs on a copy stream into one
    # of two device tables while the previous synthesis runs
    # (the host's cores but two, shared among the ranks, draw one realisation
    # per worker, and the ring holds a slot for every worker beside those whose
    # uploads are in flight: a small field's step is otherwise bound by the
    # host's drawing rate)
    workers = max(1, ((os.cpu_count() or 4) - 2) // max(1, world))
    pf = F.ModePrefetcher(params_for(F, w, dim, base_seed), depth=min(64, workers + 4), threads=workers)
    ps = F.PreparedSynth(params_for(F, w, dim, base_seed), plan, 0, maps)
    out = ps.out
    tabs = [F.ModeTable.device_only(N, dim) for _ in range(2)]
    st = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    used = [torch.cuda.Event(), torch.cuda.Event()]  # last synthesis reading tabs[k] has run
    up = [torch.cuda.Event(), torch.cuda.Event()]
    kev = []  # (start, end) events around each synthesis kernel

    def step(i):
        k = i % 2
        copy.wait_event(used[k])
        pf.next(tabs[k], stream=copy)
        up[k].record(copy)
        st.wait_event(up[k])
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        ps(tabs[k])
        b.record(st)
        used[k].record(st)
        kev.append((a, b))

    take_paths(F)  # reset
    l0 = F.launch_count()
    ms = timed_steps(torch, world, steps, warmup, step)
    launches = F.launch_count() - l0
    torch.cuda.synchronize()
    pf.close()
    paths = take_paths(F)
    kern_all = [a.elapsed_time(b) for a, b in kev[warmup:]]
    kern_ms = float(np.mean(kern_all))
    assert plan.status() == 0
    # field of the workload's own seed, for the accuracy check against the FP64 oracle
    p0 = params_for(F, w, dim, w["seed"])
    m0 = F.gen_modes(p0)
    ring = [F.ModeTable.from_modes(m0)]
    o0 = F.synth(ring[0], p0, plan, 0, F.MapSpec(y=True, thresholds=thr, facies=len(thr) > 0))
    y_seed = o0["Y"].cpu().numpy()
    fac_seed = o0["facies"].cpu().numpy() if "facies" in o0 else None
    per_step = launches / float(steps + warmup)
    res = {"workload": label or (name if shuffle_seed is None else "%s, cells in seeded random order (seed %d)"
                                 % (name, shuffle_seed)), "cells": M, "modes": N, "dim": dim, "ms_per_step": ms,
           "kernel_ms": max_over_ranks(torch, world, kern_ms),
           "kernel_ms_median": max_over_ranks(torch, world, float(np.median(kern_all))),
           "kernel_ms_best": max_over_ranks(torch, world, float(np.min(kern_all))), "plan_ms": plan_ms,
           "cell_modes_per_step": float(M) * N, "launches_in_timed_region": int(round(per_step * steps)),
           "launches_per_step": per_step, "y_seed": y_seed, **path_fields(paths)}
    if check and rank == 0:
        res["fp64_check"] = fp64_check(cells, y_seed, oracle_modes_for(w, dim, w["seed"]), w["mean"], sig,
                                       thresholds=thr, facies=fac_seed)
    if with_e2e:
        res["e2e"] = bench_forward_e2e(torch, F, W, w, cells, maps, dim, base_seed, world, max(5, steps))
        res["s1_host"] = bench_gen_modes(F, w, dim, base_seed)
        res["map_standalone"] = bench_map(torch, F, maps, out["Y"], w, steps)
    return res


def bench_gen_modes(F, w, dim, seed, reps=10):
    """S1 on the host: mode drawing (grf_gen_modes) and table packing, per realisation."""
    import ctypes
    from paper_2212_10961_gb300 import _abi
    p = params_for(F, w, dim, seed)
    t0 = time.perf_counter()
    for k in range(reps):
        m = F.gen_modes(params_for(F, w, dim, seed + k))
    t1 = time.perf_counter()
    nb = _abi.lib().grf_table_bytes(p.n_modes)
    buf = (ctypes.c_uint8 * nb)()
    ms = F._modes_struct(p.n_modes, dim, m)
    for k in range(reps):
        _abi.check(_abi.lib().grf_pack_table(ctypes.byref(ms), buf, nb))
    t2 = time.perf_counter()
    return {"gen_modes_ms": (t1 - t0) / reps * 1e3, "pack_table_ms": (t2 - t1) / reps * 1e3,
            "modes": p.n_modes, "note": "host C++, overlapped with the previous kernel in the step"}


def bench_map(torch, F, maps, Y, w, steps):
    """Standalone HBM-bound map of an existing field (grf_map_property)."""
    sig = math.sqrt(w["sigma2"])
    m2 = F.MapSpec(y=False, lognormal=maps.lognormal, thresholds=maps.thresholds, facies=maps.facies)
    out = m2.allocate(Y.numel(), Y.device)
    st = torch.cuda.current_stream()
    for _ in range(3):
        F.map_property(Y, m2, w["mean"], sig, out)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=Y.device)  # larger than L2
    times = []
    for _ in range(max(5, steps)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        F.map_property(Y, m2, w["mean"], sig, out)
        b.record(st)
        times.append((a, b))
    torch.cuda.synchronize()
    ms = float(np.median([a.elapsed_time(b) for a, b in times]))
    nbytes = Y.numel() * (4 + (4 if m2.lognormal else 0) + (1 if m2.facies else 0))
    gbs = nbytes / (ms * 1e-3) / 1e9
    peak, kind = hbm_peak()
    return {"ms": ms, "bytes": nbytes, "achieved_gbs": gbs, "peak_gbs": peak, "peak_kind": kind,
            "frac": gbs / peak, "bound": "hbm",
            "note": "L2 flushed (256 MB write) before every launch; median of launches"}


def bench_forward_e2e(torch, F, W, w, cells, maps, dim, base_seed, world, steps):
    """Same step through the public API with host buffers: pinned host cell
    centres copied in, plan, modes, synthesis, outputs copied back.

    Two slots of device buffers alternate between steps: right after step i's
    synthesis is enqueued, the copy-in and the plan of step i + 1 go to a side
    stream (so step i + 1 finds its plan complete and the host does not wait
    for it), and the copy-back of step i to another; a slot is reused only
    after its previous step's outputs have reached the host (events).  The
    modes of every step are a new realisation, drawn ahead by the native
    prefetcher (grf_prefetch_*) and uploaded on the main stream."""
    M = len(cells[0])
    host_cells = [torch.from_numpy(c).pin_memory() for c in cells]
    keys = [k for k in ("Y", "K", "facies")
            if (k == "Y" and maps.y) or (k == "K" and maps.lognormal) or (k == "facies" and maps.facies)]
    dtypes = {"Y": torch.float32, "K": torch.float32, "facies": torch.uint8}
    N = w["n_modes"]
    slots = []
    for _ in range(2):
        slots.append({
            "cells": [torch.empty(M, dtype=torch.float32, device="cuda") for _ in cells],
            "host_out": {k: torch.empty(M, dtype=dtypes[k], pin_memory=True) for k in keys},
            "dev_out": maps.allocate(M, torch.device("cuda")),
            "tab": F.ModeTable.device_only(N, dim),
            "plan": None, "planned": torch.cuda.Event(), "done": torch.cuda.Event()})
    workers = max(1, ((os.cpu_count() or 4) - 2) // max(1, world))  # the host's cores, shared among the ranks
    pf = F.ModePrefetcher(params_for(F, w, dim, base_seed), depth=min(64, workers + 4), threads=workers)
    p = params_for(F, w, dim, base_seed)
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()  # copy-in and planning of the next step
    back = torch.cuda.Stream()  # copy-back of the current step
    for sl in slots:
        sl["done"].record(main)
        sl["synthesised"] = torch.cuda.Event()

    def copy_in_and_plan(sl):
        side.wait_event(sl["done"])  # the slot's previous step has finished on the device
        with torch.cuda.stream(side):
            for h, d in zip(host_cells, sl["cells"]):
                d.copy_(h, non_blocking=True)
            sl["plan"] = F.CellPlan(*sl["cells"], stream=side)
            sl["planned"].record(side)

    copy_in_and_plan(slots[0])

    def step(i):
        sl = slots[i % 2]
        pf.next(sl["tab"], stream=main)
        main.wait_event(sl["planned"])
        F.synth(sl["tab"], p, sl["plan"], 0, maps, sl["dev_out"], stream=main)
        sl["synthesised"].record(main)
        copy_in_and_plan(slots[(i + 1) % 2])  # the next step's inputs
        back.wait_event(sl["synthesised"])
        with torch.cuda.stream(back):
            for k, h in sl["host_out"].items():
                h.copy_(sl["dev_out"][k], non_blocking=True)
        sl["done"].record(back)

    ms = timed_steps(torch, world, steps, 3, step)
    torch.cuda.synchronize()
    pf.close()
    for sl in slots:
        assert sl["plan"].status() == 0
    h2d = 4 * M * len(cells)
    d2h = sum(M * (1 if k == "facies" else 4) for k in keys)
    return {"ms_per_step": ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "pipelined": "copy-in and plan of step i+1 and copy-back of step i on side streams during "
                         "step i's synthesis; modes of every step drawn ahead by the native prefetcher"}


def bench_fwd_bwd(torch, F, W, rank, world, steps, warmup, scale):
    """Forward + backward of the calibration loss on the 128^3 cube, N = 2048:
    per step the fused forward (field, K = exp(Y), L = mean (K - T)^2 and
    dL/dY in one kernel, grf_synth_mismatch) and the adjoint
    (grf_synth_backward); tables fixed, events on the stream."""
    w = W.WORKLOADS["diff128"]
    cells = W.workload_cells("diff128", scale)
    M = len(cells[0])
    N = w["n_modes"]
    plan = F.CellPlan(*[torch.from_numpy(c).cuda() for c in cells])
    pt = F.FieldParams(family=w["family"], sigma2=w["sigma2"], ell=w["ell"], dim=3, n_modes=N,
                       seed=w["target_seed"] + 1000 * rank)
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    base = w["seed"] + 1000 * rank
    ring = [F.ModeTable.from_modes(F.gen_modes(params_for(F, w, 3, base + k))) for k in range(2)]
    st = torch.cuda.current_stream()
    kev = []

    def step(i):
        p = params_for(F, w, 3, base + (i % 2))
        tab = ring[i % 2]
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        c = torch.cuda.Event(enable_timing=True)
        a.record(st)
        loss, gY, _ = F.synth_mismatch(tab, p, plan, T)
        b.record(st)
        F.backward(tab, p, plan, gY)
        c.record(st)
        kev.append((a, b, c))

    take_paths(F)  # reset
    F.take_adjoint_path_counts()
    F.take_grid_adjoint_units()
    l0 = F.launch_count()
    ms = timed_steps(torch, world, steps, warmup, step)
    launches = F.launch_count() - l0
    paths = take_paths(F)
    bgen, blat = F.take_adjoint_path_counts()
    bgrid = F.take_grid_adjoint_units()
    fwd_ms = float(np.mean([a.elapsed_time(b) for a, b, c in kev[warmup:]]))
    bwd_ms = float(np.mean([b.elapsed_time(c) for a, b, c in kev[warmup:]]))
    res = {"workload": "diff128" if scale == 1 else "diff128/%d" % scale, "cells": M, "modes": N,
           "ms_per_step": ms, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "cell_modes_per_step": float(M) * N,
           "launches_per_step": launches / float(steps + warmup),
           "forward": "fused synthesis + lognormal mismatch loss and gradient (grf_synth_mismatch)",
           **path_fields(paths),
           "adjoint_path_tiles": {"general": bgen, "lattice": blat, "grid_units": bgrid},
           "adjoint_lattice_share": blat / float(bgen + blat) if bgen + blat else 0.0,
           "adjoint_grid_path": bgrid > 0 and bgen + blat == 0}
    if rank == 0:
        res["fp64_check"] = grad_check_40(torch, F, W, grid=res["adjoint_grid_path"])
    return res


def grad_check_40(torch, F, W, grid=False):
    """Loss and per-family gradient errors of the fused forward + adjoint on a
    40^3 grid with the 128^3 workload's parameters, against the FP64 oracle's
    own loss gradient (relative to each family's largest oracle value).  grid:
    the timed step ran on the grid path, so this check does too (40^3 is
    below the automatic threshold)."""
    from oracle import field as of
    from oracle import native
    w = W.WORKLOADS["diff128"]
    cells = W.grid_centres((40, 40, 40))
    c = np.stack(cells, axis=-1)
    plan = F.CellPlan(*[torch.from_numpy(x).cuda() for x in cells])
    p = params_for(F, w, 3, w["seed"])
    pt = params_for(F, w, 3, w["target_seed"])
    gf = F.GaussianField(p)
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    if grid:
        F.grid_path("always")
    try:
        loss, gY, out = F.synth_mismatch(gf.table, p, plan, T, want_Y=True)
        g = F.backward(gf.table, p, plan, gY)
        torch.cuda.synchronize()
    finally:
        F.grid_path(GRID_SETTING)
    om = oracle_modes_for(w, 3, w["seed"])
    y_or = native.synth(om["a"], om["amp"], om["psi"], w["mean"], c)
    l_or, g_or = of.mismatch_loss(np.exp(y_or), T.cpu().numpy().astype(np.float64))
    ref = of.grads_reparam(*native.mode_sums(om["a"], om["psi"], c, g_or), om["kappa"], om["rho"],
                           math.sqrt(w["sigma2"]), w["ell"], g_or)
    errs = {}
    for k in ("dA", "dpsi", "da", "dmu", "dsigma", "dsigma2", "dell", "drot", "drho", "dkappa"):
        r = np.asarray(ref[k], dtype=np.float64)
        errs[k] = float(np.max(np.abs(g[k].cpu().numpy().reshape(r.shape) - r)) / np.max(np.abs(r)))
    return {"grid": "40^3 with the 128^3 parameters", "path": "grid (tensor cores)" if grid else "CUDA cores",
            "grad_err_rel": errs, "tol_rel": 1e-4,
            "within_tol": bool(max(errs.values()) <= 1e-4),
            "loss_err_rel": abs(loss.item() - l_or) / abs(l_or),
            "max_abs_err_sigma": float(np.max(np.abs(out["Y"].cpu().numpy() - y_or))) / math.sqrt(w["sigma2"])}


def bench_calibration_autograd(torch, F, W, rank, world, steps, warmup, scale):
    """The calibration step as a user writes it: loss = spectral_mismatch(...)
    (parameters mu, sigma^2, l, rho, psi, kappa as CPU float64 tensors that
    require grad; Sec. 4.1 reparameterisation and packing in the library),
    then loss.backward(), on the 128^3 workload.  Host work, the table
    upload and the gradients' copy back to the parameters' device are inside
    the step."""
    w = W.WORKLOADS["diff128"]
    cells = W.workload_cells("diff128", scale)
    M, N = len(cells[0]), w["n_modes"]
    plan = F.CellPlan(*[torch.from_numpy(c).cuda() for c in cells])
    pt = params_for(F, w, 3, w["target_seed"] + 1000 * rank)
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    m = F.gen_modes(params_for(F, w, 3, w["seed"] + 1000 * rank))
    dt = torch.float64
    prm = [torch.tensor(w["mean"], dtype=dt), torch.tensor(w["sigma2"], dtype=dt), torch.tensor(w["ell"], dtype=dt),
           torch.tensor(m["rho"]), torch.tensor(m["psi"]), torch.tensor(m["kappa"])]
    for t in prm:
        t.requires_grad_(True)
    losses = []

    def step(i):
        for t in prm:
            t.grad = None
        loss = F.spectral_mismatch(*prm, plan, T)
        loss.backward()
        losses.append(loss.detach())

    l0 = F.launch_count()
    ms = timed_steps(torch, world, steps, warmup, step)
    launches = F.launch_count() - l0
    return {"workload": "diff128" if scale == 1 else "diff128/%d" % scale, "cells": M, "modes": N,
            "ms_per_step": ms, "cell_modes_per_step": float(M) * N,
            "launches_per_step": launches / float(steps + warmup),
            "api": "F.spectral_mismatch(mu, sigma2, ell, rho, psi, kappa, plan, T).backward(), CPU parameters"}


def bench_bitruncated(torch, F, W, rank, world, steps, warmup, scale):
    """Bitruncated pluri-Gaussian facies (Sec. 3.1, Appendix B) on the 256^3
    cube: two fields of 4096 modes on generator streams 0 and 1 (the
    headline's exponential field and a Gaussian one), a 3 x 2 truncation
    rule and per-facies values; per step both syntheses and the rule map
    (tables fixed; events on the stream around the whole step)."""
    w = W.WORKLOADS["grid3d_256"]
    cells = W.workload_cells("grid3d_256", scale)
    M, N = len(cells[0]), w["n_modes"]
    plan = F.CellPlan(*[torch.from_numpy(c).cuda() for c in cells])
    seed = w["seed"] + 1000 * rank
    p1 = F.FieldParams(family=w["family"], sigma2=w["sigma2"], ell=w["ell"], dim=3, n_modes=N, seed=seed)
    p2 = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1, 0.1), dim=3, n_modes=N, seed=seed)
    pg = F.PluriGaussianField(p1, p2)
    t = W.quantile_thresholds(0.0, math.sqrt(w["sigma2"]), (1.0 / 3.0, 2.0 / 3.0))
    rule = [[0, 1], [2, 3], [4, 5]]
    values = [0.01, 0.1, 1.0, 10.0, 100.0, 1000.0]
    take_paths(F)  # reset
    l0 = F.launch_count()
    ms = timed_steps(torch, world, steps, warmup, lambda i: pg.synth(plan, t, (0.0,), rule, values))
    launches = F.launch_count() - l0
    paths = take_paths(F)
    res = {"workload": "grid3d_256 bitruncated: exponential l=(0.2,0.2,0.05) x Gaussian l=0.1, 3 x 2 rule",
           "cells": M, "modes_per_field": N, "ms_per_step": ms, "cell_modes_per_step": 2.0 * M * N,
           "launches_per_step": launches / float(steps + warmup), "kernel_ms": ms, **path_fields(paths)}
    if rank == 0:
        # both fields against the oracle's own draws (streams 0 and 1), and the
        # merged facies against the rule applied to the oracle fields
        from oracle import field as of
        from oracle import modes as om
        from oracle import native
        o = pg.synth(plan, t, (0.0,), rule, values)
        y1, y2, fac = o["Y1"].cpu().numpy(), o["Y2"].cpu().numpy(), o["facies"].cpu().numpy()
        idx = np.sort(np.random.default_rng(12345).choice(M, min(M, ERR_SAMPLE_CELLS), replace=False))
        c = np.stack([cc[idx] for cc in cells], axis=-1)
        m1 = om.gen_modes(1, w["sigma2"], w["ell"], 3, N, seed, stream=0)
        m2 = om.gen_modes(0, 1.0, (0.1, 0.1, 0.1), 3, N, seed, stream=1)
        o1 = native.synth(m1["a"], m1["amp"], m1["psi"], 0.0, c)
        o2 = native.synth(m2["a"], m2["amp"], m2["psi"], 0.0, c)
        lab = of.bitruncated(o1, o2, t, (0.0,), rule)
        band = (np.min(np.abs(o1[:, None] - np.asarray(t)[None, :]), axis=1) <= 2e-5 * math.sqrt(w["sigma2"])) | \
            (np.abs(o2) <= 2e-5)
        res["fp64_check"] = {
            "max_abs_err_sigma": max(float(np.max(np.abs(y1[idx] - o1))) / math.sqrt(w["sigma2"]),
                                     float(np.max(np.abs(y2[idx] - o2)))),
            "cells": int(len(idx)), "of_cells": int(M), "tol_sigma": 1e-5,
            "facies_mismatch_outside_band": int(np.sum((fac[idx] != lab) & ~band)), "facies_in_band": int(band.sum())}
        res["fp64_check"]["within_tol"] = bool(res["fp64_check"]["max_abs_err_sigma"] <= 1e-5)
    return res


def bench_batched(torch, F, W, rank, world, steps, warmup, scale, tile="auto"):
    recipe = W.ensemble_recipe(seed=4 + rank)
    segs, xs, ys, zs = [], [], [], []
    for r in recipe:
        shape = tuple(max(1, s // scale) for s in r["shape"])
        c = W.grid_centres(shape)
        if len(c) == 2:
            c = c + [np.zeros_like(c[0])]
        xs.append(c[0])
        ys.append(c[1])
        zs.append(c[2])
        segs.append(len(c[0]))
    cells = [np.concatenate(v) for v in (xs, ys, zs)]
    plan = F.CellPlan(*[torch.from_numpy(c).cuda() for c in cells], dim=3, segments=segs)
    items = []
    cm = 0.0
    for s, r in enumerate(recipe):
        p = F.FieldParams(family=r["family"], sigma2=r["sigma2"], mean=r["mean"], ell=r["ell"], dim=r["dim"],
                          n_modes=r["n_modes"], seed=r["seed"] + 100000 * rank)
        gf = F.GaussianField(p)
        maps = F.MapSpec(y=True, lognormal=True)
        out = maps.allocate(segs[s], torch.device("cuda"))
        items.append((gf.table, p, s, maps, out))
        cm += float(segs[s]) * r["n_modes"]
    batch = F.Batch(plan, items, tile_cells=tile)
    batch.launch()
    batch.capture()
    take_paths(F)  # reset
    l0 = F.launch_count()
    ms = timed_steps(torch, world, steps, warmup, lambda i: batch.replay())
    paths = take_paths(F)
    res = {"workload": "ensemble256", "realisations": len(recipe), "cells": int(sum(segs)), **path_fields(paths),
           "ms_per_step": ms, "cell_modes_per_step": cm, "launches_per_step": 1,
           "tile_cells": batch.tile_cells, "autotune_ms": batch.tuned_ms,
           # one cell per lane takes its cosine from the FMA-pipe polynomial
           "mufu_share": 1.0 - 1.0 / (batch.tile_cells // 32)}
    if rank == 0:
        # every realisation on a seeded sample (about 2^20 cells in all), its
        # Y against the oracle's own draw of its modes
        from oracle import native
        torch.cuda.synchronize()
        rng = np.random.default_rng(12345)
        per = max(1, ERR_SAMPLE_CELLS // len(recipe))
        err, checked, t0 = 0.0, 0, time.perf_counter()
        off = 0
        for s_, r in enumerate(recipe):
            n = segs[s_]
            idx = np.arange(n) if n <= per else np.sort(rng.choice(n, per, replace=False))
            c = np.stack([cc[off + idx] for cc in cells[:r["dim"]]], axis=-1)
            om = oracle_modes_for(dict(r, seed=r["seed"] + 100000 * rank), r["dim"], r["seed"] + 100000 * rank)
            y = items[s_][4]["Y"].cpu().numpy()[idx]
            err = max(err, float(np.max(np.abs(y - native.synth(om["a"], om["amp"], om["psi"], r["mean"], c))))
                      / math.sqrt(r["sigma2"]))
            checked += len(idx)
            off += n
        res["fp64_check"] = {"max_abs_err_sigma": err, "cells": checked, "of_cells": int(sum(segs)),
                             "tol_sigma": 1e-5, "within_tol": bool(err <= 1e-5), "oracle_s": time.perf_counter() - t0}
    return res


def cpu_baseline(W, name, scale, target_s=10.0, y_gpu=None):
    """FP64 C oracle (OpenMP, all host cores) on a seeded sample of the workload.
    With y_gpu (the GPU field of the workload's own seed) the sample also gives
    the max-abs error of the GPU field against the oracle on those cells."""
    from oracle import modes as om
    from oracle import native
    w = W.WORKLOADS[name]
    cells = W.workload_cells(name, scale)
    c = np.stack(cells, axis=-1)
    fam = {"gaussian": 0, "exponential": 1, "matern": 2}[w["family"]]
    m = om.gen_modes(fam, w["sigma2"], w["ell"], c.shape[1], w["n_modes"], w["seed"], nu=w.get("nu", 1.5))
    rng = np.random.default_rng(12345)
    n = 2048
    while True:
        idx = rng.choice(len(c), min(n, len(c)), replace=False)
        t0 = time.perf_counter()
        y_or = native.synth(m["a"], m["amp"], m["psi"], w["mean"], c[idx])
        dt = time.perf_counter() - t0
        if dt > target_s / 4 or n >= len(c):
            break
        n = int(min(len(c), n * max(2.0, min(16.0, target_s / 4 / max(dt, 1e-3)))))
    rate = len(idx) * float(w["n_modes"]) / dt
    cores = native.threads()
    res = {"value": rate / 1e9, "unit": "Gcell.mode/s", "cores": cores, "kind": "oracle",
           "sample": "%d random cells of %s x %d modes, FP64 C + OpenMP, %.1f s" % (len(idx), name, w["n_modes"], dt)}
    # the same oracle on one core, on a sample sized for about the same time per core
    n1 = max(64, int(len(idx) / max(1, cores)))
    native.set_threads(1)
    try:
        t0 = time.perf_counter()
        native.synth(m["a"], m["amp"], m["psi"], w["mean"], c[idx[:n1]])
        dt1 = time.perf_counter() - t0
    finally:
        native.set_threads(cores)
    res["single_core"] = {"value": n1 * float(w["n_modes"]) / dt1 / 1e9, "unit": "Gcell.mode/s",
                          "sample": "%d of those cells, %.1f s" % (n1, dt1)}
    if y_gpu is not None:
        err = float(np.max(np.abs(y_gpu[idx].astype(np.float64) - y_or)))
        res["gpu_max_abs_err_sigma"] = err / math.sqrt(w["sigma2"])
        res["gpu_err_cells"] = int(len(idx))
    return res


# dram__bytes_read.sum + dram__bytes_write.sum of one full-size call of the
# headline's grid-path kernels (grid_prep_kernel + grid_mma_kernel, 256^3
# cells, 4096 modes), one ncu capture (`--metrics dram__bytes_read.sum,
# dram__bytes_write.sum -k regex:grid`): 0.252 + 0.027 MB and 26.95 + 91.10 MB.
# Algorithmic: 9 B written per cell (Y, K, facies) = 151 MB plus 26 MB of
# tables; part of the writes was still in L2 when the launch ended.
HEAD_TRAFFIC_BYTES = 0.25242e6 + 0.02688e6 + 26.95e6 + 91.10e6


# FP32 instructions per cell-mode of the lattice path (lanes of 4-cell grid
# rows): per (lane, mode) the complex corner term (3 FFMA phase, 2 FMUL
# radian scaling inside the hardware sine/cosine, 2 FMUL by A), the C/4 - 1
# row phasors (4 each) and per cell 2 FFMA (1 FADD on the first of a row):
# (7 + 12 + 28) / 16 = 2.94 in 3-D and (6 + 4 + 14) / 8 = 3.0 in 2-D.
LATTICE_FP32_PER_CELL_MODE = 3.0
FP32_PER_CLK_PER_SM = 128
# FP32 instructions per cell-mode of the adjoint's lattice tiles: per (row of
# 4 cells, mode) the row phasor (4, on 3 rows of 4), H and H' from the powers
# (4 chains of 3), R H (4), Im(R H') (2), the sums (Sr, Si, the row weight,
# the plane sum: 4): 25 per 4 cells, plus the plane phasors and the
# per-brick and per-tile terms: 6.6.
ADJOINT_LATTICE_FP32_PER_CELL_MODE = 6.6


# Tensor-core work of the grid path per cell-mode: the real part of a complex
# product is a 2-term dot product (2 multiply-adds = 4 flops), evaluated as
# three FP16 products (hi.hi, hi.lo, lo.hi) for FP32-level accuracy.
GRID_TENSOR_FLOPS_PER_CELL_MODE = 12.0
# The grid adjoint: per cell-mode the cosine and the sine product of g and of
# the x-weighted g (4 multiply-adds = 8 flops), each as three FP16 products.
GRID_ADJ_TENSOR_FLOPS_PER_CELL_MODE = 24.0

# Grid-path setting of this run (--grid-path), restored after checks that
# force the grid path on grids below the automatic threshold.
GRID_SETTING = True


def roofline(kern_ms, cell_modes, clocks, sms, traffic=None, lattice_share=0.0, grid=False):
    """Roofline of a synthesis kernel.  General path: the MUFU pipe, 1
    hardware cosine per cell-mode.  Lattice path (lattice_share >= 1/2 of the
    warp tiles): the FP32 pipe at LATTICE_FP32_PER_CELL_MODE instructions per
    cell-mode (1/8 MUFU per cell-mode); the MUFU fraction is kept beside it.
    Grid path: the tensor cores at GRID_TENSOR_FLOPS_PER_CELL_MODE FP16 flops
    per cell-mode against the measured dense BF16 peak (kern_ms covers the
    call's two kernels: table preparation and the tensor-core kernel)."""
    mufu_peak = MUFU_PER_CLK_PER_SM * sms * 2070e6 / 1e9  # Gcell.mode/s at the maximum SM clock
    achieved = cell_modes / (kern_ms * 1e-3) / 1e9
    if grid:
        tpk, kind = tensor_peak()
        tf = cell_modes * GRID_TENSOR_FLOPS_PER_CELL_MODE / (kern_ms * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": tf, "peak": tpk, "unit": "TFLOP/s", "frac": tf / tpk,
                "traffic": traffic, "peak_kind": kind,
                "peak_basis": ("tensor-core grid path: %.0f FP16 tensor flops per cell-mode (a 2-term real dot "
                               "product as three FP16 products hi.hi + hi.lo + lo.hi) against the %s dense BF16 "
                               "cuBLAS burst peak (FP16 runs at the BF16 rate)" %
                               (GRID_TENSOR_FLOPS_PER_CELL_MODE, kind)),
                "gcell_modes_per_s": achieved, "frac_of_mufu_roofline": achieved / mufu_peak,
                "frac_of_lattice_fp32_roofline": achieved / (FP32_PER_CLK_PER_SM * sms * 2070e6 /
                                                             LATTICE_FP32_PER_CELL_MODE / 1e9)}
    if lattice_share >= 0.5:
        peak_max = FP32_PER_CLK_PER_SM * sms * 2070e6 / LATTICE_FP32_PER_CELL_MODE / 1e9
        basis = ("lattice path (%.3f of the warp tiles): %d FP32 lanes/clk/SM x %d SMs x 2070 MHz / %.1f FP32 "
                 "instructions per cell-mode" % (lattice_share, FP32_PER_CLK_PER_SM, sms, LATTICE_FP32_PER_CELL_MODE))
        per_clk = FP32_PER_CLK_PER_SM / LATTICE_FP32_PER_CELL_MODE
    else:
        peak_max = mufu_peak
        basis = "%d MUFU cos/clk/SM x %d SMs x 2070 MHz (1 MUFU per cell-mode)" % (MUFU_PER_CLK_PER_SM, sms)
        per_clk = MUFU_PER_CLK_PER_SM
    out = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "Gcell.mode/s",
           "frac": achieved / peak_max, "traffic": traffic, "peak_basis": basis,
           "frac_of_mufu_roofline": achieved / mufu_peak}
    if clocks.get("sm_mhz"):
        peak_meas = per_clk * sms * clocks["sm_mhz"] * 1e6 / 1e9
        out["frac_at_measured_clock"] = achieved / peak_meas
    return out


HEAD_METRIC = "Gcell.mode/s forward (fused Y, lognormal K, 3 facies) at <=1e-5 sigma vs FP64"


def head_config(scale, cells, modes):
    return {"workload": "grid3d_256" if scale == 1 else "grid3d_256/%d" % scale,
            "cells": cells, "modes": modes, "covariance": "exponential", "ell": [0.2, 0.2, 0.05],
            "sigma2": 4.0, "outputs": "Y,K,facies(3)",
            "l2": "inputs (sorted coordinates 201 MB + permutation 67 MB) exceed the 129 MB L2"}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on the host cores.

    Every step evaluates the same seeded sample of the headline workload's
    cells (sized once, during warm-up, for about one second of oracle work)
    with the oracle's own modes; ms_per_step is the measured time of that
    sample, and the rate is cells x modes of the sample per second."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2212_10961_gb300 import workloads as W
    from oracle import native
    native.build()
    name = "grid3d_256"
    w = W.WORKLOADS[name]
    cells = W.workload_cells(name, args.scale)
    c_all = np.stack(cells, axis=-1)
    M, N = len(c_all), w["n_modes"]
    m = oracle_modes_for(w, 3, w["seed"])
    rng = np.random.default_rng(12345)
    # size the sample: grow until one evaluation takes about a second
    n = 1024
    while True:
        idx = rng.choice(M, min(n, M), replace=False)
        t0 = time.perf_counter()
        native.synth(m["a"], m["amp"], m["psi"], w["mean"], c_all[idx])
        dt = time.perf_counter() - t0
        if dt > 0.5 or n >= M:
            break
        n = int(min(M, n * max(2.0, min(16.0, 1.0 / max(dt, 1e-3)))))
    sample = c_all[idx]
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        native.synth(m["a"], m["amp"], m["psi"], w["mean"], sample)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = float(np.mean(times)) * 1e3
    val = len(sample) * float(N) / (ms * 1e-3) / 1e9
    desc = "%d random cells of %s x %d modes per step, FP64 C + OpenMP" % (len(sample), name, N)
    line = {"impl": "reference", "metric": HEAD_METRIC, "value": val,
            "unit": "Gcell.mode/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "sampled_cells": int(len(sample)),
            "extrapolated_ms_full_size": ms * M / len(sample),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": head_config(args.scale, M, N),
            "cpu_baseline": {"value": val, "unit": "Gcell.mode/s", "cores": native.threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": val, "unit": "Gcell.mode/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(args, line)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import __graft_entry__
    world, rank, local = dist_setup(torch)
    if rank == 0:
        __graft_entry__.build()
    barrier(torch, world)
    __graft_entry__.build()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    if rank == 0:
        from oracle import native
        native.build()  # the FP64 accuracy checks run outside every timed region

    sms, _ = F.device_info()
    global GRID_SETTING
    GRID_SETTING = {"auto": True, "off": False, "always": "always"}[args.grid_path]
    F.grid_path(GRID_SETTING)
    clocks = ClockSampler(local)
    extra = {}
    head = None
    clocks.start()
    if args.only in ("all", "fwd"):
        head = bench_forward(torch, F, W, "grid3d_256", rank, world, args.steps, args.warmup, args.scale)
    if args.only in ("all", "bwd"):
        extra["fwd_bwd"] = bench_fwd_bwd(torch, F, W, rank, world, args.steps, args.warmup, args.scale)
        extra["calibration_autograd"] = bench_calibration_autograd(torch, F, W, rank, world, args.steps,
                                                                   args.warmup, args.scale)
    if args.only in ("all", "batched"):
        extra["batched"] = bench_batched(torch, F, W, rank, world, max(3, args.steps // 2), args.warmup, args.scale,
                                         "auto" if args.batched_tile == "auto" else int(args.batched_tile))
    if args.only in ("all", "jitter"):
        extra["jitter3d_2m"] = bench_forward(torch, F, W, "jitter3d_2m", rank, world, args.steps, args.warmup,
                                             args.scale, with_e2e=False)
        extra["jitter3d_2m_shuffled"] = bench_forward(torch, F, W, "jitter3d_2m", rank, world, args.steps,
                                                      args.warmup, args.scale, with_e2e=False, shuffle_seed=5)
    if args.only in ("all", "hrl"):
        extra["hrl2d"] = bench_forward(torch, F, W, "hrl2d", rank, world, args.steps, args.warmup, 1,
                                       with_e2e=False)
    if args.only in ("all", "next"):
        extra["bitruncated_256"] = bench_bitruncated(torch, F, W, rank, world, max(3, args.steps // 2), args.warmup,
                                                     args.scale)
        c30, s30 = math.cos(math.pi / 6), math.sin(math.pi / 6)
        extra["periodic_rotated_256"] = bench_forward(
            torch, F, W, "grid3d_256", rank, world, max(3, args.steps // 2), args.warmup, args.scale,
            with_e2e=False, override={"period": (1.0, 1.0, 1.0), "rot": ((c30, s30, 0.0), (-s30, c30, 0.0),
                                                                        (0.0, 0.0, 1.0))},
            label="grid3d_256 with periodic = (1, 1, 1) and the anisotropy rotated 30 degrees about z")
    if args.only == "all":
        extra["grid2d_64"] = bench_forward(torch, F, W, "grid2d_64", rank, world, args.steps, args.warmup, 1,
                                           with_e2e=False)
    ck = clocks.stop()
    if rank != 0:
        return
    if head is not None:
        head.pop("y_seed", None)
    for v in extra.values():
        v.pop("y_seed", None)
    for k, v in extra.items():
        v["gcell_modes_per_s"] = v["cell_modes_per_step"] * world / (v["ms_per_step"] * 1e-3) / 1e9
        if "kernel_ms" in v:
            v["roofline"] = roofline(v["kernel_ms"], v["cell_modes_per_step"], ck, sms,
                                     lattice_share=v.get("lattice_share", 0.0), grid=v.get("grid_path", False))
    if k_b := extra.get("batched"):
        # one cosine per lane of the general path comes from the FMA pipe: the
        # MUFU pipe's share of that path's work; the lattice lanes (the 64^3
        # realisations) need 1/8 MUFU per cell-mode, so the MUFU fraction of
        # this mixed launch is a fraction of the general path's bound only
        r = roofline(k_b["ms_per_step"], k_b["cell_modes_per_step"], ck, sms, lattice_share=k_b["lattice_share"])
        r["mufu_frac"] = r["frac_of_mufu_roofline"] * k_b["mufu_share"]
        r["peak_basis"] += ("; %.3f of the warp tiles took the lattice path; mufu_frac counts only the %.4f of the "
                            "general path's cosines on the MUFU pipe" % (k_b["lattice_share"], k_b["mufu_share"]))
        k_b["roofline"] = r
    if (k_ca := extra.get("calibration_autograd")) and (k_fb := extra.get("fwd_bwd")):
        k_ca["vs_fwd_bwd_device_ms"] = k_ca["ms_per_step"] / (k_fb["fwd_ms"] + k_fb["bwd_ms"])
    if k_fb := extra.get("fwd_bwd"):
        # forward+backward SFU roofline: 3 MUFU per cell-mode (cos; sin and cos)
        k_fb["roofline_fwd_bwd"] = {
            "achieved": k_fb["cell_modes_per_step"] / ((k_fb["fwd_ms"] + k_fb["bwd_ms"]) * 1e-3) / 1e9,
            "peak": MUFU_PER_CLK_PER_SM * sms * 2070e6 / 3 / 1e9, "unit": "Gcell.mode/s"}
        k_fb["roofline_fwd_bwd"]["frac"] = k_fb["roofline_fwd_bwd"]["achieved"] / k_fb["roofline_fwd_bwd"]["peak"]
        k_fb["roofline_fwd_bwd"]["peak_basis"] = ("3 MUFU per cell-mode (1 forward cosine, adjoint sine and "
                                                  "cosine); the forward's own bound is in fwd_roofline")
        # each half against its own bound
        k_fb["fwd_roofline"] = roofline(k_fb["fwd_ms"], k_fb["cell_modes_per_step"], ck, sms,
                                        lattice_share=k_fb.get("lattice_share", 0.0),
                                        grid=k_fb.get("grid_path", False))
        bw = k_fb["cell_modes_per_step"] / (k_fb["bwd_ms"] * 1e-3) / 1e9
        bmufu = MUFU_PER_CLK_PER_SM * sms * 2070e6 / 2 / 1e9
        if k_fb.get("adjoint_grid_path", False):
            tpk, kind = tensor_peak()
            tf = k_fb["cell_modes_per_step"] * GRID_ADJ_TENSOR_FLOPS_PER_CELL_MODE / (k_fb["bwd_ms"] * 1e-3) / 1e12
            k_fb["bwd_roofline"] = {
                "bound": "tensor", "achieved": tf, "peak": tpk, "unit": "TFLOP/s", "frac": tf / tpk,
                "peak_kind": kind, "gcell_modes_per_s": bw, "frac_of_mufu_roofline": bw / bmufu,
                "peak_basis": ("tensor-core grid adjoint: %.0f FP16 tensor flops per cell-mode (cos and sin "
                               "products of g and of x-weighted g, three FP16 products each) against the %s dense "
                               "BF16 burst peak" % (GRID_ADJ_TENSOR_FLOPS_PER_CELL_MODE, kind)),
                "note": "scan, table preparation, tensor-core kernel and the two reductions"}
        elif k_fb.get("adjoint_lattice_share", 0.0) >= 0.5:
            bpk = FP32_PER_CLK_PER_SM * sms * 2070e6 / ADJOINT_LATTICE_FP32_PER_CELL_MODE / 1e9
            basis = ("lattice tiles (%.3f of the tiles): %d FP32 lanes/clk/SM x %d SMs x 2070 MHz / %.1f FP32 "
                     "instructions per cell-mode" % (k_fb["adjoint_lattice_share"], FP32_PER_CLK_PER_SM, sms,
                                                     ADJOINT_LATTICE_FP32_PER_CELL_MODE))
        else:
            bpk, basis = bmufu, "2 MUFU per cell-mode (sine and cosine)"
        if not k_fb.get("adjoint_grid_path", False):
            k_fb["bwd_roofline"] = {"bound": "alu", "achieved": bw, "peak": bpk, "unit": "Gcell.mode/s",
                                    "frac": bw / bpk, "peak_basis": basis, "frac_of_mufu_roofline": bw / bmufu,
                                    "note": "adjoint kernel and its two reductions"}
    if head is None:
        head = next(iter(extra.values()))
        emit(args, {"partial": args.only, "results": extra, "clocks": ck})
        return
    value = head["cell_modes_per_step"] * world / (head["ms_per_step"] * 1e-3) / 1e9
    e2e = head.get("e2e")
    line = {
        "metric": HEAD_METRIC,
        "value": value, "unit": "Gcell.mode/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": head_config(args.scale, head["cells"], head["modes"]),
        "plan_ms_once_per_mesh": head["plan_ms"],
        "roofline": roofline(head["kernel_ms"], head["cell_modes_per_step"], ck, sms,
                             HEAD_TRAFFIC_BYTES if args.scale == 1 and HEAD_TRAFFIC_BYTES else None,
                             head.get("lattice_share", 0.0), grid=head.get("grid_path", False)),
        "grid_path": head.get("grid_path", False),
        "path_warps": head.get("path_warps"),
        "kernel_ms": head["kernel_ms"], "kernel_ms_median": head["kernel_ms_median"],
        "kernel_ms_best": head["kernel_ms_best"],
        "gpu_launches": head["launches_in_timed_region"],
        "clocks": ck,
    }
    for k in ("s1_host", "map_standalone", "fp64_check"):
        if k in head:
            line[k] = head[k]
    if e2e:
        line["e2e"] = {"value": head["cell_modes_per_step"] * world / (e2e["ms_per_step"] * 1e-3) / 1e9,
                       "unit": "Gcell.mode/s", "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e2e["d2h_bytes_per_step"], "ms_per_step": e2e["ms_per_step"]}
    line.update(extra)
    if world == 1 and not args.no_cpu_baseline:
        from oracle import native
        native.build()
        line["cpu_baseline"] = cpu_baseline(W, "grid3d_256", args.scale)
    emit(args, line)


if __name__ == "__main__":
    main()

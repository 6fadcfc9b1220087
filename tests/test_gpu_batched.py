"""GPU checks of the batched ensemble path (S6): one persistent launch over
realisations of uneven size, dimension, mode count and covariance, against
the single-realisation path and the FP64 oracle (Y, lognormal K and the
facies of every item); CUDA-graph replay."""
import math

import numpy as np
import pytest

from helpers import check_facies, check_forward, check_lognormal, gpu_env, oracle_field, oracle_modes, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    return torch, F, W


def _ensemble(env, recipe, tile_cells=0):
    torch, F, W = env
    segs = []
    xs, ys, zs = [], [], []
    for r in recipe:
        c = W.grid_centres(r["shape"])
        if len(c) == 2:
            c = c + [np.zeros_like(c[0])]
        xs.append(c[0])
        ys.append(c[1])
        zs.append(c[2])
        segs.append(len(c[0]))
    cells = [np.concatenate(v) for v in (xs, ys, zs)]
    plan = F.CellPlan(*to_dev(torch, cells), dim=3, segments=segs)
    items = []
    fields = []
    for s, r in enumerate(recipe):
        p = F.FieldParams(family=r["family"], sigma2=r["sigma2"], mean=r["mean"], ell=r["ell"], dim=r["dim"],
                          n_modes=r["n_modes"], seed=r["seed"])
        gf = F.GaussianField(p)
        maps = F.MapSpec(y=True, lognormal=True, thresholds=(0.0,), facies=True)
        out = maps.allocate(segs[s], plan.buf.device)
        items.append((gf.table, p, s, maps, out))
        fields.append(gf)
    batch = F.Batch(plan, items, tile_cells=tile_cells)
    return plan, batch, items, fields


SMALL = [dict(shape=(40, 33), dim=2, n_modes=300, family="gaussian"),
         dict(shape=(16, 12, 9), dim=3, n_modes=1024, family="exponential"),
         dict(shape=(7, 5), dim=2, n_modes=129, family="exponential"),
         dict(shape=(100, 64), dim=2, n_modes=640, family="gaussian"),
         dict(shape=(3, 3, 3), dim=3, n_modes=1, family="gaussian")]


def _recipe():
    out = []
    for i, r in enumerate(SMALL):
        out.append(dict(r, ell=(0.1,) * r["dim"], sigma2=1.0 + 0.5 * i, mean=0.1 * i, seed=77 + i))
    return out


@pytest.mark.parametrize("tile_cells", [0, 256, 128, 512])
def test_batched_matches_single_and_oracle(env, tile_cells):
    torch, F, W = env
    recipe = _recipe()
    plan, batch, items, fields = _ensemble(env, recipe, tile_cells)
    batch.launch()
    torch.cuda.synchronize()
    for s, (table, p, seg, maps, out) in enumerate(items):
        single = F.synth(table, p, plan, seg, maps, workspace=False)
        torch.cuda.synchronize()
        yb = out["Y"].cpu().numpy()
        ys = single["Y"].cpu().numpy()
        # the batched kernel evaluates one cosine per lane on the FMA pipe, so
        # it agrees with the single-realisation kernel to rounding
        assert np.max(np.abs(yb - ys)) <= 2 * 1e-5 * p.sigma
        r = recipe[s]
        om = oracle_modes(r["family"], r["sigma2"], r["ell"], r["dim"], r["n_modes"], r["seed"])
        cells = W.grid_centres(r["shape"])
        y_or = oracle_field(om, r["mean"], cells)
        check_forward(yb, y_or, p.sigma, "batch item %d" % s)
        # K and the facies of the persistent kernel against the oracle field
        # (Sec. 3.1 truncation rule), with the band of the single path
        check_lognormal(out["K"].cpu().numpy(), y_or, p.sigma)
        check_facies(out["facies"].cpu().numpy(), y_or, (0.0,), p.sigma)


def test_graph_replay(env):
    torch, F, W = env
    recipe = _recipe()
    plan, batch, items, fields = _ensemble(env, recipe)
    batch.launch()
    torch.cuda.synchronize()
    ref = [it[4]["Y"].clone() for it in items]
    for it in items:
        it[4]["Y"].zero_()
    batch.capture()
    batch.replay()
    batch.replay()
    torch.cuda.synchronize()
    for r, it in zip(ref, items):
        assert torch.equal(r, it[4]["Y"])


def test_ensemble256_sampled(env):
    # the whole 256-realisation ensemble in one graph-replayed launch; every
    # realisation checked on up to 4000 sampled cells (0.93M cells in all)
    torch, F, W = env
    recipe = W.ensemble_recipe()
    plan, batch, items, fields = _ensemble(env, recipe)
    batch.capture()
    batch.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    for s in range(len(recipe)):
        r = recipe[s]
        cells = W.grid_centres(r["shape"])
        idx = rng.choice(len(cells[0]), min(4000, len(cells[0])), replace=False)
        om = oracle_modes(r["family"], r["sigma2"], r["ell"], r["dim"], r["n_modes"], r["seed"])
        out = items[s][4]
        y_or = oracle_field(om, r["mean"], cells, idx)
        sig = math.sqrt(r["sigma2"])
        check_forward(out["Y"].cpu().numpy()[idx], y_or, sig, "ensemble %d" % s)
        check_lognormal(out["K"].cpu().numpy()[idx], y_or, sig)
        check_facies(out["facies"].cpu().numpy()[idx], y_or, (0.0,), sig)


def test_autotune_picks_a_candidate_and_stays_correct(env):
    torch, F, W = env
    recipe = _recipe()
    plan, batch, items, fields = _ensemble(env, recipe, tile_cells="auto")
    assert batch.tile_cells in (128, 256, 512) and batch.tuned_ms > 0
    batch.launch()
    torch.cuda.synchronize()
    for s_, (table, p, seg, maps, out) in enumerate(items):
        r = recipe[s_]
        om = oracle_modes(r["family"], r["sigma2"], r["ell"], r["dim"], r["n_modes"], r["seed"])
        check_forward(out["Y"].cpu().numpy(), oracle_field(om, r["mean"], W.grid_centres(r["shape"])), p.sigma,
                      "autotuned item %d" % s_)
    # the same layout again hits the cache and keeps the choice
    _, batch2, _, _ = _ensemble(env, recipe, tile_cells="auto")
    assert batch2.tile_cells == batch.tile_cells

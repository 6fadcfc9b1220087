"""GPU parity of the bitruncated (pluri-Gaussian) facies map (Sec. 3.1,
Appendix B `bitruncated`): two fields on generator streams 0 and 1 of one
seed, binned by t and s, regions merged by a rule, against the FP64 oracle."""
import math

import numpy as np
import pytest

from helpers import FACIES_BAND_SIGMA, check_forward, gpu_env, oracle_field, oracle_modes, to_dev

pytestmark = pytest.mark.gpu


def test_bitruncated_matches_oracle():
    torch = gpu_env()
    from oracle import field as of
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    cells = W.grid_centres((96, 80))
    plan = F.CellPlan(*to_dev(torch, cells))
    p1 = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=700, seed=31)
    p2 = F.FieldParams(family="exponential", sigma2=2.0, mean=0.5, ell=(0.2, 0.1), dim=2, n_modes=900, seed=31)
    pg = F.PluriGaussianField(p1, p2)
    t = [-0.5, 0.7]
    s = [0.2]
    rule = [[0, 1], [2, 1], [3, 3]]  # six Cartesian regions merged into four facies
    values = [1e-12, 5e-12, 2e-11, 1e-13]
    out = pg.synth(plan, t, s, rule, values)
    torch.cuda.synchronize()
    assert plan.status() == 0
    m1 = oracle_modes("gaussian", 1.0, (0.1, 0.1), 2, 700, 31, stream=0)
    m2 = oracle_modes("exponential", 2.0, (0.2, 0.1), 2, 900, 31, stream=1)
    y1 = oracle_field(m1, 0.0, cells)
    y2 = oracle_field(m2, 0.5, cells)
    check_forward(out["Y1"].cpu().numpy(), y1, 1.0, "field 1")
    check_forward(out["Y2"].cpu().numpy(), y2, math.sqrt(2.0), "field 2")
    want = of.bitruncated(y1, y2, t, s, rule)
    got = out["facies"].cpu().numpy()
    d1 = np.min(np.abs(y1[:, None] - np.asarray(t)[None, :]), axis=1)
    d2 = np.min(np.abs(y2[:, None] - np.asarray(s)[None, :]), axis=1)
    band = (d1 <= FACIES_BAND_SIGMA * 1.0) | (d2 <= FACIES_BAND_SIGMA * math.sqrt(2.0))
    assert np.array_equal(got[~band], want[~band])
    assert np.array_equal(out["prop"].cpu().numpy()[~band], np.asarray(values, dtype=np.float32)[want[~band]])
    assert len(np.unique(got)) == 4

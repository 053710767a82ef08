"""Full-physics acceptance on the headline configuration: the robust
influence-matrix plan on the synthetic head (three fields with range shifter
and brass apertures through skull, brain and air cavities; Sec. 2.D.3,
Sec. 2.E), GPU against the FP64 oracle with independent seeds.

Plan: every 20th spot of the benchmarked plan (261 spots, all three fields),
three scenarios -- nominal, a 3 mm isocentre shift along y, and the same
shift with the stopping-power ratios scaled by 1.035.  For each scenario the
composite is the dose of 40 histories per spot: on the GPU the
influence-matrix columns (dose per primary, threshold 0) times 40, summed by
the library's own sparse product; in the oracle its dose grid.

Acceptance (reading c22 of the full-mode criterion): 100 batches per side of
the same size; per voxel, z = |mean_gpu - mean_oracle| / sqrt(se_gpu^2 +
se_oracle^2) over tissue voxels at or above 10 % of the maximum; at most
0.5 % of them beyond 3 and none beyond 5.  Equal batch sizes matter: a
voxel's batch dose is right-skewed at 10^4 histories, and unequal batches
bias z upward.  Gamma 2 %/2 mm/10 % >= 99.5 % with the GPU composite of
40,000 histories per spot as the reference (about 1 % uncertainty in the
high-dose region) and the oracle's 4,000 per spot (about 3 %) as the
evaluated dose.  Doses count inside the tissue mask only: in the air around
and inside the head, dose-to-medium of a few deposits exceeds the tissue
maximum by orders of magnitude and would set the threshold."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STRIDE = 20
SCEN_IDX = (0, 3, 9)
NB, NH = 100, 40                  # batches per side, histories per spot per batch
REF_CALLS, REF_NH = 20, 2000      # GPU gamma reference: 40,000 histories per spot


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


class _Moments:
    """Running sum and sum of squares of batch doses (FP64): the mean and
    its standard error over the batches."""

    def __init__(self, n):
        self.n, self.s, self.ss = 0, np.zeros(n), np.zeros(n)

    def add(self, d):
        self.n += 1
        self.s += d
        self.ss += d * d

    def mean_se(self):
        m = self.s / self.n
        var = np.maximum(self.ss - self.n * m * m, 0.0) / (self.n - 1)
        return m, np.sqrt(var / self.n)


def _gpu_composites(eng, sub, scens, nh, seed, torch):
    from paper_2307_01416_gb300 import vpmc
    s = sub.copy()
    s["n_hist"] = nh
    mats, st = eng.influence_matrix(s, scens, W.Options(seed=seed), rel_threshold=0.0)
    assert st["errors"] == 0
    x = torch.full((len(s),), float(nh), dtype=torch.float32, device="cuda")
    return [vpmc.weights_dose(m, x).double().cpu().numpy() for m in mats]


def test_head_plan_full_physics_statistical(torch_cuda):
    torch = torch_cuda
    from paper_2307_01416_gb300 import vpmc
    pb, spots, _, _ = W.im_set_plan()
    idx = np.arange(0, len(spots), STRIDE)
    sub = spots[idx].copy()
    all_scens = W.robust_scenarios()
    scens = [all_scens[i] for i in SCEN_IDX]
    assert scens[1].shift == (0.0, 3.0, 0.0) and scens[2].shift == (0.0, 3.0, 0.0)
    assert scens[1].spr_scale == 1.0 and scens[2].spr_scale == pytest.approx(1.035)
    mask = W.tissue_mask(pb)
    rho = O.scoring_density(pb)
    g = pb.scoring
    shp = (g.shape[2], g.shape[1], g.shape[0])

    eng = vpmc.Engine(pb)
    gb = [_Moments(g.nvox) for _ in scens]
    for b in range(NB):
        for k, d in enumerate(_gpu_composites(eng, sub, scens, NH, 10_000 + b, torch)):
            gb[k].add(np.where(mask, d, 0.0))
    ref = [np.zeros(g.nvox) for _ in scens]
    for b in range(REF_CALLS):
        for k, d in enumerate(_gpu_composites(eng, sub, scens, REF_NH, 50_000 + b, torch)):
            ref[k] += np.where(mask, d, 0.0) * (NH / REF_NH / REF_CALLS)
    eng.close()

    sp = O.oracle_spots(sub, spot_keys=idx, n_hist=np.full(len(idx), NH))
    results = []
    for k, sc in enumerate(scens):
        ob = _Moments(g.nvox)
        for b in range(NB):
            q, tl, _ = O.run(pb, sp, sc, W.Options(seed=90_000 + b))
            assert tl["errors"] == 0
            ob.add(np.where(mask, O.dose_from_q(pb, q, 24, rho), 0.0))
        (mg, sg), (mo, so) = gb[k].mean_se(), ob.mean_se()
        sel = ref[k] >= 0.1 * ref[k].max()
        z = np.abs(mg - mo)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2)
        gam = O.gamma_pass_rate(ref[k].reshape(shp), mo.reshape(shp), g.spacing)
        # the GPU reference against the GPU batches' mean: same engine, same physics
        gam_gg = O.gamma_pass_rate(ref[k].reshape(shp), mg.reshape(shp), g.spacing)
        results.append((k, int(sel.sum()), float(np.mean(z > 3.0)), float(z.max()), gam, gam_gg))
    for k, nsel, frac3, zmax, gam, gam_gg in results:
        assert nsel > 5000, results
        assert frac3 <= 0.005 and zmax < 5.0, results
        assert gam >= 99.5, results

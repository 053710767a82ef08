"""Energy-layer-specific (dynamic) apertures (the authors' future work,
Sec. 4): one beam entry per (field, energy layer), each with the target's
cross-section at the layer's depth plus the margin as its opening.  On the
GPU against the oracle: per history in deterministic mode on the head plan,
with divergent walls too; the influence-matrix columns of a plan with many
entries summing to its dose; and the intended effect: less dose in the ring
around the target for the same spots."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W
from tests.test_gpu_parity import _dense, _per_history_parity

pytestmark = pytest.mark.gpu

DET = W.Options(seed=2718, mcs=False, straggling=False, nuclear=True)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _subset(spots, every, n_hist=None):
    sub = spots[::every].copy()
    if n_hist is not None:
        sub["n_hist"] = n_hist
    return sub


@pytest.mark.parametrize("sad", [0.0, 2000.0], ids=["parallel", "divergent"])
def test_dynamic_aperture_head_per_history(torch_cuda, sad):
    pb, spots, _, _ = W.head_plan(8.4, dynamic_aperture=True, ap_sad=sad)
    assert len(pb.beams) > 16
    sub = _subset(spots, 17, n_hist=60)
    assert len(np.unique(sub["beam"])) > 16
    _per_history_parity(pb, sub, W.Scenario((1.5, -2.0, 0.5), 1.02), DET, max_flagged=0.03)


def test_dynamic_aperture_columns_sum_to_dose(torch_cuda):
    from paper_2307_01416_gb300 import vpmc
    pb, spots, _, _ = W.head_plan(8.4, dynamic_aperture=True)
    sub = _subset(spots, 23, n_hist=300)
    op = W.Options(seed=12)
    eng = vpmc.Engine(pb)
    mats, st = eng.influence_matrix(sub, [W.Scenario()], op, rel_threshold=0.0)
    dose, _, _ = eng.run_spots(sub, W.Scenario(), op)
    eng.close()
    g = _dense(mats[0]) * sub["n_hist"][None, :].astype(np.float64)
    d = dose.cpu().numpy().ravel().astype(np.float64)
    assert np.allclose(g.sum(axis=1), d, rtol=1e-5, atol=1e-6 * d.max())


def test_dynamic_aperture_spares_the_ring(torch_cuda):
    """Same spots, seeds and histories through the static and the dynamic
    apertures (full physics): the mean dose in the 10 mm ring around the
    target drops by more than 5 %, and so does the dose outside the ring
    and the target; the target keeps at least 80 % of its mean dose (the
    layers' openings follow the target's cross-section plus 5 mm)."""
    from paper_2307_01416_gb300 import vpmc
    res = {}
    for dyn in (False, True):
        pb, spots, center, r_t = W.head_plan(8.4, dynamic_aperture=dyn)
        cls = W.structure_classes(pb.scoring, center, r_t)
        sub = _subset(spots, 3)
        eng = vpmc.Engine(pb)
        d, st, _ = eng.run_spots(sub, W.Scenario(), W.Options(seed=99))
        eng.close()
        assert st["errors"] == 0
        d = d.cpu().numpy().ravel().astype(np.float64)
        rho = O.scoring_density(pb)
        body = rho > 0.5
        res[dyn] = (d[cls == 1].mean(), d[cls == 2].mean(), d[(cls == 0) & body].sum())
    assert res[True][0] >= 0.8 * res[False][0], res
    assert res[True][1] < 0.95 * res[False][1], res
    assert res[True][2] < 0.95 * res[False][2], res

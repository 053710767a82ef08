"""Divergent aperture walls (the authors' next step, Sec. 4) on the GPU
against the oracle: per history in deterministic mode and statistically in
full physics, for a strongly divergent block (virtual source 300 mm above
the isocentre: the opening grows by 15 % through the block) and a realistic
one (2000 mm), with and without the range shifter; and the refusal of the
learned surrogate, which is trained on parallel walls."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W
from tests.test_gpu_parity import _per_history_parity, _statistical_parity

pytestmark = pytest.mark.gpu

DET = W.Options(seed=4321, mcs=False, straggling=False, nuclear=True)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _divergent_case(sad, rs, opening=12.0, hist_per_layer=4000, max_layers=3, shape=(40, 40, 80)):
    pb, spots = W.water_aperture_case(opening, rs, hist_per_layer=hist_per_layer, max_layers=max_layers,
                                      shape=shape, spacing=(2.0, 2.0, 2.0))
    pb.beams[0].ap_sad = sad
    return pb, spots


@pytest.mark.parametrize("rs", [False, True], ids=["AP", "APRS"])
@pytest.mark.parametrize("sad", [300.0, 2000.0])
def test_divergent_aperture_per_history(torch_cuda, sad, rs):
    pb, spots = _divergent_case(sad, rs)
    # protons moving along a tilted wall approach it gradually, so more step
    # starts fall within 10 um of it than with parallel walls (1.8 % at 300 mm)
    _, st, rec, _, orec = _per_history_parity(pb, spots, W.Scenario(), DET, max_flagged=0.03)
    assert st["e_aperture"] > 0.05 * st["e_in"]


def test_divergence_changes_the_transmission(torch_cuda):
    """The same spots through a parallel and a strongly divergent block: the
    opening at the entrance shrinks by 15 %, so fewer protons pass, on the
    GPU as in the oracle."""
    from paper_2307_01416_gb300 import vpmc
    out = {}
    for sad in (0.0, 300.0):
        pb, spots = _divergent_case(sad, False)
        eng = vpmc.Engine(pb)
        _, st, rec = eng.run_spots(spots, W.Scenario(), DET, records=int(spots["n_hist"].sum()))
        eng.close()
        _, tl, orec = O.run(pb, O.oracle_spots(spots), W.Scenario(), DET, records=int(spots["n_hist"].sum()))
        out[sad] = (np.mean(rec["fate"] != O.FATE_AP), np.mean(orec["fate"] != O.FATE_AP))
    assert out[300.0][0] < out[0.0][0] - 0.015           # oracle: 0.141 -> 0.120
    for sad in out:
        assert abs(out[sad][0] - out[sad][1]) < 2e-3


def test_divergent_aperture_full_physics_statistical(torch_cuda):
    pb, spots = _divergent_case(300.0, True, opening=20.0, hist_per_layer=6000, max_layers=2, shape=(50, 50, 100))
    frac3, zmax, gam, nsel = _statistical_parity(pb, spots, 3000, 7000)
    assert nsel > 200
    assert frac3 <= 0.005 and zmax < 5.0, (frac3, zmax)
    assert gam >= 99.5, gam


def test_surrogate_refused_for_divergent_blocks(torch_cuda):
    from paper_2307_01416_gb300 import vpmc
    pb, spots = _divergent_case(2000.0, False, hist_per_layer=100, max_layers=1)
    eng = vpmc.Engine(pb)
    eng.surrogate_init(1)
    with pytest.raises(RuntimeError):
        eng.run_spots(spots, W.Scenario(), W.Options(seed=1, surrogate=True))
    d, st, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=1))
    assert st["errors"] == 0
    eng.close()

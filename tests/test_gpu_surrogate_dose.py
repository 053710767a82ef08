"""Dose error of the learned aperture surrogate against the plain aperture
transport (the learned part is pinned by the plain path, not by the paper).

The network is trained on the GPU from plain training tracks, then each case
runs plain and surrogate transport in 8 paired batches.  A pair shares its
seed, so histories that never enter the brass are identical in both and the
difference isolates the surrogate.  Inside the 10 % isodose (tissue voxels,
density >= 0.5 g/cc) the largest voxel error of the batch mean must stay
within 1 % of the maximum dose, the mean error within 0.5 %, and the
2 %/2 mm/10 % gamma pass rate at or above 99.5 %."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weights():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2307_01416_gb300 import vpmc
    w, losses = vpmc.train_surrogate(tracks_per_beam=12_500_000, epochs=7, batch=16384, lr=2e-3, lr_min=2e-5)
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
    return w


def _paired(pb, spots, w, nb=8, seed=4242, scen=None, eng=None):
    from paper_2307_01416_gb300 import vpmc
    scen = scen or W.Scenario()
    e = eng or vpmc.Engine(pb)
    e.surrogate_set_weights(w)
    refs, diffs, ms = [], [], []
    for b in range(nb):
        d0, s0, _ = e.run_spots(spots, scen, W.Options(seed=seed + 17 * b))
        d1, s1, _ = e.run_spots(spots, scen, W.Options(seed=seed + 17 * b, surrogate=True))
        a0 = d0.cpu().numpy().astype(np.float64)
        refs.append(a0)
        diffs.append(d1.cpu().numpy().astype(np.float64) - a0)
        ms.append((s0["ms"], s1["ms"]))
        assert s1["errors"] == 0
    if eng is None:
        e.close()
    D, dd = np.mean(refs, 0), np.mean(diffs, 0)
    rho = O.scoring_density(pb).reshape(D.shape)
    m = (D >= 0.1 * D.max()) & (rho >= 0.5)
    dmax = D[m].max()
    return {"max_err": np.abs(dd)[m].max() / dmax, "mean_err": dd[m].sum() / D[m].sum(),
            "gamma": O.gamma_pass_rate(D, D + dd, pb.scoring.spacing), "ms": np.median(np.array(ms), 0)}


def test_head_plan_dose_error_all_scenarios(weights):
    """Every 10th spot of the benchmarked plan in each of the 13 robust
    scenarios (shifts move the field across skull and cavities, range scaling
    moves the Bragg peaks)."""
    from paper_2307_01416_gb300 import vpmc
    pb, spots, _, _ = W.im_set_plan()
    eng = vpmc.Engine(pb)
    out = []
    for k, sc in enumerate(W.robust_scenarios()):
        r = _paired(pb, spots[::10], weights, nb=6, scen=sc, eng=eng)
        out.append((k, r["max_err"], r["mean_err"], r["gamma"]))
    eng.close()
    for k, max_err, mean_err, gam in out:
        assert max_err <= 0.01, out
        assert abs(mean_err) <= 0.005, out
        assert gam >= 99.5, out


@pytest.mark.parametrize("opening", [10.0, 20.0])
def test_beams_without_range_shifter_keep_the_plain_path(weights, opening):
    """Without a range shifter the network's dose error reached 1.1-2.2 % of
    the maximum (10 and 20 mm openings, different trainings): such beams
    take the plain aperture transport with opts.surrogate = 1, so the
    patient dose is the plain one, bit for bit."""
    from paper_2307_01416_gb300 import vpmc
    pb, spots = W.water_aperture_case(opening, False, hist_per_layer=20_000, max_layers=4)
    e = vpmc.Engine(pb)
    e.surrogate_set_weights(weights)
    d0, s0, _ = e.run_spots(spots, W.Scenario(), W.Options(seed=77))
    d1, s1, _ = e.run_spots(spots, W.Scenario(), W.Options(seed=77, surrogate=True))
    e.close()
    assert np.array_equal(d0.cpu().numpy(), d1.cpu().numpy())
    assert s0["e_dep"] == s1["e_dep"] and s0["e_leak"] == s1["e_leak"]
    # brass entries that can reach neither the opening nor the exit face are
    # absorbed at once on the surrogate path: the same energy, fewer steps
    assert abs(s1["e_aperture"] / s0["e_aperture"] - 1.0) < 1e-6


@pytest.mark.parametrize("opening", [10.0, 20.0, 40.0])
def test_water_aperture_dose_error(weights, opening):
    pb, spots = W.water_aperture_case(opening, True, hist_per_layer=300_000)
    r = _paired(pb, spots, weights)
    assert r["max_err"] <= 0.01, r
    assert abs(r["mean_err"]) <= 0.005, r
    assert r["gamma"] >= 99.5, r

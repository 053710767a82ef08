"""Single-beamlet edge sweep (Sec. 2.D.1): one beamlet along the beam axis
centred on the edge of a 1 cm opening in 30 mm brass, water phantom on a
1 mm grid, with (APRS) and without (AP) the 45 mm-WET range shifter, at the
paper's 97 energies from 71.3 to 228.8 MeV.  The paper compares its engine
with MCsquare; here the GPU path is compared with the FP64 oracle.

* the three energies the paper illustrates (82.0, 140.2, 228.8 MeV) on both
  machines: per history in deterministic mode, and statistically in full
  physics (3D dose within the combined batch uncertainty, 2%/2mm/10% gamma,
  integrated depth dose);
* all 97 x 2 beamlets on the GPU: properties that hold at any size (energy
  conservation, the distal edge of the depth dose moving deeper with energy,
  the range shifter pulling it back by about its water-equivalent
  thickness, the block stopping the protons that hit it below about
  155 MeV)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W
from tests.test_gpu_parity import _per_history_parity

pytestmark = pytest.mark.gpu

PAPER_ENERGIES = (82.0, 140.2, 228.8)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _depth_mm(energy, rs):
    return float(np.ceil(W.bk_range_for_energy(energy) - (45.0 if rs else 0.0) + 20.0))


@pytest.mark.parametrize("rs", [False, True], ids=["AP", "APRS"])
@pytest.mark.parametrize("energy", PAPER_ENERGIES)
def test_edge_beamlet_per_history(torch_cuda, energy, rs):
    pb = W.edge_beamlet_problem(rs, depth_mm=_depth_mm(energy, rs))
    spots = W.edge_beamlet_spot(energy, 3000)
    det = W.Options(seed=2024, mcs=False, straggling=False, nuclear=True)
    _, st, rec, _, orec = _per_history_parity(pb, spots, W.Scenario(), det, max_flagged=0.02)
    # the beamlet is centred on the rim of the opening: about 70 % of it meets
    # the brass, which stops it below about 155 MeV (after the range shifter
    # for APRS) and lets it through, slowed down, at the top energy
    stopped = np.mean(orec["fate"] == O.FATE_AP)
    assert np.mean(rec["fate"] == O.FATE_AP) == pytest.approx(stopped, abs=1e-3)
    if energy < 150.0:
        assert 0.5 < stopped < 0.85, stopped
    else:
        assert stopped < 0.2, stopped
    assert st["e_aperture"] > 0.1 * st["e_in"]


@pytest.mark.parametrize("rs", [False, True], ids=["AP", "APRS"])
@pytest.mark.parametrize("energy", PAPER_ENERGIES)
def test_edge_beamlet_full_physics_statistical(torch_cuda, energy, rs):
    """Doses per history, 20 batches per side.  Per voxel, above 10 % of the
    maximum on the 1 mm grid: GPU batches of 1e4 histories against oracle
    batches of 1e4, |z| (difference over the combined batch standard error)
    above 3 in at most 1 % of the voxels and above 6 nowhere.  The batch
    sizes are equal because a voxel's batch dose is right-skewed at this size:
    against a 10x larger batch the small batches' low draws pair with low
    standard errors and bias z upward (GPU 1e5 batches against GPU 1e4 batches
    put 5.9 % of the voxels above 3; equal GPU and oracle batches put 0.2 %).
    Integrated depth dose: GPU batches of 1e5 against the oracle's, within 5
    combined standard errors in every 1 mm bin (a bin sums thousands of
    voxels), peaks within 1 mm.  The paper's 2%/2mm/10% gamma needs both
    doses below 0.5 % uncertainty; with the oracle at 2e5 histories (6.6 %
    per-voxel uncertainty near the peak) it measures the oracle's noise:
    oracle against oracle at these sizes gave 94.6-99.6 %, GPU against oracle
    92.4-99.8 % (lowest at 228.8 MeV with the shifter, the widest low-dose
    region), so gamma is asserted at >= 90 % only as a coarse check."""
    from paper_2307_01416_gb300 import vpmc
    pb = W.edge_beamlet_problem(rs, depth_mm=_depth_mm(energy, rs))
    rho = O.scoring_density(pb)
    g = pb.scoring
    shp = (g.shape[2], g.shape[1], g.shape[0])
    eng = vpmc.Engine(pb)
    big, small, orc = [], [], []
    for b in range(20):
        d, st, _ = eng.run_spots(W.edge_beamlet_spot(energy, 100_000), W.Scenario(), W.Options(seed=7000 + b))
        assert st["errors"] == 0
        big.append(d.cpu().numpy().astype(np.float64).ravel() / 100_000)
        d, st, _ = eng.run_spots(W.edge_beamlet_spot(energy, 10_000), W.Scenario(), W.Options(seed=8000 + b))
        assert st["errors"] == 0
        small.append(d.cpu().numpy().astype(np.float64).ravel() / 10_000)
        q, tl, _ = O.run(pb, O.oracle_spots(W.edge_beamlet_spot(energy, 10_000)), W.Scenario(),
                         W.Options(seed=9000 + b))
        assert tl["errors"] == 0
        orc.append(O.dose_from_q(pb, q, 24, rho) / 10_000)
    eng.close()
    big, small, orc = np.stack(big), np.stack(small), np.stack(orc)
    n = orc.shape[0]
    mo, so = orc.mean(0), orc.std(0, ddof=1) / math.sqrt(n)
    ms, ss = small.mean(0), small.std(0, ddof=1) / math.sqrt(n)
    sel = mo >= 0.1 * mo.max()
    assert sel.sum() > 500
    z = np.abs(ms - mo)[sel] / np.sqrt(ss[sel] ** 2 + so[sel] ** 2)
    assert np.mean(z > 3.0) <= 0.01 and z.max() < 6.0, (np.mean(z > 3.0), z.max())
    mb = big.mean(0)
    gam = O.gamma_pass_rate(mo.reshape(shp), mb.reshape(shp), g.spacing)
    assert gam >= 90.0, gam
    # integrated depth dose per 1 mm bin (dose x density: energy per depth), batch by batch
    ib = (big * rho).reshape(n, *shp).sum(axis=(2, 3))
    io = (orc * rho).reshape(n, *shp).sum(axis=(2, 3))
    mib, mio = ib.mean(0), io.mean(0)
    se = np.sqrt(ib.var(0, ddof=1) / n + io.var(0, ddof=1) / n)
    keep = mio >= 0.1 * mio.max()
    zi = np.abs(mib - mio)[keep] / se[keep]
    assert zi.max() < 5.0, zi.max()
    assert abs(int(np.argmax(mib)) - int(np.argmax(mio))) <= 1


def _distal_depth_mm(dose, pb, level=0.2):
    """Deepest depth (mm) whose integrated depth dose is at least level x its
    maximum: the beamlet's open part sets it even when the part that went
    through the brass makes the higher, shallower peak."""
    g = pb.scoring
    idd = dose.reshape(g.shape[2], g.shape[1], g.shape[0]).sum(axis=(1, 2))
    if not idd.max() > 0.0:
        return 0.0
    return (np.flatnonzero(idd >= level * idd.max())[-1] + 0.5) * g.spacing[2]


def test_sweep_97_energies_both_machines(torch_cuda):
    """All 194 beamlets (1e5 histories each) on one geometry per machine."""
    from paper_2307_01416_gb300 import vpmc
    energies = W.machine_energies()
    assert energies.size == 97 and energies[0] == 71.3 and energies[-1] == 228.8
    peaks, frac_ap, reach = {}, {}, {}
    for rs in (False, True):
        pb = W.edge_beamlet_problem(rs)
        eng = vpmc.Engine(pb)
        pk, fa, rw = [], [], []
        for e in energies:
            d, st, _ = eng.run_spots(W.edge_beamlet_spot(e, 100_000), W.Scenario(), W.Options(seed=11))
            assert st["errors"] == 0
            tot = st["e_dep"] + st["e_leak"] + st["e_rs"] + st["e_aperture"]
            assert abs(tot / st["e_in"] - 1.0) < 1e-6
            pk.append(_distal_depth_mm(d.cpu().numpy().astype(np.float64), pb))
            fa.append(st["e_aperture"] / st["e_in"])
            rw.append(st["e_dep"] / st["e_in"] > 0.01)
        eng.close()
        peaks[rs], frac_ap[rs], reach[rs] = np.array(pk), np.array(fa), np.array(rw)
    # every AP beamlet reaches the water; with the 45 mm-WET shifter the lowest
    # energies (water range below the shifter's) stop in it
    assert reach[False].all()
    assert not reach[True][0] and reach[True][energies > 90.0].all()
    for rs in (False, True):
        # the distal edge moves deeper with energy (1 mm bins), over the beamlets that reach the water
        p = peaks[rs][reach[rs]]
        assert np.all(np.diff(p) >= -1.0), p
        assert p[-1] - p[0] > 200.0
    # the range shifter pulls it back by ~45 mm of water (PMMA WET, 1 mm bins)
    deep = (peaks[False] > 60.0) & reach[True]
    shift = peaks[False][deep] - peaks[True][deep]
    assert np.all(np.abs(shift - 45.0) <= 3.0), shift
    # below ~155 MeV the 30 mm block stops what hits it: about 70 % of the beamlet's energy
    low = energies < 150.0
    assert np.all((frac_ap[False][low] > 0.55) & (frac_ap[False][low] < 0.85)), frac_ap[False][low]
    # at the top energies part of it goes through the brass and deposits downstream
    assert frac_ap[False][-1] < frac_ap[False][low].min()

"""The benchmarked workload at full size, in the launch configuration the
benchmark times (autotuned, all 13 scenarios of the head plan, 5,220 spots
per scenario, full physics, seed of the benchmark's first rank):

* properties that hold at any size: CSR structure, the column threshold
  rule, energy bookkeeping, and the columns x histories summing to the dose
  of the same spots;
* outputs the oracle computes one by one: the columns of sampled spots in
  two scenarios, and the histories of sampled spots.  The random numbers are
  counter-based (key: seed and spot; counter: history, step, slot), so the
  oracle draws the same numbers for the same history; only histories whose
  path is ill-conditioned in FP32 (a step-count change re-aligns every later
  draw) differ, and the comparison is built on that."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SEED = 1234                     # bench.rank_seed(0)
SAMPLE = (97, 1411, 2050, 3333, 4780)
SCEN_SAMPLE = (0, 9)


@pytest.fixture(scope="module")
def fullset():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2307_01416_gb300 import vpmc
    pb, spots, _, _ = W.im_set_plan()
    scens = W.robust_scenarios()
    eng = vpmc.Engine(pb)
    mats, st = eng.influence_matrix(spots, scens, W.Options(seed=SEED))
    dose, _, _ = eng.run_spots(spots, scens[0], W.Options(seed=SEED))
    eng.close()
    return pb, spots, scens, mats, st, dose.cpu().numpy().ravel().astype(np.float64)


def _column(m, j):
    import torch
    sel = torch.nonzero(m["col"] == j).flatten()
    rows = torch.searchsorted(m["row_ptr"], sel, right=True) - 1
    out = np.zeros(int(m["shape"][0]))
    out[rows.cpu().numpy()] = m["val"][sel].cpu().numpy()
    return out


def test_structure_threshold_and_energy(fullset):
    pb, spots, scens, mats, st, _ = fullset
    assert len(mats) == 13 and st["errors"] == 0
    tot = st["e_dep"] + st["e_leak"] + st["e_rs"] + st["e_aperture"]
    assert abs(tot / st["e_in"] - 1.0) < 1e-6
    assert st["histories"] == 13 * int(spots["n_hist"].sum())
    for m in mats:
        rp = m["row_ptr"].cpu().numpy()
        col = m["col"].cpu().numpy()
        val = m["val"].cpu().numpy()
        assert m["shape"] == (pb.scoring.nvox, len(spots))
        assert rp[0] == 0 and rp[-1] == val.size and np.all(np.diff(rp) >= 0)
        assert col.min() >= 0 and col.max() < len(spots) and np.all(np.isfinite(val)) and val.min() > 0
        # per column, no kept entry below 1e-4 of the column maximum
        cmax = np.zeros(len(spots), dtype=np.float32)
        np.maximum.at(cmax, col, val)
        assert np.all(val >= 1e-4 * cmax[col] * (1 - 1e-6))


def test_column_boxes_hold_the_deposits(fullset):
    """Each spot's column box ends at its energy layer's reach along the field
    (rays marched through the CT per scenario, water range behind the range
    shifter + 5 % + 3 mm).  A deposit beyond its box is recorded and merged
    into the CSR, so the bound changes no value (the columns-sum-to-dose and
    sampled-column tests hold with it); it must only add few records.  The
    records are the lateral tails beyond the boxes' 25 mm margin: measured
    4,335,001 per set with full-depth boxes and 4,349,642 with the cut ones
    (2.7e-5 of the patient steps), while the scratch fell from 131.7 to
    88.2 GB.  Bound: 5e-5 of the patient steps."""
    pb, spots, scens, mats, st, _ = fullset
    patient_steps = st["steps"] - st["steps_rs"] - st["steps_aperture"]
    assert st["ovf_records"] < 5e-5 * patient_steps, (st["ovf_records"], patient_steps)
    assert st["scratch_bytes"] > 0


def test_columns_sum_to_the_dose(fullset):
    """Nominal scenario: with no entry dropped (threshold 0) the columns x
    n_hist summed over the spots equal the dose of the same spots and seed to
    1e-5 above 10 % of its maximum (measured 9e-8: FP32 rounding of the
    column values); with the benchmark's threshold the sum stays below the
    dose (only entries are dropped)."""
    from paper_2307_01416_gb300 import vpmc
    pb, spots, scens, mats, st, dose = fullset
    eng = vpmc.Engine(pb)
    exact, _ = eng.influence_matrix(spots, [scens[0]], W.Options(seed=SEED), rel_threshold=0.0)
    eng.close()
    sel = dose >= 0.1 * dose.max()
    assert sel.sum() > 5000
    for m, tol_lo, tol_hi in ((exact[0], 1e-5, 1e-5), (mats[0], 0.05, 1e-5)):
        col = m["col"].cpu().numpy()
        val = m["val"].cpu().numpy().astype(np.float64)
        rows = np.repeat(np.arange(m["shape"][0]), np.diff(m["row_ptr"].cpu().numpy()))
        tot = np.zeros(m["shape"][0])
        np.add.at(tot, rows, val * spots["n_hist"][col].astype(np.float64))
        rel = (tot[sel] - dose[sel]) / dose[sel]
        assert rel.min() > -tol_lo and rel.max() < tol_hi, (rel.min(), rel.max())


def test_sampled_columns_against_the_oracle(fullset):
    """The columns of five spots in two scenarios, recomputed by the oracle
    with the same seed and spot keys (the same random numbers), and with the
    next seed (an independent sample): against the same-seed oracle the
    column's energy (dose x mass) agrees to 1e-3 and, above 10 % of the
    column maximum, the median voxel to 5e-3 and to a twentieth of the
    independent sample's median difference.  Measured: energy within 4e-4,
    medians 2e-7 to 2e-3, against 0.11 to 1.0 between independent samples."""
    pb, spots, scens, mats, st, _ = fullset
    rho = O.scoring_density(pb)
    vol = pb.scoring.voxel_mm3 * 1e-3
    idx = np.array(SAMPLE)
    sub = spots[idx]
    for s in SCEN_SAMPLE:
        ds = []
        for seed in (SEED, SEED + 1):
            q, tl, _ = O.run(pb, O.oracle_spots(sub, spot_keys=idx), scens[s], W.Options(seed=seed), mode=1)
            d = q.astype(np.float64) * 2.0 ** -24 * O.MEV_PER_G_TO_GY / vol / rho[None, :]
            ds.append(d / sub["n_hist"].astype(np.float64)[:, None])
        for k, j in enumerate(idx):
            o, o2 = ds[0][k], ds[1][k]
            if o.max() <= 0.0:
                continue
            o = np.where(o >= 1e-4 * o.max(), o, 0.0)
            o2 = np.where(o2 >= 1e-4 * o2.max(), o2, 0.0)
            g = _column(mats[s], int(j))
            assert abs((g * rho).sum() / (o * rho).sum() - 1.0) < 1e-3, (s, j)
            sel = o >= 0.1 * o.max()
            same = np.median(np.abs(g[sel] - o[sel]) / o[sel])
            indep = np.median(np.abs(o2[sel] - o[sel]) / o[sel])
            assert same < 5e-3 and same < 0.05 * indep, (s, j, same, indep)


def test_sampled_histories_full_physics(fullset):
    """The histories of the sampled spots (nominal scenario, full physics,
    same random numbers as the oracle): fates agree for 99.9 %, scored
    energies to 1e-4 for 99.5 %, end points to 1e-3 of the track for 95 %.
    Measured: 99.99 %, 99.8 %, 97.3 %; 91 % keep the oracle's step count
    exactly -- a step-count change (an FP32 tie of two step limits)
    re-aligns every later draw, after which the history is an independent
    sample of the same distribution."""
    from paper_2307_01416_gb300 import vpmc
    pb, spots, scens, mats, st, _ = fullset
    only = spots.copy()
    keep = np.zeros(len(spots), dtype=bool)
    keep[list(SAMPLE)] = True
    only["n_hist"] = np.where(keep, np.minimum(spots["n_hist"], 3000), 0)
    n = int(only["n_hist"].sum())
    # the whole spot list with zero histories elsewhere keeps every spot's RNG
    # key; the GPU takes the plain brass steps of the oracle (no range rejection)
    eng = vpmc.Engine(pb)
    _, _, rec = eng.run_spots(only, scens[0], W.Options(seed=SEED, range_rejection=False), records=n)
    eng.close()
    _, _, orec = O.run(pb, O.oracle_spots(only), scens[0], W.Options(seed=SEED), records=n)
    fate = rec["fate"] == orec["fate"]
    energy = np.abs(rec["e_dep"] - orec["e_dep"]) / np.maximum(np.abs(orec["e_dep"]), 1.0) < 1e-4
    pos = np.linalg.norm(rec["pos"] - orec["pos"], axis=1) / np.maximum(orec["track"], 1.0) < 1e-3
    assert fate.mean() >= 0.999 and energy.mean() >= 0.995 and pos.mean() >= 0.95, (fate.mean(), energy.mean(),
                                                                                   pos.mean())


def test_the_set_reaches_half_a_percent_uncertainty(fullset):
    """The benchmarked set's histories meet the metric's 0.5 %: the batch
    estimate (10 independent runs, each a tenth of every spot's histories)
    of the nominal composite's relative standard error, averaged over the
    tissue voxels at or above half the maximum."""
    from paper_2307_01416_gb300 import uncertainty as U, vpmc
    pb, spots, scens, _, _, _ = fullset
    sub = spots.copy()
    sub["n_hist"] = U.split_histories(spots["n_hist"], 10)
    eng = vpmc.Engine(pb)
    doses = [eng.run_spots(sub, W.Scenario(), W.Options(seed=SEED + 100003 * (b + 1)))[0].reshape(-1).double()
             .cpu().numpy() for b in range(10)]
    eng.close()
    s, nvox = U.batch_sigma_rel(np.stack(doses), W.tissue_mask(pb), level=0.5)
    assert nvox > 1000
    assert 0.004 < s <= 0.005, s

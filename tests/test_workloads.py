"""The seeded input generators follow their stated recipes: the 13 robust
scenarios (Sec. 2.E), energy layers 3 mm WET apart, polygonal circular
openings (Sec. 2.D.2), the spot-size law and spot grids, the machine energies
of the edge sweep (Sec. 2.D.1), the coplanar gantry frames and the synthetic
head and its plan (Sec. 2.D.3 sizes).  These generators hold no transport
arithmetic; both the CUDA path and the oracle read their output."""
import math

import numpy as np
import pytest

from paper_2307_01416_gb300 import workloads as W


def test_thirteen_robust_scenarios():
    sc = W.robust_scenarios()
    assert len(sc) == 13
    assert sc[0].shift == (0.0, 0.0, 0.0) and sc[0].spr_scale == 1.0
    keys = {(tuple(s.shift), round(s.spr_scale, 6)) for s in sc}
    assert len(keys) == 13
    for ax in range(3):
        for sgn in (1.0, -1.0):
            shift = tuple(sgn * 3.0 if k == ax else 0.0 for k in range(3))
            assert (shift, 1.0) in keys                                  # setup error alone
            assert (shift, round(1.0 + sgn * 0.035, 6)) in keys          # with the range error of the same sign


def test_layer_energies_three_mm_wet_apart():
    e = W.layer_energies(100.0, 160.0, 3.0)
    r = W.bk_range_for_energy(e)
    assert e[0] == pytest.approx(100.0, rel=1e-12)
    assert np.allclose(np.diff(r), 3.0, rtol=0, atol=1e-9)
    assert e[-1] <= 160.0 + 1e-9
    assert W.bk_energy_for_range(r[-1] + 3.0) > 160.0
    # Bragg-Kleeman recipe: R = 0.022 mm E^1.77 and its inverse
    assert W.bk_range_for_energy(100.0) == pytest.approx(0.022 * 100.0 ** 1.77, rel=1e-12)
    assert W.bk_energy_for_range(W.bk_range_for_energy(137.0)) == pytest.approx(137.0, rel=1e-12)


def test_regular_polygon_openings():
    r, n = 10.0, 256
    p = W.regular_polygon(r, n)
    assert p.shape == (n, 2)
    assert np.allclose(np.hypot(p[:, 0], p[:, 1]), r, rtol=0, atol=1e-12)
    x, y = p[:, 0], p[:, 1]
    area = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    assert area == pytest.approx(0.5 * n * r * r * math.sin(2.0 * math.pi / n), rel=1e-12)
    # the 256-gon's area deficit against the circle is about 1e-4
    assert 0.5e-4 < 1.0 - area / (math.pi * r * r) < 1.5e-4


def test_spot_size_law_and_machine_energies():
    assert W.spot_sigma_mm(71.3) == pytest.approx(5.0)
    assert W.spot_sigma_mm(228.8) == pytest.approx(2.0)
    assert W.spot_sigma_mm(150.05) == pytest.approx(3.5)
    e = W.machine_energies()
    assert e.size == 97 and e[0] == 71.3 and e[-1] == 228.8
    assert np.allclose(np.diff(e), (228.8 - 71.3) / 96.0)


def test_spot_grid_in_disk_is_the_whole_lattice_inside():
    r, a = 13.0, 3.0
    xy = W.grid_spots_in_disk(r, a)
    assert np.all(np.hypot(xy[:, 0], xy[:, 1]) <= r + 1e-9)
    assert np.allclose(xy / a, np.round(xy / a))
    lattice = {(i, j) for i in range(-5, 6) for j in range(-5, 6) if math.hypot(a * i, a * j) <= r}
    assert {(int(round(x / a)), int(round(y / a))) for x, y in xy} == lattice


@pytest.mark.parametrize("gantry, axis", [(0.0, (0.0, 1.0, 0.0)), (90.0, (-1.0, 0.0, 0.0)), (270.0, (1.0, 0.0, 0.0))])
def test_gantry_frames(gantry, axis):
    b = W.gantry_beam(gantry, (1.0, 2.0, 3.0), 245.0)
    w, u = np.array(b.direction), np.array(b.bev_x)
    assert np.allclose(w, axis, atol=1e-15)
    assert abs(np.dot(w, u)) < 1e-15 and abs(np.linalg.norm(u) - 1.0) < 1e-15
    assert b.iso == (1.0, 2.0, 3.0)


def test_synthetic_head_ct():
    g, hu, cav = W.head_ct(1234)
    assert g.shape == (256, 256, 160) and g.spacing == (1.0, 1.0, 1.5)
    assert hu.shape == (160, 256, 256) and hu.dtype == np.int16
    x = g.centers(0)[None, None, :]
    y = g.centers(1)[None, :, None]
    z = g.centers(2)[:, None, None]
    a, b, c = W.HEAD_SEMI_AXES
    outer = (x / a) ** 2 + (y / b) ** 2 + (z / c) ** 2 <= 1.0
    inner = (x / (a - 6)) ** 2 + (y / (b - 6)) ** 2 + (z / (c - 6)) ** 2 <= 1.0
    assert np.all(hu[~outer] == -1000)
    skull = hu[outer & ~inner]
    assert skull.min() >= 900 and skull.max() <= 1500
    in_cav = np.zeros(hu.shape, dtype=bool)
    assert len(cav) == 2
    for cx, cy, cz, r in cav:
        assert 10.0 <= r <= 20.0 and cy < -20.0          # anterior brain, where the 0 deg beam enters
        in_cav |= (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= r * r
    assert np.all(hu[in_cav & inner] == -1000)
    brain = hu[inner & ~in_cav].astype(np.float64)
    assert abs(brain.mean() - 30.0) < 0.05 and abs(brain.std() - 10.0) < 0.1


def test_head_plan_sizes():
    pb, spots, center, r_t = W.head_plan(8.4)
    assert r_t == pytest.approx((3.0 * 8.4e3 / (4.0 * math.pi)) ** (1.0 / 3.0))
    assert len(pb.beams) == 3 and len(spots) == 5220
    for b in pb.beams:
        rad = np.hypot(b.polygon[:, 0], b.polygon[:, 1])
        assert b.polygon.shape == (64, 2) and np.allclose(rad, r_t + 5.0)
        assert b.rs_present and b.rs_wet == 45.0 and b.ap_thickness == 30.0 and b.ap_down_to_iso == 150.0
    assert spots["n_hist"].min() >= 1000 and spots["n_hist"].max() <= 20000
    # log-uniform: the median near sqrt(1e3 * 2e4)
    assert abs(math.log(np.median(spots["n_hist"])) - 0.5 * math.log(1000 * 20000)) < 0.1
    assert pb.scoring.spacing == (2.0, 2.0, 2.0) and pb.scoring.shape == (128, 128, 120)
    assert np.all(spots["div_mrad"] == 2.0)
    assert np.allclose(spots["sigma"], W.spot_sigma_mm(spots["energy"]))


def test_tissue_mask_follows_the_ct_at_scoring_voxel_centres():
    """A 2 mm scoring voxel is tissue when the 1 mm CT voxel at its centre
    is; air (-1000 HU) and lung-like -600 HU are not, -400 HU is."""
    g = W.Grid((8, 4, 6), (1.0, 1.0, 1.5), (0.0, 0.0, 0.0))
    hu = np.zeros((6, 4, 8), dtype=np.int16)
    hu[:, :, :4] = -1000            # x < 4 mm: air
    hu[:, :, 5] = -600              # the CT column holding the centre of scoring x-voxel 2
    hu[:3, :, 7] = -400
    sg = W.Grid((4, 2, 4), (2.0, 2.0, 2.25), (0.0, 0.0, 0.0))
    pb = W.Problem(ct=g, hu=hu, curve=W.HUCurve(), scoring=sg, beams=[])
    m = W.tissue_mask(pb).reshape(4, 2, 4)
    assert not m[:, :, :2].any()
    assert not m[:, :, 2].any()
    # scoring x-voxel 3 has its centre at 7 mm (CT column 7): -400 HU in the
    # first three CT slices (z < 4.5 mm: scoring z-voxels 0 and 1), water above
    assert m[:, :, 3].all()
    pb2, _ = W.pencil_beam_water(n_hist=1, shape=(10, 10, 10))
    assert W.tissue_mask(pb2).all()

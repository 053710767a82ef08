"""The batch estimate of a dose's statistical uncertainty and the history
rescaling that brings a plan to 0.5 % (Sec. 2.D.3), against data whose
uncertainty is known by construction."""
import math

import numpy as np
import pytest

from paper_2307_01416_gb300 import uncertainty as U


def test_known_gaussian_noise():
    """Batches D + N(0, (0.05 D)^2): the mean of 10 batches has SE/D =
    0.05/sqrt(10); the sample standard deviation of 10 values averages
    c4(10) = 0.9727 of the true one (Gaussian sampling)."""
    rng = np.random.default_rng(1)
    d = rng.uniform(0.1, 1.0, 200_000)
    b = d[None, :] * (1.0 + 0.05 * rng.standard_normal((10, d.size)))
    s, n = U.batch_sigma_rel(b, level=0.5)
    c4 = math.sqrt(2.0 / 9.0) * math.gamma(5.0) / math.gamma(4.5)
    assert abs(c4 - 0.9727) < 1e-4
    assert n > 50_000
    assert s == pytest.approx(0.05 / math.sqrt(10) * c4, rel=0.01)


def test_poisson_counting_and_the_inverse_square_root_law():
    """A voxel that collects Poisson(lambda) equal deposits per batch has a
    relative standard error 1/sqrt(B lambda) on the mean of B batches;
    scaling the histories by (sigma/target)^2 brings a fresh run to target."""
    rng = np.random.default_rng(2)
    lam = rng.uniform(200.0, 400.0, 50_000)
    b = rng.poisson(lam[None, :], (20, lam.size)).astype(np.float64)
    s, _ = U.batch_sigma_rel(b, level=0.5)
    sel = lam >= 0.5 * lam.max()
    expect = np.mean(1.0 / np.sqrt(20.0 * lam[sel]))
    assert s == pytest.approx(expect, rel=0.02)
    n, f = U.histories_for_target(np.array([1000, 20000]), s, 0.005)
    assert f == pytest.approx((s / 0.005) ** 2) and n[0] == math.ceil(1000 * f)
    b2 = rng.poisson(f * lam[None, :], (20, lam.size)).astype(np.float64)
    s2, _ = U.batch_sigma_rel(b2, level=0.5)
    assert s2 == pytest.approx(0.005, rel=0.03)


def test_level_and_mask_select_the_voxels():
    """Low-dose voxels (below level x max) and voxels outside the mask (air,
    whose dose-to-medium can exceed the tissue maximum) do not count."""
    rng = np.random.default_rng(3)
    d = np.concatenate([np.full(1000, 1.0), np.full(1000, 0.1), np.full(10, 50.0)])
    noise = np.concatenate([np.full(1000, 0.01), np.full(1000, 0.5), np.full(10, 0.9)])
    b = d[None, :] * (1.0 + noise[None, :] * rng.standard_normal((40, d.size)))
    mask = np.arange(d.size) < 2000
    s, n = U.batch_sigma_rel(b, mask=mask, level=0.5)
    assert n == 1000 and s == pytest.approx(0.01 / math.sqrt(40), rel=0.1)
    with pytest.raises(ValueError):
        U.batch_sigma_rel(b[:1])


def test_batch_split_keeps_empty_spots_empty():
    assert U.split_histories(np.array([0, 1, 10, 11]), 10).tolist() == [0, 1, 1, 2]

"""Seeded optimisation problems shared by the optimiser's oracle and GPU
tests (inputs only: matrices, voxel classes, initial weights)."""
import numpy as np

from paper_2307_01416_gb300 import workloads as W

DP = 2.0

# name: (grid shape, spots, scenarios, seed, initial mean target dose / D_p)
CASES = {
    "13 scenarios, start 1.3 D_p": ((36, 36, 40), 300, 13, 11, 1.3),
    "13 scenarios, start 1.6 D_p": ((36, 36, 40), 300, 13, 11, 1.6),
    "3 scenarios, ragged grid": ((33, 29, 37), 257, 3, 5, 0.8),
}


def scipy_csr(m):
    import scipy.sparse as sp
    return sp.csr_matrix((m["val"].astype(np.float64), m["col"], m["row_ptr"]), shape=m["shape"])


def case(shape, n_spots, n_scen, seed, level, r_target=7.0, empty=2):
    """(matrices, classes, FP32 initial weights scaled so that the nominal
    scenario's mean target dose is level x D_p)."""
    mats = W.synthetic_spot_matrices(shape=shape, n_spots=n_spots, n_scen=n_scen, seed=seed, empty_spots=empty)
    cls = W.synthetic_structure_classes(shape=shape, r_target=r_target)
    x0 = np.random.default_rng(seed + 1).uniform(0.5, 1.5, n_spots)
    d = scipy_csr(mats[0]) @ x0
    return mats, cls, (x0 * level * DP / np.mean(d[cls == 1])).astype(np.float32)

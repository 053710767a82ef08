"""The 21-bit uniform lattice of a condensed-history step (reading c17).

Both engines draw the six uniforms of a step from one Philox block, 21 bits
each, u = (v + 1/2) 2^-21, so a Box-Muller normal never exceeds
sqrt(-2 ln 2^-22) = 5.5 sigma (about 3.8e-8 of a normal's probability lies
beyond).  This study reruns the oracle with the step's uniforms at 32-bit
resolution from two Philox blocks (normals up to 6.8 sigma) and checks that
the dose cannot tell them apart: a 150 MeV pencil beam in water (Sec. 2.A
physics: Highland scattering, Bohr straggling, nuclear removal), 10 batches
of 12,000 histories per lattice, compared per depth bin, in the distal
fall-off and tail, and in the lateral spread.  The streams differ, so the
comparison is statistical: combined standard errors of the batch means.
The tests have the power to see a physics change: against the same 21-bit
run with straggling off, the depth-dose z reaches 266 and the distal R20 z
246; with scattering off, the lateral second moment at 141 mm differs by
46 standard errors.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_01416_gb300 import workloads as W

NB, NH = 10, 12_000


def _batches(pb, spots, fine):
    g = pb.scoring
    out = []
    for b in range(NB):
        sp = O.oracle_spots(spots, h_begin=np.array([b * NH]), n_hist=np.array([NH]))
        q, tl, _ = O.run(pb, sp, W.Scenario(), W.Options(seed=77), fine_uniforms=fine)
        assert tl["errors"] == 0
        out.append(q.astype(np.float64).reshape(g.shape[2], g.shape[1], g.shape[0]))
    return np.stack(out)


def _mean_se(x):
    return x.mean(axis=0), x.std(axis=0, ddof=1) / np.sqrt(x.shape[0])


@pytest.fixture(scope="module")
def lattices():
    pb, spots = W.pencil_beam_water(n_hist=NH, energy=150.0)
    return pb, _batches(pb, spots, False), _batches(pb, spots, True)


def test_depth_dose_is_the_same_with_32_bit_uniforms(lattices):
    pb, a, b = lattices
    da, db = a.sum(axis=(2, 3)), b.sum(axis=(2, 3))          # (batch, depth)
    (ma, sa), (mb, sb) = _mean_se(da), _mean_se(db)
    sel = ma >= 0.01 * ma.max()
    z = np.abs(ma - mb)[sel] / np.sqrt(sa[sel] ** 2 + sb[sel] ** 2)
    assert sel.sum() > 50
    assert z.max() < 4.5 and np.mean(z > 3.0) <= 0.02, (z.max(), np.mean(z > 3.0))


def test_distal_falloff_and_tail_are_the_same_with_32_bit_uniforms(lattices):
    """R80 and R20 behind the Bragg peak (the straggling tails shape them)
    and the energy beyond R20 (the far tail of the range distribution)."""
    pb, a, b = lattices
    dz = pb.scoring.spacing[2]

    def stats(x):
        d = x.sum(axis=(1, 2))
        k = int(np.argmax(d))
        z = (np.arange(d.size) + 0.5) * dz

        def r_at(level):
            lev = level * d[k]
            j = k + int(np.argmax(d[k:] < lev))
            return z[j - 1] + (d[j - 1] - lev) / (d[j - 1] - d[j]) * dz

        r20 = r_at(0.2)
        tail = d[z > r20 + 2.0].sum() / d.sum()
        return r_at(0.8), r20, tail

    sa = np.array([stats(x) for x in a])
    sb = np.array([stats(x) for x in b])
    (ma, ea), (mb, eb) = _mean_se(sa), _mean_se(sb)
    z = np.abs(ma - mb) / np.sqrt(ea ** 2 + eb ** 2)
    assert np.all(z < 4.0), (ma, mb, z)
    assert abs(ma[0] - mb[0]) < 0.1 and abs(ma[1] - mb[1]) < 0.1        # mm


def test_lateral_spread_is_the_same_with_32_bit_uniforms(lattices):
    """Second moment of the lateral dose at a third and at nine tenths of the
    range (multiple scattering's Gaussian core and its tails)."""
    pb, a, b = lattices
    g = pb.scoring
    x = g.origin[0] + (np.arange(g.shape[0]) + 0.5) * g.spacing[0]
    y = g.origin[1] + (np.arange(g.shape[1]) + 0.5) * g.spacing[1]
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    for zi in (26, 70):                                         # 53 mm and 141 mm deep
        ma, ea = _mean_se(np.array([(s[zi] * r2).sum() / s[zi].sum() for s in a]))
        mb, eb = _mean_se(np.array([(s[zi] * r2).sum() / s[zi].sum() for s in b]))
        assert abs(ma - mb) / np.hypot(ea, eb) < 4.0, (zi, ma, mb, ea, eb)

"""Error paths of the C ABI, injected from the host.

Each case hands the library an input it must refuse, or a limit it must
report, and checks the status code (and that the context stays usable):
polygons that are too small or not simple (Sec. 2.B's crossing-number test
needs a simple opening contour), spot energies that are NaN or outside the
tables, spots of a beam entry that was never set, history counts outside
[0, 2^32), and histories that reach a small iteration cap -- reported by the
call itself when it reads its statistics, and otherwise by the next call on
the context, which reads the status word the earlier call left latched.
"""
import dataclasses

import numpy as np
import pytest

from paper_2307_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

VPMC_ERR_ARG, VPMC_ERR_TIMEOUT, VPMC_ERR_STATE = -1, -4, -5


@pytest.fixture(scope="module")
def vpmc_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2307_01416_gb300 import vpmc
    return vpmc


def _raises(vpmc, status, fn, *args, **kw):
    with pytest.raises(vpmc.VpmcError) as err:
        fn(*args, **kw)
    assert err.value.status == status, str(err.value)
    return str(err.value)


def test_polygons_that_are_not_simple_are_refused(vpmc_mod):
    vpmc = vpmc_mod
    pb, spots = W.water_aperture_case(20.0, False, hist_per_layer=2000, max_layers=1, shape=(30, 30, 40))
    eng = vpmc.Engine(pb)
    good = pb.beams[0]
    bad = {
        "two vertices": np.array([[-5.0, 0.0], [5.0, 0.0]]),
        "bow tie": np.array([[-5.0, -5.0], [5.0, 5.0], [5.0, -5.0], [-5.0, 5.0]]),
        "repeated vertex": np.array([[-5.0, -5.0], [5.0, -5.0], [5.0, -5.0], [5.0, 5.0], [-5.0, 5.0]]),
        "edge folding back": np.array([[-5.0, -5.0], [5.0, -5.0], [0.0, -5.0], [0.0, 5.0]]),
        "vertex on another edge": np.array([[-5.0, -5.0], [5.0, -5.0], [5.0, 5.0], [0.0, -5.0], [-5.0, 5.0]]),
        "non-finite vertex": np.array([[-5.0, -5.0], [5.0, -5.0], [np.nan, 5.0]]),
    }
    for name, poly in bad.items():
        msg = _raises(vpmc, VPMC_ERR_ARG, eng.set_beam, 0, dataclasses.replace(good, polygon=poly))
        assert "polygon" in msg or "vertices" in msg, (name, msg)
    # the entry keeps its previous (valid) opening: the same dose as a fresh context
    d1, _, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=3))
    eng.close()
    eng2 = vpmc.Engine(pb)
    d2, _, _ = eng2.run_spots(spots, W.Scenario(), W.Options(seed=3))
    eng2.close()
    assert np.array_equal(d1.cpu().numpy(), d2.cpu().numpy())
    # a concave (simple) opening and collinear vertices along an edge are accepted
    eng = vpmc.Engine(pb)
    concave = np.array([[-6.0, -6.0], [6.0, -6.0], [6.0, 6.0], [0.0, 0.0], [-6.0, 6.0]])
    eng.set_beam(0, dataclasses.replace(good, polygon=concave))
    collinear = np.array([[-5.0, -5.0], [0.0, -5.0], [5.0, -5.0], [5.0, 5.0], [-5.0, 5.0]])
    eng.set_beam(0, dataclasses.replace(good, polygon=collinear))
    eng.close()


def test_bad_spots_are_refused(vpmc_mod):
    vpmc = vpmc_mod
    pb, spots = W.pencil_beam_water(n_hist=100, shape=(20, 20, 40))
    eng = vpmc.Engine(pb)
    cases = [("energy", np.nan, VPMC_ERR_ARG), ("energy", 300.0, VPMC_ERR_ARG), ("energy", 0.4, VPMC_ERR_ARG),
             ("energy", -10.0, VPMC_ERR_ARG), ("n_hist", -1, VPMC_ERR_ARG), ("n_hist", 1 << 32, VPMC_ERR_ARG),
             ("sigma", -1.0, VPMC_ERR_ARG), ("sigma", np.nan, VPMC_ERR_ARG), ("x", np.inf, VPMC_ERR_ARG),
             ("weight", -2.0, VPMC_ERR_ARG), ("beam", 5, VPMC_ERR_STATE), ("beam", -1, VPMC_ERR_STATE),
             ("beam", 64, VPMC_ERR_STATE)]
    for field, value, status in cases:
        bad = spots.copy()
        bad[field] = value
        _raises(vpmc, status, eng.run_spots, bad, W.Scenario(), W.Options())
        if status == VPMC_ERR_STATE or field != "weight":
            _raises(vpmc, status, eng.influence_matrix, bad, [W.Scenario()], W.Options())
    _raises(vpmc, VPMC_ERR_ARG, eng.run_spots, spots, W.Scenario(), W.Options(), timeout_iters=-5)
    # the context is still usable
    d, st, _ = eng.run_spots(spots, W.Scenario(), W.Options())
    assert st["histories"] == 100 and st["errors"] == 0 and float(d.max()) > 0.0
    eng.close()


def test_iteration_cap_is_reported_by_the_call_and_latched_for_the_next(vpmc_mod):
    """A 100 MeV proton takes about 500 steps in water, so a cap of 50
    iterations stops every history.  With statistics the call itself returns
    VPMC_ERR_TIMEOUT.  Without, it returns at once and the next call on the
    context reports the latched status word and does not run; the call after
    that runs normally (the word was read and is cleared)."""
    vpmc = vpmc_mod
    pb, spots = W.pencil_beam_water(n_hist=300, shape=(20, 20, 60))
    eng = vpmc.Engine(pb)
    ref, st_ref, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=9))
    assert st_ref["errors"] == 0
    ref = ref.cpu().numpy()
    _raises(vpmc, VPMC_ERR_TIMEOUT, eng.run_spots, spots, W.Scenario(), W.Options(seed=9), timeout_iters=50)
    d, none, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=9), stats=False, timeout_iters=50)
    assert none is None
    msg = _raises(vpmc, VPMC_ERR_TIMEOUT, eng.run_spots, spots, W.Scenario(), W.Options(seed=9))
    assert "earlier asynchronous call" in msg
    d, st, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=9))
    assert st["errors"] == 0 and np.array_equal(d.cpu().numpy(), ref)
    # a cap above every history's iterations changes nothing
    d, st, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=9), timeout_iters=100000)
    assert st["errors"] == 0 and np.array_equal(d.cpu().numpy(), ref)
    # the influence-matrix path reports the cap too
    _raises(vpmc, VPMC_ERR_TIMEOUT, eng.influence_matrix, spots, [W.Scenario()], W.Options(seed=9),
            timeout_iters=50)
    eng.close()


def test_failing_output_allocator_is_out_of_memory(vpmc_mod):
    """An output allocator that returns NULL makes vpmc_influence_matrix fail
    with VPMC_ERR_OOM, leaves every output struct zeroed (the library frees
    nothing it did not allocate) and the context usable; a NULL context is
    VPMC_ERR_ARG."""
    import ctypes as C
    vpmc = vpmc_mod
    assert vpmc.lib().vpmc_set_csr_allocator(None, vpmc.ALLOC_FN(lambda n, u: None), None) == VPMC_ERR_ARG
    pb, spots = W.pencil_beam_water(n_hist=50, shape=(20, 20, 40))
    eng = vpmc.Engine(pb)
    calls = []

    def refuse(nbytes, _user):
        calls.append(int(nbytes))
        return None

    cb = vpmc.ALLOC_FN(refuse)
    vpmc._check(vpmc.lib().vpmc_set_csr_allocator(eng._ctx, cb, None))
    scs = (vpmc.vpmc_scenario * 1)(vpmc.scenario_struct(W.Scenario()))
    out = (vpmc.vpmc_csr * 1)()
    st = vpmc.vpmc_stats()
    o = vpmc.make_opts(W.Options())
    status = vpmc.lib().vpmc_influence_matrix(eng._ctx, vpmc.spot_array(spots), len(spots), scs, 1, C.byref(o),
                                              1e-4, out, C.byref(st))
    assert status == -3 and calls and all(n > 0 for n in calls)          # VPMC_ERR_OOM
    assert out[0].row_ptr is None and out[0].col is None and out[0].val is None and out[0].nnz == 0
    # the engine's own allocator back in place: the context still works
    vpmc._check(vpmc.lib().vpmc_set_csr_allocator(eng._ctx, eng._alloc_cb, None))
    mats, st = eng.influence_matrix(spots, [W.Scenario()], W.Options())
    assert st["errors"] == 0 and mats[0]["val"].numel() > 0
    eng.close()

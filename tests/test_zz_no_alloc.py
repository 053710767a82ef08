"""The dose entry point that allocates nothing (vpmc_run_spots_noalloc),
called through the C ABI, against vpmc_run_spots.

It serves callers that cannot let a call allocate device memory (work
recorded into a stream capture, latency-bound serving loops, hosts whose
memory pool owns the device).  Its scratch is one fixed device array shared
by all calls, so two calls in a row check that each call starts from a
cleared array.  This file sorts last so that a run stopping at the first
failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2307_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def test_no_alloc_dose_matches_run_spots_on_two_calls(torch_cuda):
    torch = torch_cuda
    from paper_2307_01416_gb300 import vpmc
    pb, spots = W.water_aperture_case(20.0, True, hist_per_layer=20000, max_layers=2, shape=(40, 40, 60))
    scen = W.Scenario((1.0, 0.0, -2.0), 1.02)
    op = W.Options(seed=7)
    eng = vpmc.Engine(pb)
    ref, st_ref, _ = eng.run_spots(spots, scen, op)
    ref = ref.cpu().numpy()
    L = vpmc.lib()
    arr = vpmc.spot_array(spots)
    sc = vpmc.scenario_struct(scen)
    opts = vpmc.make_opts(op)
    for call in range(2):
        out = torch.full(ref.shape, -1.0, dtype=torch.float32, device="cuda")
        st = vpmc.vpmc_stats()
        rc = L.vpmc_run_spots_noalloc(eng._ctx, arr, len(spots), C.byref(sc), C.byref(opts),
                                      C.c_void_p(out.data_ptr()), C.byref(st))
        assert rc == 0, L.vpmc_last_error().decode()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=0.0)
        assert st.steps == st_ref["steps"] and st.histories == st_ref["histories"]
        assert abs(st.e_dep - st_ref["e_dep"]) <= 1e-9 * st_ref["e_dep"]
    eng.close()


def test_no_alloc_rejects_grids_beyond_its_array(torch_cuda):
    torch = torch_cuda
    from paper_2307_01416_gb300 import vpmc
    pb, spots = W.pencil_beam_water(n_hist=100, shape=(160, 160, 100))      # 2,560,000 voxels
    eng = vpmc.Engine(pb)
    out = torch.zeros((100, 160, 160), dtype=torch.float32, device="cuda")
    with pytest.raises(vpmc.VpmcError) as err:
        eng.run_spots_noalloc(spots, out)
    assert err.value.status == -1 and "at most" in str(err.value)
    eng.close()


def test_no_alloc_reports_latched_errors_and_refuses_the_surrogate(torch_cuda):
    """The fixed array holds a status word too.  A call with statistics
    reports a history that reached the iteration cap itself; a call without
    leaves the word to the next call on the device, which reports it and does
    not run.  The learned surrogate is not available on this entry point."""
    torch = torch_cuda
    from paper_2307_01416_gb300 import vpmc
    pb, spots = W.pencil_beam_water(n_hist=200, shape=(20, 20, 60))
    eng = vpmc.Engine(pb)
    ref, _, _ = eng.run_spots(spots, W.Scenario(), W.Options(seed=4))
    ref = ref.cpu().numpy()
    out = torch.zeros(ref.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(vpmc.VpmcError) as err:
        eng.run_spots_noalloc(spots, out, W.Scenario(), W.Options(seed=4), timeout_iters=50)
    assert err.value.status == -4
    assert eng.run_spots_noalloc(spots, out, W.Scenario(), W.Options(seed=4), stats=False, timeout_iters=50) is None
    with pytest.raises(vpmc.VpmcError) as err:
        eng.run_spots_noalloc(spots, out, W.Scenario(), W.Options(seed=4))
    assert err.value.status == -4 and "earlier asynchronous call" in str(err.value)
    st = eng.run_spots_noalloc(spots, out, W.Scenario(), W.Options(seed=4))
    assert st["errors"] == 0
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-6, atol=0.0)
    with pytest.raises(vpmc.VpmcError) as err:
        eng.run_spots_noalloc(spots, out, W.Scenario(), W.Options(seed=4, surrogate=True))
    assert err.value.status == -1
    eng.close()

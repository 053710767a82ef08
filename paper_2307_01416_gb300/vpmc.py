"""Python binding of the C ABI in include/vpmc.h (argument marshalling only).

Every step of transport and scoring runs in libvpmc.so's CUDA kernels; this
module converts workloads.* inputs to the ABI structs, hands torch device
buffers to the library and wraps its outputs.  It raises if the library is
missing or no CUDA device is present: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvpmc.so")

VPMC_OK = 0
_STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_TIMEOUT", -5: "ERR_STATE",
           -6: "ERR_DEVICE_FLAG"}

FATE_STOP, FATE_NUC, FATE_LEAK, FATE_RS, FATE_AP, FATE_ERR = range(6)


class VpmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("vpmc %s: %s" % (_STATUS.get(status, str(status)), message))
        self.status = status


class vpmc_hu_curve(C.Structure):
    _fields_ = [("hu", C.c_double * 5), ("density", C.c_double * 5), ("spr", C.c_double * 5)]


class vpmc_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("origin", C.c_double * 3)]


class vpmc_beam(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("bev_x", C.c_double * 3), ("iso", C.c_double * 3),
                ("source_to_iso_mm", C.c_double),
                ("rs_present", C.c_int), ("rs_wet_mm", C.c_double), ("rs_radius_mm", C.c_double),
                ("rs_down_to_iso_mm", C.c_double),
                ("ap_present", C.c_int), ("ap_thickness_mm", C.c_double), ("ap_down_to_iso_mm", C.c_double),
                ("poly_xy", C.POINTER(C.c_double)), ("n_vertices", C.c_int), ("ap_sad_mm", C.c_double)]


class vpmc_spot(C.Structure):
    _fields_ = [("beam", C.c_int), ("energy_mev", C.c_double), ("x_mm", C.c_double), ("y_mm", C.c_double),
                ("sigma_mm", C.c_double), ("div_mrad", C.c_double), ("n_hist", C.c_int64), ("weight", C.c_double)]


class vpmc_scenario(C.Structure):
    _fields_ = [("shift_mm", C.c_double * 3), ("spr_scale", C.c_double)]


class vpmc_opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("mcs", C.c_int), ("straggling", C.c_int), ("nuclear", C.c_int),
                ("frac_bits", C.c_int), ("aggregate", C.c_int), ("block_size", C.c_int),
                ("blocks_per_sm", C.c_int), ("chunk", C.c_int), ("history_out", C.c_void_p),
                ("history_cap", C.c_int64), ("range_rejection", C.c_int), ("surrogate", C.c_int),
                ("timeout_iters", C.c_int64)]


class vpmc_opt_params(C.Structure):
    _fields_ = [("prescription", C.c_float), ("w_under", C.c_float), ("w_over", C.c_float), ("w_ring", C.c_float),
                ("over_frac", C.c_float), ("ring_frac", C.c_float), ("lr", C.c_float), ("iterations", C.c_int)]


class vpmc_stats(C.Structure):
    _fields_ = [("histories", C.c_int64), ("steps", C.c_int64), ("errors", C.c_int64), ("e_in", C.c_double),
                ("e_dep", C.c_double), ("e_leak", C.c_double), ("e_rs", C.c_double), ("e_aperture", C.c_double),
                ("e_nuc", C.c_double), ("ms", C.c_float), ("launches", C.c_int64),
                ("ovf_records", C.c_int64), ("steps_rs", C.c_int64), ("steps_aperture", C.c_int64),
                ("ms_devices", C.c_float), ("ms_patient", C.c_float), ("scratch_bytes", C.c_int64)]


class vpmc_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


RECORD_DTYPE = np.dtype([("q_dep", np.int64), ("fate", np.int32), ("steps", np.int32), ("e_dep", np.float32),
                         ("e_end", np.float32), ("pos", np.float32, (3,)), ("pad", np.float32)])
assert RECORD_DTYPE.itemsize == 40

EXPORTED = ["vpmc_default_opts", "vpmc_create_geometry", "vpmc_set_aperture", "vpmc_run_spots",
            "vpmc_run_spots_noalloc", "vpmc_influence_matrix", "vpmc_free_csr", "vpmc_destroy", "vpmc_last_error",
            "vpmc_surrogate_init", "vpmc_surrogate_set_weights", "vpmc_surrogate_get_weights",
            "vpmc_surrogate_tracks", "vpmc_surrogate_forward", "vpmc_surrogate_gradient", "vpmc_surrogate_train",
            "vpmc_robust_optimize", "vpmc_target_indices", "vpmc_weights_dose", "vpmc_measure_l2_atomics",
            "vpmc_set_csr_allocator"]

# void* (*)(size_t bytes, void* user): the CSR output allocator (vpmc_set_csr_allocator)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)

SUR_NPARAMS = 23213            # VPMC_SUR_NPARAMS
SUR_IN, SUR_OUT, SUR_Y = 6, 45, 5

_lib = None


def lib():
    """Load libvpmc.so (built by __graft_entry__.build() / build_ext.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libvpmc.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`"
                           % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.vpmc_default_opts.argtypes = [C.POINTER(vpmc_opts)]
    L.vpmc_default_opts.restype = None
    L.vpmc_last_error.argtypes = []
    L.vpmc_last_error.restype = C.c_char_p
    L.vpmc_create_geometry.argtypes = [C.POINTER(vp), vp, C.c_int, C.POINTER(vpmc_grid), C.POINTER(vpmc_hu_curve),
                                       C.POINTER(vpmc_grid), vp]
    L.vpmc_set_aperture.argtypes = [vp, C.c_int, C.POINTER(vpmc_beam)]
    L.vpmc_run_spots.argtypes = [vp, C.POINTER(vpmc_spot), C.c_int, C.POINTER(vpmc_scenario), C.POINTER(vpmc_opts),
                                 vp, C.POINTER(vpmc_stats)]
    L.vpmc_run_spots_noalloc.argtypes = [vp, C.POINTER(vpmc_spot), C.c_int, C.POINTER(vpmc_scenario),
                                         C.POINTER(vpmc_opts), vp, C.POINTER(vpmc_stats)]
    L.vpmc_influence_matrix.argtypes = [vp, C.POINTER(vpmc_spot), C.c_int, C.POINTER(vpmc_scenario), C.c_int,
                                        C.POINTER(vpmc_opts), C.c_float, C.POINTER(vpmc_csr), C.POINTER(vpmc_stats)]
    L.vpmc_free_csr.argtypes = [C.POINTER(vpmc_csr), C.c_int]
    L.vpmc_set_csr_allocator.argtypes = [vp, ALLOC_FN, vp]
    L.vpmc_set_csr_allocator.restype = C.c_int
    L.vpmc_destroy.argtypes = [vp]
    L.vpmc_destroy.restype = None
    fp = C.POINTER(C.c_float)
    L.vpmc_surrogate_init.argtypes = [vp, C.c_uint64]
    L.vpmc_surrogate_set_weights.argtypes = [vp, fp]
    L.vpmc_surrogate_get_weights.argtypes = [vp, fp]
    L.vpmc_surrogate_tracks.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.c_int64, C.POINTER(vpmc_opts), C.c_int,
                                        vp, vp, vp]
    L.vpmc_surrogate_forward.argtypes = [vp, vp, C.c_int64, vp]
    L.vpmc_surrogate_gradient.argtypes = [vp, vp, vp, vp, C.c_int64, vp, C.POINTER(C.c_double)]
    L.vpmc_surrogate_train.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, C.c_int, C.c_float, C.c_float, fp]
    L.vpmc_robust_optimize.argtypes = [C.POINTER(vpmc_csr), C.c_int, vp, C.POINTER(vpmc_opt_params), vp,
                                       C.POINTER(C.c_float), C.POINTER(C.c_float), vp]
    L.vpmc_target_indices.argtypes = [C.POINTER(vpmc_csr), C.c_int, vp, C.c_float, vp, C.POINTER(C.c_double), vp]
    L.vpmc_weights_dose.argtypes = [C.POINTER(vpmc_csr), vp, vp, vp]
    L.vpmc_measure_l2_atomics.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64), vp]
    L.vpmc_measure_l2_atomics.restype = C.c_int
    for f in ("vpmc_robust_optimize", "vpmc_target_indices", "vpmc_weights_dose"):
        getattr(L, f).restype = C.c_int
    for f in ("vpmc_create_geometry", "vpmc_set_aperture", "vpmc_run_spots", "vpmc_run_spots_noalloc",
              "vpmc_influence_matrix", "vpmc_free_csr", "vpmc_surrogate_init", "vpmc_surrogate_set_weights",
              "vpmc_surrogate_get_weights", "vpmc_surrogate_tracks", "vpmc_surrogate_forward",
              "vpmc_surrogate_gradient", "vpmc_surrogate_train"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(status: int):
    if status != VPMC_OK:
        raise VpmcError(status, lib().vpmc_last_error().decode())


def _grid(g: W.Grid) -> vpmc_grid:
    return vpmc_grid(g.shape[0], g.shape[1], g.shape[2], g.spacing[0], g.spacing[1], g.spacing[2],
                     (C.c_double * 3)(*g.origin))


def _curve(c: W.HUCurve) -> vpmc_hu_curve:
    return vpmc_hu_curve((C.c_double * 5)(*c.hu), (C.c_double * 5)(*c.density), (C.c_double * 5)(*c.spr))


def make_opts(o: W.Options, aggregate: int = -1, block_size: int = 0, chunk: int = 0,
              timeout_iters: int = 0) -> vpmc_opts:
    v = vpmc_opts()
    lib().vpmc_default_opts(C.byref(v))
    v.seed, v.mcs, v.straggling, v.nuclear, v.frac_bits = int(o.seed), int(o.mcs), int(o.straggling), int(o.nuclear), \
        int(o.frac_bits)
    v.aggregate, v.block_size, v.chunk = aggregate, block_size, chunk
    v.timeout_iters = int(timeout_iters)
    v.range_rejection = int(getattr(o, "range_rejection", True))
    v.surrogate = int(getattr(o, "surrogate", False))
    return v


def spot_array(spots: np.ndarray):
    arr = (vpmc_spot * max(len(spots), 1))()
    for i, s in enumerate(spots):
        arr[i] = vpmc_spot(int(s["beam"]), float(s["energy"]), float(s["x"]), float(s["y"]), float(s["sigma"]),
                           float(s["div_mrad"]), int(s["n_hist"]), float(s["weight"]))
    return arr


def scenario_struct(sc: W.Scenario) -> vpmc_scenario:
    return vpmc_scenario((C.c_double * 3)(*sc.shift), float(sc.spr_scale))


class Engine:
    """One geometry (CT + scoring grid + fields) on the current CUDA device."""

    def __init__(self, problem: W.Problem, stream=None, host_ct: bool = False, torch_outputs: bool = True):
        """host_ct: hand the library the host CT array (it copies it to the
        device) instead of a device tensor.  torch_outputs: the influence
        matrices' CSR buffers are allocated by torch's caching allocator
        through vpmc_set_csr_allocator and returned without a copy; False
        lets the library allocate them, and they are copied into torch
        tensors and freed (vpmc_free_csr)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("vpmc needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.problem = problem
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._ctx = C.c_void_p()
        ct, sg, cv = _grid(problem.ct), _grid(problem.scoring), _curve(problem.curve)
        hu_host = np.ascontiguousarray(problem.hu, dtype=np.int16)
        if host_ct:
            ptr, on_dev, keep = hu_host.ctypes.data, 0, hu_host
        else:
            keep = torch.from_numpy(hu_host).to(self.device)
            ptr, on_dev = keep.data_ptr(), 1
        _check(lib().vpmc_create_geometry(C.byref(self._ctx), C.c_void_p(ptr), on_dev, C.byref(ct), C.byref(cv),
                                          C.byref(sg), C.c_void_p(self.stream.cuda_stream)))
        del keep
        self._outputs = None
        if torch_outputs:
            outputs, device = {}, self.device

            def _alloc(nbytes, _user):
                try:
                    t = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
                except RuntimeError:
                    return None
                outputs[t.data_ptr()] = t
                return t.data_ptr()

            self._outputs = outputs
            self._alloc_cb = ALLOC_FN(_alloc)          # the library keeps the pointer: keep the object
            _check(lib().vpmc_set_csr_allocator(self._ctx, self._alloc_cb, None))
        for i, b in enumerate(problem.beams):
            self.set_beam(i, b)

    def set_beam(self, beam_id: int, b: W.Beam):
        poly = None
        nv = 0
        if b.ap_present:
            poly = np.ascontiguousarray(b.polygon, dtype=np.float64)
            nv = len(poly)
        s = vpmc_beam((C.c_double * 3)(*b.direction), (C.c_double * 3)(*b.bev_x), (C.c_double * 3)(*b.iso),
                      float(b.source_to_iso), int(b.rs_present), float(b.rs_wet), float(b.rs_radius),
                      float(b.rs_down_to_iso), int(b.ap_present), float(b.ap_thickness), float(b.ap_down_to_iso),
                      poly.ctypes.data_as(C.POINTER(C.c_double)) if poly is not None else None, nv,
                      float(getattr(b, "ap_sad", 0.0)))
        _check(lib().vpmc_set_aperture(self._ctx, int(beam_id), C.byref(s)))

    def run_spots(self, spots: np.ndarray, scenario: Optional[W.Scenario] = None, opts: Optional[W.Options] = None,
                  records: int = 0, dose_out=None, stats: bool = True, **launch):
        """Dose (Gy, float32 tensor shaped (nz, ny, nx) on the device), stats
        dict (if stats) and per-history records (numpy, if records > 0)."""
        torch = self.torch
        o = make_opts(opts or W.Options(), **launch)
        g = self.problem.scoring
        dose = dose_out if dose_out is not None else torch.empty((g.shape[2], g.shape[1], g.shape[0]),
                                                                 dtype=torch.float32, device=self.device)
        rec = None
        if records:
            rec = torch.zeros((records, RECORD_DTYPE.itemsize), dtype=torch.uint8, device=self.device)
            o.history_out = rec.data_ptr()
            o.history_cap = records
        arr = spot_array(spots)
        sc = scenario_struct(scenario) if scenario is not None else None
        st = vpmc_stats()
        _check(lib().vpmc_run_spots(self._ctx, arr, len(spots), C.byref(sc) if sc is not None else None, C.byref(o),
                                    C.c_void_p(dose.data_ptr()), C.byref(st) if stats else None))
        out_stats = _stats_dict(st) if stats else None
        out_rec = None
        if rec is not None:
            self.stream.synchronize()
            out_rec = rec.cpu().numpy().view(RECORD_DTYPE).reshape(records)
        return dose, out_stats, out_rec

    def run_spots_noalloc(self, spots: np.ndarray, dose_out, scenario: Optional[W.Scenario] = None,
                          opts: Optional[W.Options] = None, stats: bool = True, **launch):
        """Dose into the caller's float32 device tensor dose_out through the
        entry point that allocates nothing (fixed scratch; see include/vpmc.h
        for its limits).  Returns the stats dict (if stats)."""
        o = make_opts(opts or W.Options(), **launch)
        arr = spot_array(spots)
        sc = scenario_struct(scenario) if scenario is not None else None
        st = vpmc_stats()
        _check(lib().vpmc_run_spots_noalloc(self._ctx, arr, len(spots), C.byref(sc) if sc is not None else None,
                                            C.byref(o), C.c_void_p(dose_out.data_ptr()),
                                            C.byref(st) if stats else None))
        return _stats_dict(st) if stats else None

    def influence_matrix(self, spots: np.ndarray, scenarios: Sequence[W.Scenario], opts: Optional[W.Options] = None,
                         rel_threshold: float = 1e-4, **launch):
        """Per-scenario CSR (dict of torch device tensors row_ptr int64, col
        int32, val float32) and the stats dict."""
        torch = self.torch
        o = make_opts(opts or W.Options(), **launch)
        arr = spot_array(spots)
        scs = (vpmc_scenario * len(scenarios))(*[scenario_struct(s) for s in scenarios])
        out = (vpmc_csr * len(scenarios))()
        st = vpmc_stats()
        if self._outputs is None:
            _check(lib().vpmc_influence_matrix(self._ctx, arr, len(spots), scs, len(scenarios), C.byref(o),
                                               float(rel_threshold), out, C.byref(st)))
            mats = []
            try:
                for m in out:
                    mats.append(_csr_to_torch(m, self.device))
            finally:
                lib().vpmc_free_csr(out, len(scenarios))
            return mats, _stats_dict(st)
        self._outputs.clear()
        try:
            _check(lib().vpmc_influence_matrix(self._ctx, arr, len(spots), scs, len(scenarios), C.byref(o),
                                               float(rel_threshold), out, C.byref(st)))
            mats = [_csr_from_outputs(m, self._outputs, self.device) for m in out]
        finally:
            self._outputs.clear()
        return mats, _stats_dict(st)

    # ---------------------------------------------------- learned aperture surrogate
    def surrogate_init(self, seed: int = 0):
        _check(lib().vpmc_surrogate_init(self._ctx, int(seed)))

    def surrogate_set_weights(self, params: np.ndarray):
        w = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if w.size != SUR_NPARAMS:
            raise ValueError("expected %d parameters, got %d" % (SUR_NPARAMS, w.size))
        _check(lib().vpmc_surrogate_set_weights(self._ctx, w.ctypes.data_as(C.POINTER(C.c_float))))

    def surrogate_get_weights(self) -> np.ndarray:
        w = np.zeros(SUR_NPARAMS, dtype=np.float32)
        _check(lib().vpmc_surrogate_get_weights(self._ctx, w.ctypes.data_as(C.POINTER(C.c_float))))
        return w

    def surrogate_tracks(self, beam_ids: Sequence[int], tracks_per_beam: int, opts: Optional[W.Options] = None,
                         use_surrogate: bool = False):
        """Training (plain transport) or evaluation (network draws) tracks:
        device tensors feat (n, 6), target (n, 5), label (n,) int32."""
        torch = self.torch
        n = len(beam_ids) * int(tracks_per_beam)
        feat = torch.empty((n, SUR_IN), dtype=torch.float32, device=self.device)
        target = torch.empty((n, SUR_Y), dtype=torch.float32, device=self.device)
        label = torch.empty(n, dtype=torch.int32, device=self.device)
        ids = (C.c_int * len(beam_ids))(*[int(b) for b in beam_ids])
        o = make_opts(opts or W.Options(seed=W.SURROGATE_SEED))
        _check(lib().vpmc_surrogate_tracks(self._ctx, ids, len(beam_ids), int(tracks_per_beam), C.byref(o),
                                           int(use_surrogate), C.c_void_p(feat.data_ptr()),
                                           C.c_void_p(target.data_ptr()), C.c_void_p(label.data_ptr())))
        return feat, target, label

    def surrogate_forward(self, feat):
        z = self.torch.empty((feat.shape[0], SUR_OUT), dtype=self.torch.float32, device=self.device)
        _check(lib().vpmc_surrogate_forward(self._ctx, C.c_void_p(feat.data_ptr()), int(feat.shape[0]),
                                            C.c_void_p(z.data_ptr())))
        return z

    def surrogate_gradient(self, feat, target, label):
        g = self.torch.empty(SUR_NPARAMS, dtype=self.torch.float32, device=self.device)
        loss = C.c_double()
        _check(lib().vpmc_surrogate_gradient(self._ctx, C.c_void_p(feat.data_ptr()), C.c_void_p(target.data_ptr()),
                                             C.c_void_p(label.data_ptr()), int(feat.shape[0]),
                                             C.c_void_p(g.data_ptr()), C.byref(loss)))
        return g, loss.value

    def surrogate_train(self, feat, target, label, batch: int = 8192, epochs: int = 1, lr: float = 1e-3,
                        lr_min: float = 1e-5) -> np.ndarray:
        losses = np.zeros(int(epochs), dtype=np.float32)
        _check(lib().vpmc_surrogate_train(self._ctx, C.c_void_p(feat.data_ptr()), C.c_void_p(target.data_ptr()),
                                          C.c_void_p(label.data_ptr()), int(feat.shape[0]), int(batch), int(epochs),
                                          float(lr), float(lr_min), losses.ctypes.data_as(C.POINTER(C.c_float))))
        return losses

    def close(self):
        if self._ctx:
            lib().vpmc_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stats_dict(st: vpmc_stats) -> dict:
    return {f: getattr(st, f) for f, _ in vpmc_stats._fields_}


class _DeviceView:
    """Zero-copy view of a library-owned device buffer for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                          "version": 3, "strides": None}


def _csr_from_outputs(m: vpmc_csr, outputs: dict, device):
    """The CSR of one scenario as typed views of the torch buffers the output
    allocator handed to the library (no copy)."""
    import torch
    out = {}
    for name, ptr, n, dt in (("row_ptr", m.row_ptr, m.n_rows + 1, torch.int64), ("col", m.col, m.nnz, torch.int32),
                             ("val", m.val, m.nnz, torch.float32)):
        if n == 0:
            out[name] = torch.empty(0, dtype=dt, device=device)
        else:
            out[name] = outputs.pop(int(ptr)).view(dt)[:n]
    out["shape"] = (int(m.n_rows), int(m.n_cols))
    return out


def _csr_to_torch(m: vpmc_csr, device):
    """Copy library-owned CSR buffers into torch-owned tensors (device to device)."""
    import torch
    out = {}
    for name, ptr, n, ts, dt in (("row_ptr", m.row_ptr, m.n_rows + 1, "<i8", torch.int64),
                                 ("col", m.col, m.nnz, "<i4", torch.int32),
                                 ("val", m.val, m.nnz, "<f4", torch.float32)):
        if n == 0:
            out[name] = torch.empty(0, dtype=dt, device=device)
        else:
            out[name] = torch.as_tensor(_DeviceView(ptr, n, ts), device=device).clone()
    out["shape"] = (int(m.n_rows), int(m.n_cols))
    return out


def surrogate_training_problem(radii=W.SURROGATE_RADII) -> W.Problem:
    """A small water phantom with the surrogate's training geometries as its
    beams (aperture only); the tracks never reach the phantom."""
    g, hu = W.water_phantom((8, 8, 8), (2.0, 2.0, 2.0), (-8.0, -8.0, 0.0))
    return W.Problem(ct=g, hu=hu, curve=W.HUCurve(), scoring=g, beams=W.surrogate_training_beams(radii))


def train_surrogate(tracks_per_beam: int = 2_000_000, epochs: int = 4, batch: int = 16384, lr: float = 2e-3,
                    lr_min: float = 2e-5, seed: int = W.SURROGATE_SEED, init_seed: int = 7, engine: "Engine" = None):
    """Generate training tracks with the plain aperture transport and train the
    network on the GPU.  Returns (parameters float32[SUR_NPARAMS], per-epoch
    mean losses)."""
    own = engine is None
    eng = engine or Engine(surrogate_training_problem())
    try:
        nb = len(eng.problem.beams)
        feat, target, label = eng.surrogate_tracks(list(range(nb)), tracks_per_beam, W.Options(seed=seed))
        eng.surrogate_init(init_seed)
        losses = eng.surrogate_train(feat, target, label, batch=batch, epochs=epochs, lr=lr, lr_min=lr_min)
        return eng.surrogate_get_weights(), losses
    finally:
        if own:
            eng.close()


# ------------------------------------------------------------------ robust optimisation
def _csr_array(mats):
    """vpmc_csr structs over torch CSR dicts (row_ptr int64, col int32, val float32, shape)."""
    arr = (vpmc_csr * len(mats))()
    for i, m in enumerate(mats):
        arr[i].n_rows, arr[i].n_cols = int(m["shape"][0]), int(m["shape"][1])
        arr[i].nnz = int(m["val"].numel())
        arr[i].row_ptr = m["row_ptr"].data_ptr()
        arr[i].col = m["col"].data_ptr() if arr[i].nnz else None
        arr[i].val = m["val"].data_ptr() if arr[i].nnz else None
    return arr


def robust_optimize(mats, voxel_class, x, prescription: float, iterations: int = 200, lr: float = 0.05,
                    w_under: float = 1.0, w_over: float = 0.5, w_ring: float = 0.2, over_frac: float = 1.05,
                    ring_frac: float = 0.6, stream=None):
    """Optimise the weights x (float32 device tensor, in place) over the
    scenarios' matrices; returns (worst-case objective per iteration, device ms
    of the iterations, device ms of the setup)."""
    import torch
    arr = _csr_array(mats)
    p = vpmc_opt_params(float(prescription), float(w_under), float(w_over), float(w_ring), float(over_frac),
                        float(ring_frac), float(lr), int(iterations))
    hist = np.zeros(max(int(iterations), 1), dtype=np.float32)
    ms = (C.c_float * 2)()
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().vpmc_robust_optimize(arr, len(mats), C.c_void_p(voxel_class.data_ptr()), C.byref(p),
                                      C.c_void_p(x.data_ptr()), hist.ctypes.data_as(C.POINTER(C.c_float)),
                                      ms, C.c_void_p(st.cuda_stream)))
    return hist[:int(iterations)], ms[0], ms[1]


def target_indices(mats, voxel_class, prescription: float, x, stream=None) -> np.ndarray:
    """(n_scen, 4): V100, D_min / D_p, CI100, RHI100 of the dose A_s x."""
    import torch
    arr = _csr_array(mats)
    out = np.zeros(4 * len(mats), dtype=np.float64)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().vpmc_target_indices(arr, len(mats), C.c_void_p(voxel_class.data_ptr()), float(prescription),
                                     C.c_void_p(x.data_ptr()), out.ctypes.data_as(C.POINTER(C.c_double)),
                                     C.c_void_p(st.cuda_stream)))
    return out.reshape(len(mats), 4)


def measure_l2_atomics(n_entries: int = 1 << 22, iters: int = 256, stream=None) -> dict:
    """The device's rate of 64-bit atomic adds resolved in L2 (adds/s), with
    the adds of the timed pass and the buffer's sum after both passes."""
    import torch
    rate = C.c_double(0.0)
    adds = C.c_int64(0)
    total = C.c_int64(0)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().vpmc_measure_l2_atomics(int(n_entries), int(iters), C.byref(rate), C.byref(adds), C.byref(total),
                                         C.c_void_p(st.cuda_stream)))
    return {"adds_per_s": rate.value, "adds": adds.value, "sum": total.value, "n_entries": int(n_entries)}


def weights_dose(mat, x, stream=None):
    """Dose A x of one CSR matrix (float32 device tensor)."""
    import torch
    arr = _csr_array([mat])
    d = torch.empty(int(mat["shape"][0]), dtype=torch.float32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().vpmc_weights_dose(arr, C.c_void_p(x.data_ptr()), C.c_void_p(d.data_ptr()), C.c_void_p(st.cuda_stream)))
    return d

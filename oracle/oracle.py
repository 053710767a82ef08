"""Python access to the FP64 CPU oracle (vpmc_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py.  It never imports the CUDA path; it
shares with it only the seeded input generators in
paper_2307_01416_gb300.workloads.

The influence-matrix assembly here (Sec. 2.C: sparse matrix, voxels x spots)
follows its plain definition: per spot column, dose per primary in FP64,
entries below rel_threshold x column maximum dropped, stored as FP32 CSR.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vpmc_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")

FATE_STOP, FATE_NUC, FATE_LEAK, FATE_RS, FATE_AP, FATE_ERR = range(6)
NTALLY = 9
TALLY_NAMES = ["e_in", "e_dep", "e_leak", "e_rs", "e_ap", "e_nuc", "histories", "steps", "errors"]
MEV_PER_G_TO_GY = 1.602176634e-10


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, OpenMP)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class _Curve(C.Structure):
    _fields_ = [("hu", C.c_double * 5), ("rho", C.c_double * 5), ("spr", C.c_double * 5)]


class _Beam(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("bevx", C.c_double * 3), ("iso", C.c_double * 3),
                ("source_to_iso", C.c_double),
                ("rs_present", C.c_int), ("rs_wet", C.c_double), ("rs_radius", C.c_double), ("rs_down_to_iso", C.c_double),
                ("ap_present", C.c_int), ("ap_thickness", C.c_double), ("ap_down_to_iso", C.c_double),
                ("poly_offset", C.c_int), ("nvert", C.c_int), ("ap_sad", C.c_double)]


class _Scen(C.Structure):
    _fields_ = [("shift", C.c_double * 3), ("spr_scale", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("mcs", C.c_int), ("straggling", C.c_int), ("nuclear", C.c_int),
                ("frac_bits", C.c_int), ("fine_uniforms", C.c_int)]


SPOT_DTYPE = np.dtype([("beam", np.int32), ("spot_key", np.int32), ("energy", np.float64), ("x", np.float64),
                       ("y", np.float64), ("sigma", np.float64), ("div_mrad", np.float64),
                       ("h_begin", np.int64), ("n_hist", np.int64), ("weight", np.float64)], align=True)
RECORD_DTYPE = np.dtype([("fate", np.int32), ("steps", np.int32), ("e_dep", np.float64), ("e_end", np.float64),
                         ("pos", np.float64, (3,)), ("q_dep", np.int64), ("flags", np.int32), ("pad", np.int32),
                         ("path", np.float64), ("track", np.float64)], align=True)
FLAG_NEAR_WALL, FLAG_NEAR_RIM, FLAG_NUC_LOW_DENSITY, FLAG_GRAZING_FACE = 1, 2, 4, 8

_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_box_muller.argtypes = [C.c_double, C.c_double, dp]
            L.orc_stopping_power.argtypes = [C.c_int, C.c_double]
            L.orc_stopping_power.restype = C.c_double
            for name in ("orc_table_R", "orc_table_Einv"):
                getattr(L, name).argtypes = [C.c_int, C.c_int]
                getattr(L, name).restype = C.c_double
            L.orc_table_dR.argtypes = [C.c_int]
            L.orc_table_dR.restype = C.c_double
            for name in ("orc_range", "orc_energy"):
                getattr(L, name).argtypes = [C.c_int, C.c_double]
                getattr(L, name).restype = C.c_double
            L.orc_spr_pmma.argtypes = [C.c_double]
            L.orc_spr_pmma.restype = C.c_double
            L.orc_hu_props.argtypes = [C.POINTER(_Curve), C.c_double, dp, dp]
            L.orc_point_in_polygon.argtypes = [dp, C.c_int, C.c_double, C.c_double]
            L.orc_point_in_polygon.restype = C.c_int
            L.orc_first_wall_hit.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_first_wall_hit.restype = C.c_double
            L.orc_wall_distance.argtypes = [dp, C.c_int, C.c_double, C.c_double]
            L.orc_wall_distance.restype = C.c_double
            L.orc_highland.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_highland.restype = C.c_double
            L.orc_bohr_var.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_bohr_var.restype = C.c_double
            L.orc_init_tables.argtypes = []
            L.orc_run.argtypes = [C.POINTER(_Grid), C.c_void_p, C.POINTER(_Curve), C.POINTER(_Grid),
                                  C.POINTER(_Beam), C.c_void_p, C.c_void_p, C.c_int, C.POINTER(_Scen),
                                  C.POINTER(_Opts), C.c_int, C.c_void_p, dp, C.c_void_p, C.c_int64, C.c_int]
            L.orc_run.restype = C.c_int
            L.orc_max_threads.restype = C.c_int
            L.orc_scoring_density.argtypes = [C.POINTER(_Grid), C.c_void_p, C.POINTER(_Curve), C.POINTER(_Grid), dp]
            L.orc_dose_from_q.argtypes = [C.c_void_p, C.c_int64, dp, C.c_double, C.c_int, dp]
            L.orc_gamma_pass_rate.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int64)]
            L.orc_gamma_pass_rate.restype = C.c_double
            L.orc_nearest_edge.argtypes = [dp, C.c_int, C.c_double, C.c_double, dp]
            L.orc_aperture_query.argtypes = [C.POINTER(_Beam), dp, dp, dp, dp]
            L.orc_surrogate_features.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double, dp, C.c_double,
                                                 dp, dp]
            L.orc_surrogate_tracks.argtypes = [C.POINTER(_Beam), C.c_void_p, C.c_int, C.c_int64, C.POINTER(_Opts),
                                               dp, C.c_void_p, dp, C.c_void_p, C.c_void_p, C.c_int]
            L.orc_surrogate_tracks.restype = C.c_int
            L.orc_init_tables()
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(x: int) -> float:
    return lib().orc_uniform(int(x) & 0xFFFFFFFF)


def step_uniforms(hist: int, step: int, key):
    """The six 21-bit uniforms of one condensed-history step."""
    L = lib()
    if not hasattr(L, "_su_ready"):
        L.orc_step_uniforms.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_double)]
        L._su_ready = True
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_double * 6)()
    L.orc_step_uniforms(int(hist) & 0xFFFFFFFF, int(step) & 0xFFFFFFFF, k, o)
    return list(o)


def box_muller(u1: float, u2: float):
    z = (C.c_double * 2)()
    lib().orc_box_muller(u1, u2, z)
    return z[0], z[1]


WATER, PMMA, BRASS = 0, 1, 2
NE, NR = 2501, 4096


def stopping_power(mat: int, e: float) -> float:
    return lib().orc_stopping_power(mat, float(e))


def range_table(mat: int) -> np.ndarray:
    L = lib()
    return np.array([L.orc_table_R(mat, k) for k in range(NE)])


def energy_table(mat: int) -> np.ndarray:
    L = lib()
    return np.array([L.orc_table_Einv(mat, j) for j in range(NR)])


def table_dR(mat: int) -> float:
    return lib().orc_table_dR(mat)


def csda_range(mat: int, e: float) -> float:
    return lib().orc_range(mat, float(e))


def energy_at_range(mat: int, r: float) -> float:
    return lib().orc_energy(mat, float(r))


def spr_pmma(e: float) -> float:
    return lib().orc_spr_pmma(float(e))


def _curve(c) -> _Curve:
    cv = _Curve()
    for i in range(5):
        cv.hu[i], cv.rho[i], cv.spr[i] = c.hu[i], c.density[i], c.spr[i]
    return cv


def hu_props(curve, hu: float):
    r, s = C.c_double(), C.c_double()
    lib().orc_hu_props(C.byref(_curve(curve)), float(hu), C.byref(r), C.byref(s))
    return r.value, s.value


def point_in_polygon(poly: np.ndarray, x: float, y: float) -> bool:
    p = np.ascontiguousarray(poly, dtype=np.float64)
    return bool(lib().orc_point_in_polygon(_dp(p), len(p), float(x), float(y)))


def first_wall_hit(poly: np.ndarray, x, y, dx, dy) -> float:
    p = np.ascontiguousarray(poly, dtype=np.float64)
    return lib().orc_first_wall_hit(_dp(p), len(p), float(x), float(y), float(dx), float(dy))


def wall_distance(poly: np.ndarray, x, y) -> float:
    p = np.ascontiguousarray(poly, dtype=np.float64)
    return lib().orc_wall_distance(_dp(p), len(p), float(x), float(y))


def highland(e, s_mm, rho, x0_gcm2) -> float:
    return lib().orc_highland(float(e), float(s_mm), float(rho), float(x0_gcm2))


def bohr_var(e, s_mm, rho, za) -> float:
    return lib().orc_bohr_var(float(e), float(s_mm), float(rho), float(za))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------- transport
def _grid(g) -> _Grid:
    return _Grid(g.shape[0], g.shape[1], g.shape[2], g.spacing[0], g.spacing[1], g.spacing[2],
                 g.origin[0], g.origin[1], g.origin[2])


def _beams(beams):
    arr = (_Beam * len(beams))()
    polys, off = [], 0
    for i, b in enumerate(beams):
        a = arr[i]
        for k in range(3):
            a.dir[k], a.bevx[k], a.iso[k] = b.direction[k], b.bev_x[k], b.iso[k]
        a.source_to_iso = b.source_to_iso
        a.rs_present = int(b.rs_present)
        a.rs_wet, a.rs_radius, a.rs_down_to_iso = b.rs_wet, b.rs_radius, b.rs_down_to_iso
        a.ap_present = int(b.ap_present)
        a.ap_thickness, a.ap_down_to_iso = b.ap_thickness, b.ap_down_to_iso
        a.ap_sad = float(getattr(b, "ap_sad", 0.0))
        if b.ap_present:
            p = np.ascontiguousarray(b.polygon, dtype=np.float64)
            polys.append(p)
            a.poly_offset, a.nvert = off, len(p)
            off += len(p)
        else:
            a.poly_offset, a.nvert = 0, 0
    xy = np.ascontiguousarray(np.concatenate(polys) if polys else np.zeros((1, 2)), dtype=np.float64)
    return arr, xy


def oracle_spots(spots: np.ndarray, spot_keys=None, h_begin=None, n_hist=None) -> np.ndarray:
    """Convert public spot rows to the oracle's layout.  spot_keys defaults to
    the row index (the RNG key of a spot is its index in the full list)."""
    o = np.zeros(len(spots), dtype=SPOT_DTYPE)
    for f in ("beam", "energy", "x", "y", "sigma", "div_mrad", "weight"):
        o[f] = spots[f]
    o["spot_key"] = np.arange(len(spots)) if spot_keys is None else spot_keys
    o["h_begin"] = 0 if h_begin is None else h_begin
    o["n_hist"] = spots["n_hist"] if n_hist is None else n_hist
    return o


def run(problem, spots_o: np.ndarray, scenario, opts, mode: int = 0, records: int = 0,
        nthreads: int = 0, fine_uniforms: bool = False):
    """Transport all histories of spots_o (oracle layout) for one scenario.

    mode 0 returns the weighted fixed-point grid (int64, scoring-grid size);
    mode 1 returns unweighted per-spot columns, shape (n_spots, nvox).
    fine_uniforms: the step's six uniforms at 32-bit resolution from two
    Philox blocks instead of the engines' 21-bit lattice (reading c17), for
    the study of the lattice's Box-Muller tail; not the engines' stream.
    Returns (q, tallies dict, records array or None)."""
    L = lib()
    ct, sg = _grid(problem.ct), _grid(problem.scoring)
    hu = np.ascontiguousarray(problem.hu, dtype=np.int16)
    assert hu.size == problem.ct.nvox
    cv = _curve(problem.curve)
    beams, xy = _beams(problem.beams)
    sc = _Scen((C.c_double * 3)(*scenario.shift), scenario.spr_scale)
    op = _Opts(int(opts.seed), int(opts.mcs), int(opts.straggling), int(opts.nuclear), int(opts.frac_bits),
               int(fine_uniforms))
    nv = problem.scoring.nvox
    sp = np.ascontiguousarray(spots_o, dtype=SPOT_DTYPE)
    q = np.zeros(nv if mode == 0 else len(sp) * nv, dtype=np.int64)
    tl = np.zeros(NTALLY, dtype=np.float64)
    rec = np.zeros(records, dtype=RECORD_DTYPE) if records else None
    rc = L.orc_run(C.byref(ct), hu.ctypes.data, C.byref(cv), C.byref(sg), beams, xy.ctypes.data,
                   sp.ctypes.data, len(sp), C.byref(sc), C.byref(op), mode, q.ctypes.data, _dp(tl),
                   rec.ctypes.data if rec is not None else None, records, int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle run failed")
    if mode == 1:
        q = q.reshape(len(sp), nv)
    return q, dict(zip(TALLY_NAMES, tl.tolist())), rec


def scoring_density(problem) -> np.ndarray:
    ct, sg = _grid(problem.ct), _grid(problem.scoring)
    hu = np.ascontiguousarray(problem.hu, dtype=np.int16)
    out = np.zeros(problem.scoring.nvox, dtype=np.float64)
    lib().orc_scoring_density(C.byref(ct), hu.ctypes.data, C.byref(_curve(problem.curve)), C.byref(sg), _dp(out))
    return out


def dose_from_q(problem, q: np.ndarray, frac_bits: int, rho: Optional[np.ndarray] = None) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int64)
    rho = scoring_density(problem) if rho is None else rho
    out = np.zeros(q.size, dtype=np.float64)
    lib().orc_dose_from_q(q.ctypes.data, q.size, _dp(rho), problem.scoring.voxel_mm3, int(frac_bits), _dp(out))
    return out


def gamma_pass_rate(ref: np.ndarray, ev: np.ndarray, spacing, dd_frac=0.02, dta_mm=2.0, thr_frac=0.10,
                    subdiv=5) -> float:
    """Global 3D gamma pass rate (%), arrays shaped (nz, ny, nx)."""
    r = np.ascontiguousarray(ref, dtype=np.float64)
    e = np.ascontiguousarray(ev, dtype=np.float64)
    nz, ny, nx = r.shape
    n = C.c_int64()
    return lib().orc_gamma_pass_rate(_dp(r), _dp(e), nx, ny, nz, float(spacing[0]), float(spacing[1]),
                                     float(spacing[2]), dd_frac, dta_mm, thr_frac, int(subdiv), C.byref(n))


def influence_matrix(problem, spots: np.ndarray, scenarios, opts, rel_threshold: float = 1e-4,
                     nthreads: int = 0):
    """Per-scenario influence matrices (voxels x spots) as scipy CSR, FP32
    values of dose per primary proton (Gy); per column, entries below
    rel_threshold x the column maximum are dropped (decided in FP64)."""
    import scipy.sparse as sps
    rho = scoring_density(problem)
    vol_cm3 = problem.scoring.voxel_mm3 * 1e-3
    out = []
    for sc in scenarios:
        q, tl, _ = run(problem, oracle_spots(spots), sc, opts, mode=1, nthreads=nthreads)
        d = q.astype(np.float64) * (2.0 ** -opts.frac_bits) * MEV_PER_G_TO_GY / vol_cm3
        d /= rho[None, :]
        d /= spots["n_hist"].astype(np.float64)[:, None]
        cmax = d.max(axis=1, keepdims=True)
        keep = (d >= rel_threshold * cmax) & (d > 0)
        dense = np.where(keep, d, 0.0).astype(np.float32)
        out.append(sps.csr_matrix(dense.T))
    return out


def step_sample(table, kappa, rho, za, x0, e, s_geom=float("inf"), mcs=True, straggling=True, nuclear=False,
                nlam=float("inf"), seed=1234, spot_key=0, hist=0, step=0):
    """One condensed-history step from (origin, +z, E); returns a dict."""
    L = lib()
    if not hasattr(L, "_step_ready"):
        L.orc_step_sample.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_int,
                                      C.c_uint32, C.c_uint32, C.POINTER(C.c_double)]
        L._step_ready = True
    o = (C.c_double * 11)()
    L.orc_step_sample(int(table), float(kappa), float(rho), float(za), float(x0), float(e), float(s_geom),
                      int(mcs), int(straggling), int(nuclear), float(nlam), int(seed), int(spot_key),
                      int(hist) & 0xFFFFFFFF, int(step) & 0xFFFFFFFF, o)
    v = list(o)
    return {"s": v[0], "dE": v[1], "limiter": int(v[2]), "killed": int(v[3]), "E": v[4],
            "d": np.array(v[5:8]), "disp": np.array(v[8:11])}


# ------------------------------------------------------------ learned surrogate
def aperture_query(beam, p, d):
    """(in the opening, first wall hit distance, wall distance) of the point
    p and direction d (BEV, t along the beam from the isocentre) for the
    beam's aperture, parallel or divergent walls."""
    arr, xy = _beams([beam])
    out = np.zeros(3)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    lib().orc_aperture_query(C.byref(arr[0]), _dp(xy), _dp(pp), _dp(dd), _dp(out))
    return bool(out[0]), float(out[1]), float(out[2])


def nearest_edge(poly: np.ndarray, x: float, y: float):
    """(distance, nearest x, nearest y, curvature there) of the polygon boundary."""
    p = np.ascontiguousarray(poly, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_nearest_edge(_dp(p), len(p), float(x), float(y), _dp(out))
    return tuple(out.tolist())


def surrogate_features(poly: np.ndarray, thickness: float, x: float, y: float, d, E: float):
    """Six surrogate inputs and the edge frame (n_x, n_y, u_n, u_t) of a proton
    on the block's entrance plane."""
    p = np.ascontiguousarray(poly, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    f, fr = np.zeros(6), np.zeros(4)
    lib().orc_surrogate_features(_dp(p), len(p), float(thickness), float(x), float(y), _dp(dd), float(E),
                                 _dp(f), _dp(fr))
    return f, fr


def surrogate_tracks(beams, n_tracks: int, opts, nthreads: int = 0):
    """Training tracks of the plain aperture transport, n_tracks per geometry
    (beams: aperture-only beams).  Returns dict of feat (N, 6), label (N,),
    target (N, 5), fate (N,) (-1: left through the exit plane) and flags (N,)."""
    L = lib()
    arr, xy = _beams(beams)
    op = _Opts(int(opts.seed), int(opts.mcs), int(opts.straggling), int(opts.nuclear), int(opts.frac_bits))
    n = len(beams) * int(n_tracks)
    feat, target = np.zeros((n, 6)), np.zeros((n, 5))
    label, fate, flags = (np.zeros(n, dtype=np.int32) for _ in range(3))
    rc = L.orc_surrogate_tracks(arr, xy.ctypes.data, len(beams), int(n_tracks), C.byref(op), _dp(feat),
                                label.ctypes.data, _dp(target), fate.ctypes.data, flags.ctypes.data, int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle surrogate_tracks failed")
    return {"feat": feat, "label": label, "target": target, "fate": fate, "flags": flags}

#!/usr/bin/env python
"""Benchmark of the robust influence-matrix set (one step = one 13-scenario set).

Workload: synthetic heterogeneous head (256x256x160 CT at 1x1x1.5 mm, 2 mm
scoring grid), 8.4 cc spherical target, three coplanar fields (0/90/270 deg)
with 45 mm WET range shifter and brass apertures conformed to the target
projection + 5 mm, 3 mm spot grid, layers 3 mm WET apart, 1e3-2e4 histories
per spot (log-uniform), 13 robust scenarios (nominal, +/-3 mm shifts, +/-3.5 %
range with each shift sign).  Full physics (Highland, Bohr, nuclear removal).

metric: protons/s (histories of the whole set / time) and seconds per set.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2307_01416_gb300 import workloads as W  # noqa: E402

METRIC = "protons/s; s per 13-scenario influence-matrix set at 0.5% unc."
WORKLOAD = ("13-scenario robust influence-matrix set, synthetic head 256x256x160 CT (1x1x1.5 mm), 2 mm scoring grid, "
            "8.4 cc target, 3 fields 0/90/270 deg, 45 mm WET range shifter, brass apertures (target + 5 mm), "
            "3 mm spots, log-uniform 1e3-2e4 histories/spot scaled to 0.5% uncertainty of the nominal composite")
# Lane-operations of one condensed-history step of the full-physics method,
# counted for a minimal implementation of the step's formulas.  In the
# patient: one Philox4x32-10 block 80, six uniforms 22, three Box-Muller
# pairs 24, four table interpolations 32, step selection 12, two-grid DDA 33,
# Bohr 15, Highland 10, rotation and displacement 45, scoring 11, position
# update 6 and voxel confinement 9.  In a homogeneous slab (range shifter,
# brass block) there is no voxel grid: no DDA, scoring or confinement, and the
# geometry limit is the distance to the slab's exit plane (4); in the brass
# the opening test adds a raster look-up (8).
OPS_PER_STEP = 299
OPS_PER_STEP_RS = 299 - 33 - 11 - 9 + 4
OPS_PER_STEP_BRASS = OPS_PER_STEP_RS + 8


def algorithmic_ops(st: dict) -> float:
    """Lane-operations of the condensed-history steps a call counted, by medium."""
    rs, ap = st["steps_rs"], st["steps_aperture"]
    return (st["steps"] - rs - ap) * OPS_PER_STEP + rs * OPS_PER_STEP_RS + ap * OPS_PER_STEP_BRASS
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["vpmc", "reference"], default="vpmc")
    ap.add_argument("--small", action="store_true", help="reduced history counts (quick check, not a bench line)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-aperture leg")
    ap.add_argument("--no-optimizer", action="store_true", help="skip the robust-optimisation leg")
    ap.add_argument("--no-edge-sweep", action="store_true", help="skip the single-beamlet edge sweep leg")
    ap.add_argument("--no-divergent", action="store_true", help="skip the divergent-aperture leg")
    ap.add_argument("--no-dynamic", action="store_true", help="skip the energy-layer-specific aperture leg")
    ap.add_argument("--divergent-sad", type=float, default=2000.0)
    ap.add_argument("--edge-hist", type=int, default=1_000_000, help="histories per beamlet of the edge sweep")
    ap.add_argument("--opt-iterations", type=int, default=50)
    ap.add_argument("--ncu-case", nargs="?", const="dose", choices=["dose", "im", "im13", "opt", "sur"], default=None,
                    help="small fixed-launch transport case for ncu captures (every 10th spot): 'dose' scores one "
                         "grid of the nominal scenario, 'im' its influence-matrix columns, 'im13' the columns of all "
                         "13 scenarios (the set's structure: one beam-line pass, 13 patient copies); 'opt' runs the "
                         "robust optimisation (--opt-iterations per step) over a 13-scenario set of every "
                         "--opt-stride-th spot; 'sur' the surrogate network's tensor-core kernels (per step one "
                         "forward pass over 2^22 rows and one training epoch over 2^20 tracks)")
    ap.add_argument("--opt-stride", type=int, default=1)
    return ap.parse_args()


def build_workload(small: bool):
    pb, spots, center, r = W.im_set_plan()
    if small:
        spots = spots.copy()
        spots["n_hist"] = np.maximum(spots["n_hist"] // 50, 20)
    return pb, spots, W.robust_scenarios(), (center, r)


# ----------------------------------------------------------------------------- clocks
REASONS = ["clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
           "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = "index,clocks.sm,clocks.max.sm,power.draw," + ",".join(REASONS)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 4 + len(REASONS):
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        active = set()
        for r in rows:
            for name, v in zip(REASONS, r[4:4 + len(REASONS)]):
                if v.lower() == "active":
                    active.add(name.split(".")[-1])
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(active), "samples": len(rows)}


def transport_traffic(patient_steps: float, beamline_histories: float):
    """DRAM bytes (read + write) of one set's transport: the bytes per patient
    step (k_patient) and per history handed through the beam line
    (k_source_rs + k_aperture, with the scenarios' copies) that an ncu capture
    of the 13-scenario small case measured (dram__bytes_read.sum +
    dram__bytes_write.sum), scaled by the set's patient steps and beam-line
    histories; None when the kernels changed since that capture (source hash)."""
    path = os.path.join(ROOT, "profiles", "k_transport_traffic.txt")
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    if kv.get("transport_sha256") != transport_source_digest():
        return None
    return (float(kv["patient_dram_bytes_per_step"]) * patient_steps
            + float(kv["beamline_dram_bytes_per_history"]) * beamline_histories)


TRANSPORT_SOURCES = ("transport_common.cuh", "devices.cu", "patient.cu")


def transport_source_digest() -> str:
    """sha256 over the transport kernels' sources and their compile flags, in a
    fixed order."""
    import hashlib
    from paper_2307_01416_gb300 import build_ext
    h = hashlib.sha256()
    for name in TRANSPORT_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2307_01416_gb300", "csrc", name), "rb").read())
        h.update(" ".join(build_ext.NVCC_FLAGS[:5] + build_ext.FILE_FLAGS.get(name, [])).encode())
    return h.hexdigest()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------------------- statistical uncertainty
SIGMA_TARGET = 0.005


def nominal_sigma_rel(eng, pb, spots, seed: int, n_batches: int = 10):
    """Statistical uncertainty of the set's nominal composite dose (every
    spot, weight 1 per history) by the batch method: n_batches independent
    dose runs, each with 1/n_batches of every spot's histories; sigma_rel =
    mean SE / D over tissue voxels at or above half the maximum."""
    from paper_2307_01416_gb300 import uncertainty as U
    mask = W.tissue_mask(pb)
    sub = spots.copy()
    sub["n_hist"] = U.split_histories(spots["n_hist"], n_batches)
    doses = []
    for b in range(n_batches):
        d, _, _ = eng.run_spots(sub, W.Scenario(), W.Options(seed=seed + 100003 * (b + 1)))
        doses.append(d.reshape(-1).double().cpu().numpy())
    s, nvox = U.batch_sigma_rel(np.stack(doses), mask, level=0.5)
    return {"sigma_rel": s, "target": SIGMA_TARGET, "voxels": nvox, "batches": n_batches,
            "histories": n_batches * int(sub["n_hist"].sum()), "hist_scale": W.IM_SET_HIST_SCALE,
            "method": "batch method: %d independent dose runs of the nominal scenario, each 1/%d of every spot's "
                      "histories; mean SE/D over tissue voxels (HU >= -500) at >= 50%% of the maximum"
                      % (n_batches, n_batches)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(pb, spots, target_hist: int, seed: int = 1234):
    """Deterministic subset: every k-th spot of the nominal scenario with its
    full history count, about target_hist histories in total."""
    k = max(1, int(round(spots["n_hist"].sum() / max(target_hist, 1))))
    idx = np.arange(0, len(spots), k)
    return idx


def time_oracle(pb, spots, idx, opts):
    from oracle import oracle as O
    O.lib()
    sp = O.oracle_spots(spots[idx], spot_keys=idx)
    t0 = time.perf_counter()
    _, tl, _ = O.run(pb, sp, W.Scenario(), opts, mode=0)
    dt = time.perf_counter() - t0
    return tl, dt, O.max_threads()


def cpu_baseline(pb, spots, seconds: float):
    from oracle import oracle as O
    opts = W.Options(seed=1234)
    # calibrate on a small subset, then run a subset sized for `seconds`
    idx = oracle_sample(pb, spots, 20000)
    tl, dt, cores = time_oracle(pb, spots, idx, opts)
    rate = tl["histories"] / dt
    idx = oracle_sample(pb, spots, int(rate * seconds))
    tl, dt, cores = time_oracle(pb, spots, idx, opts)
    return {"value": tl["histories"] / dt, "unit": "protons/s", "cores": cores, "kind": "oracle",
            "sample": "nominal scenario, every %d-th spot (%d spots, %d histories, %.1f s FP64 C oracle, OpenMP)"
                      % (max(1, len(spots) // max(len(idx), 1)), len(idx), int(tl["histories"]), dt)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pb, spots, scens, _ = build_workload(False)
    from oracle import oracle as O
    O.lib()
    opts = W.Options(seed=1234)
    idx0 = oracle_sample(pb, spots, 20000)
    tl, dt, cores = time_oracle(pb, spots, idx0, opts)
    rate = tl["histories"] / dt
    idx = oracle_sample(pb, spots, int(rate * 8.0))
    for _ in range(args.warmup):
        time_oracle(pb, spots, idx0, opts)
    hist, tot = 0.0, 0.0
    for _ in range(args.steps):
        tl, dt, cores = time_oracle(pb, spots, idx, opts)
        hist += tl["histories"]
        tot += dt
    value = hist / tot
    set_hist = float(spots["n_hist"].sum()) * len(scens)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "protons/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "every %d-th spot of the nominal scenario, %d histories per step"
                       % (max(1, len(spots) // len(idx)), int(hist / args.steps))},
            "s_per_im_set": set_hist / value,
            "cpu_baseline": {"value": value, "unit": "protons/s", "cores": cores, "kind": "oracle",
                             "sample": "%d histories per step" % int(hist / args.steps)},
            "e2e": {"value": value, "unit": "protons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- ranks
def rank_seed(rank: int) -> int:
    """Each rank computes its own independent set (weak scaling)."""
    return 1234 + 7919 * rank


def reduce_over_ranks(t: float, hist: float, world: int, device: str):
    """(max of the ranks' timed seconds, sum of their histories): the job's
    time is its slowest rank's, its throughput every rank's work."""
    if world <= 1:
        return float(t), float(hist)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    hh = torch.tensor([float(hist)], dtype=torch.float64, device=device)
    dist.all_reduce(hh)
    return float(tt.item()), float(hh.item())


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return run_ncu_case(args)
    import torch
    import torch.distributed as dist
    from paper_2307_01416_gb300 import vpmc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pb, spots, scens, target = build_workload(args.small)
    free_b, total_b = torch.cuda.mem_get_info()
    print("device memory: %.1f GB free of %.1f GB" % (free_b / 1e9, total_b / 1e9), file=sys.stderr)
    # independent problems per rank (weak scaling): each rank computes its own set
    opts = W.Options(seed=rank_seed(rank))
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        eng = vpmc.Engine(pb, stream=stream)
        launches = 0
        for _ in range(args.warmup):
            mats, st = eng.influence_matrix(spots, scens, opts)
            del mats
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        kern_ms, steps, hist, nnz, ops, ms_patient, patient_steps, scratch_b, ovf = 0.0, 0, 0, 0, 0.0, 0.0, 0, 0, 0
        for _ in range(args.steps):
            flush.fill_(1.0)                       # evict L2 between sets
            mats, st = eng.influence_matrix(spots, scens, opts)
            kern_ms += st["ms"]
            steps += st["steps"]
            ops += algorithmic_ops(st)
            ms_patient += st["ms_patient"]
            patient_steps += st["steps"] - st["steps_rs"] - st["steps_aperture"]
            scratch_b += st["scratch_bytes"]
            ovf += st["ovf_records"]
            hist += st["histories"]
            launches += st["launches"] + 1
            nnz = sum(int(m["val"].numel()) for m in mats)
            last_mats = mats
            del mats
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ck = clocks.stop()
        t = ev0.elapsed_time(ev1) / 1000.0
        unc = nominal_sigma_rel(eng, pb, spots, opts.seed) if rank == 0 else None   # untimed
        eng.close()                                # frees the set's column scratch before the e2e leg
    t, hist_all = reduce_over_ranks(t, hist, world, "cuda")
    value = hist_all / t
    ms_per_step = 1000.0 * t / args.steps

    out = None
    if rank == 0:
        peaks = measured_peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        peak_tops = nsm * 4 * 32 * sm_max * 1e6 / 1e12
        achieved = ops / (kern_ms / 1000.0) / 1e12
        traffic = transport_traffic(patient_steps / args.steps, hist / args.steps / len(scens))
        l2 = vpmc.measure_l2_atomics()                 # untimed: the secondary bound's peak
        # the influence-matrix assembly outside the transport: its time, and its
        # bytes (column scratch zeroed once and read three times, CSR written)
        # against 16 algorithmic bytes per stored entry (8 read, 8 written)
        nrows = int(pb.scoring.nvox)
        csr_b = nnz * 8 + len(scens) * (nrows + 1) * 8
        fin_ms = ms_per_step - kern_ms / args.steps
        fin_b = 4 * scratch_b / args.steps + csr_b
        finalise = {"ms_per_set": fin_ms, "bytes_per_set": fin_b, "nnz_per_set": nnz,
                    "scratch_bytes_per_set": scratch_b / args.steps, "out_of_box_records_per_set": ovf / args.steps,
                    "algorithmic_bytes_per_set": 16.0 * nnz,
                    "gbs": fin_b / (fin_ms * 1e-3) / 1e9 if fin_ms > 0 else None,
                    "note": "set time minus the transport kernels' CUDA-event time; scratch = dense per-(scenario, "
                            "spot) column boxes cut at each energy layer's reach along its field, zeroed, scanned for "
                            "column maxima, then read by the count and fill passes of the CSR; deposits beyond a box "
                            "are out-of-box records, merged into the CSR"}
        adds_rate = patient_steps / (ms_patient / 1000.0) if ms_patient > 0 else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved / peak_tops, "traffic": traffic, "kernel": "k_source_rs+k_aperture+k_patient",
                "peak_note": "%d SMs x 4 sub-partitions x 32 lanes x %.0f MHz (max SM clock) lane-ops/s; "
                             "lane-ops per condensed-history step: %d in the patient, %d in the range shifter, "
                             "%d in the brass" % (nsm, sm_max, OPS_PER_STEP, OPS_PER_STEP_RS, OPS_PER_STEP_BRASS),
                "kernel_ms_per_step": kern_ms / args.steps, "steps_per_launch": steps / args.steps,
                "ops_per_step": ops / max(steps, 1),
                "l2_atomic": {"kernel": "k_patient", "unit": "adds/s",
                              "achieved": adds_rate, "peak": l2["adds_per_s"],
                              "frac": adds_rate / l2["adds_per_s"] if adds_rate else None,
                              "k_patient_ms_per_step": ms_patient / args.steps,
                              "note": "one 64-bit scoring add per patient step (plain atomics; warp aggregation "
                                      "would issue fewer) over k_patient's CUDA-event time; peak = "
                                      "vpmc_measure_l2_atomics over a 32 MiB buffer"}}
        e2e = _leg(lambda: e2e_leg(pb, spots, scens, opts, args), not args.no_e2e)
        cpu = _leg(lambda: cpu_baseline(pb, spots, args.cpu_seconds), not args.no_cpu_baseline and world == 1)
        opt = _leg(lambda: optimizer_leg(pb, target, last_mats, args), not args.no_optimizer and world == 1)
        del last_mats
        edge = _leg(lambda: edge_sweep_leg(args, peak_tops), not args.no_edge_sweep and world == 1)
        div = _leg(lambda: divergent_leg(pb, spots, scens, opts, args, value, peak_tops),
                   not args.no_divergent and world == 1)
        dyn = _leg(lambda: dynamic_leg(scens, opts, value, peak_tops), not args.no_dynamic and world == 1)
        sur = _leg(lambda: surrogate_leg(pb, spots, scens, opts, args, value),
                   not args.no_surrogate and world == 1 and not args.small)
        set_hist = float(spots["n_hist"].sum()) * len(scens)
        out = {"metric": METRIC, "value": value, "unit": "protons/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD + (" (reduced histories)" if args.small else ""),
                          "scenarios": len(scens), "spots_per_scenario": int(len(spots)),
                          "histories_per_set": int(set_hist), "nnz_per_set": nnz,
                          "sigma_rel": unc["sigma_rel"] if unc else None, "uncertainty": unc,
                          "finalise": finalise,
                          "l2": "512 MiB buffer written between sets; the set's 100+ GB column scratch exceeds L2",
                          "parallelism": "independent sets per GPU" if world > 1 else "1 GPU"},
               "s_per_im_set": ms_per_step / 1000.0,
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck,
               "surrogate": sur, "optimizer": opt, "edge_sweep": edge, "divergent_aperture": div,
               "dynamic_aperture": dyn}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _leg(fn, enabled: bool):
    """One secondary leg of the bench line: its dict, None when disabled, or
    {"error": ...} when it raised (the main measurement still prints)."""
    if not enabled:
        return None
    try:
        return fn()
    except Exception as e:                                      # noqa: BLE001
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": "%s: %s" % (type(e).__name__, e)}


def run_sur_case(args):
    """The surrogate network's tcgen05 kernels on 2^20 plain training tracks
    (8 edge geometries): per step one forward pass over 2^22 rows (the tracks'
    inputs four times; k_sur_forward) and one training epoch in batches of
    16,384 (k_sur_train and k_sur_adam per batch), each timed with CUDA
    events."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    torch.cuda.set_device(0)
    tr = vpmc.Engine(vpmc.surrogate_training_problem())
    feat, target, label = tr.surrogate_tracks(list(range(8)), 1 << 17, W.Options(seed=W.SURROGATE_SEED))
    tr.surrogate_init(7)
    x = feat.repeat(4, 1).contiguous()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for i in range(args.warmup + args.steps):
        ev[0].record()
        tr.surrogate_forward(x)
        ev[1].record()
        tr.surrogate_train(feat, target, label, batch=16384, epochs=1, lr=2e-3, lr_min=2e-3)
        ev[2].record()
        torch.cuda.synchronize()
        fwd_ms, train_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        print(json.dumps({"case": "ncu-sur", "iter": i, "forward_rows": int(x.shape[0]), "forward_ms": fwd_ms,
                          "forward_tflops": x.shape[0] * SUR_FWD_FLOP / (fwd_ms * 1e-3) / 1e12,
                          "train_rows": int(feat.shape[0]), "train_ms": train_ms,
                          "train_tflops": feat.shape[0] * SUR_TRAIN_FLOP / (train_ms * 1e-3) / 1e12}))
    tr.close()
    return 0


def run_ncu_case(args):
    """Every 10th spot of the set's nominal scenario (about 3.3e6 histories,
    full physics) with a fixed launch (k_source_rs 768 threads, k_aperture 512, k_patient 896,
    chunk 32): one launch of each transport kernel per step.  'dose' scores a
    16 MB grid (warp-aggregated atomics); 'im' scores the spots' influence-matrix
    columns (about 1 GB of column scratch, plain atomics), the bench's own
    scoring path, small enough for an ncu capture."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    if args.ncu_case == "sur":
        return run_sur_case(args)
    pb, spots, scens, target = build_workload(False)
    if args.ncu_case == "opt":
        return run_opt_case(args, pb, spots, scens, target)
    sub = spots[::10]
    torch.cuda.set_device(0)
    eng = vpmc.Engine(pb)
    opts = W.Options(seed=1234)
    for i in range(args.warmup + args.steps):
        if args.ncu_case in ("im", "im13"):
            sc = scens if args.ncu_case == "im13" else [W.Scenario()]
            mats, st = eng.influence_matrix(sub, sc, opts, block_size=896, aggregate=0, chunk=32)
            del mats
        else:
            dose, st, _ = eng.run_spots(sub, W.Scenario(), opts, block_size=896, aggregate=1, chunk=32)
        print(json.dumps({"case": "ncu-" + args.ncu_case, "iter": i, "histories": st["histories"],
                          "steps": st["steps"], "steps_rs": st["steps_rs"], "steps_aperture": st["steps_aperture"],
                          "kernel_ms": st["ms"], "ms_devices": st["ms_devices"], "ms_patient": st["ms_patient"],
                          "ops_per_step": algorithmic_ops(st) / max(st["steps"], 1),
                          "steps_per_s": st["steps"] / (st["ms"] / 1000.0)}))
    eng.close()
    return 0


def run_opt_case(args, pb, spots, scens, target):
    """The robust optimisation over the 13-scenario set of every
    opt_stride-th spot (stride 1: the bench's full set, 4.7 GB of CSR; stride
    4: about 1.2 GB): the set is computed once, then warmup + steps calls of
    opt_iterations iterations."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    torch.cuda.set_device(0)
    sub = spots[::args.opt_stride]
    eng = vpmc.Engine(pb)
    mats, _ = eng.influence_matrix(sub, scens, W.Options(seed=1234))
    eng.close()
    cls_np = W.structure_classes(pb.scoring, target[0], target[1])
    cls = torch.from_numpy(cls_np).cuda()
    rl = np.diff(mats[0]["row_ptr"].cpu().numpy())
    nzr = rl[rl > 0]
    print("rows %d, non-empty %d, nnz/row over non-empty: mean %.1f, p50 %d, p90 %d, p99 %d, max %d; "
          "target+ring rows %d with %d nnz" % (rl.size, nzr.size, nzr.mean(), np.percentile(nzr, 50),
                                               np.percentile(nzr, 90), np.percentile(nzr, 99), nzr.max(),
                                               int(np.sum(cls_np > 0)), int(rl[cls_np > 0].sum())), file=sys.stderr)
    x0 = torch.ones(len(sub), dtype=torch.float32, device="cuda")
    x0 *= 1.0 / float(vpmc.weights_dose(mats[0], x0)[cls == 1].mean())
    b = optimizer_bytes(mats, cls_np)
    for i in range(args.warmup + args.steps):
        x = x0.clone()
        hist, ms, setup_ms = vpmc.robust_optimize(mats, cls, x, 1.0, iterations=args.opt_iterations)
        per = ms / args.opt_iterations
        print(json.dumps({"case": "ncu-opt", "iter": i, "spots": int(len(sub)), "ms_per_iteration": per, "setup_ms": setup_ms,
                          "bytes_per_iteration": b, "GB_per_s": b / per / 1e6, "objective_last": float(hist[-1])}))
    return 0


# algorithmic FLOPs per row of the surrogate network (6 -> 128 -> 128 -> 45):
# forward 2 (6*128 + 128*128 + 128*45); a training row adds the backward GEMMs
# dh2, dW3, dh1, dW2 (with db2) and dW1 (with db1)
SUR_FWD_FLOP = 2 * (6 * 128 + 128 * 128 + 128 * 45)
SUR_TRAIN_FLOP = SUR_FWD_FLOP + 2 * (45 * 128 + 45 * 128 + 128 * 128 + 128 * 129 + 128 * 7)


def surrogate_leg(pb, spots, scens, opts, args, plain_value):
    """The same set with the learned aperture surrogate: the network is
    trained on the GPU first (plain training tracks, Adam; not timed), then
    one warm-up set and min(steps, 2) timed sets with opts.surrogate.  Also
    the throughput of the tensor-core forward and training kernels."""
    import dataclasses
    import torch
    from paper_2307_01416_gb300 import vpmc
    tpb, epochs, batch = 12_500_000, 7, 16384
    tr = vpmc.Engine(vpmc.surrogate_training_problem())
    t0 = time.perf_counter()
    feat, target, label = tr.surrogate_tracks(list(range(8)), tpb, W.Options(seed=W.SURROGATE_SEED))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    tr.surrogate_init(7)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    losses = tr.surrogate_train(feat, target, label, batch=batch, epochs=epochs, lr=2e-3, lr_min=2e-5)
    ev1.record()
    torch.cuda.synchronize()
    train_s = ev0.elapsed_time(ev1) / 1000.0
    rows = float(feat.shape[0]) * epochs
    x = feat[: 1 << 22].contiguous()
    tr.surrogate_forward(x)
    ev0.record()
    for _ in range(5):
        tr.surrogate_forward(x)
    ev1.record()
    torch.cuda.synchronize()
    fwd_s = ev0.elapsed_time(ev1) / 1000.0 / 5
    w = tr.surrogate_get_weights()
    del feat, target, label, x
    tr.close()
    peaks = measured_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    fwd_tf = (1 << 22) * SUR_FWD_FLOP / fwd_s / 1e12
    train_tf = rows * SUR_TRAIN_FLOP / train_s / 1e12
    sopts = dataclasses.replace(opts, surrogate=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        eng = vpmc.Engine(pb, stream=stream)
        eng.surrogate_set_weights(w)
        mats, _ = eng.influence_matrix(spots, scens, sopts)
        del mats
        torch.cuda.synchronize()
        n = max(1, min(args.steps, 2))
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        hist, kern_ms, steps = 0, 0.0, 0
        for _ in range(n):
            mats, st = eng.influence_matrix(spots, scens, sopts)
            hist += st["histories"]
            kern_ms += st["ms"]
            steps += st["steps"]
            del mats
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1000.0
        eng.close()
    value = hist / t
    return {"value": value, "unit": "protons/s", "s_per_im_set": t / n, "sets": n,
            "speedup_vs_plain": value / plain_value, "kernel_ms_per_set": kern_ms / n, "steps_per_set": steps / n,
            "training": {"tracks": 8 * tpb, "epochs": epochs, "batch": batch, "generate_s": gen_s,
                         "train_s": train_s, "final_loss": float(losses[-1]),
                         "note": "plain brass transport tracks of 8 circular-edge geometries, E 40-230 MeV; "
                                 "dose error vs the plain path is checked in tests/test_gpu_surrogate_dose.py"},
            "tensor_roofline": {"bound": "tensor", "unit": "TFLOP/s", "peak": bf16_peak,
                                "forward": {"achieved": fwd_tf, "frac": fwd_tf / bf16_peak, "rows": 1 << 22,
                                            "flop_per_row": SUR_FWD_FLOP},
                                "train": {"achieved": train_tf, "frac": train_tf / bf16_peak, "rows": rows,
                                          "flop_per_row": SUR_TRAIN_FLOP},
                                "peak_note": "bf16_tflops of MEASURED_PEAKS.json (cuBLAS burst)"}}


def optimizer_bytes(mats, cls: np.ndarray) -> float:
    """Algorithmic HBM bytes of one robust-optimisation iteration on the
    compact target/ring rows the optimiser builds once per call (rows whose
    voxel is neither target nor ring do not enter the objective): forward,
    per scenario, 2 B spot index + 4 B value per entry and 8 B row pointer +
    4 B dose written + 1 B class per row; gradient, the same per entry and 8 B
    row pointer + 4 B dose + 1 B class per row of the worst scenario (the mean
    over scenarios stands for it; rows with f'(d) = 0, which the kernel skips,
    are counted); Adam: x, m, v read and written (24 B per spot).  Padding
    entries and the gradient blocks' partial sums are not counted."""
    n_cols = int(mats[0]["shape"][1])
    tr = (cls == 1) | (cls == 2)
    n_tr = float(tr.sum())
    nnz_tr = []
    for m in mats:
        rp = m["row_ptr"].cpu().numpy()
        nnz_tr.append(float(np.sum(np.diff(rp)[tr])))
    fwd = sum(6.0 * z + 13.0 * n_tr for z in nnz_tr)
    bwd = 6.0 * float(np.mean(nnz_tr)) + 13.0 * n_tr
    return fwd + bwd + 24.0 * n_cols


def optimizer_leg(pb, target, mats, args):
    """Robust spot-weight optimisation over the timed set's 13 influence
    matrices (target = the 8.4 cc sphere, ring = 10 mm shell around it):
    3 warm-up iterations, then args.opt_iterations timed on the device."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    center, r_t = target
    cls_np = W.structure_classes(pb.scoring, center, r_t)
    cls = torch.from_numpy(cls_np).cuda()
    x = torch.ones(int(mats[0]["shape"][1]), dtype=torch.float32, device="cuda")
    d0 = vpmc.weights_dose(mats[0], x)
    x *= 1.0 / float(d0[cls == 1].mean())
    vpmc.robust_optimize(mats, cls, x.clone(), 1.0, iterations=3)
    hist, ms, setup_ms = vpmc.robust_optimize(mats, cls, x, 1.0, iterations=args.opt_iterations)
    idx = vpmc.target_indices(mats, cls, 1.0, x)
    n_tr = int(np.sum(cls_np > 0))
    per_it = ms / 1000.0 / args.opt_iterations
    b = optimizer_bytes(mats, cls_np)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    gbs = b / per_it / 1e9
    return {"iterations": args.opt_iterations, "ms_per_iteration": 1000.0 * per_it, "setup_ms": setup_ms,
            "target_ring_rows": n_tr,
            "objective_first": float(hist[0]), "objective_last": float(hist[-1]),
            "worst_V100": float(idx[:, 0].min()), "worst_Dmin": float(idx[:, 1].min()),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "bytes_per_iteration": b, "traffic": None,
                         "kernel": "k_fwd (13 scenarios) + k_bwd_fixed + k_adam_fixed",
                         "peak_note": "hbm_gbs of MEASURED_PEAKS.json (STREAM-style copy)"},
            "note": "per iteration: 13 products on the compact target/ring rows (built once per call, "
                    "setup_ms), worst-case selection, the transposed product and the Adam step, all on the "
                    "device; target 8.4 cc sphere, ring = 10 mm shell"}


def edge_sweep_leg(args, peak_tops):
    """The single-beamlet edge sweep (Sec. 2.D.1): 97 energies from 71.3 to
    228.8 MeV, one beamlet on the rim of a 1 cm opening in 30 mm brass, water
    on a 1 mm grid (40 x 40 x 350 mm), without (AP) and with (APRS) the 45 mm
    range shifter; args.edge_hist histories per beamlet, full physics.  Two
    ways, each timed on the device after one untimed call per machine:
    'per_beamlet': one dose call per beamlet (194 dose grids);
    'batched': one influence-matrix call per machine whose 97 columns are the
    beamlets' doses (one transport launch per machine)."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    energies = W.machine_energies()
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        for mode in ("per_beamlet", "batched"):
            total_s, hist, steps, kern_ms, launches, ops = 0.0, 0, 0, 0.0, 0, 0.0
            for rs in (False, True):
                pb = W.edge_beamlet_problem(rs)
                eng = vpmc.Engine(pb, stream=stream)
                spots = W.make_spots([tuple(W.edge_beamlet_spot(e, args.edge_hist)[0]) for e in energies])
                if mode == "per_beamlet":
                    eng.run_spots(W.edge_beamlet_spot(150.0, args.edge_hist), W.Scenario(), W.Options(seed=5))
                else:
                    m, _ = eng.influence_matrix(spots, [W.Scenario()], W.Options(seed=5))
                    del m
                torch.cuda.synchronize()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                if mode == "per_beamlet":
                    for k, e in enumerate(energies):
                        d, st, _ = eng.run_spots(W.edge_beamlet_spot(e, args.edge_hist), W.Scenario(),
                                                 W.Options(seed=100 + k))
                        hist += st["histories"]
                        steps += st["steps"]
                        ops += algorithmic_ops(st)
                        kern_ms += st["ms"]
                        launches += st["launches"]
                        del d
                else:
                    m, st = eng.influence_matrix(spots, [W.Scenario()], W.Options(seed=100))
                    hist += st["histories"]
                    steps += st["steps"]
                    ops += algorithmic_ops(st)
                    kern_ms += st["ms"]
                    launches += st["launches"] + 1
                    del m
                ev1.record(stream)
                torch.cuda.synchronize()
                total_s += ev0.elapsed_time(ev1) / 1000.0
                eng.close()
            achieved = ops / (kern_ms / 1000.0) / 1e12
            out[mode] = {"s_per_sweep": total_s, "value": hist / total_s, "histories": hist,
                         "gpu_launches": launches,
                         "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                                      "frac": achieved / peak_tops, "kernel": "k_source_rs+k_aperture+k_patient"}}
    best = min(out, key=lambda k: out[k]["s_per_sweep"])
    return {"beamlets": 2 * int(energies.size), "histories_per_beamlet": args.edge_hist, "unit": "protons/s",
            "value": out[best]["value"], "s_per_sweep": out[best]["s_per_sweep"], "best": best, **out,
            "note": "97 energies 71.3-228.8 MeV x (AP, APRS), beamlet on the rim of a 1 cm opening in 30 mm "
                    "brass, water 40x40x350 mm at 1 mm; parity vs the oracle in tests/test_gpu_edge_sweep.py"}


def divergent_leg(pb, spots, scens, opts, args, plain_value, peak_tops):
    """The same 13-scenario set with divergent aperture walls (virtual source
    args.divergent_sad mm upstream of the isocentre; the polygons are the
    openings at the blocks' downstream faces): one untimed and one timed set."""
    import copy
    import torch
    from paper_2307_01416_gb300 import vpmc
    dpb = copy.deepcopy(pb)
    for b in dpb.beams:
        b.ap_sad = float(args.divergent_sad)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        eng = vpmc.Engine(dpb, stream=stream)
        mats, _ = eng.influence_matrix(spots, scens, opts)
        del mats
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        mats, st = eng.influence_matrix(spots, scens, opts)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1000.0
        nnz = sum(int(m["val"].numel()) for m in mats)
        del mats
        eng.close()
    achieved = algorithmic_ops(st) / (st["ms"] / 1000.0) / 1e12
    return {"sad_mm": float(args.divergent_sad), "value": st["histories"] / t, "unit": "protons/s",
            "s_per_im_set": t, "relative_to_parallel": st["histories"] / t / plain_value, "nnz_per_set": nnz,
            "gpu_launches": st["launches"] + 1,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                         "frac": achieved / peak_tops, "kernel": "k_source_rs+k_aperture+k_patient"},
            "note": "same workload and seeds as the main line, divergent brass walls; parity vs the oracle in "
                    "tests/test_gpu_divergent.py"}


def dynamic_leg(scens, opts, plain_value, peak_tops):
    """The 13-scenario set with energy-layer-specific apertures: the same
    spots and histories, one beam entry per (field, layer) whose opening is
    the target's cross-section at the layer's depth plus 5 mm (36 entries):
    one untimed and one timed set."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    pb, spots, _, _ = W.im_set_plan(dynamic_aperture=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        eng = vpmc.Engine(pb, stream=stream)
        mats, _ = eng.influence_matrix(spots, scens, opts)
        del mats
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        mats, st = eng.influence_matrix(spots, scens, opts)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1000.0
        nnz = sum(int(m["val"].numel()) for m in mats)
        del mats
        eng.close()
    achieved = algorithmic_ops(st) / (st["ms"] / 1000.0) / 1e12
    return {"beam_entries": len(pb.beams), "value": st["histories"] / t, "unit": "protons/s", "s_per_im_set": t,
            "relative_to_static": st["histories"] / t / plain_value, "nnz_per_set": nnz,
            "e_aperture_fraction": st["e_aperture"] / st["e_in"], "gpu_launches": st["launches"] + 1,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                         "frac": achieved / peak_tops, "kernel": "k_source_rs+k_aperture+k_patient"},
            "note": "same spots, histories and seeds as the main line; per-layer openings; parity vs the oracle "
                    "in tests/test_gpu_dynamic_aperture.py"}


def e2e_leg(pb, spots, scens, opts, args):
    """The same metric through the public API from host buffers: each step
    creates the geometry from the host CT, sets the fields, computes the set
    and copies every CSR back to pinned host memory."""
    import torch
    from paper_2307_01416_gb300 import vpmc
    steps = max(1, min(args.steps, 2))
    host = None
    t_tot, h2d, d2h = 0.0, 0, 0
    hist = 0
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eng = vpmc.Engine(pb, host_ct=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        mats, st = eng.influence_matrix(spots, scens, opts)
        t2 = time.perf_counter()
        if host is None:
            host = [{k: torch.empty(m[k].shape, dtype=m[k].dtype, pin_memory=True) for k in ("row_ptr", "col", "val")}
                    for m in mats]
        nb, realloc = 0, 0
        torch.cuda.synchronize()
        t2b = time.perf_counter()
        for m, h in zip(mats, host):
            for k in ("row_ptr", "col", "val"):
                if h[k].numel() != m[k].numel():
                    h[k] = torch.empty(m[k].shape, dtype=m[k].dtype, pin_memory=True)
                    realloc += 1
                h[k].copy_(m[k], non_blocking=True)
                nb += m[k].numel() * m[k].element_size()
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        print("e2e step %d: %d pinned reallocations; %.1f GB back in %.3f s after %.3f s of queued device work"
              % (i, realloc, nb / 1e9, t3 - t2b, t2b - t2), file=sys.stderr)
        eng.close()
        dt = time.perf_counter() - t0
        print("e2e step %d: context %.3f s, influence matrices %.3f s (device %.3f s), copy back %.3f s, close %.3f s"
              % (i, t1 - t0, t2 - t1, st["ms"] / 1000.0, t3 - t2, time.perf_counter() - t3), file=sys.stderr)
        if i == 0:
            continue                                   # first pass allocates the pinned buffers
        t_tot += dt
        hist += st["histories"]
        d2h = nb
        h2d = pb.hu.nbytes + len(spots) * 56 + len(scens) * 32
    return {"value": hist / t_tot, "unit": "protons/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps}


if __name__ == "__main__":
    sys.exit(main())

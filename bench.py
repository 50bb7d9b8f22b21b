"""Throughput benchmark of the fused FDTD leapfrog (arXiv 2401.07416) on GB300.

Workload (default): the 512 x 512 x 1024 throughput run (h = 0.05 bohr, 4-layer
16 x 16 softened-Coulomb slab, cos^2 absorbing layers at the z ends, detector
flux every step, norm/energy reductions every 20 steps), psi and V stored in FP32
with Kahan-compensated updates, two time steps fused per kernel launch.  One
bench step = one leapfrog time step of the whole grid.  Inputs are synthetic
(seeded), larger than L2 (the state alone is ~10 GB), so no L2 flush is needed.

Metric: grid-cell updates per second (cells x steps / device time), whole job.
Also reported: the FP64 unfused GPU step on the same grid and the FP32 variants,
the roofline of the dominant kernel (HBM bytes of the algorithm per launch over
the launch's CUDA-event time, against the measured HBM copy bandwidth), the FP64
oracle timed on this host's cores (a baseline, not the target), and the same
metric end to end through the C ABI from pinned host buffers, over complete
runs of the workload (1000 steps each, set-up and result read-back included).

Multi-GPU (torchrun): each rank advances its own replica (weak scaling, no data
exchange), the time is the max over ranks.  `--impl reference` times the FP64
CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

from paper_2401_07416_gb300 import workloads as W

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
FALLBACK_HBM = 6800.0
METRIC = "3D FDTD cell-updates/s & %HBM roofline; FP32/batched/adjoint vs FP64 plain"

# algorithmic HBM bytes per grid node and fused launch: fields read + written once
BYTES_PER_NODE = {W.FP64: 40, W.FP32: 20, W.FP32_KAHAN: 36}
PREC_NAME = {W.FP64: "f64", W.FP32: "f32", W.FP32_KAHAN: "f32+kahan"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="kahan", choices=["kahan", "fp32", "fp64"])
    ap.add_argument("--tblock", type=int, default=0, help="steps fused per launch (0: autotuned)")
    ap.add_argument("--ncu-case", action="store_true", help="mid-size run of the fused kernel for ncu")
    ap.add_argument("--variant", type=int, default=None,
                    help="kernel variant (with --tblock) instead of the autotuner's pick; "
                         "--ncu-case default 0")
    ap.add_argument("--chunk", type=int, default=None,
                    help="z-planes per work item with --variant (default: the makespan model's)")
    ap.add_argument("--no-extras", action="store_true", help="skip variants, e2e and CPU baseline")
    ap.add_argument("--batch-case", action="store_true",
                    help="the 48-film batch (FP32+Kahan, variant and z-chunk fixed by --variant / "
                         "--chunk, default 0 and the model's) for ncu: two launches, then --steps steps")
    ap.add_argument("--adjoint-case", action="store_true",
                    help="one FP32+Kahan forward and adjoint of the 96x96x192 case (--steps steps) for ncu")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_time_and_value(ms_local: float, cells: int, steps: int, world: int, reduce_max):
    """Max over ranks of the timed region (ms) and the whole-job value: every rank
    advances its own replica of `cells` nodes for `steps` steps (weak scaling)."""
    t_max = float(reduce_max(ms_local))
    return t_max, world * cells * steps / (t_max * 1e-3)


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.count(",") >= 8]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ("step_common.cuh", "tmem_common.cuh", "step_kernels.cu", "step_tmem.cu", "step_slim.cu")


def kernel_source_hash() -> str:
    """Hash of the fused-step kernel sources the traffic figures were taken on."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2401_07416_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_function(variant: str) -> str:
    """CUDA kernel that a fused-step variant launches (its name in ncu listings)."""
    layout = variant.split("_")[2] if variant.count("_") >= 2 else ""
    if layout in ("roll", "slim", "hyb", "split"):
        return "fused_step_slim_kernel"
    if layout in ("tmem", "ws"):
        return "fused_step_tmem_kernel"
    return "fused_step_kernel"


def ncu_traffic(variant: str, cells: int):
    """(DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    scaled to `cells` grid nodes, or None; why it is None)."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except OSError as e:
        return None, f"no traffic file: {e}"
    if variant not in d:
        return None, f"no ncu capture of variant {variant}"
    e = d[variant]
    h = kernel_source_hash()
    if e.get("source_hash") != h:
        return None, f"kernel sources changed since the capture ({e.get('source_hash')} != {h})"
    if e["cells"] == cells:
        return e["dram_bytes_per_launch"], f"single-pass ncu capture of this grid ({e.get('z_chunk')}-plane z-chunks)"
    return (e["dram_bytes_per_launch"] * cells / e["cells"],
            f"single-pass ncu capture of a {e['cells']}-node grid, scaled by nodes")


# ------------------------------------------------------------------ CPU oracle timing

def cpu_sample_workload():
    """A bounded slab of the 512x512x1024 workload: 512 x 512 x 16 planes around the
    packet start, the workload's atoms, walls at the slab faces."""
    wl = W.config5()
    g = wl.grid
    z0 = int(round(wl.packet.r0[2] / g.hz)) - 8
    sub = W.Grid(nx=g.nx, ny=g.ny, nz=16, hx=g.hx, hy=g.hy, hz=g.hz, dt=g.dt,
                 bc=(W.PERIODIC, W.PERIODIC, W.DIRICHLET), obs_every=20)
    return wl, sub, z0


def oracle_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_state():
    import oracle
    wl, sub, z0 = cpu_sample_workload()
    g = wl.grid
    origin = (0.0, 0.0, z0 * g.hz)
    period = [l if b == W.PERIODIC else 0.0 for l, b in zip(g.lengths, g.bc)]
    V = oracle.potential_atoms_window(sub, origin, period, wl.atoms, rc=0.5 * min(period[:2]))
    R0, I0 = oracle.wavepacket_window(sub, origin, wl.packet.r0, wl.packet.sigma, wl.packet.k0)
    return sub, V, R0, oracle.init_half(sub, V, R0, I0)


def time_oracle(seconds: float, serial_seconds: float = 4.0):
    """FP64 oracle steps on the bounded sample until `seconds` of wall time on all
    host cores, then `serial_seconds` on one thread (the paper's serial comparison)."""
    import oracle
    sub, V, R0, I0 = oracle_sample_state()

    def timed(limit):
        R, I = R0, I0
        steps = 0
        t0 = time.perf_counter()
        while True:
            R, I, _, _ = oracle.run(sub, V, R, I, 2, use_mask=False, flux=False)
            steps += 2
            el = time.perf_counter() - t0
            if el >= limit:
                return steps, el

    cores = oracle_cores()
    oracle.set_threads(cores)
    steps, el = timed(seconds)
    value = sub.cells * steps / el
    oracle.set_threads(1)
    s1, e1 = timed(serial_seconds)
    oracle.set_threads(cores)
    v1 = sub.cells * s1 / e1
    return {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "ns_per_cell_update": 1e9 / value,
            "sample": f"{steps} FP64 oracle steps on a 512x512x16 z-slab of the 512x512x1024 "
                      f"workload ({sub.cells} nodes), {el:.1f} s wall, OpenMP {cores} threads",
            "serial": {"value": v1, "unit": "cell-updates/s", "cores": 1,
                       "ns_per_cell_update": 1e9 / v1,
                       "sample": f"{s1} steps of the same sample on one thread, {e1:.1f} s wall"}}


def reference_arm(args):
    """The FP64 CPU oracle as the reference implementation: W untimed and K timed
    steps on the bounded sample of the workload (rank 0 only)."""
    import oracle
    rank, world, _ = dist_info()
    if rank != 0:
        return
    sub, V, R, I = oracle_sample_state()
    if args.warmup > 0:
        R, I, _, _ = oracle.run(sub, V, R, I, args.warmup, use_mask=False, flux=False)
    t0 = time.perf_counter()
    R, I, _, _ = oracle.run(sub, V, R, I, args.steps, use_mask=False, flux=False)
    el = time.perf_counter() - t0
    value = sub.cells * args.steps / el
    cores = oracle_cores()
    sample = (f"{args.steps} timed FP64 oracle steps (after {args.warmup} untimed) on a "
              f"512x512x16 z-slab of the 512x512x1024 workload ({sub.cells} nodes), "
              f"OpenMP {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512x1024 grid, h=0.05, 4x16x16 softened-Coulomb slab "
                               "(FP64 CPU oracle on a 16-plane sample)",
                   "nx": 512, "ny": 512, "nz": 1024, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def make_ctx(T, wl, precision, tblock, V_dev=None, autotune=True):
    """Context for one workload: potential from atoms (or a device V), packet set,
    kernel variants autotuned on this grid."""
    from paper_2401_07416_gb300.sim import Sim
    s = Sim(wl.grid, precision=precision, tblock=tblock)
    if V_dev is None:
        s.set_atoms(0, wl.atoms)
    else:
        s.set_potential(0, V_dev)
    s.set_packet(0, wl.packet)
    if autotune:   # trials on the workload's own state (saved and restored by the library)
        s.autotune(4)
    return s


def align_to_depth(T, s):
    """Untimed single steps until the step counter is a multiple of the fused depth in
    use: every step sequence between two reductions (the reduction period is a
    multiple of the depth) then consists of launches of that depth only, whatever
    warm-up count came before."""
    tb = s.tuning()["tblock"]
    extra = (-int(T.tdse_observables(s.ctx, 0)["step"])) % tb
    if extra:
        s.step(extra)
    return extra


def timed_steps(torch, T, s, steps, warmup, barrier):
    """W untimed steps (plus up to T-1 to align the step counter to the fused depth
    T), then K steps between CUDA events on the library's stream.  The steps are
    replayed from their CUDA graphs; the library's profiling records events around
    each replay (one depth per replay), which gives the device time per launch of
    every depth without host synchronisation inside the timed region."""
    s.step(warmup)
    align_to_depth(T, s)
    torch.cuda.synchronize()
    barrier()
    T.tdse_set_profiling(s.ctx, True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = T.tdse_get_profile(s.ctx)
    T.tdse_set_profiling(s.ctx, False)
    return ms, prof


def launch_stats(prof, depth):
    """(launches, mean device ms per launch) of the fused step at the given depth."""
    n = prof["launches_at_depth"].get(depth, 0)
    return n, (prof["ms_at_depth"][depth] / n if n else float("nan"))


def ncu_case(args):
    """A mid-size (256x256x512, ~1.3 GB) run of the fused kernel for ncu captures:
    the 512x512x1024 workload's spacing, slab geometry scaled, two warm-up launches
    then `--steps` steps, kernel variant fixed by --variant (z-chunk by --chunk)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2401_07416_gb300 import build as B
    B.build()
    from paper_2401_07416_gb300 import tdse as T
    from paper_2401_07416_gb300.sim import Sim
    prec = {"kahan": W.FP32_KAHAN, "fp32": W.FP32, "fp64": W.FP64}[args.precision]
    tb = 1 if prec == W.FP64 else max(1, args.tblock)
    g = W.Grid(nx=256, ny=256, nz=512, hx=0.05, hy=0.05, hz=0.05, dt=5e-4, mask_lo=20,
               mask_hi=20, det_k=180, obs_every=10 ** 6)
    atoms = W.square_slab(8, 4, 1.6, 0.4 * 25.6, 12.8, 12.8, W.rng_for(5), 0.05)
    with Sim(g, precision=prec, tblock=tb) as s:
        T.tdse_set_variant(s.ctx, tb, args.variant or 0)
        if args.chunk is not None:
            T.tdse_set_chunk(s.ctx, tb, args.chunk)
        s.set_atoms(0, atoms)
        s.set_packet(0, W.Packet((6.4, 6.4, 12.74), (0.0, 0.0, 2.0), (0.0, 0.0, -1.9)))
        s.step(2 * tb)
        s.step(args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": True, "cells": g.cells, "precision": args.precision,
                          "tblock": tb, "tuning": s.tuning()}))


def batch_throughput(torch, T, steps, warmup):
    """48-member film batch (uneven grids) in one context: aggregate cell-updates/s."""
    from paper_2401_07416_gb300.sim import Sim
    members = W.config3(48, W.FP32_KAHAN)
    with Sim([m.grid for m in members], precision=W.FP32_KAHAN) as s:
        for i, m in enumerate(members):
            s.set_atoms(i, m.atoms)
            s.set_packet(i, m.packet)
        s.autotune(2)
        ms, prof = timed_steps(torch, T, s, steps, warmup, lambda: None)
        tun = s.tuning()
    cells = sum(m.grid.cells for m in members)
    tb = tun["tblock"]
    nl, lms = launch_stats(prof, tb)
    # the same members one at a time, each in its own autotuned context: the batch's
    # gain over running them back to back
    solo_steps = max(10, steps // 2 // 2 * 2)
    solo_ms = 0.0
    for m in members:
        with Sim(m.grid, precision=W.FP32_KAHAN) as s1:
            s1.set_atoms(0, m.atoms)
            s1.set_packet(0, m.packet)
            s1.autotune(2)
            ms1, _ = timed_steps(torch, T, s1, solo_steps, warmup, lambda: None)
        solo_ms += ms1 * steps / solo_steps
    return {"value": cells * steps / (ms * 1e-3), "unit": "cell-updates/s", "members": 48,
            "cells": cells, "steps": steps, "precision": "f32+kahan", "tuning": tun,
            "graphs": True, "steps_per_launch": tb, "launches": nl, "avg_launch_ms": lms,
            "timed_ms": ms, "reduce_ms": prof["reduce_ms"], "reduce_launches": prof["reduce_launches"],
            "hbm_frac_of_algorithmic_bytes": BYTES_PER_NODE[W.FP32_KAHAN] * cells / (lms * 1e-3) / 1e9
                                             / measured_peaks()[0],
            "solo_sum_value": cells * steps / (solo_ms * 1e-3),
            "batch_over_solo": solo_ms / ms,
            "solo": f"each member alone, {solo_steps} steps, autotuned, same timing method"}


def absorber_reflection(torch, T):
    """Reflection coefficients of the absorbing layers.  A packet that is a plane wave
    in x, y (sigma_z = 2 bohr, k = 1.9 bohr^-1, kinetic energy 1.8 Ha, as in the
    diffraction runs) starts 12 bohr above a layer at the bottom of a 32 x 32 x
    (W + 300) grid (h = 0.1, walls in z, V = 0) and runs 28000 steps (14 a.u.).  The
    time-integrated flux through the face 2 bohr above the layer is the net downward
    transfer Phi, so the absorbed fraction is -Phi / Q0 and the reflection
    R = 1 + Phi / Q0 (FP64)."""
    from paper_2401_07416_gb300.sim import Sim
    out = {}
    cases = [("cos2_W20_eta0.1", W.MASK_COS2, 20, 0.1), ("cos2_W20_eta0.3", W.MASK_COS2, 20, 0.3),
             ("cos2_W100_eta0.1", W.MASK_COS2, 100, 0.1), ("cap_W100_0.5Ha", W.MASK_CAP, 100, 0.5),
             ("cap_W100_2Ha", W.MASK_CAP, 100, 2.0), ("cap_W100_8Ha", W.MASK_CAP, 100, 8.0)]
    for name, kind, width, eta in cases:
        g = W.Grid(nx=32, ny=32, nz=width + 300, hx=0.1, hy=0.1, hz=0.1, dt=5e-4,
                   bc=(W.PERIODIC, W.PERIODIC, W.DIRICHLET), mask_lo=width, mask_hi=0,
                   mask_eta=eta, mask_kind=kind, det_k=width + 20, obs_every=10 ** 6)
        p = W.Packet((1.6, 1.6, width * g.hz + 12.0), (0.0, 0.0, 2.0), (0.0, 0.0, -1.9))
        with Sim(g, precision=W.FP64, tblock=1) as s:
            s.set_packet(0, p)
            q0 = s.observables(0)["Q"]
            s.step(28000)
            q1 = s.observables(0)["Q"]
            phi = float(s.flux_map(0).sum()) * g.hx * g.hy
        out[name] = {"reflection": 1.0 + phi / q0, "norm_left": q1 / q0}
    return out


def paper_cu111_throughput(torch, T, steps=400, warmup=8):
    """The paper's benchmark geometry (Sec. 3.1: 240 x 240 x 420 + 100 absorbing
    planes = 29,952,000 nodes, anisotropic spacing, Eq. 11 time step, Eq. 4 packet)
    with the synthetic Cu(111)-like slab, FP32 + Kahan, autotuned; cell-updates/s
    over `steps` steps (context: the paper reports about 6 ns per node and step on
    its Quadro K620)."""
    wl = W.cu111(W.FP32_KAHAN)
    g = wl.grid
    s = make_ctx(T, wl, W.FP32_KAHAN, 0)
    ms, prof = timed_steps(torch, T, s, steps, warmup, lambda: None)
    tun = s.tuning()
    s.close()
    return {"nodes": g.cells, "steps": steps, "value": g.cells * steps / (ms * 1e-3),
            "unit": "cell-updates/s", "ns_per_node_step": ms * 1e6 / (g.cells * steps),
            "variant": tun["name"][tun["tblock"]], "steps_per_launch": tun["tblock"]}


def interpolation_cost(torch, T):
    """Sec. 2.3's expansion + interpolation of a cell potential onto the paper's mesh
    size (240 x 240 x 520 nodes, FP64 context) from a 96 x 96 x 560 periodic cell
    lattice on the device: the whole tdse_set_potential_grid call (interpolation,
    d build, ghost zones), wall clock after a warm-up call."""
    from paper_2401_07416_gb300.sim import Sim
    g = W.Grid(nx=240, ny=240, nz=520, hx=0.322, hy=0.322, hz=0.3149, dt=0.0,
               bc=(W.PERIODIC, W.PERIODIC, W.PERIODIC), obs_every=10 ** 6)
    Vc = torch.from_numpy(np.random.default_rng(23).normal(size=(560, 96, 96))).cuda()
    cell = (g.nx * g.hx / 15 * 6, g.ny * g.hy / 15 * 6, g.nz * g.hz)
    with Sim(g, precision=W.FP64) as s:
        s.set_potential_grid(0, Vc, cell)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_potential_grid(0, Vc, cell)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
    return {"nodes": g.cells, "cell_lattice": [96, 96, 560], "ms": el * 1e3,
            "nodes_per_s": g.cells / el}


def dissimilarity_cost(torch, T, K=48, M=100, ny=128, nx=128):
    """Eq. 16 over a batch of K synthetic detector-density trajectories (M frames of
    ny x nx pixels, seeded, on the device), the whole window: FP64 pairwise kernel."""
    rng = np.random.default_rng(16)
    frames = torch.from_numpy(rng.uniform(0.0, 1e-3, size=(K, M, ny * nx))).cuda()
    t = np.arange(M) * 20 * 5e-4
    stream = torch.cuda.current_stream()
    T.tdse_dissimilarity(frames, t, t[0], t[-1], 0.01, stream_ptr=stream.cuda_stream)   # warm-up
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    T.tdse_dissimilarity(frames, t, t[0], t[-1], 0.01, stream_ptr=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    terms = K * (K + 1) // 2 * M * ny * nx
    del frames
    return {"trajectories": K, "frames": M, "pixels": ny * nx, "ms": ms,
            "pair_frame_pixels_per_s": terms / (ms * 1e-3),
            "fp64_gflops": 3 * terms / (ms * 1e-3) / 1e9,
            "includes": "pairwise FP64 sums of squared differences and the time sums "
                        "(allocation of the scratch on the stream included)"}


def adjoint_cost(torch, T):
    """96x96x192, 3000 steps: forward with FP64 checkpoints every 100 steps, then the
    adjoint of the detector-flux loss (dL/dV and the 32 atoms), with the fused
    backward step (default) and with the three in-place passes; wall time of each
    call and, from the library's profile, device time of the backward steps."""
    from paper_2401_07416_gb300.sim import Sim
    out = {}
    for prec in (W.FP32_KAHAN, W.FP64):
        wl = W.config4(prec)
        g = wl.grid
        for fused in (True, False):
            with Sim(g, precision=prec, ckpt_every=100) as s:
                s.set_atoms(0, wl.atoms)
                s.set_packet(0, wl.packet)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.step(wl.steps)
                torch.cuda.synchronize()
                t_fwd = time.perf_counter() - t0
                gF = 2 * s.flux_map(0)
                gV = np.zeros((g.nz, g.ny, g.nx))
                ga = np.zeros_like(wl.atoms)
                T.tdse_set_adjoint_fused(s.ctx, fused)
                T.tdse_set_profiling(s.ctx, True)
                t0 = time.perf_counter()
                T.tdse_adjoint(s.ctx, 0, gF, gV, ga)
                t_adj = time.perf_counter() - t0
                prof = T.tdse_get_profile(s.ctx)
            key = PREC_NAME[prec] + ("" if fused else "_three_pass")
            out[key] = {"forward_s": t_fwd, "adjoint_s": t_adj, "adjoint_over_forward": t_adj / t_fwd,
                        "adjoint_cell_steps_per_s": g.cells * wl.steps / t_adj,
                        "backward_step_us": prof["adjoint_ms"] * 1e3 / max(1, prof["adjoint_steps"]),
                        "backward_steps": prof["adjoint_steps"]}
    out["fused_256x256x512"] = adjoint_roofline(torch, T)
    out["three_pass_256x256x512"] = adjoint_roofline(torch, T, fused=False)
    return out


def adjoint_roofline(torch, T, steps=200, fused=True):
    """The fused backward step on a grid larger than L2 (256x256x512, the 512^3
    workload's spacing, FP32 + Kahan context, checkpoints every 100 steps): device
    time per backward step from the library's profile against its algorithmic bytes
    (R, I, P, Q and d read, R, I, P, Q written, FP32; dL/dV read and written, FP64:
    52 B per node), and the forward step's time per step on the same grid."""
    from paper_2401_07416_gb300.sim import Sim
    g = W.Grid(nx=256, ny=256, nz=512, hx=0.05, hy=0.05, hz=0.05, dt=5e-4, mask_lo=20,
               mask_hi=20, det_k=180, obs_every=20)
    atoms = W.square_slab(8, 4, 1.6, 0.4 * 25.6, 12.8, 12.8, W.rng_for(5), 0.05)
    packet = W.Packet((6.4, 6.4, 12.74), (0.0, 0.0, 2.0), (0.0, 0.0, -1.9))
    peak = measured_peaks()[0]
    with Sim(g, precision=W.FP32_KAHAN, tblock=2, ckpt_every=100) as s:
        s.set_atoms(0, atoms)
        s.set_packet(0, packet)
        T.tdse_set_profiling(s.ctx, True)
        s.step(steps)
        pf = T.tdse_get_profile(s.ctx)
        fwd_ms_per_step = pf["step_ms"] / steps
        gF = 2 * s.flux_map(0)
        T.tdse_set_profiling(s.ctx, False)
        T.tdse_set_profiling(s.ctx, True)
        T.tdse_set_adjoint_fused(s.ctx, fused)
        T.tdse_adjoint(s.ctx, 0, gF, None, None)
        pa = T.tdse_get_profile(s.ctx)
    ms = pa["adjoint_ms"] / max(1, pa["adjoint_steps"])
    # the fused step moves each field once (52 B per node); the three passes read
    # d, R, I, P, Q, then d, P, I, Q, R, gV and write R, Q, then gV, P, I (72 B)
    bytes_step = (52 if fused else 72) * g.cells
    achieved = bytes_step / (ms * 1e-3) / 1e9
    return {"nodes": g.cells, "steps": steps, "backward_step_ms": ms,
            "forward_step_ms": fwd_ms_per_step, "adjoint_over_forward_device": ms / fwd_ms_per_step,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "bytes_per_node": 52 if fused else 72,
                         "kernel": "adj_fused_kernel<float> (one z-march per backward step)" if fused
                                   else "adj_b_kernel, adj_flux_q_kernel, adj_de_kernel <float> (three passes)"}}


def adjoint_case(args):
    """The adjoint of adjoint_cost's 96x96x192 FP32+Kahan case over --steps steps
    (checkpoints every 100), for profiling its kernels."""
    import torch
    torch.cuda.set_device(0)
    from paper_2401_07416_gb300 import build, tdse as T
    build.build()
    from paper_2401_07416_gb300.sim import Sim
    wl = W.config4(W.FP32_KAHAN)
    g = wl.grid
    with Sim(g, precision=W.FP32_KAHAN, ckpt_every=100) as s:
        s.set_atoms(0, wl.atoms)
        s.set_packet(0, wl.packet)
        s.step(args.steps)
        gF = 2 * s.flux_map(0)
        gV = np.zeros((g.nz, g.ny, g.nx))
        ga = np.zeros_like(wl.atoms)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.tdse_adjoint(s.ctx, 0, gF, gV, ga)
        el = time.perf_counter() - t0
    print(json.dumps({"adjoint_case": True, "cells": g.cells, "steps": args.steps,
                      "adjoint_s": el, "us_per_step": el / args.steps * 1e6}), flush=True)


def batch_case(args):
    """The 48-film batch of uneven grids (FP32+Kahan, two steps per launch) for ncu
    captures of its fused launches: kernel variant fixed by --variant (z-chunk by
    --chunk), one untimed two-step launch and a reduction, then `--steps` steps."""
    import torch
    torch.cuda.set_device(0)
    from paper_2401_07416_gb300 import build as B
    B.build()
    from paper_2401_07416_gb300 import tdse as T
    from paper_2401_07416_gb300.sim import Sim
    members = W.config3(48, W.FP32_KAHAN)
    with Sim([m.grid for m in members], precision=W.FP32_KAHAN, tblock=2) as s:
        T.tdse_set_variant(s.ctx, 2, args.variant or 0)
        if args.chunk is not None:
            T.tdse_set_chunk(s.ctx, 2, args.chunk)
        for i, m in enumerate(members):
            s.set_atoms(i, m.atoms)
            s.set_packet(i, m.packet)
        s.step(2)
        s.step(args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"batch_case": True, "members": len(members),
                          "cells": sum(m.grid.cells for m in members), "tuning": s.tuning()}))


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.ncu_case:
        return ncu_case(args)
    if args.batch_case:
        return batch_case(args)
    if args.adjoint_case:
        return adjoint_case(args)

    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = dist.barrier
    else:
        torch.cuda.set_device(0)
        barrier = lambda: None

    from paper_2401_07416_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        barrier()
    from paper_2401_07416_gb300 import tdse as T

    prec = {"kahan": W.FP32_KAHAN, "fp32": W.FP32, "fp64": W.FP64}[args.precision]
    tblock = 1 if prec == W.FP64 else args.tblock
    wl = W.config5(prec)
    g = wl.grid
    cells = g.cells
    hbm_peak, peak_kind = measured_peaks()

    # headline: the fused step on the full grid, autotuned on it (or a fixed variant,
    # e.g. to profile exactly the kernel a plain run picks)
    fixed = args.variant is not None
    if fixed and tblock == 0:
        tblock = 2
    s = make_ctx(T, wl, prec, tblock, autotune=not fixed)
    if fixed:
        T.tdse_set_variant(s.ctx, tblock, args.variant)
        if args.chunk is not None:
            T.tdse_set_chunk(s.ctx, tblock, args.chunk)
    tuning = s.tuning()
    V_dev = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
    T.tdse_get_potential(s.ctx, 0, V_dev)
    with ClockSampler(local) as clk:
        ms, prof = timed_steps(torch, T, s, args.steps, args.warmup, barrier)
    clocks = clk.summary()
    obs = s.observables(0)
    s.close()

    def reduce_max(x):
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    t_max, value = job_time_and_value(ms, cells, args.steps, world, reduce_max)

    # the dominant kernel: the fused step at the depth in use (launches of other
    # depths, if K is not a multiple of it, are left out of its roofline)
    tb = tuning["tblock"]
    nlaunch, launch_ms = launch_stats(prof, tb)
    bytes_launch = BYTES_PER_NODE[prec] * cells
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    variant = tuning["name"][tb]
    traffic, traffic_note = ncu_traffic(variant, cells)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "traffic_source": traffic_note,
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS hbm_gbs)",
                "kernel": f"{kernel_function(variant)} {variant} ({tb} steps per launch)",
                "algorithmic_bytes_per_launch": bytes_launch,
                "bytes_per_node_per_launch": BYTES_PER_NODE[prec],
                "avg_launch_ms": launch_ms, "launches": nlaunch,
                "launches_other_depths": int(prof["step_launches"] - nlaunch),
                "timing": "CUDA events on the library's stream around each CUDA-graph replay "
                          "(one reduction period of launches of one depth) inside the timed region",
                "reduce_ms_total": prof["reduce_ms"],
                "effective_frac_vs_unfused_fp32": value / world * 20 / 1e9 / hbm_peak}

    extras = {}
    e2e = None
    cpu = None
    if not args.no_extras:
        # end to end through the C ABI from pinned host buffers: potential in,
        # packet set-up, the steps, flux map and observables out, over one complete
        # run of the workload (its own length, 1000 steps, whatever --steps is)
        run_steps = wl.steps
        V_host = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, pin_memory=True)
        V_host.copy_(V_dev.cpu())
        F_host = torch.empty((g.ny, g.nx), dtype=torch.float64, pin_memory=True)
        from paper_2401_07416_gb300.sim import Sim
        se = Sim(g, precision=prec, tblock=tblock)
        se.set_potential(0, V_host)       # first call allocates; not timed
        se.set_packet(0, wl.packet)
        se.autotune(2)
        se.step(4)
        torch.cuda.synchronize()
        # five complete runs (the host-to-device copy of V shares the host's memory
        # system with other work on this machine and varies run to run); the median
        # run is reported, every run is listed
        runs = []
        for _ in range(5):
            barrier()
            t0 = time.perf_counter()
            T.tdse_set_potential(se.ctx, 0, V_host)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            se.set_packet(0, wl.packet)
            t2 = time.perf_counter()
            se.step(run_steps)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            T.tdse_get_flux_map(se.ctx, 0, F_host)
            se.observables(0)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            runs.append({"value": world * cells * run_steps / el,
                         "phases_ms": {"set_potential_h2d": (t1 - t0) * 1e3,
                                       "set_wavepacket": (t2 - t1) * 1e3,
                                       "steps": (t3 - t2) * 1e3,
                                       "flux_and_observables_d2h": (time.perf_counter() - t3) * 1e3}})
        barrier()
        se.close()
        med = sorted(runs, key=lambda r: r["value"])[len(runs) // 2]
        e2e = {"value": med["value"], "unit": "cell-updates/s",
               "steps": run_steps,
               "h2d_bytes_per_step": V_host.numel() * 8 / run_steps,
               "d2h_bytes_per_step": (F_host.numel() * 8 + 64) / run_steps,
               "includes": "tdse_set_potential (pinned host V, FP64), tdse_set_wavepacket, "
                           "tdse_step (CUDA-graph replay), tdse_get_flux_map, tdse_observables",
               "phases_ms": med["phases_ms"], "runs": [r["value"] for r in runs],
               "set_potential_h2d_ms_per_run": [r["phases_ms"]["set_potential_h2d"] for r in runs],
               "statistic": f"median of {len(runs)} complete runs"}
        del V_host
        # FP64 unfused step and the FP32 variants on the same grid (same potential)
        variants = [(W.FP64, 1)] + [(p, t) for p in (W.FP32, W.FP32_KAHAN) for t in (1, 2, 3, 4)]
        for vp, vt in variants:
            steps_v = max(10, args.steps // (8 if vp == W.FP64 else 2))
            sv = make_ctx(T, W.config5(vp), vp, vt, V_dev)
            vname = sv.tuning()["name"][vt]
            vms, vprof = timed_steps(torch, T, sv, steps_v, min(args.warmup, 6), barrier)
            sv.close()
            _, vlaunch = launch_stats(vprof, vt)
            extras[f"{PREC_NAME[vp]}_t{vt}"] = {
                "value": cells * steps_v / (vms * 1e-3), "unit": "cell-updates/s",
                "steps": steps_v, "variant": vname, "avg_launch_ms": vlaunch,
                "ms_per_step_of_launches": vlaunch / vt,
                "hbm_frac_of_algorithmic_bytes": BYTES_PER_NODE[vp] * cells / (vlaunch * 1e-3) / 1e9 / hbm_peak}
        extras["speedup_vs_fp64_plain"] = value / world / extras["f64_t1"]["value"]
        extras["batched_48_films"] = batch_throughput(torch, T, max(20, args.steps // 2),
                                                      min(args.warmup, 6))
        extras["adjoint_96x96x192_3000"] = adjoint_cost(torch, T)
        extras["dissimilarity_48x100x128x128"] = dissimilarity_cost(torch, T)
        extras["absorbing_layer_reflection"] = absorber_reflection(torch, T)
        extras["potential_interp_240x240x520"] = interpolation_cost(torch, T)
        extras["paper_cu111_240x240x520"] = paper_cu111_throughput(torch, T)

        if rank == 0 and world == 1:
            cpu = time_oracle(args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32+kahan": "f32", "f32": "f32", "f64": "f64"}[PREC_NAME[prec]],
        "data": "synthetic",
        "config": {"workload": "512x512x1024 grid, h=0.05, 4x16x16 softened-Coulomb slab, "
                               "cos^2 absorbing layers, detector flux every step, "
                               "Q/E every 20 steps",
                   "precision": PREC_NAME[prec], "steps_per_launch": tb, "variant": variant,
                   "z_chunk": tuning["chunk"][tb], "nx": g.nx, "ny": g.ny, "nz": g.nz, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (state ~10 GB), no flush"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(prof["step_launches"] + prof["reduce_launches"]),
        "clocks": clocks,
        "variants": extras,
        "final_obs": {"Q": obs["Q"], "energy": obs["energy"],
                      "flux_integrated": obs["flux_integrated"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark of the fused RLBM stream-collide step on GB300.

Metric: GLUPS (10^9 lattice-node updates per second) of the stream-collide
step, and its fraction of the measured HBM bandwidth.  Default workload: the
largest single-GPU configuration of the suite, an 8192 x 8192 periodic
lattice, FP32 populations, tau = 0.505, stirring force on the shell
16 <= |k| <= 18 (amplitude 2e-6, redrawn every 100 steps), started at rest
-- the paper's stirred-turbulence runs (Sec. 5) scaled to a GB300.  The
1024^2, 4096^2, 128^2 and ensemble configurations are timed in `configs`.

Timing: W untimed warm-up steps made of the same calls as the timed ones
(so every CUDA graph the timed calls replay exists before the first event),
then K steps, launch by launch, each launch bracketed by CUDA events on the
lattice's stream, and the whole region by one more pair.  Lattices whose
state is smaller than twice the 129 MB L2 get an L2 flush (a 256 MB write,
then a 256 MB read) between launches; larger ones (the 8192^2 headline:
9.7 GB) need none.  Multi-GPU (torchrun): each rank advances its own
independent replica (no data exchange; weak scaling); value = sum over
ranks, time = max over ranks.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 129 << 20
# Algorithmic bytes per node update (one read and one write of the 17 stored
# classes plus the force read), whatever the kernel actually moves.
ALGO_BYTES_PER_UPDATE = {"f64": 288, "f32": 144, "bf16": 76, "f16": 76}
# The CPU sample of the oracle: the workload's node, relaxation time and
# forcing on a 2048^2 lattice (the oracle lattice of the 8192^2 run).
CPU_SAMPLE_SIDE = 2048
METRIC = "GLUPS of the fused stream-collide step (and fraction of HBM peak)"
# FP64 form: FP64 flops per node of the forced step (ncu: adds + multiplies
# + 2 x FMAs of one launch / nodes, one-node-per-thread kernel, 1024^2 stirred)
# and the FP64 peak derived from the unit count and clock (152 SMs x 2 FP64
# FMA per clock x 2 flops x 2.07 GHz).
FP64_FLOPS_PER_NODE = 627.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e nominal, for context beside the measured copy bandwidth
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--landau", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--kernel", default="auto", choices=["auto", "gather", "vec", "vec2", "packed", "tma", "twopass",
                                                               "fused2", "packed4"])
    ap.add_argument("--launch", default="", metavar="KERNEL,BX,BY,BUDGET",
                    help="pin one launch shape of the autotuner's list instead of tuning (profiling runs)")
    ap.add_argument("--workload", default="large8192", choices=sorted(WORKLOADS),
                    help="workload of the headline line (profiling runs use the smaller ones)")
    ap.add_argument("--n", type=int, default=0, help="override lattice side (default: the workload's)")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-form table, e2e and CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--stencil", default="sph26", choices=["sph26", "ring8"],
                    help="time the 2D ring variant instead of the paper's node (profiling runs)")
    ap.add_argument("--nz", type=int, default=0,
                    help="time a 3D lattice of n x n x nz nodes instead of the one-layer lattice (profiling runs)")
    ap.add_argument("--ensemble-only", type=int, default=0, metavar="NRUNS",
                    help="time only an ensemble of NRUNS members with sides up to 512 (profiling runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Sources each fused-step variant compiles from (kernel id -> files).
_STEP_SOURCES = ("rlbm_device.cuh", "packed.cuh", "k_step_gather.cuh", "k_step_vec.cuh", "k_step_pair.cuh",
                 "k_launch.cuh", "k_step_f32.cu", "k_step_f64.cu", "k_step_h16.cu", "k_step_bf16.cu", "k_step_f16.cu",
                 "k_step_dfl.cu")
_TMA_SOURCES = ("rlbm_device.cuh", "packed.cuh", "k_step_vec.cuh", "k_step_tma.cuh", "k_step_tma.cu")
_FUSED2_SOURCES = ("rlbm_device.cuh", "packed.cuh", "k_step_vec.cuh", "k_step_pair.cuh", "k_step_fused2.cuh",
                   "k_fused2_launch.cuh", "k_fused2_inst.cuh", "k_step_fused2.cu", "k_fused2_f32.cu", "k_fused2_bf16.cu",
                   "k_fused2_f16.cu", "k_fused2_sub_f32.cu", "k_fused2_sub_bf16.cu", "k_fused2_sub_f16.cu",
                   "k_step_dfl.cu")
_QUAD_SOURCES = ("rlbm_device.cuh", "packed.cuh", "k_step_vec.cuh", "k_step_pair.cuh", "k_step_quad.cuh",
                 "k_quad_inst.cuh", "k_quad_f32.cu", "k_quad_bf16.cu", "k_quad_f16.cu", "k_quad_dfl_f32.cu",
                 "k_quad_dfl_bf16.cu", "k_quad_dfl_f16.cu")


def step_kernel_source_hash(kernel_id=4):
    """SHA-256 over the sources a fused-step variant compiles from (the
    per-node device code, the kernel bodies and their launchers), in name
    order: a stored DRAM-traffic figure counts only while it matches."""
    import hashlib
    src = os.path.join(ROOT, "paper_2101_06187_gb300", "csrc")
    files = {5: _TMA_SOURCES, 7: _FUSED2_SOURCES, 8: _QUAD_SOURCES}.get(kernel_id, _STEP_SOURCES)
    hsh = hashlib.sha256()
    for fn in sorted(files):
        with open(os.path.join(src, fn), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


WORKLOADS = {"large8192": workloads.LARGE_8192, "stirred1024": workloads.STIRRED_1024,
             "precision4096": workloads.PRECISION_4096}


def workload_for(args):
    w = WORKLOADS[getattr(args, "workload", "large8192")]
    n = args.n or w.nx
    return w, n


def workload_config(w, n, form):
    """The workload as both arms name it (identical keys and values)."""
    return {"workload": w.name if n == w.nx else "%s (side %d)" % (w.name, n), "nx": n, "ny": n, "form": form,
            "tau": w.tau, "forcing": "shell %d..%d amp %g redraw %d" % (w.kmin, w.kmax, w.amp, w.redraw),
            "l2": l2_policy(n, form)}


def state_bytes(n, form):
    return ALGO_BYTES_PER_UPDATE[form] * n * n


def needs_flush(n, form):
    """The L2 is flushed between timed launches unless the lattice state is
    larger than twice the L2."""
    return state_bytes(n, form) < 2 * L2_BYTES


def l2_policy(n, form):
    if needs_flush(n, form):
        return "flushed between timed launches (256 MB write, then 256 MB read)"
    return "not flushed: the state (%.1f GB) is larger than L2 (129 MB)" % (state_bytes(n, form) / 1e9)


def forcing_of(w):
    return dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw)


class L2Flush:
    """Evict the lattice from L2 between timed steps: write a buffer larger
    than L2, then read a second one, so that the lines left in L2 are clean
    and the next step neither finds its inputs there nor pays for writing
    back the flush's own dirty lines."""

    def __init__(self, torch, nbytes):
        self.w = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(nbytes // 4, dtype=torch.float32, device="cuda")
        self.sink = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.fill_(1.0)
        self.sink.copy_(self.r.sum())


def launch_units(lat, steps):
    """Split `steps` into the step counts of single launches of the chosen
    kernel: 2 for a two-step kernel (an odd remainder is a single step)."""
    spl = max(1, int(lat.info()["steps_per_launch"]))
    return [spl] * (steps // spl) + ([steps % spl] if steps % spl else [])


def time_steps(torch, lat, steps, flush, with_units=False, region=None):
    """CUDA-event timing on the lattice stream of each launch (one step, or
    two for a two-step kernel), with an L2 flush in between when `flush` is
    given.  Returns the time of every step in ms (a launch's time shared by
    its steps) and, with with_units, the launch unit of every step.  region:
    a list that receives the elapsed ms of the whole timed region (one event
    pair around all launches; without flushes it includes the gaps between
    launches)."""
    stream = lat._torch_stream
    sizes = launch_units(lat, steps)
    evs = []
    with torch.cuda.stream(stream):
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for size in sizes:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            if flush is not None:
                flush()
            a.record(stream)
            lat.step(size)
            b.record(stream)
            evs.append((a, b))
        r1.record(stream)
    stream.synchronize()
    if region is not None:
        region.append(r0.elapsed_time(r1))
    ms = np.concatenate([np.full(size, a.elapsed_time(b) / size) for (a, b), size in zip(evs, sizes)])
    if not with_units:
        return ms
    return ms, np.repeat(np.arange(len(sizes)), sizes)


def warm_up(lat, warmup, flush=None):
    """Untimed warm-up with the timed calls themselves: at least two
    launch-sized calls, so the CUDA graphs of both buffer parities that the
    timed calls replay are captured and instantiated here (graphs are keyed
    by step count and starting buffer).  Returns the steps advanced (a
    whole number of launches, so timed launches start on a launch
    boundary)."""
    spl = max(1, int(lat.info()["steps_per_launch"]))
    calls = max(2, -(-warmup // spl))
    for _ in range(calls):
        if flush is not None:
            flush()
        lat.step(spl)
    lat.synchronize()
    return calls * spl


def measure_form(torch, rl, w, n, form, landau, kernel, steps, warmup, flush, init=None, tune=True, stencil="sph26",
                 nz=0, launch=""):
    if nz > 0:
        lat = rl.Lattice3D(n, n, nz, w.tau, dtype=form, landau=landau, kernel=kernel, forcing=forcing_of(w))
    else:
        lat = rl.Lattice(n, n, w.tau, dtype=form, landau=landau, kernel=kernel, forcing=forcing_of(w), stencil=stencil)
    if init is not None:
        lat.init_fields(*init)
    else:
        lat.init_fields()
    if launch:
        k, bx, by, budget = launch.split(",")
        lat.set_launch(k, int(bx), int(by), int(budget))
    elif tune:
        lat.autotune(10)
    fl = flush if needs_flush(n, form) else None
    warmup = warm_up(lat, warmup, fl)
    region = []
    ms, unit = time_steps(torch, lat, steps, fl, with_units=True, region=region)
    info = lat.info()
    info["timed_launches"] = int(unit[-1]) + 1 if len(unit) else 0
    info["region_ms"] = region[0]
    # launches that started a forcing epoch also carry the force re-synthesis
    redraw = w.redraw
    first = warmup
    starts = np.array([((first + i) % redraw) == 0 for i in range(steps)])
    epoch_units = set(unit[starts].tolist())
    is_epoch = np.isin(unit, list(epoch_units))
    kernel_ms = ms[~is_epoch].mean() if (~is_epoch).any() else ms.mean()
    lat.close()
    return ms, kernel_ms, info, len(epoch_units)


def measure_ensemble(torch, rl, flush, steps=20, warmup=5, nruns=64, sides=None, kernel="auto", tune=True):
    """The 64-member ensemble (sides 256..1024): per-step timing with an L2
    flush between steps, and the throughput of a replayed 100-step graph.
    kernel / tune: pin the ensemble body and skip the autotuner (profiling
    runs)."""
    members = workloads.ensemble(nruns) if sides is None else workloads.ensemble(nruns, sides=sides)
    runs = [dict(nx=w.nx, ny=w.ny, tau=w.tau,
                 forcing=dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw))
            for w in members]
    ens = rl.Ensemble(runs, dtype="f32", landau="fp32", kernel=kernel)
    if tune:
        bx, by, grid = ens.autotune(5)
    else:
        i0 = ens.info()
        bx, by, grid = i0["block_x"], i0["block_y"], i0["grid"]
    spl = int(ens.info()["steps_per_launch"])  # 2 for the two-step body: time whole launches
    for _ in range(max(2, -(-warmup // spl))):  # the timed calls themselves: both graph parities captured
        flush()
        ens.step(spl)
    ens.synchronize()
    stream = ens._torch_stream
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(max(1, steps // spl)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            flush()
            a.record(stream)
            ens.step(spl)
            b.record(stream)
            evs.append((a, b))
    stream.synchronize()
    ms = np.array([a.elapsed_time(b) / spl for a, b in evs])  # per step
    info = ens.info()
    # a full forcing epoch replayed as one graph (starts at an epoch boundary;
    # one untimed epoch first, so capture and instantiation are not timed)
    ens.step((-info["step"]) % 100 + 100)
    ens.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        ens.step(100)
        b.record(stream)
    stream.synchronize()
    graph_ms = a.elapsed_time(b)
    info = ens.info()
    ens.close()
    peak, _ = load_peaks()
    step_ms = float(np.median(ms))
    side_set = "{256,384,512,768,1024}" if sides is None else "{%s}" % ",".join(str(x) for x in sides)
    algo = ALGO_BYTES_PER_UPDATE["f32"]  # one read and one write of the 17 classes plus the force, per update
    moved = info["bytes_per_step"] / info["nodes"]  # what the chosen body moves (half per update of a two-step launch)
    return {"workload": "%d stirred runs, sides %s, tau U[0.51,0.7], bands around U[4,12]" % (nruns, side_set),
            "nodes": int(info["nodes"]), "glups": info["nodes"] / (step_ms / 1e3) / 1e9,
            "hbm_frac": algo * info["nodes"] / (step_ms / 1e3) / 1e9 / peak,
            "bytes_per_update": algo, "moved_bytes_per_update": moved,
            "frac_of_moved_bytes": info["bytes_per_step"] / (step_ms / 1e3) / 1e9 / peak,
            "glups_graph_100_steps": info["nodes"] * 100 / (graph_ms / 1e3) / 1e9,
            "block": [bx, by], "grid": grid, "tiles": int(info["ntiles"]), "launches_per_step": 1 / spl,
            "body": {v: k for k, v in rl.KERNELS.items()}[info["kernel"]]}


def parity_error(rl, oracle, form, landau):
    """Max relative error vs the FP64 oracle after 100 forced steps on a
    128 x 128 lattice started from seeded smooth fields (the parity bar)."""
    n, nsteps = 128, 100
    w = workloads.STIRRED_1024
    fields = workloads.random_smooth(n, n, seed=2024, deps=0.02, vmax=0.02)
    fz = dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp * 10, seed=w.seed, redraw_period=w.redraw // 2)
    lat = rl.Lattice(n, n, w.tau, dtype=form, landau=landau, forcing=fz)
    lat.init_fields(*fields)
    lat.step(nsteps)
    e_g, vx_g, vy_g, _ = lat.moments()
    lat.close()
    f = oracle.init(n, n, *fields)
    oracle.run(f, w.tau, nsteps, kmin=fz["kmin"], kmax=fz["kmax"], amp=fz["amp"], seed=fz["seed"],
               redraw=fz["redraw_period"])
    e_o, vx_o, vy_o = oracle.fields(f)
    err_e = float(np.max(np.abs(e_g - e_o)) / np.max(np.abs(e_o)))
    vn = max(np.max(np.abs(vx_o)), np.max(np.abs(vy_o)))
    err_v = float(max(np.max(np.abs(vx_g - vx_o)), np.max(np.abs(vy_g - vy_o))) / vn)
    return {"eps": err_e, "v": err_v, "case": "128x128, 100 forced steps from seeded smooth fields"}


def measure_configs(torch, rl, flush, hbm_peak, steps=40, warmup=6):
    """The suite's other configurations at their own sizes and parameters,
    each autotuned and timed like the headline (per-launch CUDA events, L2
    flushed between launches where the state fits twice in L2): the 128^2
    shear wave (FP64 form, unforced), the 1024^2 stirred run (FP32, tau
    0.52, shell 4..6) and the 4096^2 precision run in BF16 and FP16 storage
    (tau 0.51, shell 8..10; FP32 Landau solve, and BF16 with the FP64 solve
    that run names).  hbm_frac counts the algorithmic bytes of a node update
    (one read and one write of the 17 classes plus the force) per update,
    whatever the kernel moves."""
    out = {}
    cases = ((workloads.SHEAR_128, "f64", "fp64"), (workloads.STIRRED_1024, "f32", "fp32"),
             (workloads.PRECISION_4096, "bf16", "fp32"), (workloads.PRECISION_4096, "f16", "fp32"),
             (workloads.PRECISION_4096, "bf16", "fp64"))
    for w, form, landau in cases:
        init = workloads.shear_wave(w.nx, w.ny, w.extra["u0"]) if w.init == "shear" else None
        ms, km, info, _ = measure_form(torch, rl, w, w.nx, form, landau, "auto", steps, warmup, flush, init=init)
        nodes = w.nx * w.ny
        bp = ALGO_BYTES_PER_UPDATE[form]
        spl = int(info["steps_per_launch"])
        out["%s/%s/landau-%s" % (w.name, form, landau)] = {
            "glups": nodes / (km / 1e3) / 1e9, "kernel_ms": km, "bytes_per_update": bp,
            "hbm_frac": bp * nodes / (km / 1e3) / 1e9 / hbm_peak,
            "moved_bytes_per_update": int(info["bytes_per_node"]),
            "kernel": {v: k for k, v in rl.KERNELS.items()}[info["kernel"]], "block": [info["block_x"], info["block_y"]],
            "steps_per_launch": spl, "l2": l2_policy(w.nx, form),
            "glups_whole_region": nodes * len(ms) / (info["region_ms"] / 1e3) / 1e9}
    return out


def measure_variants(torch, rl, oracle, flush, hbm_peak, steps=50, warmup=5):
    """The lattice variants beyond the paper's one-layer node, each timed
    like the headline (per-step CUDA events, L2 flushed between steps) and
    checked against its oracle on a small case: the 2D ring (1024^2, FP32)
    and the 3D lattice (256^3, FP32), both stirred."""
    out = {}
    w = workloads.STIRRED_1024
    fz = forcing_of(w)
    cases = (("ring8_1024x1024_f32", lambda: rl.Lattice(1024, 1024, w.tau, dtype="f32", forcing=fz, stencil="ring8"),
              1024 * 1024),
             ("lattice3d_256x256x256_f32", lambda: rl.Lattice3D(256, 256, 256, w.tau, dtype="f32", forcing=fz),
              256 ** 3),
             # the paper's own time step on its lattice spacings 0.08 and 0.04 (Sec. 5): cfl 0.625 and
             # 1.25, relaxation from eta/s = 0.01 and the local temperature
             ("paper_cfl0.625_eta0.01_1024x1024_f32",
              lambda: rl.Lattice(1024, 1024, w.tau, dtype="f32", forcing=fz, cfl=0.625, eta_s=0.01, dt=0.05),
              1024 * 1024),
             ("paper_cfl1.25_eta0.01_1024x1024_f32",
              lambda: rl.Lattice(1024, 1024, w.tau, dtype="f32", forcing=fz, cfl=1.25, eta_s=0.01, dt=0.05),
              1024 * 1024))
    for name, make, nodes in cases:
        lat = make()
        lat.init_fields()
        lat.autotune(5)
        warm_up(lat, warmup, flush)
        ms = time_steps(torch, lat, steps, flush)
        info = lat.info()
        lat.close()
        km = float(np.median(ms))
        bp = int(info["bytes_per_node"])  # moved per update; algorithmic = one step's read + write + force
        algo = bp * int(info["steps_per_launch"])
        out[name] = {"glups": nodes / (km / 1e3) / 1e9, "kernel_ms": km, "bytes_per_update": algo,
                     "moved_bytes_per_update": bp, "hbm_frac": algo * nodes / (km / 1e3) / 1e9 / hbm_peak,
                     "kernel": {v: k for k, v in rl.KERNELS.items()}[info["kernel"]],
                     "block": [info["block_x"], info["block_y"]]}
    # parity on small cases (FP32 against the FP64 oracles)
    n, nsteps = 64, 50
    fields = workloads.random_smooth(n, n, seed=2024, deps=0.02, vmax=0.02)
    small = dict(kmin=2, kmax=4, amp=2e-4, seed=7, redraw_period=25)
    lat = rl.Lattice(n, n, 0.6, dtype="f32", forcing=small, stencil="ring8")
    lat.init_fields(*fields)
    lat.step(nsteps)
    got = lat.moments()
    lat.close()
    f = oracle.ring.init(n, n, *fields)
    t0 = time.perf_counter()
    oracle.ring.run(f, 0.6, nsteps, kmin=2, kmax=4, amp=2e-4, seed=7, redraw=25)
    dt = time.perf_counter() - t0
    out["ring8_1024x1024_f32"]["max_rel_err_vs_oracle"] = _field_errors(oracle.ring.fields(f), got,
                                                                       "64x64, 50 forced steps")
    out["ring8_1024x1024_f32"]["cpu_oracle"] = {"glups": n * n * nsteps / dt / 1e9, "cores": os.cpu_count(),
                                               "sample": "64x64, 50 forced steps"}
    m = 20
    fields3 = workloads.random_smooth3d(m, m, m, seed=2024, deps=0.02, vmax=0.02)
    lat = rl.Lattice3D(m, m, m, 0.6, dtype="f32", forcing=dict(small, kmax=3))
    lat.init_fields(*fields3)
    lat.step(nsteps)
    got = lat.moments()
    lat.close()
    f = oracle.lattice3d.init(m, m, m, *fields3)
    t0 = time.perf_counter()
    oracle.lattice3d.run(f, 0.6, nsteps, kmin=2, kmax=3, amp=2e-4, seed=7, redraw=25)
    dt = time.perf_counter() - t0
    out["lattice3d_256x256x256_f32"]["max_rel_err_vs_oracle"] = _field_errors(oracle.lattice3d.fields(f), got,
                                                                             "20^3, 50 forced steps")
    out["lattice3d_256x256x256_f32"]["cpu_oracle"] = {"glups": m ** 3 * nsteps / dt / 1e9, "cores": os.cpu_count(),
                                                     "sample": "20^3, 50 forced steps"}
    return out


def _field_errors(ref, got, case):
    e_r, *v_r = ref
    e_g, *v_g = got[:len(ref)]
    err_e = float(np.max(np.abs(e_g - e_r)) / np.max(np.abs(e_r)))
    vn = max(float(np.max(np.abs(v))) for v in v_r)
    err_v = float(max(np.max(np.abs(g - r)) for g, r in zip(v_g, v_r)) / vn)
    return {"eps": err_e, "v": err_v, "case": case}


def cpu_oracle_glups(oracle, w, n, budget_s):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    the full n x n lattice if a step fits the budget, else a band of rows
    (same shape per node); returns (GLUPS, description, threads)."""
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    n = min(n, CPU_SAMPLE_SIDE)
    rows = n
    f = oracle.init(n, rows)
    tmp_steps = 1
    t0 = time.perf_counter()
    oracle.run(f, w.tau, tmp_steps, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
    one = time.perf_counter() - t0
    nsteps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(f, w.tau, nsteps, step0=tmp_steps, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed,
               redraw=w.redraw)
    dt = time.perf_counter() - t0
    glups = n * rows * nsteps / dt / 1e9
    return glups, ("%dx%d lattice with the workload's tau and forcing, %d forced steps (FP64 oracle, OpenMP)"
                   % (n, rows, nsteps)), threads


def e2e_glups(rl, w, n, form, landau, reps=5, steps_per_call=100):
    """Through the public API with host buffers in pinned memory: upload the
    initial fields, advance steps_per_call steps, read the fields back
    (median over reps calls)."""
    import torch
    fields = workloads.random_smooth(n, n, seed=5, deps=0.01, vmax=0.01)
    pinned = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    inp = [pinned((n * n,)) for _ in range(3)]
    for dst, src in zip(inp, fields):
        dst[:] = np.ravel(src)
    res = (pinned((n, n)), pinned((n, n)), pinned((n, n)), pinned((3,)))
    lat = rl.Lattice(n, n, w.tau, dtype=form, landau=landau, forcing=forcing_of(w))
    lat.init_fields(*inp)
    lat.step(steps_per_call)
    lat.moments(out=res)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        lat.init_fields(*inp)
        lat.step(steps_per_call)
        out = lat.moments(out=res)
        times.append(time.perf_counter() - t0)
    lat.close()
    dt = float(np.median(times))
    h2d = 3 * n * n * 8
    d2h = 3 * n * n * 8 + 3 * 8
    del out
    return {"value": n * n * steps_per_call / dt / 1e9, "unit": "GLUPS",
            "h2d_bytes_per_step": h2d / steps_per_call, "d2h_bytes_per_step": d2h / steps_per_call,
            "steps_per_call": steps_per_call}


def aggregate_replicas(torch, local_seconds, local_updates, world):
    """Whole-job figures of independent replicas: the timed region ends when
    the slowest rank ends (max over ranks), and every rank's lattice updates
    count.  Returns (max seconds, total GLUPS)."""
    if world > 1:
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
        u = torch.tensor([float(local_updates)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.barrier()
        return float(t.item()), float(u.item()) / float(t.item()) / 1e9
    return local_seconds, local_updates / local_seconds / 1e9


def reference_arm(args):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    headline workload: its node, relaxation time and forcing on a lattice of
    side min(n, 2048), each timed step a few lattice steps of it."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle
    oracle.build()
    w, n = workload_for(args)
    m = min(n, CPU_SAMPLE_SIDE)
    total_steps = max(1, args.steps)
    warm = max(0, args.warmup)
    oracle.set_threads(os.cpu_count() or 1)
    f = oracle.init(m, m)
    t0 = time.perf_counter()
    oracle.run(f, w.tau, 1, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
    one = time.perf_counter() - t0
    per_step_budget = 60.0 / max(1, total_steps + warm)
    nsub = max(1, min(50, int(per_step_budget / max(one, 1e-6))))
    done = 1
    for _ in range(min(warm, 3)):
        oracle.run(f, w.tau, 1, step0=done, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
        done += 1
    t0 = time.perf_counter()
    steps_done = 0
    for _ in range(total_steps):
        oracle.run(f, w.tau, nsub, step0=done, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
        done += nsub
        steps_done += nsub
        if time.perf_counter() - t0 > 150:
            break
    dt = time.perf_counter() - t0
    glups = m * m * steps_done / dt / 1e9
    sample = "%dx%d lattice with the workload's tau and forcing, %d forced steps (FP64 oracle, OpenMP)" % (
        m, m, steps_done)
    line = {"impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS",
            "n_gpus": args.gpus, "steps": total_steps, "warmup": args.warmup,
            "ms_per_step": dt / steps_done * 1e3 * (n * n) / (m * m), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, n, args.form),
            "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def traffic_entry(form, landau, kernel_id, n, variant_key=""):
    """The stored ncu DRAM figure (profiles/traffic.json) of this kernel and
    lattice, if it was taken on the current sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as fh:
            tj = json.load(fh)
        ent = tj.get("%s_%s_%d_%d%s" % (form, landau, kernel_id, n, variant_key))
        if ent and ent.get("source_sha256") == step_kernel_source_hash(kernel_id):
            return ent
    except (OSError, ValueError, KeyError):
        pass
    return None


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
        __graft_entry__.build()
    import paper_2101_06187_gb300 as rl

    w, n = workload_for(args)
    K, W = args.steps, max(3, args.warmup)
    flush = L2Flush(torch, L2_FLUSH_BYTES)
    if args.ensemble_only > 0:
        res = measure_ensemble(torch, rl, flush, steps=K, warmup=W, nruns=args.ensemble_only, sides=(256, 384, 512),
                               kernel=args.kernel, tune=not args.no_tune)
        print(json.dumps({"metric": METRIC, "value": res["glups"], "unit": "GLUPS", "n_gpus": 1, "steps": K,
                          "warmup": W, "higher_is_better": True, "config": {"workload": res["workload"]},
                          "ensemble": res}), flush=True)
        return
    dev_index = torch.cuda.current_device()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(phys[dev_index]) if phys and phys[0].isdigit() and dev_index < len(phys) else dev_index

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(smi_index) as clocks:
        ms, kernel_ms, info, n_epoch = measure_form(torch, rl, w, n, args.form, args.landau, args.kernel, K, W, flush,
                                                    tune=not args.no_tune, stencil=args.stencil, nz=args.nz,
                                                    launch=args.launch)
    torch.cuda.synchronize()
    nodes = n * n * max(1, args.nz)
    variant = args.stencil != "sph26" or args.nz > 0
    # whole timed region: one event pair around all launches when nothing runs between them, else the sum of
    # the launches (the L2 flushes between launches are not the job's work)
    region_s = (info["region_ms"] if not needs_flush(n, args.form) else float(ms.sum())) / 1e3
    total_s, glups_total = aggregate_replicas(torch, region_s, nodes * K, world)
    step_ms = total_s * 1e3 / K

    hbm_peak, peak_kind = load_peaks()
    spl = int(info["steps_per_launch"])
    launch_ms = kernel_ms * spl
    moved = int(info["bytes_per_node"])  # bytes the chosen kernel moves per node update (half per update of a
    #                                     two-step launch, which moves the state once)
    algo = moved * spl if variant else ALGO_BYTES_PER_UPDATE[args.form]  # algorithmic bytes per node update
    achieved = algo * nodes * spl / (launch_ms / 1e3) / 1e9
    vkey = "_%s_nz%d" % (args.stencil, args.nz) if variant else ""
    ent = traffic_entry(args.form, args.landau, info["kernel"], n, vkey)
    kname = {v: k for k, v in rl.KERNELS.items()}[info["kernel"]]

    config = workload_config(w, n, args.form)
    if variant:
        config["workload"] += " (3D lattice %dx%dx%d)" % (n, n, args.nz) if args.nz else " (2D ring)"
    line = {
        "metric": METRIC,
        "value": glups_total, "unit": "GLUPS", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.form != "f64" else "f64", "data": "synthetic",
        "config": config,
        "launch": {"kernel": kname, "block": [info["block_x"], info["block_y"]],
                   "launch_budget": info["launch_budget"], "steps_per_launch": spl, "landau": args.landau,
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": ent["bytes_per_launch"] if ent else None,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_update": algo,
                     "moved_bytes_per_update": moved,
                     "frac_of_moved_bytes": moved * nodes * spl / (launch_ms / 1e3) / 1e9 / hbm_peak,
                     "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": achieved / HBM_NOMINAL_GBS,
                     "kernel": kname, "launch_ms": launch_ms, "updates_per_launch": nodes * spl,
                     "epoch_launches_in_timed_region": n_epoch},
        "clocks": clocks.summary(),
        # an epoch start adds the force draw and synthesis: draw, row sums and synthesis (2D), draw and
        # synthesis (3D lattice)
        "gpu_launches": int(info["timed_launches"] + (2 if args.nz > 0 else 3) * n_epoch),
    }
    if ent:
        line["roofline"]["traffic_source"] = ent.get("from")
        if ent.get("scaled_from"):
            line["roofline"]["traffic_scaled_from"] = ent["scaled_from"]
        if ent.get("limiter"):
            line["roofline"]["limiter"] = ent["limiter"]
    if args.form == "f64" and not variant:
        tf = FP64_FLOPS_PER_NODE * nodes / (kernel_ms / 1e3) / 1e12
        line["roofline"] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tf / FP64_PEAK_TFLOPS, "traffic": ent["bytes_per_launch"] if ent else None,
                            "peak_kind": "derived (FP64 units x clock)", "flops_per_node": FP64_FLOPS_PER_NODE,
                            "hbm_frac": achieved / hbm_peak, "launch_ms": launch_ms,
                            "epoch_launches_in_timed_region": n_epoch}

    if rank == 0 and not args.no_extras and not variant:
        import oracle
        oracle.build()
        oracle.set_threads(os.cpu_count() or 1)
        forms = {}
        for form, landau in (("f32", "fp32"), ("f32", "fp64"), ("f64", "fp64"), ("bf16", "fp32"), ("f16", "fp32"),
                             ("bf16", "fp64")):
            if form == args.form and landau == args.landau:
                g, km, spl_f = glups_total / world, kernel_ms, spl
            else:
                msf, km, inf, _ = measure_form(torch, rl, w, n, form, landau, args.kernel, min(K, 100), 5, flush)
                g = nodes * len(msf) / (msf.sum() / 1e3) / 1e9
                spl_f = int(inf["steps_per_launch"])
            bp = ALGO_BYTES_PER_UPDATE[form]
            err = parity_error(rl, oracle, form, landau)
            forms["%s/landau-%s" % (form, landau)] = {
                "glups": g, "hbm_gbs": bp * nodes / (km / 1e3) / 1e9,
                "hbm_frac": bp * nodes / (km / 1e3) / 1e9 / hbm_peak, "bytes_per_update": bp,
                "steps_per_launch": spl_f, "max_rel_err_vs_oracle": err}
            if form == "f64":
                tf = FP64_FLOPS_PER_NODE * nodes / (km / 1e3) / 1e12
                forms["f64/landau-fp64"]["fp64_alu"] = {"tflops": tf, "peak_tflops": FP64_PEAK_TFLOPS,
                                                       "frac": tf / FP64_PEAK_TFLOPS}
        line["forms"] = forms
        line["ensemble"] = measure_ensemble(torch, rl, flush)
        line["variants"] = measure_variants(torch, rl, oracle, flush, hbm_peak)
        line["configs"] = measure_configs(torch, rl, flush, hbm_peak)
        # a call advances 1000 steps between host round trips, the 8192^2 workload's own sampling
        # cadence (its spectra are taken every 1000 steps); calls of 100 steps are reported beside it
        line["e2e"] = e2e_glups(rl, w, n, args.form, args.landau, reps=3, steps_per_call=1000)
        line["e2e"]["calls_of_100_steps"] = e2e_glups(rl, w, n, args.form, args.landau, reps=5,
                                                      steps_per_call=100)["value"]
        g, desc, th = cpu_oracle_glups(oracle, w, n, args.cpu_seconds)
        line["cpu_baseline"] = {"value": g, "unit": "GLUPS", "cores": th, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark of the two-lattice free energy LBM step on GB300.

Workload (default): D3Q19 parallel-band shear, 512x256x256 nodes (33.5M),
droplet R = 48 centred, A = kappa = 0.04, tau_f = tau_g = 2, Gamma = 0.5,
u_wall = 0.03, FP32 populations; the FP16/BF16 deviation stores are timed on
the same lattice.  One "step" = one time step of the whole lattice (phi pass,
mu pass, fused pull + collide of f and g).  Metric: MLUPS (million lattice
node updates per second, higher is better).  The state (10.6 GB for FP32) is
far larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one rank per GPU): every rank advances its own independent
lattice (weak scaling, no collective on the data path); value = total MLUPS.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q19 FRE-LBM MLUPS & %HBM peak; FP16-store vs FP32; batched p50/p99 latency"
WORKLOAD = dict(lattice="d3q19", device="shear", nx=512, ny=256, nz=256, tau_f=2.0, tau_g=2.0,
                A=0.04, kappa=0.04, gamma_mob=0.5, u_wall=0.03, rho0=1.0)
DROPLET = (255.5, 127.5, 127.5, 48.0)
# algorithmic bytes per node update: read + write of f and g once (q = 19)
ALG_BYTES = {"fp32": 2 * 2 * 19 * 4, "fp16dev": 2 * (19 * 2 + 18 * 2 + 4),
             "bf16dev": 2 * (19 * 2 + 18 * 2 + 4), "fp64": 2 * 2 * 19 * 8}
CSRC = os.path.join(ROOT, "paper_2212_01617_gb300", "csrc")
# a precision name may carry "+rest": the 16-bit f stored against the rest
# equilibrium w_i rho0 (FRE_FLAG_REST_REFERENCE) instead of the Couette
# equilibrium of the shear walls (the default of the shear device)
FLAG_REST_REFERENCE = 8


def split_prec(name: str):
    base, _, opt = name.partition("+")
    if opt not in ("", "rest"):
        raise SystemExit(f"unknown precision variant {name!r}")
    return base, (FLAG_REST_REFERENCE if opt == "rest" else 0)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# nominal HBM3e bandwidth of a GB300 (the ~8 TB/s the hardware is quoted at)
NOMINAL_HBM_GBS = 7900.0


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


# device sources that make up the time-step kernels
STEP_SOURCES = ("lattice.cuh", "fre_internal.h", "fre_kernels.cuh", "fre_rows.cuh", "fre_pipe.cuh", "fre_ws.cuh")


def strip_comments(src: str) -> str:
    """C/C++ source without comments and trailing blanks (string literals in
    these kernel sources hold no comment markers)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_hash() -> str:
    """Hash of the code of the time-step kernel sources, comments left out
    (the ncu traffic figure is valid for that code only)."""
    h = hashlib.sha256()
    for name in STEP_SOURCES:
        with open(os.path.join(CSRC, name), encoding="utf-8") as fh:
            h.update(name.encode() + strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(precision: str):
    """DRAM bytes per launch of the update kernel from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "k_update_d3q19_dram.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        if d.get("kernel_sha") != kernel_hash():
            return None
        e = d["per_precision"][precision]
        return float(e["dram_bytes_per_node"]) * WORKLOAD["nx"] * WORKLOAD["ny"] * WORKLOAD["nz"]
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    """Ranks of a torchrun launch (one replica per GPU; NCCL on GPUs, gloo
    for the host-only tests of this logic)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    """The largest of the ranks' values (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ws: int, nodes: int, steps: int, ms_max: float) -> float:
    """Whole-job MLUPS of ws independent replicas of `nodes` nodes each, all
    done in ms_max (the slowest rank's time)."""
    return ws * nodes * steps / (ms_max * 1e-3) / 1e6


def time_steps(fre, precision, steps, warmup, ws, local):
    """Kernel-only timing of `steps` time steps with inputs resident in HBM."""
    import torch
    n = WORKLOAD["nx"] * WORKLOAD["ny"] * WORKLOAD["nz"]
    base, flags = split_prec(precision)
    # the context steps on this stream, and the events are recorded on it
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _time_steps(fre, base, flags, steps, warmup, ws, local, n, stream)


def _time_steps(fre, base, flags, steps, warmup, ws, local, n, stream):
    import torch
    sim = fre.Simulation(precision=base, flags=flags, **WORKLOAD)
    sim.init_droplet(*DROPLET)
    sim.step(warmup)
    # per-kernel times (events between the kernels of every step) on a
    # separate run of up to 100 steps; the timed region below steps plainly,
    # so that each kernel may start while its predecessor drains
    kst = max(1, min(steps, 100))
    ms_phi, ms_mu, ms_upd, ms_tot, launches = sim.step_timed(kst)
    ms_phi, ms_mu, ms_upd, ms_tot = (v * steps / kst for v in (ms_phi, ms_mu, ms_upd, ms_tot))
    launches = launches * steps // kst
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ws, ms)
    obs = sim.observables()
    path = sim.kernel_path
    sim.close()
    return dict(ms=ms_max, ms_local=ms, ms_phi=ms_phi, ms_mu=ms_mu, ms_update=ms_upd, ms_seq=ms_tot,
                launches=launches, clocks=clk, obs=obs, n=n, path=path)


def time_e2e(fre, precision, steps, obs_every=100):
    """End to end through the public C API with host buffers: upload of the
    initial fields from pinned host memory, `steps` time steps, observables
    read back to the host every `obs_every` steps and at the end."""
    import numpy as np
    import torch
    nx, ny, nz = WORKLOAD["nx"], WORKLOAD["ny"], WORKLOAD["nz"]
    n = nx * ny * nz
    cx, cy, cz, R = DROPLET
    xi = (WORKLOAD["kappa"] / WORKLOAD["A"]) ** 0.5
    host = {k: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() for k in
            ("rho", "ux", "uy", "uz", "phi")}
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2).reshape(-1)
    host["phi"][:] = np.tanh((R - r) / (np.sqrt(2.0) * xi))
    host["rho"][:] = WORKLOAD["rho0"]
    host["ux"][:] = (WORKLOAD["u_wall"] * (2.0 * (y + 0.5) / ny - 1.0)).reshape(-1)
    host["uy"][:] = 0.0
    host["uz"][:] = 0.0
    del x, y, z, r
    base, flags = split_prec(precision)
    sim = fre.Simulation(precision=base, flags=flags, **WORKLOAD)
    # one untimed pass allocates the I/O staging buffer of the context
    sim.init_fields(host["rho"], host["ux"], host["uy"], host["uz"], host["phi"])
    sim.step(2)
    sim.observables()
    torch.cuda.synchronize()
    reads = 0
    t0 = time.perf_counter()
    sim.init_fields(host["rho"], host["ux"], host["uy"], host["uz"], host["phi"])
    done = 0
    while done < steps:
        k = min(obs_every, steps - done)
        sim.step(k)
        done += k
        sim.observables()
        reads += 1
    t1 = time.perf_counter()
    sim.close()
    obs_bytes = 8 * 22 + 8 + 8
    return dict(value=n * steps / (t1 - t0) / 1e6, unit="MLUPS",
                h2d_bytes_per_step=5 * 8 * n / steps, d2h_bytes_per_step=reads * obs_bytes / steps,
                obs_every=obs_every, seconds=t1 - t0)


def _oracle_rate(threads, seconds):
    """Node updates per second of the FP64 oracle on the 1/8-scale twin with
    `threads` OpenMP threads, over about `seconds` of stepping."""
    import oracle
    nx, ny, nz = 64, 32, 32
    scale = nx / WORKLOAD["nx"]
    w = WORKLOAD
    oracle.set_num_threads(threads)
    o = oracle.Oracle(oracle.D3Q19, oracle.SHEAR, nx, ny, nz, w["tau_f"], w["tau_g"], w["A"], w["kappa"],
                      w["gamma_mob"], w["u_wall"], w["rho0"])
    o.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, DROPLET[3] * scale)
    o.step(2)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(2)
        steps += 2
    dt = time.perf_counter() - t0
    used = oracle.num_threads()
    return nx * ny * nz * steps / dt / 1e6, used, steps, dt


def cpu_baseline(seconds=15.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the
    workload: all host cores (the reported value) and one core."""
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    v_all, used, steps, dt = _oracle_rate(ncores, 0.6 * seconds)
    v_one, _, steps1, dt1 = _oracle_rate(1, 0.4 * seconds)
    oracle.set_num_threads(ncores)
    return {"value": v_all, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"D3Q19 shear 64x32x32 (1/8-scale twin, droplet R={DROPLET[3] * 64 / WORKLOAD['nx']:g}), "
                      f"FP64, {steps} steps in {dt:.1f} s on {used} threads",
            "one_core": {"value": v_one, "unit": "MLUPS", "cores": 1,
                         "sample": f"same twin, {steps1} steps in {dt1:.1f} s on 1 thread"},
            "parallel_speedup": v_all / v_one if v_one > 0 else None}


SERVE_SIZES = [(64, 64, 64), (96, 96, 96), (128, 64, 64), (192, 96, 96)]


def serving_size_rates(steps=50):
    """Step rates (G node updates per second, device-timed) of the serving
    workload's D3Q19 lattice sizes, shear and four-roller, FP32 and FP16-dev,
    on the kernels each context picks (the row kernels where they apply)."""
    import torch
    import paper_2212_01617_gb300 as fre
    out = {}
    for dev in ("shear", "four_roller"):
        for shape in SERVE_SIZES:
            nx, ny, nz = shape
            for prec in ("fp32", "fp16dev"):
                sim = fre.Simulation(lattice="d3q19", precision=prec, device=dev, nx=nx, ny=ny, nz=nz,
                                     **dict(SERVE_PHYS, u_wall=0.02))
                sim.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, ny / 5)
                sim.step(10)
                torch.cuda.synchronize()
                best = None
                for _ in range(3):
                    _, _, upd, tot, _ = sim.step_timed(steps)
                    if best is None or tot < best[0]:
                        best = (tot, upd)
                out[f"{dev} {nx}x{ny}x{nz} {prec}"] = {
                    "gnodes_per_s": nx * ny * nz * steps / (best[0] * 1e-3) / 1e9,
                    "update_frac_of_measured_hbm": ALG_BYTES[prec] * nx * ny * nz * steps / (best[1] * 1e-3) / 1e9
                    / measured_peak_gbs()[0],
                    "kernel_path": sim.kernel_path}
                sim.close()
    return out


def next_rows_summary(steps=100):
    """Device-timed figures of the rows built after the hot path: the full
    functional (model 1) and the interpolated roller walls (per-node
    kernels: step rate and update-kernel fraction of HBM at the same
    304 B/node of f and g), the consistent initialisation (time per
    iteration) and the breakup detection (connected components of phi > 0,
    time per call on the benchmark lattice)."""
    import time
    import torch
    import paper_2212_01617_gb300 as fre
    peak = measured_peak_gbs()[0]
    out = {}

    def step_rate(tag, **kw):
        nx, ny, nz = kw["nx"], kw["ny"], kw["nz"]
        sim = fre.Simulation(lattice="d3q19", precision="fp32", **kw)
        sim.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, ny / 5)
        sim.step(10)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            _, _, upd, tot, _ = sim.step_timed(steps)
            if best is None or tot < best[0]:
                best = (tot, upd)
        n = nx * ny * nz
        out[tag] = {"gnodes_per_s": n * steps / (best[0] * 1e-3) / 1e9, "ms_per_step": best[0] / steps,
                    "update_frac_of_measured_hbm": ALG_BYTES["fp32"] * n * steps / (best[1] * 1e-3) / 1e9 / peak,
                    "kernel_path": sim.kernel_path, "shape": [nx, ny, nz]}
        return sim

    phys = dict(tau_f=2.0, tau_g=2.0, A=0.04, kappa=0.04, gamma_mob=0.5, rho0=1.0)
    step_rate("full_functional_shear_fp32", device="shear", nx=128, ny=64, nz=64, u_wall=0.03,
              model=1, kappa1=0.03, kappa2=0.09, alpha=0.8, **phys).close()
    step_rate("interpolated_walls_four_roller_fp32", device="four_roller", nx=192, ny=96, nz=96, u_wall=0.02,
              flags=fre.FRE_FLAG_INTERPOLATED_WALLS, **phys).close()
    # consistent initialisation, 128x64x64 FP32
    sim = fre.Simulation(lattice="d3q19", precision="fp32", device="shear", nx=128, ny=64, nz=64, u_wall=0.03,
                         **phys)
    sim.init_droplet(63.5, 31.5, 31.5, 12.8)
    sim.init_consistent(5)
    torch.cuda.synchronize()
    iters = 50
    t0 = time.perf_counter()
    sim.init_consistent(iters)
    torch.cuda.synchronize()
    out["consistent_init_shear_fp32"] = {"ms_per_iteration": (time.perf_counter() - t0) * 1e3 / iters,
                                         "iterations": iters, "shape": [128, 64, 64]}
    sim.close()
    # breakup detection on the benchmark lattice
    w = WORKLOAD
    sim = fre.Simulation(precision="fp32", **w)
    sim.init_droplet(*DROPLET)
    sim.step(2)
    sim.components()
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        count, _, _ = sim.components()
    ms = (time.perf_counter() - t0) * 1e3 / reps
    n = w["nx"] * w["ny"] * w["nz"]
    out["components_bench_lattice"] = {"ms_per_call": ms, "gnodes_per_s": n / (ms * 1e-3) / 1e9,
                                       "components": count, "shape": [w["nx"], w["ny"], w["nz"]],
                                       "what": "host-timed call (labels on the device, counts read back)"}
    sim.close()
    return out


def base_config(precision):
    return {"workload": "D3Q19 two-lattice FRE-LBM, parallel-band shear 512x256x256 (33.5M nodes), "
                        "droplet R=48, A=kappa=0.04, tau=2, Gamma=0.5, u_w=0.03",
            "lattice": "D3Q19", "nodes": WORKLOAD["nx"] * WORKLOAD["ny"] * WORKLOAD["nz"],
            "shape": [WORKLOAD["nx"], WORKLOAD["ny"], WORKLOAD["nz"]], "precision": precision,
            "l2": "inputs larger than L2 (10.6 GB FP32 state vs 129 MB L2); no flush",
            "parallelism": "independent lattice per GPU (replicas)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nx, ny, nz = 64, 32, 32
    scale = nx / WORKLOAD["nx"]
    w = WORKLOAD
    o = oracle.Oracle(oracle.D3Q19, oracle.SHEAR, nx, ny, nz, w["tau_f"], w["tau_g"], w["A"], w["kappa"],
                      w["gamma_mob"], w["u_wall"], w["rho0"])
    o.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, DROPLET[3] * scale)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    n = nx * ny * nz
    value = n * args.steps / dt / 1e6
    sample = (f"each step: one FP64 oracle time step of the 1/8-scale twin {nx}x{ny}x{nz} "
              f"(droplet R={DROPLET[3] * scale:g}) on the host cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": base_config("fp64"),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_case(spec: str, precisions, steps: int = 3):
    """Small case of the benchmark kernels for ncu captures: a D3Q19 shear
    lattice of the given size (e.g. 512x64x32), droplet, `steps` steps.  A
    "four_roller:" prefix (e.g. four_roller:192x96x96) takes the four-roller
    device instead, at the same physical parameters (u_wall 0.02)."""
    import torch
    import paper_2212_01617_gb300 as fre
    device, _, size = spec.rpartition(":")
    nx, ny, nz = (int(v) for v in size.split("x"))
    w = dict(WORKLOAD, nx=nx, ny=ny, nz=nz)
    if device:
        if device not in ("shear", "four_roller"):
            raise SystemExit(f"unknown device {device!r} in --profile-case")
        w["device"] = device
        if device == "four_roller":
            w["u_wall"] = 0.02
    for prec in precisions:
        base, flags = split_prec(prec)
        sim = fre.Simulation(precision=base, flags=flags, **w)
        sim.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, min(ny, nz) * 0.375)
        sim.step(steps)
        torch.cuda.synchronize()
        print(f"profile case {spec} {prec}: path {sim.kernel_path}, D = {sim.observables()['D']:.6f}", flush=True)
        sim.close()
    return 0


# D2Q9 batch of uneven cases: interface A = kappa = 0.01 (xi = 1), sigma =
# sqrt(8 kappa A / 9); tau_f = 2 (dynamic viscosity rho0 cs^2 (tau_f - 1/2) = 0.5)
BATCH_PHYS = dict(tau_f=2.0, tau_g=1.0, A=0.01, kappa=0.01, gamma_mob=1.0, rho0=1.0)


def batch_case_params(c):
    """Lattice, droplet and wall speed of one drawn batch case.  Shear: H = Ny
    = Nx/2, rate G = 2 u_w / H, R = (R/H) H.  Four-roller: Ny = Nx, H = Nx/2,
    rate G = u_w / (Nx/4), R = (R/H) H.  Ca = mu G R / sigma gives
    u_w = Ca sigma / (2 mu (R/H)) for both."""
    nx = c["nx"]
    ny = nx // 2 if c["device"] == "shear" else nx
    H = ny if c["device"] == "shear" else nx / 2
    sigma = (8.0 * BATCH_PHYS["kappa"] * BATCH_PHYS["A"] / 9.0) ** 0.5
    mu_visc = BATCH_PHYS["rho0"] * (BATCH_PHYS["tau_f"] - 0.5) / 3.0
    u_w = c["ca"] * sigma / (2.0 * mu_visc * c["r_over_h"])
    params = dict(BATCH_PHYS, lattice="d2q9", device=c["device"], nx=nx, ny=ny, nz=1, u_wall=u_w)
    drop = ((nx - 1) / 2, (ny - 1) / 2, 0.0, c["r_over_h"] * H)
    return params, drop


def run_batch_workload(args):
    """64 uneven D2Q9 cases (half shear, half four-roller), FP32: one batch
    (autotuned batched, per-slot or concurrent per-slot launches, CUDA-graph
    replays) against one context per case stepped on its own (one launch per
    kernel per case)."""
    line = batch_summary(args.steps, max(args.warmup, 40), args.batch_mode)
    print(json.dumps(line), flush=True)
    return 0


def batch_summary(steps, warmup, mode=None):
    import torch
    import paper_2212_01617_gb300 as fre
    from paper_2212_01617_gb300 import inputs
    cases = [batch_case_params(c) for c in inputs.batch_cases(64)]
    nodes = sum(p["nx"] * p["ny"] for p, _ in cases)
    # one stream for the batch and for every per-case context: the events
    # bracket all the work and the per-case launches run one after another
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _batch_workload(steps, warmup, fre, cases, nodes, stream, mode)


def _batch_workload(steps, warmup, fre, cases, nodes, stream, mode=None):
    import torch
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    b = fre.Batch("d2q9", "fp32")
    if mode is not None:
        # launch mode pinned (for profiling): no autotuning
        m, _, bx = mode.partition(":")
        b.set_mode(int(m), int(bx) if bx else 64)
    for p, d in cases:
        b.add(*d, **p)
    b.step(warmup)  # includes the autotuner's timed candidates
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = ev(), ev()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_batch = e0.elapsed_time(e1)
    tuning = b.tuning()
    b.close()

    sims = []
    for p, d in cases:
        sim = fre.Simulation(precision="fp32", **{k: v for k, v in p.items() if k != "precision"})
        sim.init_droplet(*d)
        sims.append(sim)
    for sim in sims:
        sim.step(3)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for sim in sims:
        sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for sim in sims:
        sim.close()
    mode = {0: "batched", 1: "per-slot", 2: "per-slot concurrent"}[tuning["mode"]]
    peak = measured_peak_gbs()[0]
    achieved = 144.0 * nodes / (ms_batch / steps * 1e-3) / 1e9
    return {"metric": "batched D2Q9 FRE-LBM MLUPS, 64 uneven cases", "value": nodes * steps / ms_batch / 1e3,
            "unit": "MLUPS", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": ms_batch / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 D2Q9 cases, Nx uniform in 64..512 (even), shear Ny=Nx/2, four-roller "
                                   "Ny=Nx, Ca U(0.05,0.5), R/H U(0.1,0.3), FP32", "nodes": nodes,
                       "l2": "state of all cases (~0.4 GB) larger than L2; no flush"},
            "sequential": {"value": nodes * steps / ms_seq / 1e3, "unit": "MLUPS",
                           "ms_per_step": ms_seq / steps,
                           "what": "one context per case, each stepped on its own kernels"},
            "speedup_vs_sequential": ms_seq / ms_batch,
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak, "achieved": achieved,
                         "frac": achieved / peak, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "what": "whole batch step, algorithmic 144 B per D2Q9 FP32 node update"},
            "tuning": {"mode": mode, "bx": tuning["bx"],
                       "ms_per_step_candidates": dict(zip(["batched bx32", "batched bx64", "batched bx128",
                                                           "per-slot", "per-slot concurrent"],
                                                          tuning["ms_per_step"]))},
            "clocks": clk}


# D3Q19 serving requests: A = kappa = 0.01 (xi = 1), tau_f = 1.5 (dynamic
# viscosity 1/3), tau_g = 1, Gamma = 1
SERVE_PHYS = dict(tau_f=1.5, tau_g=1.0, A=0.01, kappa=0.01, gamma_mob=1.0, rho0=1.0)


def serve_case_params(c):
    """Lattice, droplet and wall speed of one request.  Shear: H = Ny, rate
    G = 2 u_w / H.  Four-roller: H = Nx/2, rate G = u_w / (Nx/4).  R = (R/H) H
    and Ca = mu G R / sigma, so u_w = Ca sigma / (2 mu (R/H)) for both."""
    nx, ny, nz = c["shape"]
    H = ny if c["device"] == "shear" else nx / 2
    sigma = (8.0 * SERVE_PHYS["kappa"] * SERVE_PHYS["A"] / 9.0) ** 0.5
    mu_visc = SERVE_PHYS["rho0"] * (SERVE_PHYS["tau_f"] - 0.5) / 3.0
    u_w = c["ca"] * sigma / (2.0 * mu_visc * c["r_over_h"])
    params = dict(SERVE_PHYS, lattice="d3q19", device=c["device"], nx=nx, ny=ny, nz=nz, u_wall=u_w)
    drop = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, c["r_over_h"] * H)
    return params, drop


def drive_server(srv, trace, cases):
    """Submit each request when its arrival time comes (server clock) and
    advance the server until every request has a result."""
    start = srv.clock()
    n = len(trace)
    i, by_id, results = 0, {}, {}
    while len(results) < n:
        now = srv.clock() - start
        while i < n and trace[i]["t_arrival"] <= now:
            p, d = cases[i]
            by_id[srv.submit(*d, **p)] = i
            i += 1
        running = srv.advance()
        for r in srv.results():
            k = by_id[r["id"]]
            r["latency"] = r["t_done"] - (start + trace[k]["t_arrival"])
            r["nodes"] = int(np.prod(trace[k]["shape"]))
            results[k] = r
        if running == 0 and srv.stats()["queued"] == 0 and i < n:
            wait = trace[i]["t_arrival"] - (srv.clock() - start)
            if wait > 0:
                time.sleep(wait)
    end = max(r["t_done"] for r in results.values())
    return results, end - start


SERVE_ARMS = {
    # the configured serving loop: FP16-dev storage, continuous batching
    "batched_fp16dev": dict(precision="fp16dev", chunk_steps=250),
    # the same requests one at a time in plain FP32 (the configured baseline)
    "sequential_fp32": dict(precision="fp32", max_running=1, chunk_steps=1000),
    # one at a time in the same FP16-dev storage: separates the gain of
    # batching from the gain of the storage format
    "sequential_fp16dev": dict(precision="fp16dev", max_running=1, chunk_steps=1000),
}


def serve_summary(n_requests, max_steps, target_nodes, arms=tuple(SERVE_ARMS)):
    """Poisson-arriving D3Q19 droplet-deformation requests through the
    serving loop, one run per arm of SERVE_ARMS on the same trace."""
    import torch
    import paper_2212_01617_gb300 as fre
    from paper_2212_01617_gb300 import inputs
    trace = inputs.serving_trace(n_requests)
    cases = [serve_case_params(c) for c in trace]
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        for name in arms:
            kw = dict(SERVE_ARMS[name])
            prec = kw["precision"]
            if "max_running" not in kw:
                kw["target_nodes"] = target_nodes
            srv = fre.Server("d3q19", budget_bytes=150 << 30, check_every=1000, tol_D=1e-4,
                             max_steps=max_steps, stream=stream.cuda_stream, **kw)
            cs = [(dict(p, precision=prec), d) for p, d in cases]
            res, wall = drive_server(srv, trace, cs)
            st = srv.stats()
            srv.close()
            lat = np.array([res[k]["latency"] for k in range(len(trace))])
            upd = sum(res[k]["steps"] * res[k]["nodes"] for k in range(len(trace)))
            outcomes = {}
            for r in res.values():
                outcomes[r["outcome"]] = outcomes.get(r["outcome"], 0) + 1
            out[name] = {"aggregate_mlups": upd / wall / 1e6, "wall_s": wall,
                         "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                         "mean_s": float(lat.mean()), "node_updates": upd, "outcomes": outcomes,
                         "mean_steps": float(np.mean([r["steps"] for r in res.values()])),
                         "contexts_created": st["contexts_created"], "contexts_reused": st["contexts_reused"],
                         "batch_mode_at_end": {0: "batched", 1: "per-slot", 2: "per-slot concurrent"}.get(
                             st["batch_mode"]),
                         "autotunes": st["tunes"], "graph_captures": st["captures"]}
            log(f"serve {name}: {json.dumps(out[name])}")
    summary = {"requests": len(trace), "max_steps": max_steps, "target_nodes": target_nodes, "arms": out}
    b = out.get("batched_fp16dev")
    for base in ("sequential_fp32", "sequential_fp16dev"):
        s_ = out.get(base)
        if b and s_:
            summary[f"vs_{base}"] = {"throughput_ratio": b["aggregate_mlups"] / s_["aggregate_mlups"],
                                     "speedup_p50": s_["p50_s"] / b["p50_s"],
                                     "speedup_p99": s_["p99_s"] / b["p99_s"]}
    return summary


def run_serve_workload(args):
    """Poisson-arriving D3Q19 droplet-deformation requests: the serving loop
    (FP16 deviation store, continuous batching under a 150 GB budget)
    against the same requests served one at a time in plain FP32 and in
    FP16-dev storage."""
    sm = serve_summary(args.serve_requests, args.serve_max_steps, args.serve_target_nodes)
    b, s_ = sm["arms"]["batched_fp16dev"], sm["arms"]["sequential_fp32"]
    line = {"metric": "serving D3Q19 FRE-LBM: aggregate MLUPS and p50/p99 time-to-result",
            "value": b["aggregate_mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": None, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16-store/f32",
            "data": "synthetic",
            "config": {"workload": f"{sm['requests']} Poisson requests (20/s), D3Q19 sizes 64^3, 96^3, "
                                   "128x64x64, 192x96x96, shear or four-roller, Ca U(0.05,0.45), R/H U(0.1,0.3), "
                                   "run until |dD| < 1e-4 per 1000 steps or breakup, 150 GB budget",
                       "max_steps": args.serve_max_steps, "target_nodes": args.serve_target_nodes},
            "p50_s": b["p50_s"], "p99_s": b["p99_s"], **{k: v for k, v in sm.items() if k != "arms"},
            **sm["arms"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precisions", default="fp32,fp16dev,bf16dev,fp16dev+rest,bf16dev+rest")
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    help="[four_roller:]NXxNYxNZ: run a few steps of a small case (ncu captures) and exit")
    ap.add_argument("--workload", choices=["lattice", "batch", "serve"], default="lattice",
                    help="lattice: the 512x256x256 D3Q19 lattice (default); batch: 64 uneven D2Q9 cases; "
                         "serve: Poisson-arriving D3Q19 requests through the serving loop")
    ap.add_argument("--batch-mode", default=None,
                    help="MODE[:BX] pins the batch's launch mode (0 batched, 1 per-slot, 2 concurrent) for profiling")
    ap.add_argument("--no-batch-serve", action="store_true",
                    help="leave the batch and serving summaries out of the default line")
    ap.add_argument("--summary-requests", type=int, default=12,
                    help="requests of the serving summary in the default line")
    ap.add_argument("--summary-max-steps", type=int, default=8000)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-target-nodes", type=int, default=8_000_000)
    ap.add_argument("--serve-max-steps", type=int, default=30000)
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch_workload(args)
    if args.workload == "serve":
        return run_serve_workload(args)
    if args.profile_case:
        return profile_case(args.profile_case, [p for p in args.precisions.split(",") if p])
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        return run_reference(args, ws, rank)

    import torch
    ws, rank, local = dist_setup()
    import paper_2212_01617_gb300 as fre
    fre.load_library()

    precisions = [p for p in args.precisions.split(",") if p]
    runs = {}
    for prec in precisions:
        runs[prec] = time_steps(fre, prec, args.steps, args.warmup, ws, local)
        r = runs[prec]
        log(f"[rank {rank}] {prec}: {r['ms'] / args.steps:.3f} ms/step, "
            f"{r['n'] * args.steps / (r['ms'] * 1e-3) / 1e6:.0f} MLUPS per GPU, update "
            f"{r['ms_update'] / args.steps:.3f} ms, phi {r['ms_phi'] / args.steps:.3f} ms, "
            f"mu {r['ms_mu'] / args.steps:.3f} ms, D={r['obs']['D']:.4f}")
    main_prec = precisions[0]
    r = runs[main_prec]
    n = r["n"]
    value = weak_scaling_value(ws, n, args.steps, r["ms"])
    peak, peak_src = measured_peak_gbs()
    t_upd = r["ms_update"] / args.steps * 1e-3
    achieved = ALG_BYTES[split_prec(main_prec)[0]] * n / t_upd / 1e9
    traffic = ncu_traffic(split_prec(main_prec)[0])
    step_achieved = ALG_BYTES[split_prec(main_prec)[0]] * n / (r["ms"] / args.steps * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(fre, main_prec, args.e2e_steps)
        e2e["value"] *= ws  # every rank ran the same job on its own GPU

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    # batch and serving summaries (one GPU, rank 0 of a single-rank run)
    batch, serve, next_rows = None, None, None
    if rank == 0 and ws == 1 and not args.no_batch_serve:
        bl = batch_summary(200, 40)
        batch = {k: bl[k] for k in ("value", "unit", "ms_per_step", "sequential", "speedup_vs_sequential",
                                    "roofline", "tuning", "config")}
        serve = serve_summary(args.summary_requests, args.summary_max_steps, args.serve_target_nodes)
        serve["step_rates_by_size"] = serving_size_rates()
        next_rows = next_rows_summary()

    if rank == 0:
        variants = {}
        for prec, rr in runs.items():
            t = rr["ms_update"] / args.steps * 1e-3
            ab = ALG_BYTES[split_prec(prec)[0]]
            variants[prec] = {
                "mlups": ws * rr["n"] * args.steps / (rr["ms"] * 1e-3) / 1e6,
                "ms_per_step": rr["ms"] / args.steps,
                "update_ms": rr["ms_update"] / args.steps, "phi_ms": rr["ms_phi"] / args.steps,
                "mu_ms": rr["ms_mu"] / args.steps,
                "update_alg_gbs": ab * rr["n"] / t / 1e9,
                "update_frac_of_measured_hbm": ab * rr["n"] / t / 1e9 / peak,
                "update_frac_of_nominal_hbm": ab * rr["n"] / t / 1e9 / NOMINAL_HBM_GBS,
                "step_alg_frac_of_measured_hbm": ab * rr["n"] / (rr["ms"] / args.steps * 1e-3)
                / 1e9 / peak,
                "D_after_run": rr["obs"]["D"], "mass": rr["obs"]["mass"], "kernel_path": rr["path"],
            }
        if "fp32" in runs and "fp16dev" in runs:
            variants["fp16dev_speedup_vs_fp32"] = variants["fp16dev"]["mlups"] / variants["fp32"]["mlups"]
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if main_prec == "fp32" else ("f16-store/f32" if main_prec == "fp16dev" else main_prec),
            "data": "synthetic", "config": base_config(main_prec),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "kernel": (f"k_wsrow<19,{main_prec},update,pull> (fused pull + collide of f and g; "
                                    "warp-specialised, bulk-copy staged x-rows)" if r["path"] == 2 else
                                    f"update kernel, path {r['path']}"),
                         "algorithmic_bytes_per_launch": ALG_BYTES[split_prec(main_prec)[0]] * n,
                         "peak_source": peak_src,
                         "step_achieved": step_achieved, "step_frac": step_achieved / peak,
                         "step_frac_of_nominal": step_achieved / NOMINAL_HBM_GBS},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "variants": variants,
        }
        if batch is not None:
            line["batch"] = batch
        if serve is not None:
            line["serve"] = serve
        if next_rows is not None:
            line["next_rows"] = next_rows
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

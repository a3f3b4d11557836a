"""Throughput of the moment-only lattice Boltzmann step on GB300.

Workload (one step = one full time step of the hot path over the box):
256^3 periodic box, D3Q19, FP32 moments, 3D Taylor-Green vortex u0 = 0.05
plus seeded U(-1e-3, 1e-3) velocity noise, tau = 0.6.  Metric: MLUPS =
nodes / (1e6 * seconds per step) (Sec. IV A, Eq. (12)), with the HBM
roofline fraction of the step kernel, and the population-storing LB of the
same library on the same box and GPU beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one independent replica per GPU (weak scaling; the step has no
data exchange between replicas).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM peak: moment-only vs stored-population LB, 1 GB300, at oracle tol"
NX = NY = NZ = 256
LATTICE = 19
TAU = 0.6
U0, NOISE, SEED = 0.05, 1e-3, 2301
WORKLOAD = "256^3 periodic D3Q19 moment-only LB, FP32, Taylor-Green u0=0.05 + U(-1e-3,1e-3) noise, tau=0.6"
# near-contact strength of the bench's droplet collision: the paper's value, with which the
# 20000-step run of the 384 x 192 x 192 pair ends as two droplets (A_h = 0: one)
OUTCOME_A_H = 0.01
L2_NOTE = "inputs larger than L2 (each FP32 state copy 671 MB vs 129 MB L2); no flush"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the D3Q27 and population lines")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tma", "tiled", "direct"],
                    help="moment-only kernel (auto = the library's choice)")
    ap.add_argument("--variant", type=int, default=0, help="kernel variant (tuning; tiled 0..5, TMA 0..2)")
    ap.add_argument("--lattice", type=int, default=19, choices=[19, 27], help="lattice of the main line")
    ap.add_argument("--cg-variant", type=int, default=0, help="two-component kernel variant (tuning)")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds the reference arm (host oracle) may spend on its timed steps")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed


def dist_setup(ngpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_available() else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def _cuda_available():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(value: float, world: int) -> float:
    """Max of a float over ranks (the slowest replica defines the job time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
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
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks / profiles


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s)"


KERNEL_SOURCES = ("moment_tiled.cuh", "moment_common.cuh", "moment_tiled_f32.cu", "lattice.cuh", "layout.cuh",
                  "storage.cuh")


def kernel_source_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2301_01622_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(key: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(key)
    if not d or d.get("source_sha") != kernel_source_sha():
        return None
    return float(d["dram_bytes_per_launch"])


# ----------------------------------------------------------------------------- GPU timing


KERNEL_CODE = {"auto": 0, "direct": 1, "tiled": 2, "tma": 3}
_KERNEL = ["auto", 0]


def make_ctx(llb, lattice, scheme, stream, storage=None):
    kern = KERNEL_CODE[_KERNEL[0]] if scheme == llb.LLB_SCHEME_MOMENT else 0
    p = llb.llb_params_default(storage=llb.LLB_F32 if storage is None else storage, scheme=scheme,
                               stream=stream, kernel=kern, variant=_KERNEL[1])
    return llb.llb_create(NX, NY, NZ, lattice, TAU, p)


def time_steps(llb, ctx, steps, warmup, world, sampler=None):
    """Device time of `steps` single-step launches (CUDA events on the context stream)."""
    import torch
    llb.llb_step(ctx, warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        llb.llb_step(ctx, 1)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(world)
    ms = e0.elapsed_time(e1)
    return ms, clocks


def gpu_arm(args, rank, world, local):
    import torch

    from paper_2301_01622_gb300 import inputs, llb

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream().cuda_stream
    rho, u = inputs.taylor_green_3d(NX, NY, NZ, u0=U0, noise=NOISE, seed=SEED)
    nodes = NX * NY * NZ
    peak, peak_src = measured_peaks()

    def run(lattice, scheme, sampler=None, storage=None):
        ctx = make_ctx(llb, lattice, scheme, stream, storage=storage)
        try:
            llb.llb_init_equilibrium(ctx, rho, u)
            kernel = llb.llb_state_device(ctx)[2]
            ms, clocks = time_steps(llb, ctx, args.steps, args.warmup, world, sampler)
            fp = llb.llb_footprint_query(NX, NY, NZ, lattice, llb.llb_params_default(
                scheme=scheme, storage=llb.LLB_F32 if storage is None else storage))
        finally:
            llb.llb_destroy(ctx)
        ms_max = reduce_max(ms, world)
        t_step = ms_max / 1e3 / args.steps
        mlups = world * nodes / t_step / 1e6
        gbs = fp.stream_bytes_per_node * nodes / (ms / 1e3 / args.steps) / 1e9
        return {"mlups": mlups, "ms_per_step": ms_max / args.steps, "achieved_gbs": gbs, "frac": gbs / peak,
                "bytes_per_node": fp.stream_bytes_per_node, "kernel": kernel, "clocks": clocks,
                "launch_ms": ms / args.steps}

    main = run(args.lattice, llb.LLB_SCHEME_MOMENT, ClockSampler(local))
    extra = {}
    if not args.no_extra:
        extra["population_d3q19"] = run(19, llb.LLB_SCHEME_POPULATION)
        extra["moment_d3q27"] = run(27, llb.LLB_SCHEME_MOMENT)
        extra["population_d3q27"] = run(27, llb.LLB_SCHEME_POPULATION)
        # 16-bit shifted/scaled storage, FP32 arithmetic (40 B/node)
        for q in (19, 27):
            extra[f"moment_d3q{q}_fp16"] = run(q, llb.LLB_SCHEME_MOMENT, storage=llb.LLB_F16S)
            extra[f"moment_d3q{q}_bf16"] = run(q, llb.LLB_SCHEME_MOMENT, storage=llb.LLB_BF16S)

    if not args.no_extra:
        extra["two_component_d3q27"] = droplet_arm(args, llb, inputs, stream, world, peak, OUTCOME_A_H,
                                                   "near-contact force on: the pair does not merge")
        extra["batched_ensemble"] = ensemble_arm(args, llb, inputs, stream, world, peak)
        extra["adjoint_two_component_d3q27"] = adjoint_arm(args, llb, inputs, stream, world, peak)

    # end to end through the C ABI with pinned host buffers
    e2e = e2e_arm(args, llb, rho, u, stream, world)

    # diagnostics pass (off the step path; reported separately)
    ctx = make_ctx(llb, LATTICE, llb.LLB_SCHEME_MOMENT, stream)
    try:
        llb.llb_init_equilibrium(ctx, rho, u)
        llb.llb_step(ctx, 2)
        llb.llb_diagnostics(ctx)
        t0 = time.perf_counter()
        for _ in range(5):
            diag = llb.llb_diagnostics(ctx)
        diag_ms = (time.perf_counter() - t0) / 5 * 1e3
    finally:
        llb.llb_destroy(ctx)
    return main, extra, e2e, {"ms": diag_ms, "mass": diag["mass"][0], "flags": diag["flags"]}, peak, peak_src


def droplet_arm(args, llb, inputs, stream, world, peak, A_h, label):
    """Two-component D3Q27 droplet collision, 384 x 192 x 192, FP32, tau = 1,
    R = 30, +-0.05 along x, impact parameter 0.5 R: MLUPS of the fused
    moment-only colour-gradient step (88 B/node), and of the colour-gradient
    LB with stored colour populations on the same field (BGK collision, the
    paper's "standard CGLB"; 432 B/node algorithmic: 2Q populations read and
    written; the implementation is the split approach, a phase-field pass and
    a collide-and-stream pass, which moves ~656 B/node)."""
    nx, ny, nz = 384, 192, 192
    r1, r2, u = inputs.droplet_pair(nx, ny, nz, 30.0, 0.05, 15.0)
    nodes = nx * ny * nz
    steps = max(10, args.steps // 4)
    out = {}
    for key, scheme, bpn in (("moment", llb.LLB_SCHEME_MOMENT, 88),
                             ("population_bgk", llb.LLB_SCHEME_POPULATION_BGK, 2 * 2 * 27 * 4)):
        p = llb.llb_params_default(ncomp=2, storage=llb.LLB_F32, A_h=A_h, A_s=0.01, beta=0.7, stream=stream,
                                   scheme=scheme, variant=getattr(args, "cg_variant", 0) if key == "moment" else 0)
        ctx = llb.llb_create(nx, ny, nz, 27, 1.0, p)
        e2e = None
        try:
            llb.llb_init_equilibrium(ctx, np.stack([r1, r2]), u)
            ms, _ = time_steps(llb, ctx, steps, max(3, args.warmup), world)
            if key == "moment":
                llb.llb_init_equilibrium(ctx, np.stack([r1, r2]), u)  # end to end from the initial field
                e2e = droplet_e2e(args, llb, ctx, (11, nz, ny, nx), world)
        finally:
            llb.llb_destroy(ctx)
        ms = reduce_max(ms, world)
        t = ms / 1e3 / steps
        gbs = bpn * nodes / t / 1e9
        out[key] = {"mlups": world * nodes / t / 1e6, "frac": gbs / peak, "achieved_gbs": gbs, "bytes_per_node": bpn,
                    "ms_per_step": ms / steps, "steps": steps}
        if e2e is not None:
            out[key]["e2e"] = e2e
    line = dict(out["moment"])
    line["workload"] = f"384x192x192 D3Q27 two-component CG, FP32, tau=1, R=30, U=+-0.05, b=0.5R, A_h={A_h} ({label})"
    line["population_bgk"] = out["population_bgk"]
    line["speedup_vs_population"] = out["moment"]["mlups"] / out["population_bgk"]["mlups"]
    return line


def droplet_e2e(args, llb, ctx, shape, world):
    """One step end to end through llb_step_host: pinned host canonical FP32
    moments (11 fields) in, one step, moments out, the slab copies overlapped
    with the per-slab steps; `args.e2e_steps` timed calls."""
    import torch
    dev = torch.empty(shape, dtype=torch.float32, device="cuda")
    llb.llb_get_moments_device(ctx, dev)
    h_in = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    h_out = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    h_in.copy_(dev)
    del dev
    torch.cuda.synchronize()
    k = max(1, args.e2e_steps)
    for _ in range(2):
        llb.llb_step_host(ctx, h_in, h_out, 1)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(k):
        llb.llb_step_host(ctx, h_in, h_out, 1)
    torch.cuda.synchronize()
    dt = reduce_max(time.perf_counter() - t0, world)
    nodes = shape[1] * shape[2] * shape[3]
    nbytes = 11 * nodes * 4
    return {"value": world * nodes * k / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": k,
            "path": "llb_step_host(host in, 1 step, host out), FP32 canonical (11 fields), pinned, copies overlapped "
                    "with per-slab steps"}


def ensemble_arm(args, llb, inputs, stream, world, peak):
    """64 two-component D3Q27 droplet-collision boxes, sizes drawn from
    {48, 64, 96, 128}^3, radius in [8, N/6], impact parameter in [0, R], head-on
    speeds in [0.02, 0.08] (seeded), FP32, tau = 1, all boxes advanced by one
    persistent launch per step replayed from a CUDA graph; the tile variant is
    chosen by the library's autotuner."""
    import torch
    rng = np.random.default_rng(2301)
    sizes = rng.choice([48, 64, 96, 128], size=64)
    dims = [(int(n), int(n), int(n)) for n in sizes]
    p = llb.llb_params_default(ncomp=2, storage=llb.LLB_F32, A_h=0.01, A_s=0.01, beta=0.7, stream=stream)
    b = llb.llb_batch_create(dims, 27, 1.0, p)
    try:
        for k, (n, _, _) in enumerate(dims):
            r = rng.uniform(8.0, n / 6.0)
            bimp = rng.uniform(0.0, r)
            v = rng.uniform(0.02, 0.08)
            r1, r2, u = inputs.droplet_pair(n, n, n, r, v / 2, bimp)
            llb.llb_init_equilibrium(llb.llb_batch_domain(b, k), np.stack([r1, r2]), u)
        variant = llb.llb_batch_autotune(b, 3)
        nodes = llb.llb_batch_nodes(b)
        steps = max(10, args.steps // 20)
        llb.llb_batch_step_graph(b, steps)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        llb.llb_batch_step_graph(b, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), world)
    finally:
        llb.llb_batch_destroy(b)
    t = ms / 1e3 / steps
    gbs = 88 * nodes / t / 1e9
    return {"mlups": world * nodes / t / 1e6, "frac": gbs / peak, "achieved_gbs": gbs, "bytes_per_node": 88,
            "ms_per_step": ms / steps, "steps": steps, "boxes": 64, "nodes": nodes, "variant": variant,
            "workload": "64 two-component D3Q27 droplet boxes, sizes from {48,64,96,128}^3, one launch per step, CUDA graph"}


def adjoint_arm(args, llb, inputs, stream, world, peak):
    """Gradient of a phase-field mismatch loss through 500 two-component D3Q27
    FP32 steps on 96^3 (off-axis droplet pair, smooth interface normal, no
    near-contact switch), checkpoints every 22 steps: one llb_adjoint call
    (forward with checkpoints, segment recomputation, adjoint steps), with the
    500 forward steps alone timed beside it to split the call.  Algorithmic
    bytes per node of one adjoint step: the cotangent pass reads 11 cotangent
    and 11 state fields and writes 11 + 3 (cotangents of the fields and of the
    phase-field gradient), the gradient-stencil pass reads 2 state, 3 + 2
    cotangent fields and writes 2: 45 FP32 values = 180 B."""
    import torch
    n, steps, every = 96, 500, 22
    prm = dict(ncomp=2, storage=llb.LLB_F32, beta=0.7, A_s=0.01, A_h=0.0, grad_eps=0.02, stream=stream)
    r1, r2, u = inputs.droplet_pair(n, n, n, 12.0, 0.05, 6.0)
    ctx = llb.llb_create(n, n, n, 27, 1.0, llb.llb_params_default(**prm))
    try:
        llb.llb_init_equilibrium(ctx, np.stack([r1, r2]), u)
        g = torch.zeros((11, n, n, n), dtype=torch.float32, device="cuda")
        g[0] = 1e-3
        gi = torch.empty_like(g)
        llb.llb_adjoint(ctx, 10, g, gi, every=5)   # warm-up (allocations, first launches)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        llb.llb_adjoint(ctx, steps, g, gi, every=every)   # synchronises
        dt = reduce_max(time.perf_counter() - t0, world)
        # the context holds the starting state again (llb_adjoint restores it)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        llb.llb_step(ctx, steps)
        llb.llb_synchronize(ctx)
        dt_fwd = reduce_max(time.perf_counter() - t0, world)
    finally:
        llb.llb_destroy(ctx)
    nodes = n ** 3
    # the call runs the forward steps twice (checkpointing, then segment recomputation)
    dt_adj = max(dt - 2 * dt_fwd, 1e-9)
    gbs = 180 * nodes * steps / dt_adj / 1e9
    return {"seconds": dt, "steps": steps, "checkpoint_every": every,
            "mlups_gradient": world * nodes * steps / dt / 1e6,
            "forward_seconds": dt_fwd, "adjoint_steps_seconds_estimate": dt_adj,
            "adjoint_bytes_per_node": 180, "adjoint_achieved_gbs": gbs, "adjoint_frac": gbs / peak,
            "workload": "96^3 D3Q27 two-component FP32, 500 steps, loss gradient w.r.t. initial moments and tau "
                        "(forward + recomputation + adjoint per step; host wall clock of one synchronising call; "
                        "adjoint share = call - 2 x forward)"}


def e2e_arm(args, llb, rho, u, stream, world):
    """Per step, through the public C ABI: pinned host canonical FP32 moments ->
    device, one step, device -> pinned host (llb_step_host, which overlaps the
    slab copies with the per-slab steps); the sequential form
    (llb_init_moments + llb_step + llb_get_moments) is timed beside it."""
    import torch

    nodes = NX * NY * NZ
    ctx = make_ctx(llb, LATTICE, llb.LLB_SCHEME_MOMENT, stream)
    try:
        llb.llb_init_equilibrium(ctx, rho, u)
        dev = torch.empty((10, NZ, NY, NX), dtype=torch.float32, device="cuda")
        llb.llb_get_moments_device(ctx, dev)
        h_in = torch.empty((10, NZ, NY, NX), dtype=torch.float32, pin_memory=True)
        h_out = torch.empty_like(h_in).pin_memory()
        h_in.copy_(dev)
        torch.cuda.synchronize()
        k = max(1, args.e2e_steps)
        times = {}
        for name in ("sequential", "overlapped"):
            def one():
                if name == "overlapped":
                    llb.llb_step_host(ctx, h_in, h_out, 1)
                else:
                    llb.llb_init_moments(ctx, h_in)
                    llb.llb_step(ctx, 1)
                    llb.llb_get_moments(ctx, h_out)
            for _ in range(2):
                one()
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(k):
                one()
            torch.cuda.synchronize()
            times[name] = reduce_max(time.perf_counter() - t0, world)
    finally:
        llb.llb_destroy(ctx)
    nbytes = 10 * nodes * 4
    dt = times["overlapped"]
    return {"value": world * nodes * k / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": k,
            "path": "llb_step_host(host in, 1 step, host out), FP32 canonical, pinned, copies overlapped with "
                    "per-slab steps",
            "sequential_mlups": world * nodes * k / times["sequential"] / 1e6,
            "sequential_path": "llb_init_moments(host) + llb_step(1) + llb_get_moments(host)"}


# ----------------------------------------------------------------------------- CPU (oracle) legs


def oracle_sample(nz_sample):
    """The bench field restricted to a 256 x 256 x nz_sample periodic slab."""
    from paper_2301_01622_gb300 import inputs
    rho, u = inputs.taylor_green_3d(NX, NY, NZ, u0=U0, noise=NOISE, seed=SEED)
    return rho[:nz_sample].copy(), u[:, :nz_sample].copy()


def _slab_step(args):
    """One oracle step of a z-slab with one halo plane on each side (runs in a
    worker process); returns the interior planes and the step's wall time."""
    from oracle import D3Q19, lb
    slab, tau = args
    t0 = time.perf_counter()
    new = lb.step_moment_only(slab, D3Q19, tau)
    return new[:, 1:-1], time.perf_counter() - t0


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(gpu_check: bool):
    """Time the FP64 oracle on one full-size step of the bench field, on one
    host core and on all host cores (the field split into z-slabs with one
    halo plane each, one oracle step per slab in parallel worker processes;
    time = the slowest worker's step, data distribution excluded), and use its
    result to check the GPU's first step per shifted field at FP32 and
    16-bit storage."""
    import multiprocessing as mp

    from oracle import D3Q19, lb
    from paper_2301_01622_gb300 import inputs, llb

    rho, u = inputs.taylor_green_3d(NX, NY, NZ, u0=U0, noise=NOISE, seed=SEED)
    m0 = lb.equilibrium_moments(rho, u)
    t0 = time.perf_counter()
    ref = lb.step_moment_only(m0, D3Q19, TAU)
    dt = time.perf_counter() - t0
    nodes = NX * NY * NZ
    cores = max(1, min(os.cpu_count() or 1, 32))
    par = None
    if cores > 1:
        bounds = [(k * NZ) // cores for k in range(cores + 1)]
        slabs = [np.take(m0, range(bounds[k] - 1, bounds[k + 1] + 1), axis=1, mode="wrap") for k in range(cores)]
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_slab_step, [(sl, TAU) for sl in slabs])
        got_par = np.concatenate([r[0] for r in res], axis=1)
        par_dt = max(r[1] for r in res)
        par = {"value": nodes / par_dt / 1e6, "unit": "MLUPS", "cores": cores, "seconds": par_dt,
               "matches_single_core": bool(np.array_equal(got_par, ref))}
    single = {"value": nodes / dt / 1e6, "unit": "MLUPS", "cores": 1, "seconds": dt}
    if par is not None:
        out = {"value": par["value"], "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"one time step of the full 256^3 D3Q19 workload, numpy FP64, split into {cores} z-slabs "
                         "(one halo plane each) stepped in parallel worker processes",
               "seconds": par["seconds"], "matches_single_core": par["matches_single_core"],
               "single_core": single, "cpu_model": _cpu_model()}
    else:
        out = {"value": single["value"], "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": "one time step of the full 256^3 D3Q19 workload, numpy FP64, single thread",
               "seconds": dt, "cpu_model": _cpu_model()}
    parity = None
    if gpu_check:
        import torch
        parity = {"vs": "FP64 oracle, one step of the full 256^3 field, per shifted field "
                        "(max |gpu - oracle| / max |oracle| of rho-1, each j, each A = P - cs^2 rho I)"}
        for name, storage, tol in (("fp32", llb.LLB_F32, 1e-5), ("fp16", llb.LLB_F16S, None),
                                   ("bf16", llb.LLB_BF16S, None)):
            ctx = make_ctx(llb, LATTICE, llb.LLB_SCHEME_MOMENT, torch.cuda.current_stream().cuda_stream,
                           storage=storage)
            try:
                llb.llb_init_equilibrium(ctx, rho, u)
                llb.llb_step(ctx, 1)
                got = llb.llb_get_moments(ctx, np.empty((10, NZ, NY, NX)))
            finally:
                llb.llb_destroy(ctx)
            errs = _field_errors(got, ref)
            parity[name] = {"max_rel_err": errs, "max": max(errs.values())}
            if tol is not None:
                parity[name]["tol"] = tol
                parity[name]["pass"] = all(v <= tol for v in errs.values())
    return out, parity


def _field_errors(got, ref):
    """Per shifted field: max |got - ref| / max |ref| (rho - 1, j, A = P - cs^2 rho I)."""
    cs2 = 1.0 / 3.0
    names = ["drho", "jx", "jy", "jz", "Axx", "Ayy", "Azz", "Axy", "Axz", "Ayz"]

    def shifted(m):
        sh = np.empty_like(m)
        sh[0] = m[0] - 1.0
        sh[1:4] = m[1:4]
        sh[4:10] = m[4:10]
        for a in range(3):
            sh[4 + a] = m[4 + a] - cs2 * m[0]
        return sh

    g, r = shifted(got), shifted(ref)
    return {nm: float(np.abs(g[k] - r[k]).max() / np.abs(r[k]).max()) for k, nm in enumerate(names)}


def reference_arm(args, rank):
    """The oracle as it stands, on the host cores, on this arm's workload: each
    step is one time step of a 256 x 256 x nz periodic slab of the bench field,
    nz chosen so the whole run ends within a few minutes."""
    from oracle import D3Q19, lb

    if rank != 0:
        return None
    budget_s = getattr(args, "ref_budget", 150.0)
    per_plane = 0.03
    nzs = int(max(1, min(NZ, budget_s / max(1, args.steps + args.warmup) / per_plane)))
    rho, u = oracle_sample(nzs)
    m = lb.equilibrium_moments(rho, u)
    for _ in range(args.warmup):
        m = lb.step_moment_only(m, D3Q19, TAU)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m = lb.step_moment_only(m, D3Q19, TAU)
    dt = time.perf_counter() - t0
    nodes = NX * NY * nzs
    val = nodes * args.steps / dt / 1e6
    sample = f"each step: one time step of a 256x256x{nzs} periodic slab of the workload (numpy FP64 oracle, 1 thread)"
    return {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_nodes_per_step": nodes},
        "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------------------------- main


def main():
    args = parse()
    _KERNEL[0] = args.kernel
    _KERNEL[1] = args.variant
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        line = reference_arm(args, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    main_r, extra, e2e, diag, peak, peak_src = gpu_arm(args, rank, world, local)
    cpu, parity = (None, None)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, parity = cpu_baseline(gpu_check=True)

    if rank != 0:
        return
    nodes = NX * NY * NZ
    traffic = ncu_traffic("moment_tiled_d3q19_f32")
    roof = {"bound": "hbm", "achieved": main_r["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": main_r["achieved_gbs"] / peak, "traffic": traffic,
            "frac_of_nominal_7900": main_r["achieved_gbs"] / 7900.0,
            "peak_source": peak_src + ", burst copy figure (the step kernel is timed alone)",
            "algorithmic_bytes_per_launch": main_r["bytes_per_node"] * nodes,
            "kernel": {1: "k_moment_direct", 2: "k_moment_tiled", 3: "k_moment_tma"}.get(main_r["kernel"], "?") + "<D3Q19,float>", "avg_launch_ms": main_r["launch_ms"]}
    line = {
        "metric": METRIC, "value": main_r["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes_per_gpu": nodes, "lattice": "D3Q19", "tau": TAU,
                   "parallelism": "replicas" if world > 1 else "single", "l2": L2_NOTE},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": main_r["clocks"],
        "parity": parity,
        "population_d3q19": _short(extra.get("population_d3q19")),
        "moment_d3q27": _short(extra.get("moment_d3q27")),
        "population_d3q27": _short(extra.get("population_d3q27")),
        "moment_d3q19_fp16": _short(extra.get("moment_d3q19_fp16")),
        "moment_d3q19_bf16": _short(extra.get("moment_d3q19_bf16")),
        "moment_d3q27_fp16": _short(extra.get("moment_d3q27_fp16")),
        "moment_d3q27_bf16": _short(extra.get("moment_d3q27_bf16")),
        "two_component_d3q27": extra.get("two_component_d3q27"),
        "batched_ensemble": extra.get("batched_ensemble"),
        "adjoint_two_component_d3q27": extra.get("adjoint_two_component_d3q27"),
        "speedup_vs_population_d3q19": (main_r["mlups"] / extra["population_d3q19"]["mlups"])
        if "population_d3q19" in extra else None,
        "diagnostics": diag,
        "paper_context": {"v100_mlups_without_populations": 622, "v100_mlups_with_populations": 277,
                          "workload": "128^3 two-component droplet collision, Tesla V100 (not this workload)"},
    }
    print(json.dumps(line), flush=True)


def _short(r):
    if not r:
        return None
    return {"mlups": r["mlups"], "frac": r["frac"], "achieved_gbs": r["achieved_gbs"],
            "bytes_per_node": r["bytes_per_node"], "ms_per_step": r["ms_per_step"]}


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark: two-flavour Wilson HMC trajectories per second on a 32^3x64
lattice (beta 5.8, kappa 0.1570, synthetic start exp(i 0.15 H) from Philox
seed 3, Omelyan 2MN with 16 steps, tau 1, CG true |r|/|b| <= 1e-10), mixed
precision (FP16+norm spinors and 12-real FP16 links in the solver, FP32
arithmetic, FP64 master fields, residuals, reductions and dH), with the plain
FP64 GPU path timed beside it.

One step = one full trajectory on the device.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (a bounded sample of the same
workload, scaled to trajectories/s).  For N > 1 (torchrun) every rank runs its
own independent chain (chain id = rank): the method has no exchange between
chains, so there is no collective on the data path.
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
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

WORKLOAD = {
    "workload": "nf2_wilson_hmc_32x32x32x64",
    "dims": [32, 32, 32, 64],
    "beta": 5.8,
    "kappa": 0.1570,
    "start": "exp(i*0.15*H), H Gell-Mann Gaussians from Philox seed 3",
    "integrator": "omelyan_2mn",
    "nsteps": 16,
    "tau": 1.0,
    "cg_tol": 1e-10,
}
SEED, EPS = 3, 0.15
ORACLE_SAMPLE_DIMS = (12, 12, 12, 24)


# ---------------------------------------------------------------- distributed

def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, use_cuda):
    if world <= 1:
        return None
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("nccl" if use_cuda else "gloo")
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        reasons = sorted({name for r in rows for name, v in zip(self.REASONS, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------- peaks, profiles

# HBM3e bandwidth of a GB300 as specified (context beside the measured copy peak)
NOMINAL_HBM_GBS = 7900.0
# the dominant class's launches carry events one in TIMER_EVERY inside the timed region
TIMER_EVERY = 13


def measured_peaks() -> dict:
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d.get("hbm_gbs"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    """hash of the hopping-term sources: a stored ncu traffic figure is only
    valid for the kernel it was taken on"""
    h = hashlib.sha256()
    base = os.path.join(HERE, "paper_1212_0785_gb300", "csrc")
    for name in ("dslash.cu", "dslash_site.cuh", "dslash_packed.cuh", "spin.cuh", "lqcd_internal.cuh", "dslash.cuh"):
        with open(os.path.join(base, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel: str, key: str = "dram_bytes_per_launch"):
    """DRAM bytes per launch from the committed ncu summary, or None if absent or stale"""
    p = os.path.join(HERE, "profiles", f"traffic_{kernel}_32x32x32x64.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    with open(p) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != kernel_source_hash():
        return None
    try:
        return float(kv[key])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- oracle baseline

def host_cpu() -> dict:
    """core count and CPU model of the host the oracle runs on"""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or "unknown",
            "arch": platform.machine()}


def oracle_sample(dims=ORACLE_SAMPLE_DIMS, wl=WORKLOAD, openmp=True):
    """Time the FP64 CPU oracle (its OpenMP or its serial build) on the
    operations of one MD force evaluation of the workload at a reduced volume
    with the same recipe: one CG solve to the workload's tolerance from a zero
    guess (time per iteration), the gauge force, the fermion force and a link
    update."""
    from oracle import oracle as orc

    prev = orc.use_openmp(openmp)
    try:
        beta, kappa, n = wl["beta"], wl["kappa"], wl["nsteps"]
        U = orc.gauge_start(dims, SEED, EPS)
        eta = orc.eta_refresh(dims, SEED, 0)
        phi = orc.mhat(dims, U, kappa, eta, dagger=True)
        P = orc.momentum_refresh(dims, SEED, 0)
        t0 = time.perf_counter()
        X, conv, iters, _ = orc.cg(dims, U, kappa, phi, tol=wl["cg_tol"])
        t1 = time.perf_counter()
        orc.gauge_force(dims, U, beta)
        t2 = time.perf_counter()
        orc.fermion_force(dims, U, kappa, X)
        t3 = time.perf_counter()
        orc.link_update(dims, U, P, 0.5 * wl["tau"] / n)
        t4 = time.perf_counter()
        threads = orc.num_threads()
    finally:
        orc.use_openmp(prev == "openmp")
    return {"dims": list(dims), "threads": threads, "cg_iters": iters, "sample_cpu_s": t4 - t0,
            "parts_s": {"cg_iteration": (t1 - t0) / max(iters, 1), "gauge_force": t2 - t1,
                        "fermion_force": t3 - t2, "link_update": t4 - t3},
            "scale": float(np.prod(wl["dims"])) / float(np.prod(dims))}


def derived_traj_s(sample, cg_iters_per_traj, wl=WORKLOAD) -> float:
    """one trajectory of the workload from the sample's per-part times:
    (2n+1) force evaluations (merged Omelyan kicks), 2n link updates and the
    given number of CG iterations, scaled by the volume ratio"""
    n, p = wl["nsteps"], sample["parts_s"]
    t = (cg_iters_per_traj * p["cg_iteration"] + (2 * n + 1) * (p["gauge_force"] + p["fermion_force"])
         + 2 * n * p["link_update"])
    return t * sample["scale"]


def oracle_trajectory_4(gpu_traj=None):
    """a full oracle trajectory at 4^4 with the workload's recipe (beta,
    kappa, Omelyan 16 steps, tau 1, start seed 3 eps 0.15), timed on the serial
    and the OpenMP build; with gpu_traj (the library's trajectory of the same
    4^4 chain in the benchmark's mixed configuration: dH, H0, plaquette,
    links) the per-result differences against the oracle"""
    from oracle import oracle as orc

    dims, wl = (4, 4, 4, 4), WORKLOAD
    U = orc.gauge_start(dims, SEED, EPS)
    out = {}
    for variant in (False, True):
        prev = orc.use_openmp(variant)
        t0 = time.perf_counter()
        Uo, o = orc.hmc_trajectory(dims, U, wl["beta"], wl["kappa"], wl["tau"], wl["nsteps"],
                                   integrator=orc.OMELYAN, seed=SEED, traj=0, cg_tol=wl["cg_tol"])
        out["openmp_s" if variant else "serial_s"] = time.perf_counter() - t0
        out["openmp_threads" if variant else "serial_threads"] = orc.num_threads()
        orc.use_openmp(prev == "openmp")
    out["oracle"] = {"dH": o["dH"], "accepted": int(o["accepted"]), "plaq": o["plaq"], "cg_iters": o["cg_iters"]}
    if gpu_traj is not None:
        g, Ug = gpu_traj
        out["mixed_gpu_minus_oracle"] = {"dH": g["dH"] - o["dH"], "H0_rel": (g["H0"] - o["H0"]) / o["H0"],
                                         "plaq": g["plaq"] - o["plaq"], "links_max": float(np.max(np.abs(Ug - Uo))),
                                         "accept_same": g["accepted"] == int(o["accepted"]),
                                         "tolerances": {"dH": 9.1e-5, "H0_rel": 1e-12, "plaq": 1e-8,
                                                        "links_max": 1e-5}}
    return out


def cpu_baseline_block(omp, serial, cg_iters_per_traj, iters_source, traj4=None) -> dict:
    d = "x".join(str(v) for v in omp["dims"])
    t_omp = derived_traj_s(omp, cg_iters_per_traj)
    t_ser = derived_traj_s(serial, cg_iters_per_traj)
    blk = {"value": 1.0 / t_omp, "unit": "trajectories/s", "cores": omp["threads"], "kind": "oracle",
           "sample": (f"FP64 oracle (OpenMP build, {omp['threads']} threads): one CG solve to 1e-10 "
                      f"({omp['cg_iters']} iterations from a zero guess), gauge force, fermion force and link "
                      f"update at {d} with the 32^3x64 recipe ({omp['sample_cpu_s']:.1f} s), derived to one "
                      f"trajectory of 33 force evaluations, 32 link updates and {cg_iters_per_traj:.0f} CG "
                      f"iterations ({iters_source}), scaled by volume x{omp['scale']:.1f}"),
           "derived": True, "host": host_cpu(),
           "single_thread": {"value": 1.0 / t_ser, "cores": 1, "sample_cpu_s": serial["sample_cpu_s"],
                             "parts_s": serial["parts_s"]},
           "parts_s": omp["parts_s"]}
    if traj4 is not None:
        blk["full_trajectory_4^4"] = traj4
    return blk


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    samples = []
    for k in range(args.warmup + args.steps):
        s = oracle_sample(openmp=True)
        if k >= args.warmup:
            samples.append(s)
    # the oracle's own iteration count: its zero-guess solve at the sample
    # volume, for each of the trajectory's 34 solves
    iters = 34 * samples[-1]["cg_iters"]
    t = float(np.mean([derived_traj_s(s, iters) for s in samples]))
    value = 1.0 / t
    serial = oracle_sample(openmp=False)
    cb = cpu_baseline_block(samples[-1], serial, iters, "the oracle's own: 34 zero-guess solves")
    cb["value"] = value
    line = {"metric": "trajectories/s", "value": value, "unit": "trajectories/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(args), "arithmetic": arithmetic_block(args, "f64", "f64", 0),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_block(args):
    """The workload both arms run: the same dict for ours and the oracle's."""
    c = dict(WORKLOAD)
    c["dims"] = list(args.dims)
    c["nsteps"] = args.nsteps
    c["parallelism"] = f"replicas{args.gpus}" if args.gpus > 1 else "single_gpu"
    c["l2"] = "inputs larger than L2 (FP64 links 1.21 GB, spinors 0.2 GB)"
    return c


def arithmetic_block(args, sloppy, force_prec, chrono):
    """How an arm computes the workload: solver storage, force precision, initial guess."""
    a = {"solver": ("fp64 CG" if sloppy == "f64" else
                    f"reliable-update mixed CG: {sloppy} spinors + 12-real {sloppy} links, fp32 math, "
                    f"float-float residual/solution, fp64 dot sums, delta {args.delta}"),
         "forces": f"{force_prec} arithmetic"}
    k = int(chrono)
    a["initial_guess"] = {0: "zero", 1: "previous solution (chronological)"}.get(
        k, f"extrapolated through the last {k} solutions (chronological)"
           + (", refined by minimal residual extrapolation" if getattr(args, "mre", 0) and sloppy != "f64" else ""))
    return a


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch

    from paper_1212_0785_gb300 import lqcd

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    dims = tuple(args.dims)
    V = int(np.prod(dims))
    sloppy = lqcd.PREC_NAMES[args.sloppy]
    wl = WORKLOAD
    cg = lqcd.cg_params(tol=wl["cg_tol"], maxiter=20000, sloppy=sloppy, delta=args.delta)
    force_prec = lqcd.PREC_NAMES[args.force_prec]
    params = lqcd.hmc_params(wl["beta"], wl["kappa"], wl["tau"], args.nsteps, lqcd.OMELYAN, n_flavors=2, cg=cg,
                             force_prec=force_prec, chrono=int(args.chrono), chrono_mre=args.mre)

    tuned = None
    if args.autotune:
        # threads per block of the tunable kernels on this lattice (paper Sec. 4),
        # before the warm-up; the timings go to --tune-file if given
        tuned = lqcd.autotune(dims, args.tune_file)
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, SEED, EPS, chain=rank)
    state = lqcd.HmcState(U, seed=SEED, chain=rank)
    warm = [state.trajectory(params) for _ in range(args.warmup)]
    warm_rejected = all(i["accepted"] == 0 for i in warm)
    torch.cuda.synchronize()
    barrier(dist, local)

    gpu_index = int((os.environ.get("CUDA_VISIBLE_DEVICES") or str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    clocks = ClockSampler(gpu_index)
    kclass = f"dslash_{args.sloppy}"
    # only the dominant class is timed inside the timed region (events on its
    # launches); the per-class breakdown comes from one more trajectory below
    plain_class = kclass + "_plain" if kclass == "dslash_f16n" else None
    # events on one launch of the class in every TIMER_EVERY (coprime to the
    # four hop variants of a CG iteration, so all are sampled alike): events
    # on every launch would slow the timed trajectories themselves
    lqcd.kernel_timers(True, only=kclass, every=TIMER_EVERY)
    launches0 = lqcd.launch_count()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    infos = [state.trajectory(params) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist, local)
    clk = clocks.stop()
    launches = lqcd.launch_count() - launches0
    t_local = ev0.elapsed_time(ev1) / 1e3
    t_max = max_over_ranks(dist, t_local, dev)
    total_traj = sum_over_ranks(dist, float(args.steps), dev)
    value = total_traj / t_max

    ms, n, nbytes = lqcd.kernel_timer_read(kclass)
    # per-class breakdown: one more trajectory with every launch of every class timed
    lqcd.kernel_timers(True, every=1)
    state.trajectory(params)
    torch.cuda.synchronize()
    timers = {k: lqcd.kernel_timer_read(k) for k in lqcd.KERNEL_CLASSES}
    lqcd.kernel_timers(False)
    # the plain variant's own events (outside the timed region, whose only
    # events are the class's: nested events would add to every plain launch)
    pms, pn, pbytes = timers[plain_class] if plain_class else (0.0, 0, 0.0)
    Vh = V // 2
    peaks = measured_peaks()
    # achieved = algorithmic bytes of the timed launches (each launch's own
    # fields: plain, axpy and CG-update variants) / their summed event time
    achieved = nbytes / (ms * 1e-3) / 1e9 if n else None
    full = tuple(dims) == (32, 32, 32, 64)
    traffic = stored_traffic(kclass) if full else None
    roofline = {"kernel": kclass, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"] if achieved else None, "traffic": traffic,
                "peak_source": peaks["source"],
                "nominal_peak": NOMINAL_HBM_GBS,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS if achieved else None,
                # DRAM bytes actually moved per second (ncu traffic / live launch time)
                "dram_achieved": traffic / (ms / n * 1e-3) / 1e9 if (traffic and n) else None,
                "algorithmic_bytes_per_launch": nbytes / n if n else None,
                "avg_launch_us": ms / n * 1e3 if n else None, "launches": n, "timed_one_in": TIMER_EVERY}
    if pn:
        # the plain hop alone (no fused epilogue), from its own event timers
        # in the breakdown trajectory
        p_ach = pbytes / (pms * 1e-3) / 1e9
        p_traffic = stored_traffic(kclass, "dram_bytes_per_launch_plain") if full else None
        roofline["plain"] = {"achieved": p_ach, "frac": p_ach / peaks["hbm_gbs"],
                             "frac_of_nominal": p_ach / NOMINAL_HBM_GBS,
                             "algorithmic_bytes_per_launch": pbytes / pn, "avg_launch_us": pms / pn * 1e3,
                             "launches": pn, "traffic": p_traffic,
                             "dram_achieved": p_traffic / (pms / pn * 1e-3) / 1e9 if p_traffic else None}
    step_ms = t_max / args.steps * 1e3
    kernel_share = {k: {"ms_per_traj": v[0], "launches_per_traj": v[1],
                        "GB_per_s": (v[2] / (v[0] * 1e-3) / 1e9) if v[2] else None}
                    for k, v in timers.items() if v[1]}

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        host_in = torch.empty(V * 4 * 9 * 2, dtype=torch.float64, pin_memory=True).numpy()
        host_out = torch.empty(V * 4 * 9 * 2, dtype=torch.float64, pin_memory=True).numpy()
        hin = host_in.view(np.complex128).reshape(V, 4, 3, 3)
        hout = host_out.view(np.complex128).reshape(V, 4, 3, 3)
        U.download(out=hin)
        # one untimed round trip first: the transfer staging buffers are
        # allocated once, like every other buffer before the timed region
        U.upload(hin)
        state.trajectory(params)
        U.download(out=hout)
        hin, hout = hout, hin
        torch.cuda.synchronize()
        barrier(dist, local)
        eclk = ClockSampler(gpu_index)
        eclk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            U.upload(hin)
            info = state.trajectory(params)
            U.download(out=hout)
            hin, hout = hout, hin
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_clk = eclk.stop()
        te = max_over_ranks(dist, e0.elapsed_time(e1) / 1e3, dev)
        nb = V * 4 * 18 * 8
        e2e = {"value": sum_over_ranks(dist, float(args.e2e_steps), dev) / te, "unit": "trajectories/s",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 96, "steps": args.e2e_steps,
               "clocks": e2e_clk}

    # FP64 GPU path beside it: same start, same chain, same trajectory counters
    # as the first timed mixed trajectories, so dH differences measure the
    # error of the mixed path
    fp64 = None
    if args.fp64_steps > 0:
        U64 = lqcd.gauge_field(dims)
        p64 = lqcd.hmc_params(wl["beta"], wl["kappa"], wl["tau"], args.nsteps, lqcd.OMELYAN, n_flavors=2,
                              cg=lqcd.cg_params(tol=wl["cg_tol"], maxiter=20000, sloppy=lqcd.F64),
                              chrono=int(args.chrono))
        lqcd.gauge_start(U64, SEED, EPS, chain=rank)
        st64 = lqcd.HmcState(U64, seed=SEED, chain=rank, traj0=args.warmup)
        for _ in range(args.fp64_warmup):  # allocations and first launches, then the same start again
            st64.trajectory(p64)
        lqcd.gauge_start(U64, SEED, EPS, chain=rank)
        st64.traj = args.warmup
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        i64 = [st64.trajectory(p64) for _ in range(args.fp64_steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        # the mixed chain's timed trajectories against the FP64 chain's, from
        # the same links and trajectory counters (hence the same momenta and
        # pseudofermions) as long as neither chain accepted a trajectory
        same_start = (all(i["accepted"] == 0 for i in infos[:args.fp64_steps])
                      and all(i["accepted"] == 0 for i in i64[:-1]) and
                      (args.warmup == 0 or warm_rejected))
        fp64 = {"trajectories_per_s": args.fp64_steps / t64, "s_per_traj": t64 / args.fp64_steps,
                "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                "cg_iters_per_traj": float(np.mean([i["cg_iters"] for i in i64])),
                "dH": [i["dH"] for i in i64], "mixed_speedup": value / world / (args.fp64_steps / t64),
                "mixed_minus_fp64_dH": ([m["dH"] - f["dH"] for m, f in zip(infos, i64)]
                                        if same_start else None),
                "mixed_minus_fp64_plaq": ([m["plaq"] - f["plaq"] for m, f in zip(infos, i64)]
                                          if same_start else None)}
        st64.close()
        del U64

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        traj4 = None
        if args.nsteps == WORKLOAD["nsteps"]:
            # the benchmark's mixed configuration on a 4^4 lattice with the same
            # recipe, for the per-result differences against the oracle
            U4 = lqcd.gauge_field((4, 4, 4, 4))
            lqcd.gauge_start(U4, SEED, EPS)
            st4 = lqcd.HmcState(U4, seed=SEED)
            g4 = st4.trajectory(params)
            traj4 = oracle_trajectory_4((g4, U4.download()))
            st4.close()
        if fp64:
            iters, src = fp64["cg_iters_per_traj"], "measured on the FP64 GPU path of this run"
        else:
            iters, src = float(np.mean([i["cg_iters"] for i in infos])), "measured on the mixed GPU path of this run"
        cpu = cpu_baseline_block(oracle_sample(openmp=True), oracle_sample(openmp=False), iters, src, traj4)

    if rank == 0:
        acc = [i["accepted"] for i in infos]
        line = {
            "metric": "trajectories/s", "value": value, "unit": "trajectories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32",
            "dtype_detail": (f"f32 math ({args.sloppy} storage in the solver, {args.force_prec} forces); f64 master "
                             f"links/momenta, residuals, dots, link update, dH"),
            "data": "synthetic",
            "config": config_block(args),
            "arithmetic": arithmetic_block(args, args.sloppy, args.force_prec, args.chrono),
            "tuning": {"threads_per_block": tuned,
                       "dslash_form": {0: "gathered", 1: "prefetched_links", 2: "prefetched_links_packed_f32x2"}.get(
                           lqcd.dslash_form(), "?")},
            "gpu_launches": launches,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "fp64_gpu_path": fp64,
            "physics": {"acceptance": float(np.mean(acc)), "dH": [i["dH"] for i in infos],
                        "plaquette": [i["plaq"] for i in infos],
                        "cg_iters_per_traj": float(np.mean([i["cg_iters"] for i in infos])),
                        "solves_per_traj": float(np.mean([i["n_solves"] for i in infos])),
                        "accurate_residuals_per_traj": float(np.mean([i["cg_accurate_residuals"] for i in infos])),
                        "failed_checks_per_traj": float(np.mean([i["cg_failed_checks"] for i in infos])),
                        "guesses_refined_per_traj": float(np.mean([i["cg_guesses_refined"] for i in infos])),
                        "cg_true_rel_res_max": max(i["cg_true_rel_res_max"] for i in infos)},
            "kernel_time_per_traj": kernel_share,
        }
        print(json.dumps(line))
    state.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- plain FP64 path, 16^3x32

FP64_16 = {"workload": "nf2_wilson_hmc_fp64_16x16x16x32", "dims": [16, 16, 16, 32], "beta": 5.6, "kappa": 0.1575,
           "start": "exp(i*0.2*H), H Gell-Mann Gaussians from Philox seed 2", "integrator": "leapfrog",
           "nsteps": 20, "tau": 1.0, "cg_tol": 1e-10, "seed": 2, "eps": 0.2}
FP64_FLOP_PER_SITE = 1320  # one half hopping term per output site
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x FP64 FMA/clock/SM x 2 flop x max SM clock


def run_fp64_16(args):
    """Config 2: the plain FP64 GPU path (FP64 hopping term, FP64 CG on
    Mhat^dag Mhat to 1e-10, FP64 forces and link update) on 16^3x32, beta 5.6,
    kappa 0.1575, start exp(i 0.2 H) from Philox seed 2, leapfrog with 20 steps,
    tau 1, 10 trajectories with plaquette and acceptance logged; beside it one
    full trajectory of the FP64 oracle on all host cores."""
    import torch

    from paper_1212_0785_gb300 import lqcd

    torch.cuda.set_device(0)
    wl = FP64_16
    dims = tuple(wl["dims"])
    steps = args.steps if args.steps is not None else 10
    stream = torch.cuda.current_stream()
    cg = lqcd.cg_params(tol=wl["cg_tol"], maxiter=20000, sloppy=lqcd.F64)
    params = lqcd.hmc_params(wl["beta"], wl["kappa"], wl["tau"], wl["nsteps"], lqcd.LEAPFROG, cg=cg,
                             chrono=int(args.chrono))
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, wl["seed"], wl["eps"])
    st = lqcd.HmcState(U, seed=wl["seed"])
    warm = [st.trajectory(params) for _ in range(args.warmup)]
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    lqcd.kernel_timers(True, only="dslash_f64")
    launches0 = lqcd.launch_count()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [st.trajectory(params) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = lqcd.launch_count() - launches0
    t = e0.elapsed_time(e1) / 1e3
    ms, n, nbytes = lqcd.kernel_timer_read("dslash_f64")
    lqcd.kernel_timers(False)
    Vh = int(np.prod(dims)) // 2
    flops = FP64_FLOP_PER_SITE * Vh * n
    achieved = flops / (ms * 1e-3) / 1e12 if n else None
    roofline = {"kernel": "dslash_f64", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flop x 2.07 GHz",
                "hbm_GB_per_s": nbytes / (ms * 1e-3) / 1e9 if n else None,
                "avg_launch_us": ms / n * 1e3 if n else None, "launches": n, "timed_one_in": TIMER_EVERY}
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as orc

        prev = orc.use_openmp(True)
        Uo = orc.gauge_start(dims, wl["seed"], wl["eps"])
        t0 = time.perf_counter()
        _, o = orc.hmc_trajectory(dims, Uo, wl["beta"], wl["kappa"], wl["tau"], wl["nsteps"],
                                  integrator=orc.LEAPFROG, seed=wl["seed"], traj=0, cg_tol=wl["cg_tol"])
        t_or = time.perf_counter() - t0
        threads = orc.num_threads()
        orc.use_openmp(prev == "openmp")
        cpu = {"value": 1.0 / t_or, "unit": "trajectories/s", "cores": threads, "kind": "oracle",
               "sample": f"one full FP64 oracle trajectory at 16^3x32 (OpenMP build, {threads} threads, "
                         f"{t_or:.1f} s, {o['cg_iters']:.0f} CG iterations from zero guesses)",
               "derived": False, "host": host_cpu(),
               "oracle_traj0": {"dH": o["dH"], "accepted": int(o["accepted"]), "plaq": o["plaq"]},
               "gpu_traj0_minus_oracle": ({"dH": warm[0]["dH"] - o["dH"], "plaq": warm[0]["plaq"] - o["plaq"]}
                                          if warm else None)}
    line = {"metric": "trajectories/s", "value": steps / t, "unit": "trajectories/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": t / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(wl, solver="fp64 CG", forces="f64 arithmetic", parallelism="single_gpu",
                           initial_guess={0: "zero", 1: "previous solution"}.get(
                               args.chrono, f"extrapolated through the last {args.chrono} solutions"),
                           l2="inputs larger than L2 (FP64 links 151 MB)"),
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "physics": {"acceptance": float(np.mean([i["accepted"] for i in infos])),
                        "plaquette": [i["plaq"] for i in infos], "dH": [i["dH"] for i in infos],
                        "accepted": [i["accepted"] for i in infos],
                        "cg_iters_per_traj": float(np.mean([i["cg_iters"] for i in infos])),
                        "cg_true_rel_res_max": max(i["cg_true_rel_res_max"] for i in infos)}}
    print(json.dumps(line))
    st.close()
    return 0


# ---------------------------------------------------------------- batched chains

CHAINS64 = [(8, 8, 8, 8)] * 32 + [(12, 12, 12, 12)] * 24 + [(16, 16, 16, 32)] * 8


def run_chains(args):
    """64 independent chains of uneven volume (32 at 8^4, 24 at 12^4, 8 at
    16^3x32), beta in [5.6, 5.9] and kappa in [0.150, 0.157] spread over the
    chains, Philox seed 100 + i, start eps 0.3, leapfrog 10 steps, tau 1,
    FP16+norm mixed solver, FP32 MD; all chains advanced together (their
    solves in shared launches) against the same chains one after another."""
    import torch

    from paper_1212_0785_gb300 import lqcd

    torch.cuda.set_device(0)
    n = len(CHAINS64)
    betas = np.linspace(5.6, 5.9, n)
    kappas = np.linspace(0.150, 0.157, n)
    cg = lqcd.cg_params(tol=1e-10, maxiter=20000, sloppy=lqcd.F16N, delta=args.delta)
    params = [lqcd.hmc_params(float(betas[i]), float(kappas[i]), 1.0, 10, lqcd.LEAPFROG, cg=cg,
                              force_prec=lqcd.F32, chrono=int(args.chrono)) for i in range(n)]

    def make():
        fields, states = [], []
        for i, dims in enumerate(CHAINS64):
            U = lqcd.gauge_field(dims)
            lqcd.gauge_start(U, 100 + i, 0.3)
            fields.append(U)
            states.append(lqcd.HmcState(U, seed=100 + i, chain=i))
        return fields, states

    stream = torch.cuda.current_stream()
    fields, states = make()
    batch = lqcd.Batch(states)
    for _ in range(args.warmup):
        batch.trajectory(params)
    torch.cuda.synchronize()
    launches0 = lqcd.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [batch.trajectory(params) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    launches = lqcd.launch_count() - launches0
    # per-class kernel time of one more batched trajectory (every class timed)
    lqcd.kernel_timers(True)
    batch.trajectory(params)
    torch.cuda.synchronize()
    kernel_time = {k: {"ms": v[0], "launches": v[1]} for k in lqcd.KERNEL_CLASSES
                   for v in [lqcd.kernel_timer_read(k)] if v[1]}
    lqcd.kernel_timers(False)
    batch.close()
    # the same chains, one trajectory after another, each alone
    fields2, states2 = make()
    for i in range(n):
        states2[i].trajectory(params[i])
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for i in range(n):
            states2[i].trajectory(params[i])
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    sites = sum(int(np.prod(d)) for d in CHAINS64)
    line = {"metric": "chain-trajectories/s", "value": n * args.steps / t_batch, "unit": "chain-trajectories/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "dtype_detail": "f32 math (f16n solver storage, f32 forces); f64 master fields, residuals, dH",
            "data": "synthetic",
            "config": {"workload": "chains64_8^4x32_12^4x24_16^3x32x8", "chains": n, "sites_total": sites,
                       "beta": [5.6, 5.9], "kappa": [0.150, 0.157], "integrator": "leapfrog", "nsteps": 10,
                       "tau": 1.0, "start_eps": 0.3, "initial_guess": {0: "zero", 1: "previous solution"}.get(
                           args.chrono, f"extrapolated through the last {args.chrono} solutions")},
            "gpu_launches": launches,
            "kernel_time_per_batch_traj": kernel_time,
            "sequential": {"value": n * args.steps / t_seq, "ms_per_step": t_seq / args.steps * 1e3},
            "batched_speedup": t_seq / t_batch,
            "physics": {"acceptance": float(np.mean([f["accepted"] for it in infos for f in it])),
                        "cg_iters_per_chain_traj": float(np.mean([f["cg_iters"] for it in infos for f in it])),
                        "cg_true_rel_res_max": max(f["cg_true_rel_res_max"] for it in infos for f in it)}}
    print(json.dumps(line))
    for st in states + states2:
        st.close()
    return 0

SERVICE_LATS = [(8, 8, 8, 8), (16, 16, 16, 32), (24, 24, 24, 48), (32, 32, 32, 64)]


def _serve(lqcd, fields, arrivals, reqs, params):
    """submit reqs at their arrival times (s after the start) to a fresh
    service; returns (results, makespan s, launches)"""
    svc = lqcd.Service(params)
    ids = [svc.add_gauge(U) for U in fields]
    # warm-up: one single-RHS request per gauge makes its link copies and work space
    for gid in ids:
        t = svc.submit(gid, 0.15, (0, 0, 0, 0), 1)
        svc.wait(t)
        svc.release(t)
    launches0 = lqcd.launch_count()
    pending, results = {}, {}
    t0 = time.perf_counter()
    i = 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and arrivals[i] <= now:
            g, kappa, site = reqs[i]
            pending[svc.submit(ids[g], kappa, site, 12)] = i
            i += 1
        for t in list(pending):
            r = svc.poll(t)
            if r is not None:
                results[pending.pop(t)] = r
                svc.release(t)
        time.sleep(2e-4)
    makespan = time.perf_counter() - t0
    launches = lqcd.launch_count() - launches0
    svc.close()
    return [results[k] for k in range(len(reqs))], makespan, launches


def run_service(args):
    """Point-source solve requests (12 spin-colour right-hand sides each) of the
    full Wilson operator on resident gauge fields of 8^4, 16^3x32, 24^3x48 and
    32^3x64 (start exp(i 0.15 H), Philox seed 200 + k), volume uniform over the
    four, kappa uniform in [0.150, 0.158], source site uniform, Poisson
    arrivals at 200/s; mixed FP16+norm CG to full |r|/|b| <= 1e-10.  The
    continuously batched service against the same service admitting one
    request at a time (FIFO)."""
    import torch

    from paper_1212_0785_gb300 import lqcd

    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    n = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n))
    arrivals -= arrivals[0]
    reqs = []
    for _ in range(n):
        g = int(rng.integers(len(SERVICE_LATS)))
        site = tuple(int(rng.integers(L)) for L in SERVICE_LATS[g])
        reqs.append((g, float(rng.uniform(0.150, 0.158)), site))
    fields = []
    for k, dims in enumerate(SERVICE_LATS):
        U = lqcd.gauge_field(dims)
        lqcd.gauge_start(U, 200 + k, 0.15)
        fields.append(U)
    sloppy = lqcd.PREC_NAMES[args.sloppy]
    prm = lqcd.service_params(tol=1e-10, sloppy=sloppy, delta=args.delta, hbm_budget=args.hbm_budget << 30)
    clocks = ClockSampler(0)
    clocks.start()
    res, span, launches = _serve(lqcd, fields, arrivals, reqs, prm)
    clk = clocks.stop()
    fifo_prm = lqcd.service_params(tol=1e-10, sloppy=sloppy, delta=args.delta, hbm_budget=args.hbm_budget << 30,
                                   max_active_rhs=12)
    fres, fspan, _ = _serve(lqcd, fields, arrivals, reqs, fifo_prm)

    def stats(rs, sp):
        lat = np.array([r["latency_s"] for r in rs])
        return {"solves_per_s": len(rs) / sp, "rhs_per_s": 12 * len(rs) / sp, "makespan_s": sp,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "queue_p50_s": float(np.percentile([r["queue_s"] for r in rs], 50)),
                "true_rel_res_max": max(r["true_rel_res_max"] for r in rs),
                "failed": sum(r["status"] != lqcd.OK for r in rs)}

    ours, fifo = stats(res, span), stats(fres, fspan)
    line = {"metric": "solves/s", "value": ours["solves_per_s"], "unit": "solves/s (12 point-source RHS each)",
            "n_gpus": 1, "steps": n, "warmup": len(SERVICE_LATS), "ms_per_step": span / n * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "dtype_detail": "f32 math (f16n solver storage); f64 residual check and solutions",
            "data": "synthetic",
            "config": {"workload": "solve_service_8^4_16^3x32_24^3x48_32^3x64", "requests": n,
                       "arrival_rate_per_s": args.rate, "rhs_per_request": 12, "kappa": [0.150, 0.158],
                       "tol_full_M": 1e-10, "hbm_budget_gib": args.hbm_budget, "start_eps": 0.15},
            "latency_p50_s": ours["latency_p50_s"], "latency_p99_s": ours["latency_p99_s"],
            "service": ours, "fifo": fifo, "gpu_launches": launches, "clocks": clk,
            "iters_per_rhs": float(np.mean([r["iters"] / 12 for r in res]))}
    print(json.dumps(line))
    return 0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; 10 trajectories for fp64_16x32, 2 for chains64)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("hmc32", "fp64_16x32", "chains64", "service"), default="hmc32",
                    help="hmc32: the 32^3x64 trajectory (default); fp64_16x32: the plain FP64 path on 16^3x32; "
                         "chains64: 64 batched chains; service: Poisson-arriving point-source solves")
    ap.add_argument("--requests", type=int, default=40, help="service: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="service: mean arrivals per second")
    ap.add_argument("--hbm-budget", type=int, default=96, help="service: admission budget, GiB")
    ap.add_argument("--sloppy", choices=("f32", "f16n", "bf16"), default="f16n")
    ap.add_argument("--delta", type=float, default=0.003)
    ap.add_argument("--force-prec", choices=("f64", "f32"), default="f32")
    ap.add_argument("--chrono", type=int, choices=(0, 1, 2, 3, 4), default=3,
                    help="initial guess of each solve after the first of a trajectory: 0 zero, 1 the previous "
                         "solution, k >= 2 extrapolated through the last k solutions (both the mixed and the "
                         "FP64 path)")
    ap.add_argument("--autotune", type=int, choices=(0, 1), default=1,
                    help="1: tune the threads per block of the tunable kernels on the lattice first")
    ap.add_argument("--tune-file", default=None, help="write the autotuner's timings to this file")
    ap.add_argument("--mre", type=int, choices=(0, 1), default=0,
                    help="1: refine the extrapolated guesses by minimal residual extrapolation")
    ap.add_argument("--dims", type=int, nargs=4, default=WORKLOAD["dims"])
    ap.add_argument("--nsteps", type=int, default=WORKLOAD["nsteps"],
                    help="MD steps per trajectory (16 for the benchmarked workload)")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed trajectories of the plain FP64 GPU path (0: skip it)")
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.steps is None and args.workload in ("hmc32", "service"):
        args.steps = 5
    elif args.steps is None and args.workload == "chains64":
        args.steps = 2
    return args


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "fp64_16x32":
        return run_fp64_16(args)
    if args.workload == "chains64":
        return run_chains(args)
    if args.workload == "service":
        return run_service(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

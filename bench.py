"""Benchmark of the fused stream + collide step (MLUPS and HBM roofline).

Workload (default): D3Q27 cumulant LBM, regularised (shear rate from
nu = 1e-3, bulk and higher-order rates 1), periodic 512^3 Taylor-Green vortex
u0 = 0.05 plus seeded uniform +-1e-3 velocity noise, populations stored as
FP32 deviations, pull streaming.  The same step is also timed with FP16- and
BF16-delta storage (reported under "forms" with its velocity error against an
FP64 run of the same steps), with the in-place patterns (AA, Esoteric Twist,
Pull, Push) and with a Guo body force.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Under torchrun (N > 1) every rank advances its own independent replica
(the method does not shard here: replicas only); the reported value is the
sum of all ranks' cell updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_02435_b300 import inputs as I  # noqa: E402

METRIC = "MLUPS and % of HBM roofline, D3Q27 cumulant 512^3, FP32 vs FP16-delta storage"
UNIT = "MLUPS"
BYTES_PER_CELL = {"f64": 432, "f32": 216, "f16_delta": 108, "bf16_delta": 108}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process
    group): the slowest rank's time defines the whole job's time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, cells_per_rank, steps, seconds):
    """Whole-job throughput of `world` independent replicas."""
    return world * cells_per_rank * steps / seconds / 1e6


def profile_value(name, key, sources=("lbm_device.cuh", "lbm_kernels.cuh")):
    """A figure `key = value` of the committed ncu summary profiles/<name>, or
    None when the kernel sources it was taken from changed since (the summary
    records the SHA-1 of those files as kernel_source_sha1)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m1 = re.search(re.escape(key) + r" = ([0-9.eE+-]+)", txt)
    m2 = re.search(r"kernel_source_sha1 = ([0-9a-f]+)", txt)
    if not (m1 and m2):
        return None
    h = hashlib.sha1()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2211_02435_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return float(m1.group(1)) if h.hexdigest() == m2.group(1) else None


def kernel_traffic_per_cell():
    """DRAM bytes per cell update of the FP32 step kernel from the committed
    ncu summary, or None when the kernel sources changed since the capture."""
    return profile_value("ncu_k_pull_d3q27_cumulant_f32_256.md", "traffic_bytes_per_cell")


def fp32_peak_tflops(sm_max_mhz):
    """FP32 CUDA-core peak of this device: SMs x 128 FP32 lanes x 2 flop (one
    fused multiply-add) x the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 128 * 2 * (sm_max_mhz or 2032.0) * 1e6 / 1e12


def alu_roof(profile, mlups, peak_tflops, sources):
    """ALU roof of a kernel: FP32 flops per cell update (ncu instruction
    counts, FFMA = 2, FFMA2 = 4, FADD / FMUL = 1, FADD2 / FMUL2 = 2) x cell
    updates per second against the FP32 CUDA-core peak; and the FMA-pipe
    lane-ops per cell (FADD2 / FMUL2 occupy two lanes like FFMA2) against the
    pipe's lane rate, peak / 2."""
    fpc = profile_value(profile, "fp32_flop_per_cell", sources)
    if fpc is None:
        return None
    ach = fpc * mlups * 1e6 / 1e12
    out = {"bound": "alu", "flop_per_cell": fpc, "achieved": ach, "peak": peak_tflops,
           "unit": "TFLOP/s", "frac": ach / peak_tflops, "profile": profile}
    ops = profile_value(profile, "fp32_lane_ops_per_cell", sources)
    if ops is not None:
        out["lane_ops_per_cell"] = ops
        out["pipe_frac"] = ops * mlups * 1e6 / (peak_tflops * 1e12 / 2)
    # instruction issue: 4 schedulers x 32 lanes per SM per clock, the same
    # SMs x 128 x clock as the FP32 lane rate
    ins = profile_value(profile, "thread_inst_per_cell", sources)
    if ins is not None:
        out["inst_per_cell"] = ins
        out["issue_frac"] = ins * mlups * 1e6 / (peak_tflops * 1e12 / 2)
    return out


def make_fields(n):
    rho, u = I.taylor_green((n, n, n), 0.05)
    u = I.add_uniform_noise(u, 1e-3, seed=1)
    return rho, u


def oracle_sample(n_cells_edge, steps, nthreads=0):
    """Time the FP64 CPU oracle on a small cube of the same method and flow:
    one call that advances a state made once by `steps` steps, so that the
    per-call set-up (marshalling, allocation, thread start-up) is paid once.
    nthreads = 0 uses every host core (the count is passed explicitly: the
    oracle's OpenMP thread count persists between calls)."""
    import oracle as O
    O.build()
    nu = 1e-3
    rates = [I.shear_viscosity_rate(nu)] + [1.0] * 5
    m = O.method(O.D3Q27, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, rates)
    dims = (n_cells_edge,) * 3
    rho, u = make_fields(n_cells_edge)
    df = O.init(m, dims, rho, u)
    threads = nthreads or (os.cpu_count() or 1)
    O.step(m, dims, df, 1, threads)  # warm: thread pool and pages
    t0 = time.perf_counter()
    O.step(m, dims, df, steps, threads)
    dt = time.perf_counter() - t0
    return n_cells_edge ** 3 * steps / dt / 1e6, dt


def cpu_baselines(edge, steps_all, steps_one):
    """The oracle on every host core and on one core (same flow and cube)."""
    v_all, dt_all = oracle_sample(edge, steps_all)
    v_one, dt_one = oracle_sample(edge, steps_one, nthreads=1)
    cores = os.cpu_count()
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{edge}^3 cells x {steps_all} steps of the same method and flow "
                      f"({dt_all:.1f} s, OpenMP over {cores} cores), one oracle call",
            "one_core": {"value": v_one, "unit": UNIT, "cores": 1,
                         "sample": f"{edge}^3 cells x {steps_one} steps ({dt_one:.1f} s)"}}


def main_config(args, cells, world):
    """The workload the cuda arm times (and the reference arm samples)."""
    key = {"f32": "f32", "f16": "f16_delta", "bf16": "bf16_delta"}[args.storage]
    return {"workload": f"D3Q27 cumulant LBM (R-: shear from nu=1e-3, bulk and orders 3-6 "
                        f"rate 1), periodic {args.size}^3 Taylor-Green u0=0.05 + uniform 1e-3 "
                        f"noise, {key} zero-centered storage, {args.streaming}"
                        + ("" if args.force == "none" else f", {args.force} body force"),
            "cells": cells, "global_batch": world, "parallelism": "replicas",
            "l2": "working set 29 GB >> 126 MB L2, no flush needed"}


def run_reference(args):
    """The oracle as it stands, on the host cores: W warm-up steps, then the K
    timed steps as one oracle call on the bounded 48^3 sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    edge = args.ref_edge
    cores = os.cpu_count()
    oracle_sample(edge, args.warmup)
    v, dt = oracle_sample(edge, args.steps)
    sample = (f"{edge}^3 cells of the same D3Q27 cumulant TGV flow, the {args.steps} timed "
              f"steps as one oracle call on {cores} cores (bounded sample of the 512^3 workload)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": main_config(args, args.size ** 3, args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, L, torch, stream, peak):
    """Ensemble of independent D3Q19 O-MRT (R-) Taylor-Green domains, edges
    from {16, 24, 32, 48, 64, 96}, per-instance viscosity log-uniform in
    [1e-4, 1e-1], FP32 storage: one persistent launch per step replayed from
    CUDA graphs, with the autotuned launch shape; compared with one launch per
    instance and with a single 512^3 domain of the same method."""
    dims, nu, u0 = I.batch_ensemble(args.batch_n, seed=4)
    om = [I.shear_viscosity_rate(v) for v in nu]
    rates = [1.0] * 6
    out = {"workload": f"{args.batch_n} periodic D3Q19 O-MRT R- TGV domains, edges "
                       "{16,24,32,48,64,96}, nu log-uniform [1e-4, 1e-1], u0 U[0.01, 0.08], "
                       "FP32, pull", "instances": args.batch_n}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    with L.Batch(L.D3Q19, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, rates, [tuple(d) for d in dims],
                 om, stream=stream) as b:
        cells = b.cells()
        tune, tune_mlups = b.autotune(trial_steps=args.autotune_steps)
        b.init_tgv(u0)
        b.step(args.warmup)
        ms = timed(b.step, args.steps)
        mlups = cells * args.steps / (ms / 1e3) / 1e6
        ach = 152 * cells / (ms / 1e3 / args.steps) / 1e9
        b.set_tuning(**dict(tune, per_instance=1))
        b.step(2)
        ksteps = max(2, args.steps // 5)
        ms_pi = timed(b.step, ksteps)
        out.update({"cells": cells, "mlups": mlups, "achieved_gbs": ach,
                    "roofline_frac": ach / peak, "tuning": tune,
                    "per_instance_launch_mlups": cells * ksteps / (ms_pi / 1e3) / 1e6,
                    "launches_per_step": 1})
    lat = L.Lattice(L.D3Q19, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, L.PULL,
                    [I.shear_viscosity_rate(1e-3)] + [1.0] * 5, (512, 512, 512), stream=stream)
    rho, u = I.taylor_green((512, 512, 512), 0.05)
    lat.init_velocity(rho.reshape(-1), u.reshape(-1))
    del rho, u
    lat.step(args.warmup)
    ms1 = timed(lat.step, args.steps)
    lat.close()
    out["single_domain_d3q19_512_mlups"] = 512 ** 3 * args.steps / (ms1 / 1e3) / 1e6
    return out


def run_learned(args, L, torch, stream):
    """Learned closure: fine 512^3 plain cumulant run (nu = 2e-4, seeded
    Fourier-mode flow) restricted to 128^3 every 4 fine steps over 1280
    coarse steps, GPU training of the rate network on K-step rollout windows
    of the first 80 %, held-out K-step loss and 64- / 256-step rollout errors
    against the plain method from the first held-out snapshot, and the fused
    learned-rate kernel's MLUPS against the plain kernel's at 128^3."""
    from paper_2211_02435_b300 import closure as C
    sc = args.learned_fine / 512  # time scale of the flow relative to 512^3
    res = C.train_and_evaluate(fine_edge=args.learned_fine, span=int(round(1280 * sc)),
                               unroll=args.learned_unroll, windows=24,
                               epochs=args.learned_epochs, lr=3e-3,
                               rollout=int(round(256 * sc)), short=int(round(64 * sc)),
                               nu_fine=2e-4, seed=5, stream=stream)
    w = res.pop("weights")
    n = args.learned_fine // 4
    omega_c = I.shear_viscosity_rate(2e-4 / 4)
    rho, u = I.fourier_modes((n, n, n), seed=5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rates = {}
    steps = max(args.steps, 20)
    for name, weights in (("plain", None), ("learned", w)):
        with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL,
                       [omega_c] + [1.0] * 5, (n, n, n), stream=stream) as lat:
            if weights is not None:
                lat.set_closure(weights)
            lat.init_velocity(rho.reshape(-1), u.reshape(-1))
            lat.step(args.warmup)
            torch.cuda.synchronize()
            e0.record(stream)
            lat.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            rates[name] = n ** 3 * steps / (e0.elapsed_time(e1) / 1e3) / 1e6
    res[f"mlups_{n}_plain_kernel"] = rates["plain"]
    res[f"mlups_{n}_learned_kernel"] = rates["learned"]
    res["learned_vs_plain_mlups"] = rates["learned"] / rates["plain"]
    return res


def run_closure_timing(args):
    """Throughput of the fused learned-rate step against the plain step
    (D3Q27 cumulant, FP32, pull) at --size^3 on the Fourier-mode flow, with a
    seeded random network (normalised on the initial state): one JSON line.
    A small, training-free case for profiling the fused kernel."""
    import torch
    from paper_2211_02435_b300 import build as B
    from paper_2211_02435_b300 import closure as C
    from paper_2211_02435_b300 import lbm as L

    B.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.size
    omega_c = I.shear_viscosity_rate(2e-4 / 4)
    rho, u = I.fourier_modes((n, n, n), seed=5)
    with L.Trainer((n, n, n), omega_c, 1.0, 2, stream=stream) as tr:
        with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL,
                       [omega_c] + [1.0] * 5, (n, n, n), stream=stream) as lat:
            lat.init_velocity(rho.reshape(-1), u.reshape(-1))
            lat.step(2)
            tr.add_snapshot(lat.get_populations())
        shift, scale = C.feature_normalisation(tr, [0])
        p = C.init_params(7, 0.3)
        p[1312:] = 0.3 * np.random.default_rng(8).standard_normal(132)
        tr.set_params(p, shift, scale)
        w = tr.export()
    out = {"metric": "fused learned-rate step MLUPS vs the plain step", "unit": UNIT,
           "cells": n ** 3, "steps": args.steps, "warmup": args.warmup}
    for name, weights in (("plain", None), ("learned", w)):
        with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL,
                       [omega_c] + [1.0] * 5, (n, n, n), stream=stream) as lat:
            if weights is not None:
                lat.set_closure(weights)
            lat.init_velocity(rho.reshape(-1), u.reshape(-1))
            lat.step(args.warmup)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            out[f"{name}_mlups"] = n ** 3 * args.steps / (e0.elapsed_time(e1) / 1e3) / 1e6
    out["learned_vs_plain"] = out["learned_mlups"] / out["plain_mlups"]
    print(json.dumps(out), flush=True)
    return 0


def run_cuda(args):
    import torch
    from paper_2211_02435_b300 import build as B
    from paper_2211_02435_b300 import lbm as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        args.gpus = world
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()

    n = args.size
    N = n ** 3
    rates = [I.shear_viscosity_rate(1e-3)] + [1.0] * 5
    stream = torch.cuda.current_stream()
    rho_h, u_h = make_fields(n)
    rho_d = torch.from_numpy(rho_h.reshape(-1)).cuda()
    u_d = torch.from_numpy(u_h.reshape(-1)).cuda()
    peak, peak_kind = measured_peaks()

    def time_form(storage, steps, warmup, streaming=L.PULL, force=None, windows=1):
        lat = L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, storage, streaming, rates,
                        (n, n, n), stream=stream)
        if streaming == L.PULL:
            lat.set_step_kernel(STEP_KERNELS[args.step_kernel])
        if force is not None:
            if force.ndim == 1:
                lat.set_force(force)
            else:
                lat.set_force_field(force)
        lat.init_velocity(rho_d, u_d)
        lat.step(warmup)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # the timed steps as consecutive windows with an event between each
        # pair (queued back to back: no gap is added between windows)
        cuts = [round(k * steps / windows) for k in range(windows + 1)]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(windows + 1)]
        ev[0].record(stream)
        for k in range(windows):
            lat.step(cuts[k + 1] - cuts[k])
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[-1])
        if windows > 1:
            win = [(cuts[k + 1] - cuts[k], ev[k].elapsed_time(ev[k + 1])) for k in range(windows)]
            return lat, ms, win
        return lat, ms

    # ---- headline: FP32 storage (or --storage), kernel-only, inputs in HBM
    main_store = {"f32": L.STORE_F32, "f16": L.STORE_F16_DELTA, "bf16": L.STORE_BF16_DELTA}[args.storage]
    main_key = {"f32": "f32", "f16": "f16_delta", "bf16": "bf16_delta"}[args.storage]
    main_stream = STREAMINGS[args.streaming]
    main_force = None
    if args.force == "uniform":
        main_force = np.array([1e-6, 0.0, 0.0])
    elif args.force == "field":
        main_force = torch.full((3, N), 1e-6, dtype=torch.float64, device="cuda")
    nwin = max(1, min(5, args.steps))
    with ClockSampler(local) as clk:
        lat32, ms32, *win = time_form(main_store, args.steps, args.warmup, streaming=main_stream,
                                      force=main_force, windows=nwin)
    win = win[0] if win else [(args.steps, ms32)]
    win_mlups = [N * k / (w / 1e3) / 1e6 for k, w in win]
    del main_force
    clocks = clk.summary()
    ms_max = max_over_ranks(ms32, dist, "cuda")
    per_step_s = ms_max / 1e3 / args.steps
    value = job_mlups(world, N, args.steps, ms_max / 1e3)
    main_bpc = BYTES_PER_CELL[main_key] + (12 if args.force == "field" else 0)
    achieved = main_bpc * N / (ms32 / 1e3 / args.steps) / 1e9
    # velocity of the timed run, copied to the host once its stream is idle
    u32 = np.empty(3 * N)
    lat32.macroscopic(None, u32)
    lat32.close()
    del lat32

    # a separate sustained run of >= 1 s of steps, median of 5 windows
    sustained = None
    if not args.no_sustained and args.sustained_steps > 0:
        lat, ms_s, win_s = time_form(main_store, args.sustained_steps, args.warmup,
                                     streaming=main_stream, windows=5)
        lat.close()
        del lat
        wm = sorted(N * k / (w / 1e3) / 1e6 for k, w in win_s)
        sustained = {"steps": args.sustained_steps, "seconds": ms_s / 1e3, "windows": 5,
                     "median_mlups": wm[2], "min_mlups": wm[0], "max_mlups": wm[-1],
                     "median_frac": main_bpc * wm[2] * 1e6 / 1e9 / peak}


    forms = {}
    if not args.no_forms:
        # FP64 reference of the same number of steps for the velocity errors
        lat64 = L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL, rates,
                          (n, n, n), stream=stream)
        lat64.init_velocity(rho_d, u_d)
        lat64.step(args.warmup + args.steps)
        u64 = np.empty(3 * N)
        lat64.macroscopic(None, u64)
        lat64.close()
        del lat64
        umax = float(np.abs(u64).max())

        def uerr(uu):
            return float(np.abs(uu - u64).max()) / umax

        forms["f32"] = {"mlups": N * args.steps / (ms32 / 1e3) / 1e6,
                        "roofline_frac": achieved / peak, "u_rel_linf_vs_f64": uerr(u32)}
        # each form is timed under its own clock sampler: the forms run one
        # after the other, and a form late in the run can meet the power cap
        for name, st in (("f16_delta", L.STORE_F16_DELTA), ("bf16_delta", L.STORE_BF16_DELTA)):
            with ClockSampler(local) as ck:
                lat, ms = time_form(st, args.steps, args.warmup)
            uu = np.empty(3 * N)
            lat.macroscopic(None, uu)
            lat.close()
            del lat
            ach = BYTES_PER_CELL[name] * N / (ms / 1e3 / args.steps) / 1e9
            forms[name] = {"mlups": N * args.steps / (ms / 1e3) / 1e6,
                           "achieved_gbs": ach, "roofline_frac": ach / peak,
                           "u_rel_linf_vs_f64": uerr(uu),
                           "vs_f32_mlups": (N * args.steps / (ms / 1e3)) / (N * args.steps / (ms32 / 1e3)),
                           "clocks": ck.summary()}
            del uu
        # in-place patterns (one buffer), FP32 and FP16 delta, even number of steps
        st_ip = 2 * (args.steps // 2)
        for key, store in (("f32", L.STORE_F32), ("f16_delta", L.STORE_F16_DELTA)):
            for name in ("aa", "et", "epull", "epush"):
                with ClockSampler(local) as ck:
                    lat, ms = time_form(store, st_ip, args.warmup + args.warmup % 2,
                                        streaming=STREAMINGS[name])
                lat.close()
                del lat
                ach = BYTES_PER_CELL[key] * N / (ms / 1e3 / st_ip) / 1e9
                forms[f"{key}_{name}"] = {
                    "mlups": N * st_ip / (ms / 1e3) / 1e6, "achieved_gbs": ach,
                    "roofline_frac": ach / peak, "buffers": 1,
                    "note": "same per-cell arithmetic as pull (bitwise equal states)",
                    "clocks": ck.summary()}
        # body force (Guo): uniform, and a per-cell field (+12 B/cell of reads)
        for name, force, bpc in (
                ("f32_force_uniform", np.array([1e-6, 0.0, 0.0]), BYTES_PER_CELL["f32"]),
                ("f32_force_field", torch.full((3 * N,), 1e-6, dtype=torch.float64,
                                               device="cuda"), BYTES_PER_CELL["f32"] + 12)):
            if not isinstance(force, np.ndarray):
                force = force.view(3, -1)
            lat, ms = time_form(L.STORE_F32, args.steps, args.warmup, force=force)
            lat.close()
            del lat
            ach = bpc * N / (ms / 1e3 / args.steps) / 1e9
            forms[name] = {"mlups": N * args.steps / (ms / 1e3) / 1e6, "achieved_gbs": ach,
                           "roofline_frac": ach / peak, "bytes_per_cell": bpc}
            del force
        del u64
    del u32

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        rho_p = torch.from_numpy(rho_h.reshape(-1)).pin_memory()
        u_p = torch.from_numpy(u_h.reshape(-1)).pin_memory()
        rho_out = torch.empty(N, dtype=torch.float64).pin_memory()
        u_out = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        lat = L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, rates,
                        (n, n, n), stream=stream)
        # one call: host fields in, the steps, host fields out; the library
        # overlaps the copies and the steps of different slabs of z-planes
        lat.run_host(rho_p.numpy(), u_p.numpy(), args.warmup, rho_out.numpy(), u_out.numpy())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        lat.run_host(rho_p.numpy(), u_p.numpy(), args.steps, rho_out.numpy(), u_out.numpy())
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        lat.close()
        e2e = {"value": job_mlups(world, N, args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": 4 * N * 8 / args.steps,
               "d2h_bytes_per_step": 4 * N * 8 / args.steps,
               "job": f"lbm_run_host: host rho,u (FP64, pinned) -> init -> {args.steps} steps "
                      "-> host rho,u, pipelined by slabs of z-planes"}

    batched = None
    if not args.no_batched:
        del rho_d, u_d
        torch.cuda.empty_cache()
        batched = run_batched(args, L, torch, stream, peak)

    learned = None
    if not args.no_learned:
        torch.cuda.empty_cache()
        learned = run_learned(args, L, torch, stream)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baselines(args.ref_edge, args.cpu_steps, args.cpu_steps_one_core)

    default_kernel = args.storage == "f32" and args.streaming == "pull" and args.force == "none"
    traffic = kernel_traffic_per_cell() if default_kernel else None
    if traffic is not None:
        traffic *= N

    # ALU roofs of the kernels that may reach it (the packed FP16 and BF16 steps and
    # the fused learned-rate step): FP32 flops per cell from ncu counts
    fp32_peak = fp32_peak_tflops(clocks.get("sm_max_mhz"))
    for form, prof in (("f16_delta", "alu_k_pull4_d3q27_cumulant_f16.md"),
                       ("bf16_delta", "alu_k_pull4_d3q27_cumulant_bf16.md")):
        if form in forms:
            forms[form]["alu"] = alu_roof(prof, forms[form]["mlups"], fp32_peak,
                                          ("lbm_device.cuh", "lbm_kernels.cuh",
                                           "lbm_packed.cuh"))
    if learned is not None:
        n_c = args.learned_fine // 4
        learned["alu"] = alu_roof("alu_k_closure_pull_d3q27_128.md",
                                  learned[f"mlups_{n_c}_learned_kernel"], fp32_peak,
                                  ("lbm_device.cuh", "lbm_closure.cu"))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "f32" else f"f32 compute, {args.storage} storage",
            "data": "synthetic",
            "config": main_config(args, N, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "bytes_per_cell": main_bpc,
                         "kernel": (("k_pull" if args.streaming == "pull" else "k_inplace")
                                    + f"<D3Q27, {args.streaming}, {main_key} storage, cumulant, "
                                    + ("regularised>" if args.force == "none"
                                       else f"{args.force} force>")),
                         "step_kernel": args.step_kernel,
                         "timed_windows_mlups": win_mlups},
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": args.steps,
            "sustained": sustained,
            "forms": forms, "batched": batched, "learned": learned}
    line["summary"] = summary(line, win_mlups)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def summary(line, win_mlups):
    """The figures a reader needs, compact and last on the line."""
    def r(x, nd=3):
        return None if x is None else round(float(x), nd)

    out = {"headline_mlups": r(line["value"], 0), "headline_frac": r(line["roofline"]["frac"]),
           "headline_window_median_mlups": r(statistics.median(win_mlups), 0)}
    if line.get("sustained"):
        out["sustained_median_mlups"] = r(line["sustained"]["median_mlups"], 0)
    f = line.get("forms") or {}
    for k in ("f16_delta", "bf16_delta"):
        if k in f:
            alu = f[k].get("alu")
            out[f"{k}_pull"] = {"mlups": r(f[k]["mlups"], 0), "frac": r(f[k]["roofline_frac"]),
                                "u_rel_linf_vs_f64": r(f[k]["u_rel_linf_vs_f64"], 8),
                                "alu_frac": r(alu["frac"]) if alu else None,
                                "alu_pipe_frac": r(alu.get("pipe_frac")) if alu else None}
    ip = {k.split("_")[-1]: r(v["roofline_frac"]) for k, v in f.items()
          if k.startswith("f16_delta_") and "roofline_frac" in v}
    if ip:
        out["f16_delta_inplace_frac"] = ip
        mhz = {k.split("_")[-1]: (v.get("clocks") or {}).get("sm_mhz") for k, v in f.items()
               if k.startswith("f16_delta_") and "roofline_frac" in v}
        if any(m is not None for m in mhz.values()):
            out["f16_delta_inplace_sm_mhz"] = mhz
    b = line.get("batched")
    if b:
        out["batched"] = {"mlups": r(b["mlups"], 0), "frac": r(b["roofline_frac"]),
                          "tuning": [b["tuning"][k] for k in ("threads", "cells_per_thread",
                                                             "blocks_per_sm")]}
    le = line.get("learned")
    if le:
        o = {}
        for key in le:
            if key.startswith("rollout") and key.endswith("_err_learned"):
                steps = key[len("rollout"):-len("_err_learned")]
                o[f"rollout{steps}_l2"] = [r(le[key], 4), r(le[f"rollout{steps}_err_plain"], 4)]
        o["heldout_loss"] = [le.get("heldout_loss_learned"), le.get("heldout_loss_plain")]
        o["kernel_mlups"] = [r(v, 0) for k, v in le.items() if k.startswith("mlups_")][::-1]
        o["alu_frac"] = r(le["alu"]["frac"]) if le.get("alu") else None
        o["alu_pipe_frac"] = r(le["alu"].get("pipe_frac")) if le.get("alu") else None
        o["issue_frac"] = r(le["alu"].get("issue_frac")) if le.get("alu") else None
        out["learned"] = o
    c = line.get("cpu_baseline")
    if c:
        out["oracle_mlups"] = {"cores": c["cores"], "all": r(c["value"], 3),
                               "one": r(c["one_core"]["value"], 4)}
    return out


STEP_KERNELS = {"auto": 0, "direct": 1, "staged": 2}  # LBM_STEP_* of include/lbm.h
# lbm_streaming of include/lbm.h: pull, AA, Esoteric Twist / Pull / Push
STREAMINGS = {"pull": 0, "aa": 1, "et": 2, "epull": 3, "epush": 4}


def run_method_survey(args):
    """Throughput of the pull step for every stencil, collision space and
    storage (not the headline): D3Q19 / D3Q27 at 512^3, D2Q9 at 8192^2, the
    regularised (R-) rates with shear from nu = 1e-3, Taylor-Green start; one
    JSON line with MLUPS and the fraction of the measured copy bandwidth at
    2 q b bytes per cell update."""
    import torch
    from paper_2211_02435_b300 import build as B
    from paper_2211_02435_b300 import lbm as L

    B.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()
    rates = [I.shear_viscosity_rate(1e-3)] + [1.0] * 5
    spaces = [("SRT", L.SPACE_POPULATIONS, L.EQ_DELTA), ("TRT", L.SPACE_TRT, L.EQ_DELTA),
              ("R-O-MRT", L.SPACE_RAW, L.EQ_DELTA), ("R-WO-MRT", L.SPACE_RAW_WEIGHTED, L.EQ_DELTA),
              ("R-CM", L.SPACE_CENTRAL, L.EQ_ABSOLUTE), ("R-K", L.SPACE_CUMULANT, L.EQ_ABSOLUTE)]
    stores = [("f32", L.STORE_F32, 4), ("f16_delta", L.STORE_F16_DELTA, 2)]
    rows = []
    for st, name, dims in ((L.D2Q9, "D2Q9", (8192, 8192, 1)), (L.D3Q19, "D3Q19", (512,) * 3),
                           (L.D3Q27, "D3Q27", (512,) * 3)):
        d = 2 if st == L.D2Q9 else 3
        rho, u = I.taylor_green(dims, 0.05, d=d)
        rho_d = torch.from_numpy(np.ascontiguousarray(rho.reshape(-1))).cuda()
        u_d = torch.from_numpy(np.ascontiguousarray(u.reshape(-1))).cuda()
        del rho, u
        N = int(np.prod(dims))
        for sname, space, eq in spaces:
            r = [1.6] * 6 if space == L.SPACE_POPULATIONS else (
                [rates[0], 1.0, 1.75, 1.0, 1.0, 1.0] if space == L.SPACE_TRT else rates)
            for kname, storage, eb in stores:
                with L.Lattice(st, space, eq, storage, L.PULL, r, dims, stream=stream) as lat:
                    lat.init_velocity(rho_d, u_d)
                    lat.step(args.warmup)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    lat.step(args.steps)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / args.steps
                bpc = 2 * lat.q * eb
                rows.append({"stencil": name, "method": sname, "storage": kname,
                             "cells": N, "mlups": N / ms / 1e3,
                             "bytes_per_cell": bpc, "roofline_frac": bpc * N / ms / 1e6 / peak})
        del rho_d, u_d
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "pull-step MLUPS per stencil, collision space and storage",
                      "unit": UNIT, "peak_gbs": peak, "peak_kind": peak_kind,
                      "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                      "rows": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--ref-edge", type=int, default=48)
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--cpu-steps-one-core", type=int, default=4)
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32",
                    help="storage of the headline form (default FP32)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-sustained", action="store_true")
    ap.add_argument("--sustained-steps", type=int, default=250,
                    help="steps of the separate >= 1 s sustained run (5 windows, median)")
    ap.add_argument("--closure-timing", action="store_true",
                    help="time the fused learned-rate step against the plain one at --size^3")
    ap.add_argument("--method-survey", action="store_true",
                    help="time the pull step of every stencil / space / storage instead")
    ap.add_argument("--learned-fine", type=int, default=512)
    ap.add_argument("--learned-unroll", type=int, default=8)
    ap.add_argument("--learned-epochs", type=int, default=4)
    ap.add_argument("--batch-n", type=int, default=4096)
    ap.add_argument("--autotune-steps", type=int, default=6,
                    help="steps per autotuner trial of the batched ensemble")
    ap.add_argument("--step-kernel", choices=list(STEP_KERNELS), default="auto",
                    help="pull step kernel of the D3Q27 forms (include/lbm.h)")
    ap.add_argument("--streaming", choices=list(STREAMINGS), default="pull",
                    help="streaming pattern of the headline run")
    ap.add_argument("--force", choices=["none", "uniform", "field"], default="none",
                    help="body force (Guo) of the headline run")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "cuda":
        args.warmup = 3
    if args.method_survey:
        return run_method_survey(args)
    if args.closure_timing:
        return run_closure_timing(args)
    return run_reference(args) if args.impl == "reference" else run_cuda(args)


if __name__ == "__main__":
    sys.exit(main())

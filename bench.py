#!/usr/bin/env python
"""Benchmark of the batched Parareal hot path on one GB300 (or N, weak scaling).

A step is one pass of the whole hot path over one batch: one call of
parareal_iterate with max_iters = 1, i.e. the serial coarse sweep, the batched
fine sweep of all time slices, the serial coarse correction sweep with the
Parareal update (Eq. 20) and the defect/Nusselt norms.

Workload (default): Ra = 1e6, Pr = 1, Lx/Lz = 2, fine 256 x 64 (Fourier x
Chebyshev), coarse 128 x 32, 32 time slices of 3125 fine steps each, all FP64,
seeded noise initial condition.  The fine and coarse time steps are the largest
stable ones of a halving ladder (the configured 2e-4 / 2e-3 blow up in the
initial plume burst); the configured number of fine steps per slice is kept.

value: fine DOF-steps per second, DOF = 2 Nx Nz per slice (psi and T), counted
over the fine sweep of all slices, divided by the wall time of the whole step.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Parareal time-to-tol vs serial fine on 1 GB300; DOF-steps/s; p50/p99 latency"
UNIT = "DOF-steps/s"

# Workloads.  dt values: largest stable on the halving ladder from the
# configured values (oracle survey: the configured steps blow up at t ~ 0.015).
WORKLOADS = {
    "rbc_ra1e6_256x64_32slices_fp64": dict(
        Ra=1e6, Pr=1.0, Lx=2.0, Nx=256, Nz=64, Nxc=128, Nzc=32, dt=1.25e-5, dtc_target=1.5625e-5,
        slices=32, steps_per_slice=3125, seed=1),
    "rbc_ra1e4_64x32_4slices_fp64": dict(
        Ra=1e4, Pr=1.0, Lx=2.0, Nx=64, Nz=32, Nxc=32, Nzc=16, dt=1e-3, dtc_target=5e-3,
        slices=4, steps_per_slice=1000, seed=0),
}
DEFAULT = "rbc_ra1e6_256x64_32slices_fp64"


def derived(w):
    slice_len = w["steps_per_slice"] * w["dt"]
    nc = max(1, int(round(slice_len / w["dtc_target"])))
    return dict(slice_len=slice_len, t_end=w["slices"] * slice_len, nc=nc, dtc=slice_len / nc,
                dof=2 * w["Nx"] * w["Nz"])


# --------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, one host thread, bounded sample.
# --------------------------------------------------------------------------
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle.rbc import RBC
from paper_2001_01609_gb300.inputs import initial_temperature
w = {w!r}
o = RBC(w["Ra"], w["Pr"], w["Lx"], w["Nx"], w["Nz"], w["dt"])
X = o.from_grid(initial_temperature(w["Nx"], w["Nz"], seed=w["seed"], Lx=w["Lx"]))
X, _ = o.step(X)
t0 = time.perf_counter(); n = 0
while True:
    X, _ = o.step(X); n += 1
    el = time.perf_counter() - t0
    if el > {budget} or n >= {max_steps}:
        break
print(json.dumps(dict(steps=n, seconds=el)))
"""


def cpu_oracle_rate(w, budget_s=12.0, max_steps=100000):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = CPU_SNIPPET.format(root=ROOT, w=w, budget=budget_s, max_steps=max_steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    rate = 2 * w["Nx"] * w["Nz"] * d["steps"] / d["seconds"]
    return rate, d


# --------------------------------------------------------------------------
# Clock sampling during the timed region.
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sm))


# --------------------------------------------------------------------------
# DRAM bytes (read + write) per launch of the stage kernels: the mean over the
# four stages of one RK443 step captured with ncu (fine: batches of 2 and 32
# slices of 256 x 64, keyed "kernel@batch"; coarse: one slice of 128 x 32; the
# stage-kernel traffic summary in profiles/), valid only while the kernel
# sources are those that were captured.
NCU_TRAFFIC_SOURCES = ("paper_2001_01609_gb300/csrc/rbc_kernels.cu", "paper_2001_01609_gb300/csrc/rbc_internal.h")
NCU_TRAFFIC_SHA256 = "bccf5326cefa87d23c30c873735b605116d20294072d2c0e5a25ffdcbd076c31"
NCU_TRAFFIC = {
    "coarse:k_zinv": 130202, "coarse:k_rows": 483123, "coarse:k_zfwd": 116864, "coarse:k_solve": 826752,
    "fine:k_zinv@32": 8907264, "fine:k_rows@32": 56720845, "fine:k_zfwd@32": 12620800, "fine:k_solve@32": 23538240,
    # batch of 2 with the heuristic shapes (the clustered row kernel; the tuned one-block-per-row
    # kernel reads and writes the same rows)
    "fine:k_zinv@2": 661350, "fine:k_rows@2": 3586304, "fine:k_zfwd@2": 821824, "fine:k_solve@2": 2441088,
}


def ncu_traffic(kernel):
    """Captured DRAM bytes per launch of `kernel`, or None if the sources changed since."""
    import hashlib
    h = hashlib.sha256()
    for f in NCU_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return NCU_TRAFFIC.get(kernel) if h.hexdigest() == NCU_TRAFFIC_SHA256 else None


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank totals over all ranks (the slowest rank times the job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(work_per_rank, world, seconds):
    """Work of all ranks (each rank runs its own problem of the same size) per second."""
    return world * work_per_rank / seconds


def fine_group_starts(N, group, first, n0=0):
    """First slice of each fine group of parareal_iterate's schedule (and N)."""
    a = [n0]
    if group >= N:
        return [n0, N]
    size = first
    while a[-1] < N:
        a.append(min(N, a[-1] + size))
        size = min(group, 2 * size)
    return a


def time_to_tolerance(rbc, w, dv, U0, stream, tol=0.01, max_iters=6, depth=1, reserve_sms=32, arms=None):
    """Parareal to a stated tolerance against the serial all-FP64 fine propagator
    on the same GPU (Sec. 3.7: iterate until Nu_k is within tol of Nu_{k-1}).

    Serial fine: one trajectory, B = 1, all FP64, every slice in turn over
    [0, t_end] (the same kernels), with the Nu_V integral of each slice.
    Parareal arms: mixed precision (fine and coarse propagators: FP32
    transforms and products, FP64 solves, correction and norms; TF32 hi/lo
    operands in the fine grid's tensor-core z transforms; RK443 in both, the
    paper's choice), "mixed_fast" (BF16 hi/lo operands in the fine transforms
    and the coarse propagator on ARS(2,2,2), Sec. 3.6, at the same coarse
    step), and all FP64 (or the given `arms`: (name, fine precision, coarse
    precision, coarse scheme, coarse dt));
    RBC_CRIT_NU with tol, iterations enqueued `depth` ahead, fine groups kept off
    `reserve_sms` SMs (the sweeps on the coarse grid use all of them).  "Equal
    Nu accuracy": each arm's Nu (time mean over the second half of the slices)
    is compared with the serial FP64 one.  Device time with CUDA events on the
    caller's stream, after one untimed warm-up iteration per arm."""
    import torch
    N, nf = w["slices"], w["steps_per_slice"]
    n_half = N // 2
    win = dv["t_end"] * (N - n_half) / N

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, r

    F64 = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nx"], w["Nz"], w["dt"])
    warm = F64.new_states(1)
    warm.copy_(U0[0:1])
    F64.step_batch(warm, 20, stream=stream)
    ser = F64.new_states(1)
    ser.copy_(U0[0:1])
    nu_ser = torch.zeros(N, dtype=torch.float64, device="cuda")

    def serial():
        for n in range(N):
            F64.step_batch(ser, nf, nu_ser[n:n + 1], stream=stream)
    serial_s, _ = timed(serial)
    if F64.check_diverged(stream) != rbc.RBC_OK:
        raise RuntimeError("serial fine run diverged")
    nu_serial = float(nu_ser[n_half:].sum().item()) / win
    out = dict(criterion=f"Nu: |Nu_k - Nu_(k-1)| <= {tol} |Nu_k| (Sec. 3.7, the paper's 1%)",
               serial_fine=dict(precision="fp64", s=serial_s, nu=nu_serial,
                                run=f"B = 1, {N} slices x {nf} steps in turn, same kernels"),
               arms={})
    pname = {rbc.RBC_MIXED: "mixed", rbc.RBC_MIXED_BF16: "mixed_bf16", rbc.RBC_FP64: "fp64"}
    sname = {rbc.RBC_RK443: "RK443", rbc.RBC_RK222: "RK222", rbc.RBC_RK111: "RK111"}
    if arms is None:
        arms = (("mixed", rbc.RBC_MIXED, rbc.RBC_MIXED, rbc.RBC_RK443, dv["dtc"]),
                ("mixed_fast", rbc.RBC_MIXED_BF16, rbc.RBC_MIXED, rbc.RBC_RK222, dv["dtc"]),
                ("fp64", rbc.RBC_FP64, rbc.RBC_FP64, rbc.RBC_RK443, dv["dtc"]))
    for name, pf, pg, scheme, dtc in arms:
        F = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nx"], w["Nz"], w["dt"], precision=pf)
        G = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nxc"], w["Nzc"], dtc, precision=pg, scheme=scheme)
        P = rbc.Parareal(F, G, 0.0, dv["t_end"], N, rbc.CRIT_NU, tol)
        P.set_depth(depth)
        group = -(-N // 4)
        first = -(-group // 4)
        P.set_schedule(group, first, 2, 1, reserve_sms)
        starts = fine_group_starts(N, group, first)
        for Bg in sorted({b - a for a, b in zip(starts, starts[1:])}):
            F.autotune(Bg)
        G.autotune(1)
        U = F.new_states(N + 1)
        P.iterate(U0[0], U, 1, stream=stream)                      # warm-up: graphs, workspaces
        el, (st, k, de, nus) = timed(lambda: P.iterate(U0[0], U, max_iters, stream=stream))
        nu = float(nus[-1]) if len(nus) else float("nan")
        out["arms"][name] = dict(
            fine_precision=pname[pf], coarse_precision=pname[pg], coarse_scheme=sname[scheme], coarse_dt=dtc,
            status={rbc.RBC_OK: "tolerance met", rbc.RBC_ENOTCONVERGED: "not converged",
                    rbc.RBC_EDIVERGED: "diverged"}.get(st, str(st)),
            iterations=int(k), s=el, speedup_vs_serial_fp64=serial_s / el, defects=[float(x) for x in de],
            nus=[float(x) for x in nus], nu=nu, nu_rel_err_vs_serial_fp64=abs(nu - nu_serial) / abs(nu_serial),
            equal_nu_accuracy=bool(abs(nu - nu_serial) <= tol * abs(nu_serial)), depth=depth,
            reserve_sms=P.coarse_sms)
        del P, F, G, U
    return out


def run_gb300(args, w):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, d = cpu_oracle_rate(w)       # before any CUDA work in this process
        cpu = dict(value=rate, unit=UNIT, cores=1, kind="oracle",
                   sample=f"oracle fine propagator, one slice, {d['steps']} RK443 steps of the "
                          f"{w['Nx']}x{w['Nz']} grid in {d['seconds']:.1f} s on one host thread")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2001_01609_gb300 import build
    if local == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature

    dv = derived(w)
    F = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nx"], w["Nz"], w["dt"])
    G = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nxc"], w["Nzc"], dv["dtc"])
    N = w["slices"]
    P = rbc.Parareal(F, G, 0.0, dv["t_end"], N)
    group = args.group if args.group else -(-N // 4)
    first = args.first_group if args.first_group else (group if group >= N else -(-group // 4))
    P.set_schedule(group, first, args.fine_streams, args.coarse_priority, args.coarse_sms)
    stream = torch.cuda.current_stream()
    # launch shapes of the batch sizes the schedule uses, picked on the device
    # (the results do not depend on them)
    starts0 = fine_group_starts(N, group, first)
    tuned = {}
    for Bg in sorted({b - a for a, b in zip(starts0, starts0[1:])}):
        tuned[f"fine_B{Bg}"] = F.autotune(Bg) + (F.tuned_shapes(Bg),)
    tuned["coarse_B1"] = G.autotune(1) + (G.tuned_shapes(1),)
    U0 = F.new_states(1)
    Th = initial_temperature(w["Nx"], w["Nz"], seed=w["seed"] + rank, Lx=w["Lx"])
    F.set_state(U0[0], Th)
    U = F.new_states(N + 1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)

    def one_step():
        st, k, de, nu = P.iterate(U0[0], U, 1)
        if st == rbc.RBC_EDIVERGED:
            raise RuntimeError("diverged")
        return de, nu

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # Timed steps.  Each step: H2D of the initial state from pinned host memory,
    # [device-timed: one Parareal iteration], D2H of the last slice state.
    # value uses the device-timed part (inputs resident); e2e the whole.
    U0h = U0.cpu().pin_memory()
    outh = torch.empty_like(U[N], device="cpu").pin_memory()
    clocks = Clocks(torch.cuda.current_device())
    times, e2e_times = [], []
    launches0 = rbc.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for si in range(args.steps):
        flush.zero_()                                         # L2 flush between timed steps
        torch.cuda.synchronize()
        # sampled kernel timing: the first 8 RK443 steps of the step's first coarse
        # call and of its first fine group are recorded kernel by kernel, on
        # their own streams; everything else runs on the graph loops
        G.profile(True, sample=True)
        F.profile(True, sample=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        U0.copy_(U0h, non_blocking=True)
        e0.record(stream)
        de, nu = one_step()
        e1.record(stream)
        outh.copy_(U[N], non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    prof_f = F.profile_read()
    prof_g = G.profile_read()
    F.profile(False)
    G.profile(False)
    ck = clocks.stop()
    gpu_launches = rbc.launch_count() - launches0
    # The batched fine propagator at the full batch (all slices in one launch):
    # per-kernel CUDA-event times of 2 RK443 steps of the 32 fine states, with
    # the library's algorithmic FP64 flops and bytes, against the FP64 peak and
    # the measured HBM copy rate.
    Fb = F.new_states(N)
    Fb.copy_(U[:N])
    F.step_batch(Fb, 1, stream=stream)
    F.profile(True)
    F.step_batch(Fb, 2, stream=stream)
    pb = F.profile_read()
    F.profile(False)
    hbm = measured_hbm_gbs()
    fine_batch = {}
    for kname, v in pb.items():
        if v["launches"]:
            sec = v["ms"] / 1e3
            fine_batch[kname] = dict(us_per_launch=1e6 * sec / v["launches"], fp64_tflops=v["flops"] / sec / 1e12,
                                     frac_fp64_peak=v["flops"] / sec / 1e12 / (152 * 4 * 2070e6 / 1e12),
                                     algorithmic_gbs=v["bytes"] / sec / 1e9, frac_hbm=v["bytes"] / sec / 1e9 / hbm)
    del Fb
    # Time to tolerance (after the timed region): Parareal iterated until the
    # Nu criterion holds, against the serial all-FP64 fine run on this GPU.
    ttt = None if args.no_time_to_tol else time_to_tolerance(rbc, w, dv, U0, stream)
    # Serving leg (the metric's p50/p99): a short stream of requests of the serving mix
    srv = None
    if not args.no_serving and rank == 0:
        sl = serve(args, "serving_leg", SERVING_LEG, cpu_leg=False, warmup=1)
        srv = dict(requests=sl["config"]["requests"], latency_s=sl["latency"], requests_per_s=sl["requests_per_s"],
                   dof_steps_per_s=sl["value"], offered_load=sl["config"]["offered_load"],
                   peak_active_requests=sl["config"]["peak_active_requests"], failed=sl["failed"],
                   classes=sorted(sl["config"]["classes"]),
                   note="Poisson arrivals of the serving mix (Ra log-uniform 1e4..1e8, grids by the N_BL rule, "
                        "4-64 slices, FP64 or mixed), 10 fine steps per slice, 2 iterations; the full 256-request "
                        "run is --workload rbc_serving_256req_poisson")
    # Sec. 2.2 diagnostics of all fine states (one rbc_diagnostics call), after the timed region
    dout = F.diagnostics(U[:N])
    for _ in range(3):
        F.diagnostics(U[:N], out=dout)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(10):
        F.diagnostics(U[:N], out=dout)
    d1.record(stream)
    torch.cuda.synchronize()
    diag_s = d0.elapsed_time(d1) / 1e3 / 10
    Mz, nm = 3 * w["Nz"] // 2, w["Nx"] // 2
    diag_flops = N * (24.0 * ((Mz + 1) // 2) * nm * w["Nz"] + 20.0 * Mz * nm)
    if world > 1:
        dist.barrier()
    t_total, e2e_total = max_over_ranks([sum(times), sum(e2e_times)], world, "cuda")
    fine_dof_steps = N * w["steps_per_slice"] * dv["dof"]
    value = whole_job_rate(fine_dof_steps * args.steps, world, t_total)
    e2e_value = whole_job_rate(fine_dof_steps * args.steps, world, e2e_total)

    # Per-kernel time over the timed steps, from the samples (8 steps each of
    # one coarse call and one fine group): mean time per launch times the
    # known launch count.  Fine: groups of `group` slices,
    # nf steps each, 4 stages per step; coarse: (2N - 1) nc steps per iteration
    # (the correction sweep reuses G(U_0)), 4 stages per step.
    # The fine groups differ in size: the sample (the first group, `first`
    # slices) gives a time per launch and slice, scaled to all N slices.
    kern = {}
    starts = fine_group_starts(N, group, first)
    f_launches = 4 * (len(starts) - 1) * w["steps_per_slice"] * args.steps
    f_slice_launches = 4 * N * w["steps_per_slice"] * args.steps
    b0 = starts[1] - starts[0]
    for k, v in prof_f.items():
        if v["launches"]:
            per = v["ms"] / v["launches"]
            kern["fine:" + k] = dict(ms=per / b0 * f_slice_launches, launches=f_launches, per_ms=per,
                                     flops_per=v["flops"] / v["launches"], bytes_per=v["bytes"] / v["launches"],
                                     sampled_launches=v["launches"], sampled_batch=b0)
    g_launches = 4 * (2 * N - 1) * dv["nc"] * args.steps
    for k, v in prof_g.items():
        if v["launches"]:
            per = v["ms"] / v["launches"]
            kern["coarse:" + k] = dict(ms=per * g_launches, launches=g_launches, per_ms=per,
                                       flops_per=v["flops"] / v["launches"], bytes_per=v["bytes"] / v["launches"],
                                       sampled_launches=v["launches"])
    dom = max(kern, key=lambda k: kern[k]["ms"])
    pk = kern[dom]
    # FP64 work is bound by the FP64 pipe: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz
    peak_fp64 = 152 * 4 * 2070e6 / 1e12
    achieved = pk["flops_per"] / (pk["per_ms"] / 1e3) / 1e12
    total_ms = sum(v["ms"] for v in kern.values())
    # the fine kernels are captured at 32 slices; a sampled fine group of another size has no figure
    # captured per launch at the batch sizes sampled here (coarse: one slice; fine: the first group)
    traffic = ncu_traffic(dom if dom.startswith("coarse:") else f"{dom}@{kern[dom].get('sampled_batch')}")
    roofline = dict(bound="alu", achieved=achieved, peak=peak_fp64, unit="TFLOP/s", frac=achieved / peak_fp64,
                    traffic=traffic, traffic_source="ncu, one RK443 step, cold cache (profiles/)", kernel=dom, peak_source="derived: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz",
                    launch_us=1e3 * pk["per_ms"], flops_per_launch=pk["flops_per"],
                    algorithmic_bytes_per_launch=pk["bytes_per"],
                    kernel_share={k: v["ms"] / total_ms for k, v in kern.items()},
                    kernel_launch_us={k: 1e3 * v["per_ms"] for k, v in kern.items()})
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=1e3 * t_total / args.steps, higher_is_better=True, scaling="weak",
                    vs_baseline=None, dtype="f64", data="synthetic",
                    config=dict(workload=args.workload, Ra=w["Ra"], grid=f"{w['Nx']}x{w['Nz']}",
                                coarse_grid=f"{w['Nxc']}x{w['Nzc']}", slices=N,
                                fine_steps_per_slice=w["steps_per_slice"], coarse_steps_per_slice=dv["nc"],
                                dt=w["dt"], dt_coarse=dv["dtc"], t_end=dv["t_end"], dof_per_slice=dv["dof"],
                                step="one Parareal iteration (coarse sweep, batched fine sweep, correction, norms)",
                                fine_group=group, first_fine_group=first, fine_streams=args.fine_streams,
                                coarse_priority=args.coarse_priority, coarse_sms=P.coarse_sms,
                                schedule=("serial order: coarse sweep, one batched fine sweep, correction sweep"
                                          if group >= N else
                                          "coarse sweep, fine groups and correction sweep overlapped on 3 streams"),
                                l2="flushed between timed steps (256 MB write)",
                                autotune={k: dict(heuristic_ms_per_step=v[0], tuned_ms_per_step=v[1],
                                                  shapes_solve_zfwd_tm_zfwd_nch_rows_cl_rows_threads_rows_lean=list(v[2]))
                                          for k, v in tuned.items()},
                                parallelism=f"{world} independent problems" if world > 1 else "single GPU"),
                    e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=int(U0h.numel() * 8),
                             d2h_bytes_per_step=int(outh.numel() * 8)),
                    gpu_launches=int(gpu_launches), roofline=roofline, cpu_baseline=cpu, clocks=ck,
                    defect=float(de[-1]) if len(de) else None, nu=float(nu[-1]) if len(nu) else None,
                    diagnostics=dict(states=N, us_per_call=1e6 * diag_s, flops_per_call=diag_flops,
                                     tflops=diag_flops / diag_s / 1e12,
                                     frac_fp64=diag_flops / diag_s / 1e12 / peak_fp64,
                                     note="rbc_diagnostics (Sec. 2.2 averages) of all slices' fine states, "
                                          "FP64 z inverse plus Parseval and Clenshaw-Curtis reductions"),
                    time_to_tol=ttt, serving=srv,
                    fine_batch_roofline=dict(
                        batch=N, kernels=fine_batch, hbm_peak_gbs=hbm,
                        note="one launch per kernel covers all 32 fine slices; FP64 peak derived "
                             "(152 SMs x 4 flop/clk x 2070 MHz), HBM of measured; the batch's working "
                             "set stays in L2, so the FP64 pipe, not HBM, bounds these kernels"))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# Reference arm: the oracle's Parareal on all host cores (the fine solves of
# the slices in a process pool, as the paper runs one slice per processor),
# one iteration per step on a bounded sample of the workload.
# --------------------------------------------------------------------------
CPU_PARAREAL_SNIPPET = r"""
import json, multiprocessing as mp, os, sys, time
sys.path.insert(0, {root!r})
w, nf, nc, iters, cores = {w!r}, {nf}, {nc}, {iters}, {cores}

def make(Nx, Nz, dt):
    from oracle.rbc import RBC
    return RBC(w["Ra"], w["Pr"], w["Lx"], Nx, Nz, dt)

def init():
    global FINE
    FINE = make(w["Nx"], w["Nz"], w["dt"])

def fine(U):
    return FINE.run(U, nf)

if __name__ == "__main__":
    from oracle.rbc import prolong, restrict
    from paper_2001_01609_gb300.inputs import initial_temperature
    N = w["slices"]
    F = make(w["Nx"], w["Nz"], w["dt"])
    G = make(w["Nxc"], w["Nzc"], w["dtc"])
    def coarse(U):
        return prolong(G.run(restrict(U, w["Nxc"], w["Nzc"]), nc)[0], w["Nx"], w["Nz"])
    U0 = F.from_grid(initial_temperature(w["Nx"], w["Nz"], seed=w["seed"], Lx=w["Lx"]))
    ctx = mp.get_context("spawn")
    out = []
    with ctx.Pool(cores, initializer=init) as pool:
        pool.map(fine, [U0] * cores)                     # workers up
        for it in range(iters):
            t0 = time.perf_counter()
            U, Gold = [U0], []
            for n in range(N):                           # U^0: serial coarse sweep
                Gold.append(coarse(U[n]))
                U.append(Gold[-1])
            Fres = pool.map(fine, U[:N])                 # fine sweep, one slice per worker task
            Unew = [U0]
            for n in range(N):                           # correction sweep (Eq. 20)
                g = coarse(Unew[n])
                Unew.append(Fres[n][0] + (g - Gold[n]))
            out.append(time.perf_counter() - t0)
    print(json.dumps(dict(seconds=out)))
"""


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def cpu_model():
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def run_reference(args, w):
    """The oracle's Parareal iteration on all host cores, per step: the coarse
    sweep U^0, the fine solves of all slices in a process pool, the correction
    sweep; a bounded sample of the workload (the slice count and grids kept,
    10 fine and 8 coarse steps per slice: the workload's 3125 : 2500 ratio)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dv = derived(w)
    cores = os.cpu_count() or 1
    nf = 10
    nc = max(1, int(round(nf * dv["nc"] / w["steps_per_slice"])))
    wd = dict(w, dtc=dv["dtc"])
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = CPU_PARAREAL_SNIPPET.format(root=ROOT, w=wd, nf=nf, nc=nc, iters=args.warmup + args.steps, cores=cores)
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:          # spawned workers import the script by path
        script = os.path.join(tmp, "oracle_parareal.py")
        with open(script, "w") as fh:
            fh.write(code)
        r = subprocess.run([sys.executable, script], capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError("oracle Parareal failed: " + r.stderr[-2000:])
    secs = json.loads(r.stdout.strip().splitlines()[-1])["seconds"][args.warmup:]
    total_s = sum(secs)
    fine_dof_steps = w["slices"] * nf * dv["dof"]
    value = fine_dof_steps * args.steps / total_s
    sample = (f"per step: one oracle Parareal iteration of {w['slices']} slices ({w['Nx']}x{w['Nz']} fine, "
              f"{w['Nxc']}x{w['Nzc']} coarse), {nf} fine and {nc} coarse steps per slice, fine solves in a "
              f"pool of {cores} processes, coarse sweeps serial; CPU: {cpu_model()}")
    cpu = dict(value=value, unit=UNIT, cores=cores, kind="oracle", sample=sample)
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=int(os.environ.get("WORLD_SIZE", "1")),
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * total_s / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, Ra=w["Ra"], grid=f"{w['Nx']}x{w['Nz']}",
                            coarse_grid=f"{w['Nxc']}x{w['Nzc']}", slices=w["slices"], dt=w["dt"],
                            dt_coarse=dv["dtc"], fine_steps_per_slice_sampled=nf,
                            coarse_steps_per_slice_sampled=nc,
                            step="one Parareal iteration (coarse sweep, fine sweep on all cores, correction)"),
                cpu_baseline=cpu, e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# Serving: many Parareal requests on one GPU (continuous batching).
SERVING = {
    "rbc_serving_256req_poisson": dict(requests=256, seed=4, fine_steps=10, coarse_ratio=2, max_iters=2,
                                       f_chunk=10, load=0.8),
}
# the serving leg of the default bench line: the same request mix, fewer requests
SERVING_LEG = dict(requests=24, seed=4, fine_steps=10, coarse_ratio=2, max_iters=2, f_chunk=10, load=0.8)


def run_serving(args, name):
    print(json.dumps(serve(args, name, SERVING[name], cpu_leg=not args.no_cpu_baseline, warmup=args.warmup)),
          flush=True)


def serve(args, name, cfgw, cpu_leg=True, warmup=1):
    """`requests` requests, Poisson arrivals at `load` x the calibrated capacity; Ra
    log-uniform in [1e4, 1e8], a grid drawn among those with >= 6 points in the
    thermal boundary layer, 4-64 slices, FP64 or mixed precision with p = 1/2,
    `fine_steps` fine steps per slice and 2 Parareal iterations per request.
    Returns the JSON line (a dict)."""
    import torch
    cpu = None
    if cpu_leg:
        w0 = dict(Ra=1e4, Pr=1.0, Lx=2.0, Nx=64, Nz=32, dt=3.125e-5, seed=0)
        rate, d = cpu_oracle_rate(w0)
        cpu = dict(value=rate, unit=UNIT, cores=1, kind="oracle",
                   sample=f"oracle fine propagator on the smallest serving grid (64x32), {d['steps']} RK443 "
                          f"steps in {d['seconds']:.1f} s on one host thread")
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc, serving
    from paper_2001_01609_gb300.inputs import initial_temperature

    def class_config(Nx, Nz, precision):
        return serving.default_class_config(Nx, Nz, precision, fine_steps=cfgw["fine_steps"],
                                            coarse_ratio=cfgw["coarse_ratio"])

    eng = serving.Engine(max_iters=cfgw["max_iters"], f_chunk=cfgw["f_chunk"], class_config=class_config)
    reqs = serving.make_requests(cfgw["requests"], cfgw["seed"], rate=1.0)
    # initial states on the host, pinned: each request's H2D copy is inside the timed run
    for r in reqs:
        cls = eng._class(r.key)
        u = cls.fine.new_states(1)
        cls.fine.set_state(u[0], initial_temperature(r.Nx, r.Nz, r.seed))
        r.U0 = u[0].cpu().pin_memory()
    # capacity: per-class fine cost per slice-step (batch of 32) and coarse cost per step (batch of 1)
    cost = {}
    for key, cls in eng.classes.items():
        B = 32
        st = cls.fine.new_states(B)
        st.copy_(reqs[[r.key for r in reqs].index(key)].U0.cuda().expand_as(st))
        cls.fine.step_batch(st, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cls.fine.step_batch(st, 4)
        torch.cuda.synchronize()
        tf = (time.perf_counter() - t0) / 4 / B
        c = cls.coarse.new_states(1)
        rbc.restrict(cls.fine, cls.coarse, st[:1], c)
        cls.coarse.step_batch(c, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cls.coarse.step_batch(c, 4)
        torch.cuda.synchronize()
        cost[key] = (tf, (time.perf_counter() - t0) / 4)
    work = []
    for r in reqs:
        cf = eng.config_for(r.key)
        tf, tc = cost[r.key]
        sweeps = cfgw["max_iters"] + 1
        work.append(sum(r.nslices - (k - 1) for k in range(1, cfgw["max_iters"] + 1)) * cf.nf * tf
                    + sweeps * r.nslices * cf.nc * tc)
    capacity = len(reqs) / sum(work)
    rate = cfgw["load"] * capacity
    g = np.random.Generator(np.random.PCG64(cfgw["seed"] + 1000))
    t = 0.0
    for r in reqs:
        t += g.exponential(1.0 / rate)
        r.arrival = t
    # warm-up: one request per class, arriving at once (graph captures, lazy setup)
    for _ in range(max(1, warmup)):
        seen, warm = set(), []
        for r in reqs:
            if r.key not in seen:
                seen.add(r.key)
                warm.append(serving.Request(rid=-1 - len(warm), Ra=r.Ra, Nx=r.Nx, Nz=r.Nz, nslices=4,
                                            precision=r.precision, U0=r.U0))
        eng.run(warm, deadline=600)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    launches0 = rbc.launch_count()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    eng.run(reqs, deadline=3600)
    torch.cuda.synchronize()
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    makespan = e0.elapsed_time(e1) / 1e3
    launches = rbc.launch_count() - launches0
    dof = serving.dof_steps(reqs, eng)
    lat = serving.latency_stats(reqs)
    bad = [r.rid for r in reqs if r.status != rbc.RBC_OK]
    value = dof / makespan
    h2d = sum(r.U0.numel() * 8 for r in reqs)
    d2h = sum((2 * (r.nslices + 1) + r.nslices * -(-eng.config_for(r.key).nf // cfgw["f_chunk"])) * 8 * r.k_done
              for r in reqs)
    classes = {f"{k[0]}x{k[1]}/{'mixed' if k[2] else 'fp64'}": dict(
        requests=sum(1 for r in reqs if r.key == k), dt=eng.config_for(k).dt_fine,
        dt_coarse=eng.config_for(k).dt_coarse, fine_ms_per_slice_step=1e3 * cost[k][0],
        coarse_ms_per_step=1e3 * cost[k][1]) for k in eng.classes}
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=1, steps=1, warmup=max(1, warmup),
                ms_per_step=1e3 * makespan, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64+mixed", data="synthetic",
                config=dict(workload=name, requests=len(reqs), seed=cfgw["seed"], arrivals="Poisson",
                            rate_per_s=rate, offered_load=cfgw["load"], capacity_per_s=capacity,
                            fine_steps_per_slice=cfgw["fine_steps"], coarse_ratio=cfgw["coarse_ratio"],
                            parareal_iterations=cfgw["max_iters"], fine_chunk=cfgw["f_chunk"],
                            mem_limit_bytes=eng.mem_limit, peak_committed_bytes=eng.peak_committed,
                            peak_active_requests=eng.peak_active, classes=classes,
                            step="the whole request stream, arrival of the first to completion of the last",
                            l2="working set of each class batch exceeds L2 for the large grids"),
                latency=lat, requests_per_s=len(reqs) / makespan, failed=bad,
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h)),
                gpu_launches=int(launches), roofline=None, cpu_baseline=cpu, clocks=ck)
    eng.close()
    return line


NCU_CASES = {
    # name: (Ra, Nx, Nz, dt, B) -- one RK443 step without graphs, for ncu captures
    "fine_b32": (1e6, 256, 64, 1.25e-5, 32),
    "fine_b2": (1e6, 256, 64, 1.25e-5, 2),       # the first fine group of the Parareal schedule
    "coarse_b1": (1e6, 128, 32, 1.5625e-5, 1),
    "parareal_small": None,   # one Parareal iteration, see run_ncu_case
    "mixed_b8": (1e7, 512, 128, 7.8125e-7, 8),   # RBC_MIXED: tensor-core z transforms
    "mixed_b32": (1e6, 256, 64, 1.25e-5, 32),    # RBC_MIXED fine batch of the Parareal workload
    "mixed_coarse_b1": (1e6, 128, 32, 1.5625e-5, 1),   # RBC_MIXED coarse slice (CUDA-core FP32 transforms)
}


# Coarsening and slice-count study (Sec. 3.6; Fig. 9 plots speedup against the
# number of slices): the 256 x 64, Ra 1e6 fine propagator over a tenth of the
# Parareal workload's horizon, with coarse propagators coarsened in space
# (CF 2, 4, 8) and in time, for several slice counts; iteration time, defects
# and final error against the serial fine run on the same GPU.
STUDY = dict(Ra=1e6, Pr=1.0, Lx=2.0, Nx=256, Nz=64, dt=1.25e-5, total_steps=9600, seed=1, iters=4,
             slices=(8, 16, 32), coarse=((128, 32, 1.5625e-5), (64, 16, 1.5625e-5), (64, 16, 3.125e-5)))


def run_coarsening_study(coarse=None, slices=None):
    import torch
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature
    s = STUDY
    F = rbc.Propagator(s["Ra"], s["Pr"], s["Lx"], s["Nx"], s["Nz"], s["dt"])
    U0 = F.new_states(1)
    F.set_state(U0[0], initial_temperature(s["Nx"], s["Nz"], seed=s["seed"], Lx=s["Lx"]))
    T = s["total_steps"] * s["dt"]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ser = F.new_states(1)
    ser.copy_(U0)
    F.step_batch(ser, 20)                                  # graphs for B = 1
    ser.copy_(U0)
    e0.record(stream)
    F.step_batch(ser, s["total_steps"])
    e1.record(stream)
    torch.cuda.synchronize()
    serial_s = e0.elapsed_time(e1) / 1e3
    nrm = torch.zeros(2, dtype=torch.float64, device="cuda")

    def finite(x):
        return float(x) if math.isfinite(float(x)) else None

    rows = []
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for Nxc, Nzc, dtc in (coarse or s["coarse"]):
        G = rbc.Propagator(s["Ra"], s["Pr"], s["Lx"], Nxc, Nzc, dtc)
        for N in (slices or s["slices"]):
            P = rbc.Parareal(F, G, 0.0, T, N)
            U = F.new_states(N + 1)
            e0.record(stream)
            st, k, de, _ = P.iterate(U0[0], U, min(s["iters"], N))
            e1.record(stream)
            torch.cuda.synchronize()
            el = e0.elapsed_time(e1) / 1e3
            rbc.l2_diff(F, U[N:N + 1], ser, nrm[0:1])
            rbc.l2_diff(F, ser, None, nrm[1:2])
            a, b = nrm.cpu().tolist()
            err = math.sqrt(a / b) if math.isfinite(a) and b > 0 else None
            rows.append(dict(coarse_grid=f"{Nxc}x{Nzc}", coarse_dt=dtc, slices=N,
                             fine_steps_per_slice=s["total_steps"] // N,
                             coarse_steps_per_slice=int(round(T / N / dtc)), iterations=k, status=st,
                             seconds=el, seconds_per_iteration=el / max(k, 1),
                             defects=[finite(x) for x in de], final_error_vs_serial=err,
                             speedup_vs_serial_fine=serial_s / el))
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            P.close()
        G.close()
    ck = clocks.stop()
    print(json.dumps(dict(study="parareal_coarsening_and_slices", Ra=s["Ra"], grid=f"{s['Nx']}x{s['Nz']}",
                          dt=s["dt"], t_end=T, total_fine_steps=s["total_steps"], serial_fine_s=serial_s,
                          iterations_max=s["iters"], clocks=ck, rows=rows)), flush=True)


def run_statistics_study():
    """Parareal with the Sec. 2.2 statistics sampled along every fine sweep and
    the statistical stopping rule (RBC_CRIT_STAT), against the same Parareal
    without sampling, on the study's fine grid: 16 slices of 600 fine steps,
    CF 2 coarse propagator."""
    import torch
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature
    s = STUDY
    N, every, K = 16, 50, 3
    Nxc, Nzc, dtc = s["coarse"][0]
    F = rbc.Propagator(s["Ra"], s["Pr"], s["Lx"], s["Nx"], s["Nz"], s["dt"])
    G = rbc.Propagator(s["Ra"], s["Pr"], s["Lx"], Nxc, Nzc, dtc)
    U0 = F.new_states(1)
    F.set_state(U0[0], initial_temperature(s["Nx"], s["Nz"], seed=s["seed"], Lx=s["Lx"]))
    T = s["total_steps"] * s["dt"]
    P = rbc.Parareal(F, G, 0.0, T, N, rbc.CRIT_STAT, 1e-2)
    P.set_sampling(every)
    U = F.new_states(N + 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_s, k_s, de_s, _ = P.iterate(U0[0], U, K)
    torch.cuda.synchronize()
    t_stat = time.perf_counter() - t0
    summary = rbc.stat_summary(s["Nz"], s["Ra"], s["Pr"], P.stat_means())
    L = rbc.Parareal(F, G, 0.0, T, N)
    U2 = F.new_states(N + 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, k, de, nus = L.iterate(U0[0], U2, k_s)
    torch.cuda.synchronize()
    t_lib = time.perf_counter() - t0
    keep = ("NuV", "Nub", "Nut", "Re", "P", "eps_U", "Nu_int", "balance", "delta_T", "N_BL", "delta_t")
    print(json.dumps(dict(study="statistical_parareal", grid=f"{s['Nx']}x{s['Nz']}", coarse_grid=f"{Nxc}x{Nzc}",
                          Ra=s["Ra"], slices=N, fine_steps_per_slice=s["total_steps"] // N, sample_every=every,
                          criterion="stat", tol=1e-2, status=st_s, iterations=k_s,
                          defects=list(map(float, de_s)), stats_at_stop={q: summary[q] for q in keep},
                          seconds=t_stat,
                          unsampled_parareal=dict(iterations=k, seconds=t_lib, defects=list(map(float, de))),
                          same_iterates_as_unsampled=bool(torch.equal(U, U2)))), flush=True)


def run_config3_study():
    """Config 3 (Ra 1e8, 1024 x 256, 128 slices, mixed precision, Nu criterion):
    the transient on 128 x 64, which survives it (t = 0.004, reading R24), is
    prolonged to 1024 x 256; then mixed-precision Parareal to the 1% Nu
    criterion against the serial all-FP64 fine run on the same GPU, over 40
    fine steps of 7.8125e-8 per slice (coarse 256 x 64, 20 steps of 1.5625e-7):
    TF32 or BF16 fine operands with the RK443 coarse propagator, and BF16 with
    the ARS(2,2,2) coarse propagator."""
    import torch
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature
    Ra, N, nf, nc, dtf, dtc = 1e8, 128, 40, 20, 7.8125e-8, 1.5625e-7
    D = rbc.Propagator(Ra, 1.0, 2.0, 128, 64, 1.5625e-7, precision=rbc.RBC_MIXED)
    x = D.new_states(1)
    D.set_state(x[0], initial_temperature(128, 64, seed=3))
    D.step_batch(x, 25600)
    if D.check_diverged() != rbc.RBC_OK:
        raise RuntimeError("the 128 x 64 transient diverged")
    F = rbc.Propagator(Ra, 1.0, 2.0, 1024, 256, dtf, precision=rbc.RBC_MIXED)
    G = rbc.Propagator(Ra, 1.0, 2.0, 256, 64, dtc, precision=rbc.RBC_MIXED)
    U0 = F.new_states(1)
    rbc.prolong(F, D, x, U0)
    T = N * nf * dtf

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, r

    F64 = rbc.Propagator(Ra, 1.0, 2.0, 1024, 256, dtf)
    warm = F64.new_states(1)
    warm.copy_(U0)
    F64.step_batch(warm, 3)
    ser = F64.new_states(1)
    ser.copy_(U0)
    nus = torch.zeros(N, dtype=torch.float64, device="cuda")

    def serial():
        for n in range(N):
            F64.step_batch(ser, nf, nus[n:n + 1])
    ts, _ = timed(serial)
    st_s = F64.check_diverged()
    nu_serial = float(nus[N // 2:].sum().item()) / (T / 2)
    arms = {}
    # TF32 fine operands with the RK443 coarse propagator; BF16 fine operands with it; BF16 with
    # the ARS(2,2,2) coarse propagator at the same coarse step (unstable there: it reports
    # RBC_EDIVERGED in the first coarse sweep)
    F16 = rbc.Propagator(Ra, 1.0, 2.0, 1024, 256, dtf, precision=rbc.RBC_MIXED_BF16)
    for name, Fa, Ga in (("parareal_mixed", F, G),
                         ("parareal_mixed_bf16", F16, G),
                         ("parareal_mixed_bf16_rk222_coarse", F16,
                          rbc.Propagator(Ra, 1.0, 2.0, 256, 64, dtc, precision=rbc.RBC_MIXED,
                                         scheme=rbc.RBC_RK222))):
        P = rbc.Parareal(Fa, Ga, 0.0, T, N, rbc.CRIT_NU, 0.01)
        P.set_depth(1)
        P.set_schedule(32, 8, 2, 1, 32)
        for Bg in (8, 16, 32):
            Fa.autotune(Bg)
        Ga.autotune(1)
        U = Fa.new_states(N + 1)
        P.iterate(U0[0], U, 1)
        tp, (st, k, de, nu) = timed(lambda: P.iterate(U0[0], U, 5))
        nu_k = float(nu[-1]) if len(nu) else float("nan")
        arms[name] = dict(s=tp, status=st, iterations=k, defects=list(map(float, de)), nus=list(map(float, nu)),
                          speedup=ts / tp, nu_rel_err=abs(nu_k - nu_serial) / abs(nu_serial))
        P.close()
        del U
    print(json.dumps(dict(study="config3", Ra=Ra, grid="1024x256", coarse_grid="256x64", slices=N,
                          fine_steps_per_slice=nf, dt=dtf, coarse_steps_per_slice=nc, dt_coarse=dtc,
                          start="128x64 transient to t = 0.004 (25600 steps of 1.5625e-7), prolonged",
                          serial_fp64=dict(s=ts, status=st_s, nu=nu_serial), **arms)), flush=True)


COARSE_NC = (625, 1000, 1250, 1600, 2000, 2500, 3125, 4000, 5000, 6250, 8000, 10000, 12500)


def run_coarse_scheme_study():
    """Lower-order coarse steppers (Sec. 3.6) on the Parareal workload (Ra 1e6,
    fine 256 x 64 RK443 with dt 1.25e-5, coarse 128 x 32, 32 slices of 3125
    fine steps).  Per scheme (RK443, RK222, RK111): the largest stable coarse
    step, found by serial coarse runs over the whole horizon from the restricted
    initial state (mixed precision, dt = slice length / nc for nc in COARSE_NC,
    largest step first; stable = every slice ends finite with |Nu_V| < 100), the
    coarse step's device time at that step, and Parareal with that coarse
    propagator to the 1% Nu criterion against the serial FP64 fine run."""
    import torch
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature
    w = WORKLOADS[DEFAULT]
    dv = derived(w)
    N = w["slices"]
    stream = torch.cuda.current_stream()
    F = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nx"], w["Nz"], w["dt"], precision=rbc.RBC_MIXED)
    U0 = F.new_states(1)
    F.set_state(U0[0], initial_temperature(w["Nx"], w["Nz"], seed=w["seed"], Lx=w["Lx"]))
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    schemes = (("RK443", rbc.RBC_RK443), ("RK222", rbc.RBC_RK222), ("RK111", rbc.RBC_RK111))
    scan, arms = {}, []
    for name, sc in schemes:
        tried = []
        for nc in COARSE_NC:
            dtc = dv["slice_len"] / nc
            G = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nxc"], w["Nzc"], dtc, precision=rbc.RBC_MIXED,
                               scheme=sc)
            x = G.new_states(1)
            rbc.restrict(F, G, U0, x)
            w0 = x.clone()
            G.step_batch(w0, 10)                               # graphs, untimed
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ok, done = True, 0
            e0.record(stream)
            for n in range(N):
                G.step_batch(x, nc)
                done += 1
                nu = G.nusselt(x[0])[0]
                if G.check_diverged() != rbc.RBC_OK or not math.isfinite(nu) or abs(nu) >= 100.0:
                    ok = False
                    break
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (done * nc)
            tried.append(dict(nc=nc, dt=dtc, stable=ok, slices_run=done, ms_per_step=ms))
            print(json.dumps(dict(scheme=name, **tried[-1])), file=sys.stderr, flush=True)
            G.close()
            if ok:
                arms.append((f"coarse_{name}", rbc.RBC_MIXED, rbc.RBC_MIXED, sc, dtc))
                break
        scan[name] = tried
    res = time_to_tolerance(rbc, w, dv, U0, stream, arms=arms)
    ck = clocks.stop()
    print(json.dumps(dict(study="coarse_schemes", Ra=w["Ra"], grid=f"{w['Nx']}x{w['Nz']}",
                          coarse_grid=f"{w['Nxc']}x{w['Nzc']}", slices=N, dt=w["dt"],
                          fine_steps_per_slice=w["steps_per_slice"], stability_scan=scan, clocks=ck, **res)),
          flush=True)


def run_config2_study():
    """Config 2 (Ra 1e7, 512 x 128, 64 slices, mixed precision): Parareal from the
    seeded IC (the ladder's fine step 7.8125e-7; 100 fine steps per slice, through
    the initial plume burst) with a 256 x 64 coarse propagator (CF 2, twice the
    fine step, 50 steps per slice), to the 1% Nu criterion, against the serial
    all-FP64 fine run on the same GPU; TF32 and BF16 fine operands."""
    import torch
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature
    Ra, N, nf, nc, dtf = 1e7, 64, 100, 50, 7.8125e-7
    dtc = nf * dtf / nc
    T = N * nf * dtf

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, r

    F64 = rbc.Propagator(Ra, 1.0, 2.0, 512, 128, dtf)
    U0 = F64.new_states(1)
    F64.set_state(U0[0], initial_temperature(512, 128, seed=2))
    warm = U0.clone()
    F64.step_batch(warm, 3)
    ser = U0.clone()
    nus = torch.zeros(N, dtype=torch.float64, device="cuda")

    def serial():
        for n in range(N):
            F64.step_batch(ser, nf, nus[n:n + 1])
    ts, _ = timed(serial)
    st_s = F64.check_diverged()
    nu_serial = float(nus[N // 2:].sum().item()) / (T / 2)
    arms = {}
    for name, prec in (("parareal_mixed", rbc.RBC_MIXED), ("parareal_mixed_bf16", rbc.RBC_MIXED_BF16)):
        F = rbc.Propagator(Ra, 1.0, 2.0, 512, 128, dtf, precision=prec)
        G = rbc.Propagator(Ra, 1.0, 2.0, 256, 64, dtc, precision=rbc.RBC_MIXED)
        P = rbc.Parareal(F, G, 0.0, T, N, rbc.CRIT_NU, 0.01)
        P.set_depth(1)
        P.set_schedule(16, 4, 2, 1, 32)
        for Bg in (4, 8, 16):
            F.autotune(Bg)
        G.autotune(1)
        U = F.new_states(N + 1)
        P.iterate(U0[0], U, 1)
        tp, (st, k, de, nu) = timed(lambda: P.iterate(U0[0], U, 6))
        nu_k = float(nu[-1]) if len(nu) else float("nan")
        arms[name] = dict(s=tp, status=st, iterations=k, defects=list(map(float, de)), nus=list(map(float, nu)),
                          speedup=ts / tp, nu_rel_err=abs(nu_k - nu_serial) / abs(nu_serial))
        P.close()
        del U, F, G
    print(json.dumps(dict(study="config2", Ra=Ra, grid="512x128", coarse_grid="256x64", slices=N,
                          fine_steps_per_slice=nf, dt=dtf, coarse_steps_per_slice=nc, dt_coarse=dtc,
                          start="seeded IC (config 2)", serial_fp64=dict(s=ts, status=st_s, nu=nu_serial), **arms)),
          flush=True)


def run_ncu_case(name):
    """A small, self-ending case for ncu: one plain (graph-free) RK443 step of a
    batch, or one short Parareal iteration on the bench's grids."""
    import torch
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature
    if name == "parareal_small":
        # the Parareal workload's grids and time steps, 8 slices of 25 fine / 20 coarse steps
        # (the coarse-to-fine step ratio of the bench workload); every kernel
        # launched from the host, so that a profiler sees each one
        w = WORKLOADS[DEFAULT]
        N, nf, nc = 8, 25, 20
        F = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nx"], w["Nz"], w["dt"], eager=True)
        G = rbc.Propagator(w["Ra"], w["Pr"], w["Lx"], w["Nxc"], w["Nzc"], nf * w["dt"] / nc, eager=True)
        P = rbc.Parareal(F, G, 0.0, N * nf * w["dt"], N)
        u0 = F.new_states(1)
        F.set_state(u0[0], initial_temperature(w["Nx"], w["Nz"], seed=w["seed"], Lx=w["Lx"]))
        U = F.new_states(N + 1)
        st, k, _, _ = P.iterate(u0[0], U, 1)
        torch.cuda.synchronize()
        assert st == rbc.RBC_OK and k == 1
        print(f"ncu case {name} ok")
        return
    Ra, Nx, Nz, dt, B = NCU_CASES[name]
    prec = rbc.RBC_MIXED if name.startswith("mixed") else rbc.RBC_FP64
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, prec, eager=True)
    st = F.new_states(B)
    for b in range(B):
        F.set_state(st[b], initial_temperature(Nx, Nz, seed=b, amplitude=0.3))
    F.step_batch(st, 1)
    torch.cuda.synchronize()
    assert F.check_diverged() == rbc.RBC_OK
    print(f"ncu case {name} ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(SERVING))
    ap.add_argument("--group", type=int, default=0,
                    help="largest fine group (default: a quarter of the slices; the number of slices gives "
                         "one fine batch after the coarse sweep)")
    ap.add_argument("--first-group", type=int, default=0,
                    help="first fine group (default: --group when it covers all slices, else a quarter of it)")
    ap.add_argument("--fine-streams", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--coarse-priority", type=int, default=1, choices=[0, 1])
    ap.add_argument("--coarse-sms", type=int, default=0, help="SMs of the coarse sweeps' own partition (0: shared)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-tol", action="store_true", help="skip the Parareal-to-tolerance runs")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg of the default line")
    ap.add_argument("--ncu-case", choices=sorted(NCU_CASES), help="run one small step for an ncu capture")
    ap.add_argument("--study", choices=["coarsening", "statistics", "config2", "config3", "coarse_schemes"],
                    help="the coarsening and slice-count study, or the statistical Parareal run (not bench lines)")
    ap.add_argument("--study-coarse", default="",
                    help="coarse propagators of the coarsening study, e.g. 32x8:3.125e-5,64x16:1.5625e-5")
    ap.add_argument("--study-slices", default="", help="slice counts of the coarsening study, e.g. 8,32")
    args = ap.parse_args()
    if args.ncu_case:
        run_ncu_case(args.ncu_case)
        return
    if args.study == "coarsening":
        coarse = [(int(g.split(":")[0].split("x")[0]), int(g.split(":")[0].split("x")[1]), float(g.split(":")[1]))
                  for g in args.study_coarse.split(",") if g]
        slices = [int(n) for n in args.study_slices.split(",") if n]
        run_coarsening_study(coarse or None, slices or None)
        return
    if args.study == "statistics":
        run_statistics_study()
        return
    if args.study == "config2":
        run_config2_study()
        return
    if args.study == "config3":
        run_config3_study()
        return
    if args.study == "coarse_schemes":
        run_coarse_scheme_study()
        return
    if args.workload in SERVING:
        if args.impl == "reference":
            print(json.dumps(dict(impl="reference", unavailable="the serving workload has no CPU reference run: "
                                  "the oracle would take hours for 256 requests")), flush=True)
        else:
            run_serving(args, args.workload)
        return
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gb300(args, w)


if __name__ == "__main__":
    main()

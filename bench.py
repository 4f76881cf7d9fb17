"""Benchmark of the consensus-ADMM calibration hot path on GB300.

One step = one full calibration of the LOFAR-shaped batch (62 stations / 1891 baselines,
5 directions of 20-source clusters, 32 subbands 115-185 MHz, 10 solution intervals of 10
samples, Bernstein degree 3, rho 10, SNR 10): coherency prediction from the sky model,
a cold start (J = I, Z = Y = 0) and 30 C-ADMM iterations with 10 LM x 4 PCG inner steps.
Metric: visibilities x directions x ADMM iterations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank calibrates its own batch (seed offset by rank): no data-path
collective, weak scaling. --impl reference times the FP64 CPU oracle on a bounded sample,
spread over every host core (one process per core, each calibrating its own subband group).
The default run also measures the batched uneven workload (256 subbands x 10 intervals, K=10,
5/10/20 samples, flagged baselines, 50 iterations) and reports it as the nested "uneven" field.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")  # the CPU oracle legs run on one core

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "lofar_n62_k5"  # the default workload; --workload picks another
N_LM, N_CG = 10, 4
METRICS = {
    "lofar_n62_k5": "ADMM vis*dir*iter/s (LOFAR-shaped: N=62, K=5, 32 subbands, 10 intervals x 10 samples)",
    "uneven_n62_k10": "ADMM vis*dir*iter/s (batched uneven: N=62, K=10, 256 subbands x 10 intervals, "
                      "5/10/20 samples per subband, 0-15 % of baselines flagged)",
}
METRIC = METRICS[WORKLOAD]
UNIT = "vis*dir*iter/s"

# DRAM traffic per launch of each sweep kernel from one ncu capture; valid only for the kernel
# source it was taken on (sha256 prefix of the kernel's .cu file), else reported as null.
NCU_TRAFFIC = {  # dram__bytes_read.sum + dram__bytes_write.sum of one full capture each (summaries in profiles/)
    ("stats_hessvec", "effefc092027"): 82.56e6,
    ("stats_trial", "7102e7ad44aa"): 181.1e6,
    ("stats_pass", "fbe001eb534e"): 592.6e6,
    ("residual", "fbe001eb534e"): 618.7e6,
}
KERNEL_SOURCE = {"sweep_residual": "sweep.cu", "sweep_hessvec": "sweep.cu", "stats_hessvec": "ss_hessvec.cu",
                 "stats_trial": "ss.cu", "stats_pass": "data.cu", "residual": "data.cu"}
# The sufficient-statistics passes do 13-17 real flops per algorithmic byte at K=5, above the FP32
# ridge (~12 flop/B): their roofline is the FP32 pipe. The direct passes are below it (HBM).
ALU_BOUND = {"stats_hessvec", "stats_trial"}
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM (4 sub-partitions x 32)


def peaks(sms: int):
    """(HBM GB/s, FP32 TFLOP/s, how the FP32 peak was derived). FP32 peak = SMs (read from the
    device) x FP32 lanes per SM x 2 flops (FMA) x the maximum SM clock measured on the box."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mp = json.load(fh)
        mhz, hbm, kind = float(mp.get("sm_max_mhz", 2070.0)), float(mp["hbm_gbs"]), "measured"
    except Exception:
        mhz, hbm, kind = 2070.0, 6800.0, "fallback"
    fp32 = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    how = (f"FP32: {sms} SMs (device attribute) x {FP32_LANES_PER_SM} lanes x 2 flops x {mhz:.0f} MHz "
           f"({kind} max SM clock) = {fp32:.1f} TFLOP/s; HBM: {hbm:.1f} GB/s ({kind} copy bandwidth)")
    return hbm, fp32, how


def source_hash(kind: str) -> str:
    with open(os.path.join(ROOT, "paper_1502_00858_gb300", "csrc", KERNEL_SOURCE[kind]), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:12]


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of each rank's value (the slowest rank's time); a collective when world > 1."""
    if world == 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_step_per_rank: float, steps: int, dt_slowest: float) -> float:
    """Whole-job throughput: every rank processes its own batch (weak scaling), the job takes as
    long as the slowest rank."""
    return world * units_per_step_per_rank * steps / dt_slowest


def units(prob) -> float:
    """Unflagged visibilities x directions per ADMM iteration."""
    keep = (prob["flags"] == 0).sum(axis=1)
    return float(np.sum(keep * prob["T"])) * prob["K"]


# ----------------------------------------------------------------------------- CPU oracle legs

ORACLE_FREQS = 4  # subbands per oracle task: one C-ADMM problem of 4 agents


def oracle_task(sub: dict) -> tuple[float, float]:
    """One C-ADMM iteration of the FP64 oracle on one task (runs in a worker process).
    Returns (seconds, vis*dir*iter)."""
    from oracle import admm as O

    t0 = time.perf_counter()
    O.admm(sub, 1, n_lm=N_LM, n_cg=N_CG)
    return time.perf_counter() - t0, units(sub)


def oracle_tasks(prob, n_tasks: int, n_freq: int = ORACLE_FREQS) -> list[dict]:
    """n_tasks sub-problems of the workload: interval iv, subbands [g n_freq, (g+1) n_freq), over
    (iv, g) in order, each a C-ADMM problem with the same per-agent data and LM/PCG schedule."""
    tasks = []
    for iv in range(prob["I"]):
        for g in range(prob["P"] // n_freq):
            if len(tasks) == n_tasks:
                return tasks
            ag = [iv * prob["P"] + g * n_freq + f for f in range(n_freq)]
            fr = slice(g * n_freq, (g + 1) * n_freq)
            tasks.append(dict(N=prob["N"], K=prob["K"], P=n_freq, M=prob["M"], I=1, A=n_freq, pq=prob["pq"],
                              rho=prob["rho"], basis=prob["basis"][fr], freqs=prob["freqs"][fr],
                              V=[np.asarray(prob["V"][a], dtype=np.complex128) for a in ag],
                              C=[np.asarray(prob["C"][a], dtype=np.complex128) for a in ag],
                              flags=prob["flags"][ag], T=prob["T"][ag]))
    return tasks


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        import platform
        return platform.processor() or platform.machine()
    except Exception:
        return "unknown"


class OraclePool:
    """The float64 oracle on every host core: a spawn-started process pool (one worker per core,
    BLAS at one thread each), each worker calibrating its own subband group."""

    def __init__(self, workers: int):
        import multiprocessing as mp

        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers)

    def run(self, tasks) -> tuple[float, float]:
        """Wall seconds and total vis*dir*iter of the tasks, one per worker."""
        t0 = time.perf_counter()
        res = self.pool.map(oracle_task, tasks, chunksize=1)
        return time.perf_counter() - t0, float(sum(u for _, u in res))

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample_text(workers: int, n_tasks: int, P: int, seconds: float) -> str:
    return (f"one C-ADMM iteration (10 LM x 4 PCG) of {n_tasks} tasks run concurrently on {workers} processes, "
            f"each task one solution interval restricted to {ORACLE_FREQS} of its {P} subbands "
            f"({seconds:.1f} s wall per sample); CPU: {cpu_model()}, nproc {cpu_cores()}")


def run_reference(args, world, rank):
    if rank != 0:
        return
    from synth import make_problem

    prob = make_problem(args.workload)
    workers = cpu_cores()
    tasks = oracle_tasks(prob, workers)
    pool = OraclePool(len(tasks))
    for _ in range(args.warmup):
        pool.run(tasks)
    tot_t, tot_u = 0.0, 0.0
    for _ in range(args.steps):
        dt, u = pool.run(tasks)
        tot_t += dt
        tot_u += u
    pool.close()
    value = tot_u / tot_t
    sample = oracle_sample_text(len(tasks), len(tasks), prob["P"], tot_t / args.steps) + ", per step"
    print(json.dumps({
        "impl": "reference", "metric": METRICS[args.workload], "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_lm": N_LM, "n_cg": N_CG, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(tasks), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- GPU leg

def run_ours(args, world, rank, local):
    import torch

    from paper_1502_00858_gb300 import Calibrator, capi
    from synth import make_problem, user_layout

    # the CPU baseline's worker processes start (spawn) while the GPU leg runs
    pool = OraclePool(cpu_cores()) if (rank == 0 and not args.no_cpu_baseline) else None
    torch.cuda.set_device(local)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    capi.load()

    t_gen = time.perf_counter()
    # the large uneven batch is generated in complex64 (its visibilities and coherencies take 6.4 GB)
    gen_kw = {"dtype": np.complex64} if args.workload != WORKLOAD else {}
    prob = make_problem(args.workload, seed=1 + rank, **gen_kw)
    ul = user_layout(prob)
    t_gen = time.perf_counter() - t_gen
    n_admm = prob["n_admm"]
    per_iter_units = units(prob)

    stream = torch.cuda.Stream()
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], n_lm=N_LM, n_cg=N_CG,
                     chunk_diagonals=args.chunk_diagonals, ctas_per_sm=args.ctas_per_sm, cuda_stream=stream.cuda_stream,
                     formulation=capi.CALIB_FORM_DIRECT if args.formulation == "direct" else capi.CALIB_FORM_STATISTICS)
    dev = torch.device("cuda", local)
    vis_d = torch.from_numpy(ul["vis"].view(np.float32)).to(dev)
    uvw_d = torch.from_numpy(np.ascontiguousarray(prob["uvw"])).to(dev)
    sky_d = torch.from_numpy(np.ascontiguousarray(prob["sky"])).to(dev)
    J_d = torch.empty(int(np.prod(cal.jones_shape)) * 2, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    capi.calib_set_data(cal.ctx, vis_d)  # device pointers: stream-ordered

    if args.kernels_only:
        # One launch of each sweep mode on the full workload (for a profiler capture), then exit.
        capi.calib_predict(cal.ctx, uvw_d, sky_d, prob["f0"])
        J = np.ascontiguousarray(prob["J_true"], dtype=np.complex64)
        cal.eval(J)
        cal.hessvec(J, J)
        capi.calib_reset(cal.ctx)
        capi.calib_admm_iter(cal.ctx, 1, want_hist=False)
        out_d = torch.empty(int(vis_d.numel()), dtype=torch.float32, device=dev)
        capi.calib_residual(cal.ctx, out_d)
        torch.cuda.synchronize()
        cal.close()
        print("kernels-only run done", flush=True)
        return

    def step():
        capi.calib_predict(cal.ctx, uvw_d, sky_d, prob["f0"])
        capi.calib_reset(cal.ctx)
        capi.calib_admm_iter(cal.ctx, n_admm, want_hist=False)

    # the sweep split the autotuner picks for this shape (what the first calib_admm_iter would do)
    capi.calib_predict(cal.ctx, uvw_d, sky_d, prob["f0"])
    split = args.ctas_per_sm if args.formulation == "statistics" else args.chunk_diagonals
    split_tr, split_ms = split, None
    if split == 0:
        split, split_tr, split_ms = capi.calib_autotune(cal.ctx)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = capi.calib_launch_count(cal.ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    dt = ev0.elapsed_time(ev1) / 1e3
    launches = capi.calib_launch_count(cal.ctx) - launches0
    dt = max_over_ranks(dt, world, dev)
    value = whole_job_rate(world, per_iter_units * n_admm, args.steps, dt)

    # per-kernel durations (CUDA events recorded on the library stream around every sweep launch).
    # The profiled graph has event records between its kernels and no programmatic dependent launch,
    # so it runs slower than the timed one: per-kernel shares are taken of its own duration.
    capi.calib_profile_enable(cal.ctx, True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        step()
    pe1.record(stream)
    torch.cuda.synchronize()
    dt_prof = pe0.elapsed_time(pe1) / 1e3
    prof = capi.calib_profile_read(cal.ctx)
    capi.calib_profile_enable(cal.ctx, False)
    dom = max((k for k in prof if prof[k]["bytes_per_launch"] > 0 and k != "stats_pass"), key=lambda k: prof[k]["total_ms"])
    avg_s = prof[dom]["total_ms"] / 1e3 / max(1, prof[dom]["launches"])
    hbm_peak, fp32_peak, peak_how = peaks(sms)
    hbm_achieved = prof[dom]["bytes_per_launch"] / avg_s / 1e9
    traffic = NCU_TRAFFIC.get((dom, source_hash(dom)))
    if dom in ALU_BOUND:
        achieved = prof[dom]["flops_per_launch"] / avg_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": traffic, "peak_source": peak_how,
                    "hbm_achieved_gbs": hbm_achieved, "hbm_frac": hbm_achieved / hbm_peak}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "traffic": traffic, "peak_source": peak_how}
    roofline["kernel"] = dom
    # the kernel that streams the visibilities: the statistics pass (HBM-bound), once per step
    sp = prof.get("stats_pass")
    if sp and sp["launches"]:
        sp_s = sp["total_ms"] / 1e3 / sp["launches"]
        sp_gbs = sp["bytes_per_launch"] / sp_s / 1e9
        roofline["hbm_kernel"] = {"kernel": "stats_pass", "bound": "hbm", "achieved": sp_gbs, "peak": hbm_peak,
                                  "unit": "GB/s", "frac": sp_gbs / hbm_peak, "avg_launch_us": sp_s * 1e6,
                                  "algorithmic_bytes_per_launch": sp["bytes_per_launch"],
                                  "traffic": NCU_TRAFFIC.get(("stats_pass", source_hash("stats_pass")))}
    roofline["algorithmic_bytes_per_launch"] = prof[dom]["bytes_per_launch"]
    roofline["algorithmic_flops_per_launch"] = prof[dom]["flops_per_launch"]
    roofline["avg_launch_us"] = avg_s * 1e6
    roofline["profiled_ms_per_step"] = 1e3 * dt_prof / args.steps  # the graph the per-kernel figures come from
    roofline["per_kernel"] = {
        k: {"avg_us": 1e3 * v["total_ms"] / max(1, v["launches"]), "launches": v["launches"],
            "GBps": v["bytes_per_launch"] / (v["total_ms"] / 1e3 / v["launches"]) / 1e9
            if v["launches"] and v["bytes_per_launch"] else None,
            "TFLOPs": v["flops_per_launch"] / (v["total_ms"] / 1e3 / v["launches"]) / 1e12
            if v["launches"] and v["flops_per_launch"] else None,
            "share_of_step": v["total_ms"] / 1e3 / dt_prof if dt_prof else None,
            "traffic": NCU_TRAFFIC.get((k, source_hash(k))) if k in KERNEL_SOURCE else None}
        for k, v in prof.items()}

    # coherency prediction (once per step), after the timed region
    for _ in range(2):
        capi.calib_predict(cal.ctx, uvw_d, sky_d, prob["f0"])
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(5):
        capi.calib_predict(cal.ctx, uvw_d, sky_d, prob["f0"])
    p1.record(stream)
    torch.cuda.synchronize()
    roofline["predict"] = {"avg_launch_us": p0.elapsed_time(p1) * 1e3 / 5,
                           "note": "coherencies of every (baseline, sample, direction) from the sky model, "
                                   "with the Jacobi weights they imply; once per step"}

    # residual visibilities of every direction at the final solutions (Section 2), after the timed
    # region: one HBM stream reading V and C and writing R once per visibility
    out_d = torch.empty(int(vis_d.numel()), dtype=torch.float32, device=dev)
    for _ in range(2):
        capi.calib_residual(cal.ctx, out_d)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r_reps = 5
    r0.record(stream)
    for _ in range(r_reps):
        capi.calib_residual(cal.ctx, out_d)
    r1.record(stream)
    torch.cuda.synchronize()
    r_s = r0.elapsed_time(r1) / 1e3 / r_reps
    r_bytes = per_iter_units / prob["K"] * (32 + 8 * prob["K"] + 32)
    roofline["residual_kernel"] = {"kernel": "residual", "bound": "hbm", "achieved": r_bytes / r_s / 1e9,
                                   "peak": hbm_peak, "unit": "GB/s", "frac": r_bytes / r_s / 1e9 / hbm_peak,
                                   "avg_launch_us": r_s * 1e6, "algorithmic_bytes_per_launch": r_bytes,
                                   "traffic": NCU_TRAFFIC.get(("residual", source_hash("residual")))}
    del out_d

    # end to end through the public API with host buffers: H2D of the visibilities, uvw and sky,
    # prediction, cold start, 30 iterations, D2H of the solutions.
    vis_h = torch.from_numpy(ul["vis"].view(np.float32)).pin_memory()
    uvw_h = torch.from_numpy(np.ascontiguousarray(prob["uvw"])).pin_memory()
    sky_h = torch.from_numpy(np.ascontiguousarray(prob["sky"])).pin_memory()
    J_h = torch.empty(int(np.prod(cal.jones_shape)) * 2, dtype=torch.float32).pin_memory()

    def e2e_step():
        capi.calib_set_data(cal.ctx, vis_h)
        capi.calib_predict(cal.ctx, uvw_h, sky_h, prob["f0"])
        capi.calib_reset(cal.ctx)
        capi.calib_admm_iter(cal.ctx, n_admm, want_hist=False)
        capi.calib_get_solutions(cal.ctx, J=J_h)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e_dt = max_over_ranks(e2e_dt, world, dev)
    e2e_value = whole_job_rate(world, per_iter_units * n_admm, args.steps, e2e_dt)
    h2d = vis_h.numel() * 4 + uvw_h.numel() * 8 + sky_h.numel() * 8
    d2h = J_h.numel() * 4

    cal.close()
    stream_mb = (ul["vis"].nbytes + ul["coh"].nbytes) / 1e6
    del vis_d, vis_h, ul

    uneven = None
    if not args.no_uneven and args.workload == WORKLOAD:
        uneven = run_uneven(args, world, local, sms, hbm_peak, fp32_peak, barrier)

    cpu = None
    if pool is not None:
        tasks = oracle_tasks(prob, pool.workers)
        pool.run(tasks[:1])  # workers have imported the oracle
        cdt, cu = pool.run(tasks)
        pool.close()
        cpu = {"value": cu / cdt, "unit": UNIT, "cores": len(tasks), "kind": "oracle",
               "sample": oracle_sample_text(pool.workers, len(tasks), prob["P"], cdt)}

    if rank == 0:
        out = {
            "metric": METRICS[args.workload], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "stations": prob["N"], "baselines": prob["B"], "directions": prob["K"],
                       "subbands": prob["P"], "intervals": prob["I"],
                       "samples": sorted(set(int(t) for t in np.asarray(prob["T"]).ravel())),
                       "flagged_fraction": round(float(np.mean(prob["flags"])), 4), "admm_iters": n_admm,
                       "n_lm": N_LM, "n_cg": N_CG, "basis": "Bernstein degree 3", "rho": 10.0,
                       "formulation": args.formulation,
                       ("ctas_per_sm" if args.formulation == "statistics" else "chunk_diagonals"): [split, split_tr],
                       "autotune_ms_hessian_trial": split_ms,
                       "step": f"predict + cold start + {n_admm} C-ADMM iterations",
                       "l2": f"inputs larger than L2: every step streams the visibilities and predicted coherencies "
                             f"({stream_mb:.0f} MB) through predict, the statistics "
                             f"pass and the first residual sweep; each LM step reads U and S "
                             f"({1e-6 * prof['stats_trial']['bytes_per_launch']:.0f} MB)",
                       "parallelism": f"replica x{world}" if world > 1 else "single GPU",
                       "generate_s": round(t_gen, 2)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "uneven": uneven,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_uneven(args, world, local, sms, hbm_peak, fp32_peak, barrier) -> dict:
    """The batched uneven workload (2560 agents: 256 subbands x 10 intervals, K=10, 5/10/20 samples
    per subband, 0-15 % of baselines flagged, 50 C-ADMM iterations) in one graph per
    calib_admm_iter, measured like the main line on fewer steps (one step takes seconds)."""
    import torch

    from paper_1502_00858_gb300 import Calibrator, capi
    from synth import make_problem

    t_gen = time.perf_counter()
    prob = make_problem("uneven_n62_k10", seed=1 + int(os.environ.get("RANK", "0")), dtype=np.complex64,
                        coherencies=False)
    vis = np.concatenate([V.reshape(-1) for V in prob["V"]]).astype(np.complex64)
    prob["V"] = None
    t_gen = time.perf_counter() - t_gen
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], n_lm=N_LM, n_cg=N_CG, cuda_stream=stream.cuda_stream)
    vis_d = torch.from_numpy(vis.view(np.float32)).to(dev)
    del vis
    uvw_d = torch.from_numpy(np.ascontiguousarray(prob["uvw"])).to(dev)
    sky_d = torch.from_numpy(np.ascontiguousarray(prob["sky"])).to(dev)
    flags_d = torch.from_numpy(np.ascontiguousarray(prob["flags"])).to(dev)
    torch.cuda.synchronize()
    capi.calib_set_data(cal.ctx, vis_d, flags=flags_d)
    n_admm = prob["n_admm"]
    keep = (prob["flags"] == 0).sum(axis=1)
    per_iter_units = float(np.sum(keep * prob["T"])) * prob["K"]

    def step():
        capi.calib_predict(cal.ctx, uvw_d, sky_d, prob["f0"])
        capi.calib_reset(cal.ctx)
        capi.calib_admm_iter(cal.ctx, n_admm, want_hist=False)

    step()  # warm-up: the autotuner and the graph capture run here
    torch.cuda.synchronize()
    steps = 2
    launches0 = capi.calib_launch_count(cal.ctx)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    dt = e0.elapsed_time(e1) / 1e3
    launches = capi.calib_launch_count(cal.ctx) - launches0
    capi.calib_profile_enable(cal.ctx, True)
    step()
    prof = capi.calib_profile_read(cal.ctx)
    capi.calib_profile_enable(cal.ctx, False)
    cal.close()
    per_kernel = {}
    for k, v in prof.items():
        if not v["launches"]:
            continue
        avg = v["total_ms"] / 1e3 / v["launches"]
        e = {"avg_us": avg * 1e6, "launches": v["launches"]}
        if v["flops_per_launch"] and k in ALU_BOUND:
            e.update(bound="alu", achieved_tflops=v["flops_per_launch"] / avg / 1e12,
                     frac=v["flops_per_launch"] / avg / 1e12 / fp32_peak)
        elif v["bytes_per_launch"]:
            e.update(bound="hbm", achieved_gbs=v["bytes_per_launch"] / avg / 1e9,
                     frac=v["bytes_per_launch"] / avg / 1e9 / hbm_peak)
        per_kernel[k] = e
    return {"metric": METRICS["uneven_n62_k10"], "value": world * per_iter_units * n_admm * steps / dt,
            "unit": UNIT, "ms_per_step": 1e3 * dt / steps, "steps": steps, "warmup": 1,
            "agents": int(prob["A"]), "directions": int(prob["K"]), "admm_iters": n_admm,
            "samples": sorted(set(int(t) for t in prob["T"])),
            "flagged_fraction": round(float(np.mean(prob["flags"])), 4),
            "gpu_launches": int(launches), "per_kernel": per_kernel, "generate_s": round(t_gen, 1),
            "step": f"predict + cold start + {n_admm} C-ADMM iterations, one graph per calib_admm_iter"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--chunk-diagonals", type=int, default=0, help="direct sweeps: diagonals per CTA (0 = tuned)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="statistics sweeps: CTAs per SM (0 = tuned)")
    ap.add_argument("--formulation", choices=["statistics", "direct"], default="statistics")
    ap.add_argument("--workload", choices=sorted(METRICS), default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uneven", action="store_true", help="skip the nested batched uneven workload")
    ap.add_argument("--kernels-only", action="store_true",
                    help="run one launch of each sweep on the workload and exit (profiler captures)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark of the macro-element HDG hot path on one GB300 (or N replicas).

One step = the whole hot path on the 128 x 128 macro mesh (32,768
macro-triangles, m = 8, p = 3, beta = 50 (cos 0.3, sin 0.3), kappa = 1,
manufactured source of u = sin(pi x) sin(pi y)): element formation and batched
condensation, right-hand-side assembly, left-preconditioned GMRES(50) to a
1e-10 true relative residual, and the back-solve for u and q. Inputs (the
source at the quadrature points) are resident in HBM before the timed region.

value = trace-operator GDoF/s over the whole step: N_tr times the number of
trace-operator applications executed in the timed steps, divided by their
device time. The solve time (time to a 1e-10 residual) and the apply-only
throughput are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trace-operator GDoF/s and time-to-1e-10 solve (FP64 vs FP32+IR, 1 GB300)"
WORKLOAD = ("2D steady advection-diffusion, 128x128 macro grid (32768 macro-triangles), m=8 (64 sub-triangles), "
            "p=3, beta=50(cos 0.3, sin 0.3), kappa=1, u=sin(pi x)sin(pi y), Dirichlet; step = condense + rhs + "
            "GMRES(restart) to 1e-10 true relative residual + back-solve")
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12     # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
CPU_SAMPLE_COND, CPU_SAMPLE_APPLY = 40, 100000     # about 12 s of single-thread oracle work
# trace-operator applications per step of the GPU path (GMRES(50) Arnoldi steps + 2 per restart)
REFERENCE_APPLIES_PER_STEP = 5250


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="c1")
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args(argv)


# ----------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(units, seconds, world):
    """Whole-job throughput over replicas: (sum of units) / (max of times)."""
    if world == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def gpu_smi_id(dev_index):
    import torch
    try:
        uuid = str(torch.cuda.get_device_properties(dev_index).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        return dev_index


def measured_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------- CPU oracle
def oracle_sample(cfg_name, n_cond, n_apply_elems, applies_per_step):
    """Time the oracle on a bounded sample of the workload, extrapolate one step.

    The oracle condenses n_cond sampled macro-elements (dense LU of the full
    3Q x 3Q local system) and applies the resulting Schur blocks element by
    element; one step is extrapolated as N condensations + applies_per_step
    element-wise applies of all N elements + N back-solves.
    """
    import numpy as np
    from oracle.hdg import HDGProblem
    from paper_2302_10917_gb300 import workloads as wl
    cfg = wl.CONFIGS[cfg_name]
    ora = HDGProblem(cfg["n"], cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"])
    msh = ora.mesh
    rng = np.random.default_rng([wl.MASTER_SEED, 99])
    els = rng.choice(msh.N, size=n_cond, replace=False)
    t0 = time.perf_counter()
    S = {}
    for e in els:
        S[int(e)], _ = ora.condense_element(int(e))
    t_cond = (time.perf_counter() - t0) / n_cond
    x = wl.random_vector(msh.N_tr, seed=3)
    y = np.zeros(msh.N_tr)
    zero_bnd = np.zeros((msh.n_bnd_edges, msh.P1))
    keys = list(S.keys())
    t0 = time.perf_counter()
    for r in range(n_apply_elems):
        e = keys[r % len(keys)]
        ora.scatter(e, S[e] @ ora.element_trace(e, x, zero_bnd), y)
    t_app = (time.perf_counter() - t0) / n_apply_elems
    # the oracle's back-solve body (a dense solve per element) on the sampled elements
    t0 = time.perf_counter()
    for e in keys:
        A, B, _, _ = ora.local_blocks(e)
        np.linalg.solve(A, -B @ ora.element_trace(e, x, zero_bnd))
    t_rec = (time.perf_counter() - t0) / len(keys)
    step_s = msh.N * (t_cond + applies_per_step * t_app + t_rec)
    return {"t_condense_elem_s": t_cond, "t_apply_elem_s": t_app, "t_recover_elem_s": t_rec,
            "step_s": step_s, "N": msh.N, "N_tr": msh.N_tr,
            "value": msh.N_tr * applies_per_step / step_s / 1e9}


def cpu_baseline(cfg_name, applies_per_step):
    """Run the oracle sample in a fresh single-threaded interpreter."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, bench; print(json.dumps(bench.oracle_sample(%r, %d, %d, %d)))"
            % (cfg_name, CPU_SAMPLE_COND, CPU_SAMPLE_APPLY, applies_per_step))
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    if res.returncode != 0:
        return {"value": None, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "error": res.stderr[-400:]}
    r = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": r["value"], "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle (numpy, 1 thread) condensing {CPU_SAMPLE_COND} sampled macro-elements (dense LU "
                       f"of the 975x975 local system each), {CPU_SAMPLE_APPLY} element-wise Schur applies and "
                       f"{CPU_SAMPLE_COND} element back-solves, extrapolated to one step: 32768 condensations + "
                       f"{applies_per_step} applies of all elements + 32768 back-solves"),
            "step_s_extrapolated": r["step_s"]}


# ---------------------------------------------------------------- reference
def run_reference(args):
    world, rank, local = dist_env()
    if world > 1 and rank != 0:
        return
    applies = REFERENCE_APPLIES_PER_STEP
    samples = []
    for _ in range(args.warmup):
        oracle_sample(args.config, 1, 300, applies)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        samples.append(oracle_sample(args.config, 4, 10000, applies))
    wall = time.perf_counter() - t0
    value = statistics.mean(s["value"] for s in samples)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: bounded sample per step, extrapolated)"},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "kind": "oracle", "cores": 1,
                             "sample": "per step: oracle condensation and back-solve of 4 sampled macro-elements "
                                       "and 10000 element-wise applies, extrapolated to 32768 elements and "
                                       f"{applies} applies"},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2302_10917_gb300 import Problem
    from paper_2302_10917_gb300 import workloads as wl
    cfg = wl.CONFIGS[args.config]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    pr = Problem(cfg["n"], cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], device=dev, stream=stream)
    N_tr, N, Q = pr.info["N_tr"], pr.info["N"], pr.info["Q"]
    xy = pr.quad_points()
    f = wl.sin_sin_source(xy, cfg["kappa"], cfg["beta"]).contiguous()
    del xy
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(rec=None):
        marks = [ev() for _ in range(4)] if rec is not None else None
        if marks:
            marks[0].record(stream)
        pr.set_source(f)
        pr.condense(keep_factors=True)
        g = pr.rhs()
        if marks:
            marks[1].record(stream)
        x, rep, st = pr.solve(g, tol=1e-10, restart=args.restart, maxit=60000)
        if marks:
            marks[2].record(stream)
        u, q = pr.recover(x)
        if marks:
            marks[3].record(stream)
            rec.append((marks, rep))
        return rep, st

    for _ in range(args.warmup):
        rep, st = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_smi_id(dev.index))
    clocks.start()
    launches0 = pr.launches()
    pr.profile(True)
    recs = []
    t_start, t_end = ev(), ev()
    t_start.record(stream)
    for _ in range(args.steps):
        rep, st = step(recs)
    t_end.record(stream)
    torch.cuda.synchronize()
    prof = pr.profile_read()
    pr.profile(False)
    launches = pr.launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_s = t_start.elapsed_time(t_end) / 1e3
    applies = prof["apply"][0]
    units, total_max = aggregate(N_tr * applies, total_s, world)
    value = units / total_max / 1e9

    cond_s = [m[0].elapsed_time(m[1]) / 1e3 for m, _ in recs]
    solve_s = [m[1].elapsed_time(m[2]) / 1e3 for m, _ in recs]
    rec_s = [m[2].elapsed_time(m[3]) / 1e3 for m, _ in recs]
    reps = [r for _, r in recs]
    apply_ms = prof["apply"][1] / max(1, prof["apply"][0])
    cond_ms = prof["condense"][1] / max(1, prof["condense"][0])

    peaks = measured_peaks()
    # dominant kernel over the timed region
    P1, n_t, n_int = cfg["m"] * cfg["p"] + 1, 3 * (cfg["m"] * cfg["p"] + 1), pr.info["n_int_edges"]
    apply_flops = 4.0 * P1 * n_t * n_int                       # 2 sides x P1 rows x n_t cols x 2 flop per edge
    apply_bytes = 8.0 * (2 * P1 * n_t * n_int + 2 * N_tr)      # Schur row-blocks + x gathers + y write
    R, Cc = Q + n_t, Q + n_t + 1
    cond_flops = N * sum(2.0 * (R - 1 - k) * (Cc - 1 - k) for k in range(Q))
    kern = {"apply": (prof["apply"][1], apply_flops, apply_ms, prof["apply"][0]),
            "condense": (prof["condense"][1], cond_flops, cond_ms, prof["condense"][0])}
    dom = max(kern, key=lambda k: kern[k][0])
    tot_ms, flops, avg_ms, cnt = kern[dom]
    achieved = flops / (avg_ms / 1e3) / 1e12
    roofline = {"kernel": "apply_kernel<double,double> (FP64 trace apply)" if dom == "apply"
                else "condense_kernel (element build + bordered LU + Schur)",
                "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived; no measured "
                               "FP64 peak in the driver's file)",
                "algorithmic_per_launch": flops, "avg_launch_ms": avg_ms, "launches": cnt,
                "hbm_view": {"bytes_per_launch": apply_bytes if dom == "apply" else None,
                             "achieved_gbs": apply_bytes / (avg_ms / 1e3) / 1e9 if dom == "apply" else None,
                             "peak_gbs": peaks.get("hbm_gbs")}}

    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("GMRES(restart)", f"GMRES({args.restart})"),
                       "N_tr": N_tr, "macro_elements": N, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2: Schur blocks 1.47 GB, factors 42 GB, source 0.42 GB per replica"},
            "time_to_solve_s": statistics.median(solve_s), "condense_s": statistics.median(cond_s),
            "recover_s": statistics.median(rec_s), "iterations": reps[-1]["iterations"],
            "restarts": reps[-1]["restarts"], "rel_residual": reps[-1]["rel_residual"],
            "apply_gdofs": N_tr / (apply_ms / 1e3) / 1e9, "apply_us": apply_ms * 1e3,
            "phases_ms": {k: v[1] / args.steps for k, v in prof.items()},
            "roofline": roofline, "gpu_launches": int(launches), "clocks": clk}

    if not args.no_e2e:
        fh = f.cpu().pin_memory()
        torch.cuda.synchronize()
        pr.run_host(fh, outputs=True)                 # warm-up of the host path
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, u, q, rep = pr.run_host(fh, outputs=True)
        e2e_s = time.perf_counter() - t0
        app_e2e = rep["iterations"] + 2 * rep["restarts"]
        eu, es = aggregate(N_tr * app_e2e, e2e_s, world)
        line["e2e"] = {"value": eu / es / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": int(fh.numel() * 8),
                       "d2h_bytes_per_step": int((x.numel() + u.numel() + q.numel()) * 8), "seconds": e2e_s,
                       "call": "hdg_run_host (pinned host f in; x, u, q out)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config, int(round(applies / args.steps)))
    pr.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

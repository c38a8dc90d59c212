#!/usr/bin/env python3
"""Benchmark of the macro-element HDG hot path on one GB300 (or N replicas).

One step = the whole hot path on the 128 x 128 macro mesh (32,768
macro-triangles, m = 8, p = 3, beta = 50 (cos 0.3, sin 0.3), kappa = 1,
manufactured source of u = sin(pi x) sin(pi y)): element formation and batched
condensation, right-hand-side assembly, left-preconditioned GMRES(80) to a
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
# split-FP32 multiply-add (Dekker product + two-sum accumulation): 1 FMUL + 3 FFMA + 8 FADD
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12
# DRAM bytes (read + write) of one apply_vdf_kernel<1,1> launch per interior edge, from an ncu
# capture at n = 64, m = 8, p = 3 (376.20 MB for 12 160 edges); the traffic scales with the
# edges. Only valid for that kernel and element (m = 8, p = 3).
APPLY_VDF1_TRAFFIC_PER_EDGE_M8P3 = 376.20e6 / 12160
# the same for apply_vdf_kernel<0,0> (FP64 blocks, FP64 vectors): 376.72 MB for 12 160 edges at n = 64
APPLY_VDF00_TRAFFIC_PER_EDGE_M8P3 = 376.72e6 / 12160
# the same for apply_fix_kernel (fixed-point rows, FP64 vectors): 376.25 + 4.69 MB for 12 160 edges at n = 64
APPLY_FIX_TRAFFIC_PER_EDGE_M8P3 = 380.94e6 / 12160
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
CPU_SAMPLE_COND, CPU_SAMPLE_APPLY = 40, 100000     # about 12 s of single-thread oracle work
# trace-operator applications per step of the GPU path (GMRES(80) Arnoldi steps + 1 per restart)
REFERENCE_APPLIES_PER_STEP = 4375


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="n128_m8_p3")
    ap.add_argument("--restart", type=int, default=80)
    ap.add_argument("--mode", type=int, default=3, choices=[0, 1, 2, 3],
                    help="Arnoldi operator of the timed solve: 0 FP64, 1 FP32 (+FP64 refinement), 2 split FP32, "
                         "3 fixed-point rows with exact integer products (FP64-accurate)")
    ap.add_argument("--basis", type=int, default=0, choices=[0, 1, 2],
                    help="Krylov basis and orthogonalisation: 0 FP64, 1 split FP32, 2 fixed-point chunks with "
                         "exact integer products (FP64-accurate)")
    ap.add_argument("--orth", type=int, default=3, choices=[0, 1, 2, 3],
                    help="Arnoldi orthogonalisation: 0 CGS2 (four passes), 1 CGS with Pythagorean norm (two passes), "
                         "2 CGS with a second projection where more than half of the vector lay in the basis, "
                         "3 the same where the single projection cancelled more than six digits")
    ap.add_argument("--augment", type=int, default=0, choices=[0, 1, 2, 3],
                    help="augmented restarts: corrections of earlier cycles in each cycle's search space (LGMRES)")
    ap.add_argument("--elim", default="tc", choices=["tc", "fp64", "split"],
                    help="local factorisation: tc = FP64 panels with the trailing updates as exact slice products "
                         "on the tensor cores (FP64-accurate), fp64 = FP64 FMAs throughout, split = split-FP32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the many-source and gradient measurements that follow the main line")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the whole-step comparison of the precision forms and preconditioners")
    ap.add_argument("--no-keep-factors", action="store_true",
                    help="do not keep the factored local systems (the back-solve condenses again; small device "
                         "footprint for profiler captures)")
    ap.add_argument("--bulk-warps", type=int, default=0,
                    help="with --mode 2 --basis 1: the pipelined bulk-copy apply with this many consumer warps per "
                         "edge instead of the autotuned shape")
    ap.add_argument("--maxit", type=int, default=60000,
                    help="GMRES operator applications per solve; a value below what the solve needs (one restart "
                         "cycle for a profiler's launch list) lets the step end unconverged: not a benchmark line")
    ap.add_argument("--n", type=int, default=0,
                    help="macro squares per side instead of the workload's (small cases for profiler captures)")
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
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return summarize_clock_lines(lines)


def summarize_clock_lines(lines):
    """Median SM clock, maximum clock and power, and the throttle reasons seen, from
    `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits` rows;
    short rows (a header, an interrupted last line) are skipped, and a row whose
    clocks do not parse still contributes its throttle reasons."""
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        # a throttle reason counts on every complete row, the clocks only where all three parse
        for name, val in zip(names, parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(name)
        try:
            vals = float(parts[1]), float(parts[2]), float(parts[3])
        except ValueError:
            continue
        sm.append(vals[0])
        smax.append(vals[1])
        power.append(vals[2])
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"] + sorted(reasons)}
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
def oracle_sample(cfg_name, n_cond, n_apply_elems, applies_per_step, seed=0):
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
    rng = np.random.default_rng([wl.MASTER_SEED, 99, seed])
    els = rng.choice(msh.N, size=n_cond + 1, replace=False)
    # one untimed element first: the oracle builds its quadrature and basis caches on first use
    ora.condense_element(int(els[-1]))
    els = els[:-1]
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


def oracle_sample_one_thread(cfg_name, n_cond, n_apply_elems, applies_per_step):
    """oracle_sample in a fresh interpreter whose BLAS / OpenMP pools have one thread
    (so the reported core count is the one used); raises if the child fails."""
    code = ("import json, bench; print(json.dumps(bench.oracle_sample(%r, %d, %d, %d)))"
            % (cfg_name, n_cond, n_apply_elems, applies_per_step))
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=_one_thread_env(), capture_output=True,
                         text=True, timeout=600)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-400:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def _one_thread_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                CUDA_VISIBLE_DEVICES="")


def oracle_sample_all_cores(cfg_name, cores, n_cond, n_apply_elems, applies_per_step):
    """The oracle sample on every host core at once: `cores` single-threaded interpreters, each
    on its own seeded element sample, started together. Their per-element times under full load
    give the oracle's throughput on the whole host: one step = N (t_cond + applies t_apply +
    t_recover) / cores."""
    code = ("import json, sys, bench; print(json.dumps(bench.oracle_sample(%r, %d, %d, %d, int(sys.argv[1]))))"
            % (cfg_name, n_cond, n_apply_elems, applies_per_step))
    procs = [subprocess.Popen([sys.executable, "-c", code, str(i + 1)], cwd=ROOT, env=_one_thread_env(),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for i in range(cores)]
    outs = []
    for pr_ in procs:
        out, err = pr_.communicate(timeout=900)
        if pr_.returncode != 0:
            raise RuntimeError(err[-400:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    mean = lambda k: statistics.mean(o[k] for o in outs)
    N, N_tr = outs[0]["N"], outs[0]["N_tr"]
    step_s = N * (mean("t_condense_elem_s") + applies_per_step * mean("t_apply_elem_s") +
                  mean("t_recover_elem_s")) / cores
    return {"step_s": step_s, "value": N_tr * applies_per_step / step_s / 1e9, "N": N}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(cfg_name, applies_per_step):
    """The oracle on the host: in a fresh single-threaded interpreter, and on every core at once."""
    try:
        r = oracle_sample_one_thread(cfg_name, CPU_SAMPLE_COND, CPU_SAMPLE_APPLY, applies_per_step)
    except (RuntimeError, subprocess.TimeoutExpired, ValueError, IndexError) as exc:
        return {"value": None, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "error": str(exc)[-400:]}
    out = {"value": r["value"], "unit": "GDoF/s", "cores": 1, "kind": "oracle",
           "sample": (f"oracle (numpy, 1 thread) condensing {CPU_SAMPLE_COND} sampled macro-elements (dense LU "
                      f"of the 975x975 local system each), {CPU_SAMPLE_APPLY} element-wise Schur applies and "
                      f"{CPU_SAMPLE_COND} element back-solves, extrapolated to one step: 32768 condensations + "
                      f"{applies_per_step} applies of all elements + 32768 back-solves"),
           "step_s_extrapolated": r["step_s"]}
    cores = host_cores()
    nc, na = max(2, CPU_SAMPLE_COND // 4), max(5000, CPU_SAMPLE_APPLY // 4)
    try:
        ra = oracle_sample_all_cores(cfg_name, cores, nc, na, applies_per_step)
        out["all_cores"] = {"value": ra["value"], "unit": "GDoF/s", "cores": cores, "kind": "oracle",
                            "sample": (f"{cores} single-threaded oracle processes at once, each condensing {nc} "
                                       f"sampled macro-elements, {na} element-wise applies and {nc} back-solves; "
                                       "one step extrapolated from their per-element times under full load"),
                            "step_s_extrapolated": ra["step_s"]}
    except (RuntimeError, subprocess.TimeoutExpired, ValueError, IndexError, OSError) as exc:
        out["all_cores"] = {"value": None, "cores": cores, "error": str(exc)[-400:]}
    return out


# ---------------------------------------------------------------- reference
def run_reference(args):
    world, rank, local = dist_env()
    if world > 1 and rank != 0:
        return
    applies = REFERENCE_APPLIES_PER_STEP
    samples = []
    # every sample in a fresh single-threaded interpreter, so "cores": 1 is what ran
    for _ in range(args.warmup):
        oracle_sample_one_thread(args.config, 1, 300, applies)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        samples.append(oracle_sample_one_thread(args.config, 4, 10000, applies))
    wall = time.perf_counter() - t0
    value = statistics.mean(s["value"] for s in samples)
    step_s = statistics.mean(s["step_s"] for s in samples)
    # a step here is one bounded sample (wall time, what a clock around the run sees); the oracle's
    # time for one whole step of the workload, extrapolated from the samples, is reported beside it
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "step_s_extrapolated": step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: bounded sample per step, extrapolated)"},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "kind": "oracle", "cores": 1,
                             "sample": "per step: oracle (numpy, 1 thread) condensation and back-solve of 4 "
                                       "sampled macro-elements and 10000 element-wise applies, extrapolated to "
                                       f"32768 elements and {applies} applies"},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tc_slice_flops(Q, R, Cc, b=32, m_tile=128, n_tile=32, products=28):
    """bf16 flops the tensor-core condensation issues per element: every 32-column panel,
    every 128-row x 32-column tile of the trailing block, 28 slice products of K = 32."""
    flops, j0 = 0, 0
    while j0 < Q:
        nb = min(b, Q - j0)
        jb = j0 + nb
        tiles = -(-(R - jb) // m_tile) * -(-(Cc - jb) // n_tile)
        flops += tiles * products * 2 * m_tile * n_tile * b
        j0 += b
    return flops


# ---------------------------------------------------------------------- ours
MODE_NAMES = {0: "fp64", 1: "fp32_ir", 2: "df64", 3: "fp64_fixed"}
# precision forms of one step: (Arnoldi operator mode, Krylov basis, local factorisation)
FORMS = {"fp64": (0, 0, "tc"), "fp64_fixed": (3, 0, "tc"), "fp64_fixed_basis": (3, 2, "tc"),
         "fp64_dfma": (0, 0, "fp64"), "fp32_ir": (1, 0, "tc"), "df64": (2, 1, "split")}
FORM_DTYPES = {(0, 0, "tc"): "f64 (tensor-core trailing updates by exact 8-bit slices, FP64-accurate)",
               (3, 0, "tc"): "f64 (trace apply on 56-bit fixed-point rows with exact integer products, one FP64 "
                             "rounding per element side; tensor-core trailing updates by exact 8-bit slices)",
               (3, 2, "tc"): "f64 (as fp64_fixed, and the Krylov basis in 56-bit fixed-point chunks with exact "
                             "integer products in the multi-dot and the updates)",
               (0, 0, "fp64"): "f64 (FP64 FMAs throughout)",
               (1, 0, "tc"): "f32 blocks (FP32 operator) + f64 factorisation, orthogonalisation and refinement",
               (2, 1, "split"): "df64 (f32x2) elimination, blocks and Krylov basis + f64 residual"}


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
    cfg = dict(wl.CONFIGS[args.config])
    if args.n > 0:
        cfg["n"] = args.n
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    pr = Problem(cfg["n"], cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], device=dev, stream=stream)
    N_tr, N, Q = pr.info["N_tr"], pr.info["N"], pr.info["Q"]
    xy = pr.quad_points()
    f = wl.sin_sin_source(xy, cfg["kappa"], cfg["beta"]).contiguous()
    del xy
    ev = lambda: torch.cuda.Event(enable_timing=True)
    split = args.elim == "split"
    tc = args.elim == "tc"

    def condense_flags(mode, elim):
        # only the blocks the solve mode needs
        return dict(keep_factors=not args.no_keep_factors, store_fp32=(mode == 1), store_df64=(mode == 2),
                    store_fix=(mode == 3), split_update=elim == "split", tc_update=elim == "tc")

    def step(rec=None, mode=args.mode, basis=args.basis, elim=args.elim, precond="d"):
        marks = [ev() for _ in range(4)] if rec is not None else None
        if marks:
            marks[0].record(stream)
        pr.set_source(f)
        pr.condense(precond=precond, **condense_flags(mode, elim))
        g = pr.rhs()
        if marks:
            marks[1].record(stream)
        x, rep, st = pr.solve(g, tol=1e-10, restart=args.restart, maxit=args.maxit, mode=mode, orth=args.orth,
                              basis=basis, check=False, augment=args.augment)
        if st != 0 and not (st == 6 and args.maxit < 60000):   # 6: HDG_ERR_NOCONV
            raise RuntimeError(f"solve did not converge: {rep} (status {st})")
        if marks:
            marks[2].record(stream)
        u, q = pr.recover(x)
        if marks:
            marks[3].record(stream)
            rec.append((marks, rep))
        return rep, x, u, q

    # the project's launch-shape autotuner runs once per problem (outside the timed region)
    step()
    tune = pr.autotune(mode=args.mode, restart=args.restart, basis=args.basis)
    if args.bulk_warps:
        pr.set_apply_shape(2, bulk_warps=args.bulk_warps)
        tune["apply_bulk"] = args.bulk_warps
    for _ in range(args.warmup - 1):
        step()
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
        step(recs)
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
    applies = prof["apply"][0] + prof["apply32"][0] + prof["resid"][0]
    units, total_max = aggregate(N_tr * applies, total_s, world)
    value = units / total_max / 1e9

    cond_s = [m[0].elapsed_time(m[1]) / 1e3 for m, _ in recs]
    solve_s = [m[1].elapsed_time(m[2]) / 1e3 for m, _ in recs]
    rec_s = [m[2].elapsed_time(m[3]) / 1e3 for m, _ in recs]
    reps = [r for _, r in recs]

    peaks = measured_peaks()
    P1 = cfg["m"] * cfg["p"] + 1
    n_t, n_int = 3 * P1, pr.info["n_int_edges"]
    R, Cc = Q + n_t, Q + n_t + 1
    avg = lambda ph: prof[ph][1] / max(1, prof[ph][0])
    # algorithmic work per launch (blocks of both sides, x once, y once)
    apply_bytes = 8.0 * (2 * P1 * n_t * n_int + 2 * N_tr)        # blocks of both sides + x once + y once
    apply_flops = 4.0 * P1 * n_t * n_int
    cond_flops = N * sum(2.0 * (R - 1 - k) * (Cc - 1 - k) for k in range(Q))
    fp64_ceiling = FP64_PEAK_TFLOPS * 1e12 / 2 * 8 / 1e9     # GB/s at one FP64 FMA per 8-byte entry
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    apply_kernels = {0: "apply_vdf_kernel<0,0> (FP64 blocks, FP64 vectors)",
                     3: "apply_fix_kernel (56-bit fixed-point rows, exact int64 products, FP64 vectors)",
                     1: "apply_vdf_kernel<2,%d> (FP32 blocks)" % (1 - args.basis),
                     2: "apply_vdf_kernel<1,%d> (split-FP32 blocks)" % (1 - args.basis)}
    rooflines = {
        "apply": {"kernel": (apply_kernels[args.mode] if not tune.get("apply_bulk")
                             else f"apply_bulk_kernel (split-FP32 blocks, bulk copies into shared-memory slots, "
                                  f"{tune['apply_bulk']} consumer warps per edge)"),
                  "bound": "hbm",
                  "launches": prof["apply32" if args.mode == 1 else "apply"][0],
                  "avg_launch_ms": avg("apply32" if args.mode == 1 else "apply")},
        "condense": {"kernel": ("condense_df_kernel (split-FP32 formation + bordered LU + Schur)" if split
                                else "condense_tc_kernel (FP64 formation, 32-column FP64 panels, trailing updates "
                                     "as exact 8-bit slice products on the tensor cores)" if tc
                                else "condense_kernel (FP64 formation + bordered LU + Schur)"),
                     "bound": "alu", "launches": prof["condense"][0], "avg_launch_ms": avg("condense")},
    }
    ra = rooflines["apply"]
    # FP32 blocks move 4 bytes per entry; the vectors are 8 bytes per entry in either basis
    # (fixed-point rows: 8 bytes per entry plus a 4-byte scale per row of each side)
    bpl = apply_bytes - (4.0 * 2 * P1 * n_t * n_int if args.mode == 1 else 0.0) + \
        (4.0 * 2 * P1 * n_int if args.mode == 3 else 0.0)
    ra.update(achieved=bpl / (ra["avg_launch_ms"] / 1e3) / 1e9, peak=hbm_peak, unit="GB/s",
              algorithmic_per_launch=bpl, peak_source=hbm_src)
    ra["frac"] = ra["achieved"] / ra["peak"]
    if args.mode == 0:
        # FP64 blocks: one FP64 FMA per 8-byte entry; GB300's FP64 pipe caps this at fp64_ceiling
        tf = apply_flops / (ra["avg_launch_ms"] / 1e3) / 1e12
        ra["fp64_pipe"] = {"achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
                           "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)",
                           "hbm_frac_at_fp64_peak": fp64_ceiling / hbm_peak}
    rc = rooflines["condense"]
    # one condensation per step (several launches when the factors are not kept: chunks)
    cond_ms = prof["condense"][1] / max(1, args.steps)
    rc["avg_launch_ms"] = cond_ms
    rc["note"] = "per condensation of all elements (launches per step: %d)" % (prof["condense"][0] // max(1, args.steps))
    if split:
        rc.update(achieved=cond_flops / (rc["avg_launch_ms"] / 1e3) / 1e12, peak=DF_PEAK_TFLOPS, unit="TFLOP/s",
                  algorithmic_per_launch=cond_flops,
                  peak_source="FP32 pipe in FP64-equivalent flop: 152 SMs x 128 lanes x 2.07 GHz / 12 FP32 "
                              "instructions per split-FP32 multiply-add x 2 flop (derived)")
    else:
        rc.update(achieved=cond_flops / (rc["avg_launch_ms"] / 1e3) / 1e12, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                  algorithmic_per_launch=cond_flops,
                  peak_source="FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)",
                  note_flops="FP64-equivalent flops of the dense bordered LU")
    rc["frac"] = rc["achieved"] / rc["peak"]
    if tc:
        # the slice products issued on the tensor cores (bf16, dense) against the measured bf16 peak
        tflop = N * tc_slice_flops(Q, R, Cc) / (rc["avg_launch_ms"] / 1e3) / 1e12
        bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)
        rc["tensor_pipe"] = {"achieved": tflop, "peak": bf16_peak, "unit": "TFLOP/s (bf16 slice products)",
                             "frac": tflop / bf16_peak,
                             "peak_source": "measured cuBLAS bf16, sustained" if "bf16_tflops_sustained" in peaks
                             else "fallback 1.7 PFLOP/s"}
    # Krylov vector passes: algorithmic bytes of every Arnoldi step of the timed solves
    # (CGS: multi-dot over nv + 1 vectors, update reading nv + 1 and writing 1; CGS2 (and the
    #  second projection of orth = 2, counted as not taken): two multi-dots and two updates)
    K = args.restart
    steps_bytes = 0.0
    for r in reps:
        its, cyc = r["iterations"], r["restarts"]
        for ci in range(cyc):
            jused = min(K, its - ci * K)
            for j in range(max(jused, 0)):
                nv = j + 1
                steps_bytes += ((4 * nv + 6) if args.orth == 0 else (2 * nv + 3)) * 8.0 * N_tr
                if args.basis == 2:
                    # the new vector is also written in FP64 (the operator's input); chunk scales are
                    # 4 bytes per 2048 entries and vector read
                    steps_bytes += 8.0 * N_tr + ((2 * nv + 1) * 4.0 * N_tr / 2048)
    vk = {0: "d_mdot_kernel + d_update_kernel", 1: "df_mdot_kernel + df_update_kernel",
          2: "fx_mdot_kernel + fx_combine_kernel (fixed-point chunks, exact int64 products)"}[args.basis]
    rooflines["ortho"] = {"kernel": vk + " (+ reduce2_givens_kernel)",
                          "bound": "hbm", "launches": prof["ortho"][0], "avg_launch_ms": avg("ortho"),
                          "achieved": steps_bytes / (prof["ortho"][1] / 1e3) / 1e9 if prof["ortho"][1] else 0.0,
                          "peak": hbm_peak, "unit": "GB/s", "peak_source": hbm_src,
                          "algorithmic_total": steps_bytes,
                          "note": "per Arnoldi step (launches = steps), all passes of that step"}
    rooflines["ortho"]["frac"] = rooflines["ortho"]["achieved"] / rooflines["ortho"]["peak"]
    if args.basis == 0:
        rooflines["ortho"]["fp64_pipe_ceiling_frac_of_hbm"] = fp64_ceiling / hbm_peak
    dom = max(("apply", "condense", "ortho"), key=lambda kname: prof["apply32" if (kname == "apply" and args.mode == 1)
                                                           else kname][1])
    roof = dict(rooflines[dom])
    roof["traffic"] = None
    traffic_per_edge = {(0, 0): APPLY_VDF00_TRAFFIC_PER_EDGE_M8P3, (2, 1): APPLY_VDF1_TRAFFIC_PER_EDGE_M8P3,
                        (3, 0): APPLY_FIX_TRAFFIC_PER_EDGE_M8P3}
    if dom == "apply" and (cfg["m"], cfg["p"]) == (8, 3) and (args.mode, args.basis) in traffic_per_edge \
            and not tune.get("apply_bulk") and traffic_per_edge[(args.mode, args.basis)]:
        roof["traffic"] = traffic_per_edge[(args.mode, args.basis)] * n_int
        roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum at n = 64, scaled by interior edges"
    roof_other = {k: v for k, v in rooflines.items() if k != dom}

    all_fp64 = args.mode in (0, 3) and args.basis in (0, 2) and not split
    dtype = "f64" if all_fp64 else FORM_DTYPES.get((args.mode, args.basis, args.elim), "mixed")
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("GMRES(restart)", f"GMRES({args.restart})").replace(
                           "128x128 macro grid (32768", f"{cfg['n']}x{cfg['n']} macro grid ({N}"),
                       "N_tr": N_tr, "macro_elements": N, "solve_mode": MODE_NAMES[args.mode],
                       "local_factorisation": {"split": "split-FP32", "fp64": "FP64 FMAs",
                                               "tc": "FP64 panels + tensor-core trailing updates by exact 8-bit "
                                                     "slices (FP64-accurate)"}[args.elim],
                       "trace_apply": {0: "FP64 blocks, FP64 FMAs", 1: "FP32 blocks, FP32 FMAs",
                                       2: "split-FP32 blocks on the FP32 pipe",
                                       3: "56-bit fixed-point rows, exact int64 products, one FP64 rounding per "
                                          "element side"}[args.mode],
                       "krylov_basis": ["FP64", "split-FP32",
                                        "fixed-point chunks of 2048 entries (56-bit, exact int64 products)"][args.basis],
                       "orthogonalisation": ["CGS2", "CGS, Pythagorean norm",
                                             "CGS + second projection where ||w - V h||^2 < ||w||^2 / 2",
                                             "CGS + second projection where ||w - V h||^2 < 1e-6 ||w||^2"][args.orth],
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2: Schur blocks 1.47 GB, factors 42 GB, source 0.42 GB per replica"},
            "time_to_solve_s": statistics.median(solve_s), "condense_s": statistics.median(cond_s),
            "recover_s": statistics.median(rec_s), "iterations": reps[-1]["iterations"],
            "restarts": reps[-1]["restarts"], "rel_residual": reps[-1]["rel_residual"],
            "apply_gdofs": N_tr / (rooflines["apply"]["avg_launch_ms"] / 1e3) / 1e9,
            "phases_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
            "roofline": roof, "roofline_other": roof_other, "gpu_launches": int(launches), "clocks": clk,
            "autotune": tune}

    # The metric compares FP64 with FP32 + refinement: the whole step of each precision form
    # (condensation + rhs + GMRES to 1e-10 + back-solve), each with its own autotuned shapes,
    # and each result's relative l2 distance from the all-FP64 step's x, u and q.
    if not args.no_forms:
        _, x64, u64, q64 = step(mode=0, basis=0, elim="fp64")
        torch.cuda.synchronize()
    forms = {}
    for name, (mode, basis, elim) in ({} if args.no_forms else FORMS).items():
        step(mode=mode, basis=basis, elim=elim)
        pr.autotune(mode=mode, restart=args.restart, basis=basis)
        recf = []
        for _ in range(2):
            rep_f, xf, uf, qf = step(recf, mode=mode, basis=basis, elim=elim)
        torch.cuda.synchronize()
        cs = [m[0].elapsed_time(m[1]) / 1e3 for m, _ in recf]
        ss = [m[1].elapsed_time(m[2]) / 1e3 for m, _ in recf]
        rs = [m[2].elapsed_time(m[3]) / 1e3 for m, _ in recf]
        dist = lambda a, b: float((a - b).norm() / b.norm())
        forms[name] = {"dtype": FORM_DTYPES[(mode, basis, elim)],
                       "step_s": statistics.median([c + s2 + r2 for c, s2, r2 in zip(cs, ss, rs)]),
                       "condense_s": statistics.median(cs), "solve_s": statistics.median(ss),
                       "recover_s": statistics.median(rs), "iterations": rep_f["iterations"],
                       "rel_residual": rep_f["rel_residual"], "converged": bool(rep_f["converged"]),
                       "rel_l2_vs_fp64_step": {"trace": dist(xf, x64), "u": dist(uf, u64), "q": dist(qf, q64)}}
    if not args.no_forms:
        # back to the timed step's blocks and launch shapes (the last form kept other blocks)
        pr.condense(**condense_flags(args.mode, args.elim))
        pr.autotune(mode=args.mode, restart=args.restart, basis=args.basis)
        del x64, u64, q64
        line["forms"] = forms

    # the same solve with the preconditioner of the inverted diagonal face blocks of S
    pcs = {}
    solve_kw = dict(tol=1e-10, restart=args.restart, maxit=60000, mode=args.mode, orth=args.orth, basis=args.basis)
    for pc in () if args.no_forms else ("d", "face_schur"):
        pr.condense(precond=pc, **condense_flags(args.mode, args.elim))
        g = pr.rhs()
        pr.solve(g, **solve_kw)
        t0, t1, t2 = ev(), ev(), ev()
        torch.cuda.synchronize()
        t0.record(stream)
        pr.condense(precond=pc, **condense_flags(args.mode, args.elim))
        g = pr.rhs()
        t1.record(stream)
        x, rep, st = pr.solve(g, **solve_kw)
        t2.record(stream)
        torch.cuda.synchronize()
        pcs[pc] = {"condense_s": t0.elapsed_time(t1) / 1e3, "solve_s": t1.elapsed_time(t2) / 1e3,
                   "iterations": rep["iterations"], "rel_residual": rep["rel_residual"],
                   "converged": bool(rep["converged"])}
    pcs["note"] = ("d: D_f^-1 of Sec. 6.1 (the timed step above); face_schur: the inverted diagonal face blocks "
                   "of S folded into the same stored rows (same apply cost), the timed step's precision form")
    line["time_to_solve_by_preconditioner"] = pcs

    if not args.no_e2e:
        # the whole step through the public end-to-end call on pinned host buffers, median of 3 calls
        fh = f.cpu().pin_memory()
        host_kw = dict(outputs=True, restart=args.restart, mode=args.mode, orth=args.orth, basis=args.basis)
        torch.cuda.synchronize()
        pr.run_host(fh, **host_kw)    # warm-up
        torch.cuda.synchronize()
        calls = []
        for _ in range(3):
            t0 = time.perf_counter()
            x, u, q, rep = pr.run_host(fh, **host_kw)
            calls.append((time.perf_counter() - t0, rep))
        e2e_s, rep = sorted(calls, key=lambda c: c[0])[1]
        app_e2e = rep["iterations"] + rep["outer"]
        eu, es = aggregate(N_tr * app_e2e, e2e_s, world)
        line["e2e"] = {"value": eu / es / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": int(fh.numel() * 8),
                       "d2h_bytes_per_step": int((x.numel() + u.numel() + q.numel()) * 8), "seconds": e2e_s,
                       "calls": [round(c[0], 4) for c in calls], "statistic": "median of 3 calls",
                       "call": "hdg_run_host (pinned host f in; x, u, q out)"}
    pr.close()
    del f
    torch.cuda.synchronize()
    if not args.no_extras:
        line["multi_rhs"] = bench_multi_rhs(stream)
        line["levels_many_source"] = bench_levels_many_source(stream)
        line["mixed_precision_n256"] = bench_mixed_precision_n256(stream)
        line["gradient"] = bench_gradient(stream)
        line["macro_vs_standard"] = bench_macro_vs_standard(stream)
        line["supg_layer"] = bench_supg_layer(stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config, int(round(applies / args.steps)))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_multi_rhs(stream, count=64):
    """64 Gaussian-bump sources on one level (n=128, m=4, p=2, kappa=1e-2, beta=(1,0)):
    one condensation with 64 load columns, the lockstep batched GMRES to 1e-10 for all
    columns, against one single-source solve of the same problem (x count = sequential)."""
    import torch
    from paper_2302_10917_gb300 import Problem
    from paper_2302_10917_gb300 import workloads as wl
    cfg = wl.CONFIGS["n128_m4_p2_64src"]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    pr = Problem(cfg["n"], cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], stream=stream)
    f = wl.gaussian_bumps(pr.quad_points(), count, seed=3).contiguous()
    a, b, c2, d = ev(), ev(), ev(), ev()
    torch.cuda.synchronize()
    a.record(stream)
    pr.set_source(f)
    pr.condense(keep_factors=True, store_df64=True, split_update=True)
    g = pr.rhs()
    b.record(stream)
    x, rep, st = pr.solve(g, tol=1e-10, restart=80, mode=2, orth=3, basis=1, maxit=40000)
    c2.record(stream)
    u, q = pr.recover(x)
    d.record(stream)
    torch.cuda.synchronize()
    batched_s = b.elapsed_time(c2) / 1e3
    # one source alone on the same mesh
    p1 = Problem(cfg["n"], cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], stream=stream)
    p1.set_source(f[0])
    p1.condense(keep_factors=True, store_df64=True, split_update=True)
    g1 = p1.rhs()
    p1.solve(g1, tol=1e-10, restart=80, mode=2, orth=3, basis=1)
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    x1, rep1, st1 = p1.solve(g1, tol=1e-10, restart=80, mode=2, orth=3, basis=1)
    e1.record(stream)
    torch.cuda.synchronize()
    single_s = e0.elapsed_time(e1) / 1e3
    out = {"workload": f"n={cfg['n']} m={cfg['m']} p={cfg['p']} kappa={cfg['kappa']} beta={cfg['beta']}, "
                       f"{count} Gaussian-bump sources (width 0.05, seeded centres), uniform level",
           "N_tr": pr.info["N_tr"], "sources": count,
           "condense_and_rhs_s": a.elapsed_time(b) / 1e3, "batched_solve_s": batched_s,
           "batched_iterations": rep["iterations"], "batched_converged": bool(rep["converged"]),
           "batched_max_rel_residual": rep["rel_residual"], "recover_s": c2.elapsed_time(d) / 1e3,
           "single_solve_s": single_s, "single_iterations": rep1["iterations"],
           "sequential_estimate_s": single_s * count, "speedup_vs_sequential": single_s * count / batched_s,
           "column0_rel_diff_to_single": float((x1 - x[0]).abs().max() / x1.abs().max())}
    pr.close()
    p1.close()
    return out


def bench_levels_many_source(stream, count=64):
    """64 Gaussian-bump sources on the banded-level mesh (n=128, p=2, kappa=1e-2, beta=(1,0);
    levels r = 1 below x = 0.7, 2, 3, r = 4 from x = 0.9 on, faces at the finer side's level):
    one condensation with 64 load columns per level plus the face lift, the lockstep batched
    GMRES to 1e-10 for all columns, the back-solve, and the element-side apply kernels alone
    (one column FP64; 64 columns FP64, split-FP32 and FP32 blocks). The preconditioner is the
    inverted diagonal face blocks of S: restarted GMRES with D^-1 stalls on this mesh."""
    import torch
    from paper_2302_10917_gb300 import Problem
    from paper_2302_10917_gb300 import workloads as wl
    cfg = wl.CONFIGS["levels_n128_p2_64src"]
    lev = wl.band_levels(cfg["n"])
    ev = lambda: torch.cuda.Event(enable_timing=True)
    pr = Problem(cfg["n"], 1, cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], stream=stream, levels=lev)
    f = wl.gaussian_bumps(pr.quad_points(), count, seed=3, width=cfg["width"]).contiguous()
    N_tr, ns = pr.info["N_tr"], pr.info["n_s_total"]
    flags = dict(keep_factors=True, store_df64=True, store_fp32=True, split_update=True, precond="face_schur")
    pr.set_source(f)
    pr.condense(**flags)            # first pass: allocations and launch set-up
    tune = pr.autotune(mode=2, restart=80)     # element-side rows per CTA, Krylov launch shapes
    a, b, c2, d = ev(), ev(), ev(), ev()
    torch.cuda.synchronize()
    a.record(stream)
    pr.set_source(f)
    pr.condense(**flags)
    g = pr.rhs()
    b.record(stream)
    x, rep, st = pr.solve(g, tol=1e-10, restart=80, mode=2, orth=3, basis=1, maxit=40000)
    c2.record(stream)
    u, q = pr.recover(x)
    d.record(stream)
    torch.cuda.synchronize()
    # the apply kernels alone (inputs of 64 x 3.7 MB: the blocks, 0.39 GB, exceed L2 for FP64)
    X = torch.randn(count, N_tr, dtype=torch.float64, device=pr.device)

    def time_apply(xx, prec, reps=10):
        xin = xx.float() if prec == 32 else xx
        for _ in range(2):
            pr.apply(xin, precond=True, prec=prec)
        ts = []
        for _ in range(reps):
            e0, e1 = ev(), ev()
            e0.record(stream)
            pr.apply(xin, precond=True, prec=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(ts)
    t1 = time_apply(X[0], 64)
    t1df = time_apply(X[0], 48)
    t64 = {prec: time_apply(X, prec) for prec in (64, 48, 32)}
    from paper_2302_10917_gb300 import OFF_SCHUR
    offs = pr.offsets(OFF_SCHUR)
    rows = int(sum(int(round(math.sqrt(int(offs[e + 1] - offs[e])))) for e in range(pr.info["N"])))
    # one column: blocks (8 B per entry, FP64 or split-FP32 pairs) + gathered x (element-side rows)
    # + element-side products written and read + one y write
    bytes1 = ns * 8 + rows * 8 + 2 * rows * 8 + N_tr * 8
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    flops64 = 2.0 * ns * count
    out = {"workload": f"n={cfg['n']} p={cfg['p']} kappa={cfg['kappa']} beta={cfg['beta']}, levels by band of x "
                       f"(r=1..4: {[int((lev == r).sum()) for r in (1, 2, 3, 4)]} elements), faces at the finer "
                       f"side, {count} Gaussian-bump sources (width {cfg['width']}, seeded centres), g_D = 0",
           "N_tr": N_tr, "element_side_rows": rows, "schur_bytes_fp64": ns * 8, "sources": count,
           "autotune": tune,
           "condense_and_rhs_s": a.elapsed_time(b) / 1e3, "batched_solve_s": b.elapsed_time(c2) / 1e3,
           "batched_iterations": rep["iterations"], "batched_converged": bool(rep["converged"]),
           "batched_max_rel_residual": rep["rel_residual"], "recover_s": c2.elapsed_time(d) / 1e3,
           "apply_1col_fp64_s": t1, "apply_1col_split_s": t1df, "apply_1col_gdofs": N_tr / t1df / 1e9,
           "apply_1col_roofline": {
               "split_fp32": {"bound": "hbm", "achieved": bytes1 / t1df / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": (bytes1 / t1df / 1e9 / hbm) if hbm else None, "traffic": None,
                              "bytes_per_launch": bytes1},
               "fp64": {"bound": "fp64 pipe", "achieved": 2.0 * ns / t1 / 1e12, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": 2.0 * ns / t1 / 1e12 / FP64_PEAK_TFLOPS}},
           "arnoldi_operator_roofline": {
               "kernel": "lv_elem_kernel<1,1,1> + lv_face_kernel (split-FP32 blocks and vectors: the GMRES operator), "
                         "best of 5 in hdg_autotune", "bound": "hbm", "launch_ms": tune["apply_ms"],
               "achieved": bytes1 / (tune["apply_ms"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
               "frac": (bytes1 / (tune["apply_ms"] / 1e3) / 1e9 / hbm) if hbm else None,
               "bytes_per_launch": bytes1},
           "apply_64col_s": {"fp64": t64[64], "split_fp32": t64[48], "fp32": t64[32]},
           "apply_64col_gdofs": {k: N_tr * count / v / 1e9 for k, v in
                                 (("fp64", t64[64]), ("split_fp32", t64[48]), ("fp32", t64[32]))},
           "apply_64col_roofline": {
               "fp64": {"bound": "fp64 pipe", "achieved": flops64 / t64[64] / 1e12, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": flops64 / t64[64] / 1e12 / FP64_PEAK_TFLOPS},
               "split_fp32": {"bound": "alu (FP32 pipe, split arithmetic)", "achieved": flops64 / t64[48] / 1e12,
                              "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s (FP64-equivalent)",
                              "frac": flops64 / t64[48] / 1e12 / DF_PEAK_TFLOPS}}}
    pr.close()
    return out


def bench_mixed_precision_n256(stream):
    """The large workload's element at n = 256 (131 072 macro-elements, N_tr = 4 902 400),
    face-block preconditioner, GMRES(80) to 1e-10, in the three precision forms: all-FP64
    (FP64 elimination, blocks, operator, Krylov basis); FP32+IR (the same FP64 elimination,
    the preconditioned blocks stored and applied in FP32 inside FP64 residual replacement, FP64
    basis and orthogonalisation); split-FP32 (split-FP32 elimination, blocks and basis). Each
    form's solution (trace, u, q) against the all-FP64 one (relative l2), and u against the
    manufactured solution at the lattice nodes."""
    import math
    import torch
    from paper_2302_10917_gb300 import Problem
    from paper_2302_10917_gb300 import workloads as wl
    cfg = wl.CONFIGS["n256_m8_p3"]
    pr = Problem(cfg["n"], cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], stream=stream)
    pr.set_source(wl.sin_sin_source(pr.quad_points(), cfg["kappa"], cfg["beta"]).contiguous())
    ev = lambda: torch.cuda.Event(enable_timing=True)
    xy = _lattice_nodes(cfg["n"], cfg["m"], cfg["p"], "cuda")
    u_ex = torch.sin(math.pi * xy[..., 0]) * torch.sin(math.pi * xy[..., 1])
    del xy
    out = {"workload": f"n={cfg['n']} m={cfg['m']} p={cfg['p']} beta=50(cos 0.3, sin 0.3) kappa=1, "
                       "u = sin(pi x) sin(pi y); face-block preconditioner, GMRES(80), orth 3",
           "N_tr": pr.info["N_tr"], "forms": {}}
    sols = {}
    for name, (mode, basis, elim) in FORMS.items():
        if name == "fp64_dfma":
            continue
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        # factors not kept (131 072 local systems would take 169 GB): chunked condensation, the
        # back-solve condenses each chunk again
        pr.condense(keep_factors=False, store_fp32=(mode == 1), store_df64=(mode == 2), store_fix=(mode == 3),
                    split_update=elim == "split", tc_update=elim == "tc", precond="face_schur")
        b.record(stream)
        g = pr.rhs()
        pr.autotune(mode=mode, restart=80, basis=basis)
        t0, t1 = ev(), ev()
        torch.cuda.synchronize()
        t0.record(stream)
        x, rep, st = pr.solve(g, tol=1e-10, restart=80, maxit=60000, mode=mode, orth=3, basis=basis)
        t1.record(stream)
        torch.cuda.synchronize()
        u, q = pr.recover(x)
        sols[name] = (x, u, q)
        out["forms"][name] = {"dtype": FORM_DTYPES[(mode, basis, elim)], "condense_s": a.elapsed_time(b) / 1e3,
                              "solve_s": t0.elapsed_time(t1) / 1e3, "iterations": rep["iterations"],
                              "rel_residual": rep["rel_residual"], "converged": bool(rep["converged"]),
                              "max_nodal_error_u": float((u - u_ex).abs().max())}
    rel = lambda a, b: float((a - b).norm() / b.norm())
    for name in sols:
        if name != "fp64":
            out["forms"][name]["rel_l2_vs_fp64"] = {
                k: rel(sols[name][i], sols["fp64"][i]) for i, k in enumerate(("trace", "u", "q"))}
    pr.close()
    return out


def _lattice_nodes(n, m, p, device):
    """Physical coordinates [N, Q, 2] of every element's lattice nodes (the "/" mesh
    conventions of the C ABI: element 2 (j n + i) + t, node (a, b) at v0 + a/P (v1 - v0)
    + b/P (v2 - v0), b-major)."""
    import torch
    P = m * p
    ab = torch.tensor([(a, b) for b in range(P + 1) for a in range(P + 1 - b)], dtype=torch.float64, device=device) / P
    h = 1.0 / n
    sq = torch.arange(n * n, device=device)
    i, j = (sq % n).double(), (sq // n).double()
    x0, x1, y0, y1 = i * h, (i + 1) * h, j * h, (j + 1) * h
    v = torch.empty(2 * n * n, 3, 2, dtype=torch.float64, device=device)
    v[0::2, 0, 0], v[0::2, 0, 1], v[0::2, 1, 0], v[0::2, 1, 1], v[0::2, 2, 0], v[0::2, 2, 1] = x1, y0, x1, y1, x0, y0
    v[1::2, 0, 0], v[1::2, 0, 1], v[1::2, 1, 0], v[1::2, 1, 1], v[1::2, 2, 0], v[1::2, 2, 1] = x0, y1, x0, y0, x1, y1
    return v[:, None, 0, :] + ab[None, :, 0:1] * (v[:, None, 1, :] - v[:, None, 0, :]) + \
        ab[None, :, 1:2] * (v[:, None, 2, :] - v[:, None, 0, :])


def bench_macro_vs_standard(stream):
    """The paper's comparison with standard HDG (Sec. 5.3; Tables 8 and 10 of Sec. 6.3-6.4) in 2D:
    the same 65 536 sub-triangles of degree 3 as n = 32 macro-squares with m = 8 (macro-element HDG) and as n = 256 squares
    with m = 1 (standard HDG), beta = 50 (cos 0.3, sin 0.3), kappa = 1, u = sin(pi x) sin(pi y);
    GMRES(80), split-FP32 operator, to 1e-10."""
    import math
    import torch
    from paper_2302_10917_gb300 import Problem
    from paper_2302_10917_gb300 import workloads as wl
    beta = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {}
    for name, (n, m) in {"macro_m8": (32, 8), "standard_m1": (256, 1)}.items():
        pr = Problem(n, m, 3, beta=beta, kappa=1.0, stream=stream)
        f = wl.sin_sin_source(pr.quad_points(), 1.0, beta).contiguous()
        pr.set_source(f)
        pr.condense(keep_factors=True, store_df64=True, split_update=True)
        g = pr.rhs()
        pr.solve(g, tol=1e-10, restart=80, mode=2, orth=3, basis=1)      # warm-up (graph capture)
        a, b, c2 = ev(), ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        pr.set_source(f)
        pr.condense(keep_factors=True, store_df64=True, split_update=True)
        g = pr.rhs()
        b.record(stream)
        x, rep, st = pr.solve(g, tol=1e-10, restart=80, mode=2, orth=3, basis=1)
        c2.record(stream)
        u, q = pr.recover(x)
        torch.cuda.synchronize()
        xy = _lattice_nodes(n, m, 3, u.device)
        err = float((u - wl.sin_sin_exact(xy)).abs().max())
        out[name] = {"n": n, "m": m, "p": 3, "sub_triangles": 2 * n * n * m * m, "N_tr": pr.info["N_tr"],
                     "condense_s": a.elapsed_time(b) / 1e3, "solve_s": b.elapsed_time(c2) / 1e3,
                     "iterations": rep["iterations"], "converged": bool(rep["converged"]),
                     "max_nodal_error": err}
        pr.close()
    return out


def bench_supg_layer(stream):
    """The paper's SUPG comparison (Sec. 3.4 and its kappa = 1e-5 figure) in 2D, as
    source-free transport: kappa = 1e-5, beta = (1, 1), f = 0, g_D = the interior-layer
    profile (1 + tanh((y - 2x + 0.4) / kappa)) / 2 on the boundary (a step), n = 32, m = 4,
    p = 3, without and with SUPG. The maximum principle bounds u to [0, 1]; reported: the
    range of the nodal values and the solve statistics."""
    import torch
    from paper_2302_10917_gb300 import Problem
    from paper_2302_10917_gb300 import workloads as wl
    n, m, p, kap, beta = 32, 4, 3, 1e-5, (1.0, 1.0)
    out = {}
    for supg in (False, True):
        pr = Problem(n, m, p, beta=beta, kappa=kap, stream=stream, supg=supg)
        f = torch.zeros(pr.info["N"], pr.info["n_qp"], dtype=torch.float64, device="cuda")
        gD = wl.tanh_layer_exact(pr.bnd_quad_points(), kap).contiguous()
        pr.set_source(f, gD)
        pr.condense(keep_factors=True, store_df64=True, split_update=True)
        x, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=80, mode=2, orth=3, basis=1, maxit=40000, check=False)
        u, q = pr.recover(x)
        out["supg" if supg else "plain"] = {"u_min": float(u.min()), "u_max": float(u.max()),
                                            "overshoot": float(max(u.max() - 1.0, -u.min(), 0.0)),
                                            "iterations": rep["iterations"], "converged": bool(rep["converged"])}
        pr.close()
    out["workload"] = (f"n={n} m={m} p={p} kappa={kap} beta={beta}, f = 0, g_D = interior-layer step; "
                       "exact range [0, 1]")
    return out


def bench_gradient(stream, fd_directions=20):
    """Adjoint gradient of J = 1/2 |u - u_obs|^2 (nodal) with respect to the per-element
    diffusivities and the source, n=256, m=4, p=2, beta=(1,0.5), kappa_e = exp(GRF); forward
    and adjoint GMRES(128) with the face blocks of S (with D^-1 the solve stalls at this size)."""
    import torch
    from paper_2302_10917_gb300 import Problem, solve_u
    from paper_2302_10917_gb300 import workloads as wl
    n, m, p, beta = 256, 4, 2, (1.0, 0.5)
    kap = torch.from_numpy(wl.grf_kappa(n, 1)).cuda()
    kobs = torch.from_numpy(wl.grf_kappa(n, 1001)).cuda()
    pr = Problem(n, m, p, beta=beta, kappa=kap.cpu().numpy(), stream=stream)
    f = wl.sin_sin_source(pr.quad_points(), 1.0, beta).contiguous()
    opts = dict(tol=1e-10, restart=128, mode=2, split_update=True, orth=3, basis=1, precond="face_schur", maxit=60000)
    with torch.no_grad():
        u_obs = solve_u(pr, kobs, f, **opts).clone()      # also the warm-up (graph capture)
    times = []
    for _ in range(1):
        k = kap.clone().requires_grad_(True)
        ff = f.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = 0.5 * ((solve_u(pr, k, ff, **opts) - u_obs) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        times.append((t1 - t0, time.perf_counter() - t1))
    out = {"workload": f"n={n} m={m} p={p} beta={beta}, kappa_e = exp(GRF std 0.5, length 0.1), "
                       "J = 1/2 |u - u_obs|^2 nodal; face-block preconditioner", "N_tr": pr.info["N_tr"],
           "forward_s": times[-1][0], "backward_s": times[-1][1], "J": float(J.detach()),
           "grad_kappa_norm": float(k.grad.norm()), "grad_f_norm": float(ff.grad.norm())}
    if fd_directions > 0:
        out["finite_differences"] = gradient_fd_check(pr, kap, f, u_obs, k.grad, ff.grad, opts, fd_directions)
    pr.close()
    return out


def gradient_fd_check(pr, kap, f, u_obs, gk, gf, opts, count, h=1e-3):
    """Central differences of J along `count` seeded directions (d_kappa, d_f) at once:
    kappa_e (1 + h z_e) and f + h |f|_max w, J(+) - J(-) over 2h against the adjoint
    gradient's dJ/dkappa . (kappa z) + dJ/df . (|f|_max w). Each perturbed solve starts from
    the unperturbed trace solution (same solve options as the gradient)."""
    import torch
    from paper_2302_10917_gb300 import workloads as wl
    fmax = float(f.abs().max())
    Z = torch.from_numpy(wl.random_directions(count, tuple(kap.shape), seed=5)).cuda()
    Wd = torch.from_numpy(wl.random_directions(count, tuple(f.shape), seed=6)).cuda()
    sk = dict(tol=opts["tol"], restart=opts["restart"], mode=opts["mode"], orth=opts["orth"],
              basis=opts["basis"], maxit=opts["maxit"])

    def J_of(kk, fv, x0):
        pr.set_kappa(kk)
        pr.set_source(fv)
        pr.condense(keep_factors=True, store_df64=opts["mode"] == 2, store_fp32=opts["mode"] == 1,
                    store_fix=opts["mode"] == 3, split_update=opts["split_update"], precond=opts["precond"])
        x, rep, st = pr.solve(pr.rhs(), x0=x0, **sk)
        if st != 0:
            raise RuntimeError(f"finite-difference solve did not converge: {rep}")
        u, _ = pr.recover(x)
        return 0.5 * float(((u - u_obs) ** 2).sum()), x

    t0 = time.perf_counter()
    _, x_base = J_of(kap, f, None)
    devs, rows = [], []
    for i in range(count):
        dk, df = kap * Z[i], fmax * Wd[i]
        jp, _ = J_of(kap + h * dk, f + h * df, x_base)
        jm, _ = J_of(kap - h * dk, f - h * df, x_base)
        fd = (jp - jm) / (2.0 * h)
        ad = float((gk * dk).sum() + (gf * df).sum())
        devs.append(abs(fd - ad) / abs(ad))
        rows.append({"fd": fd, "adjoint": ad})
    return {"directions": count, "h": h, "max_rel_deviation": max(devs), "median_rel_deviation":
            statistics.median(devs), "seconds": time.perf_counter() - t0, "first": rows[:3],
            "directions_def": "kappa_e (1 + h z_e), f + h |f|_max w; z, w seeded standard normal"}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark: CG + smoothed-aggregation AMG solve phase on 150^3 Poisson.

Workload: 3D Poisson, 7-point stencil on a 150^3 grid (3,375,000 unknowns,
23,490,000 nonzeros), f = A u* with seeded u* ~ U(-1,1), x0 = 0, CG
preconditioned by one SA-AMG V-cycle (strength 0.08, damped Jacobi 0.72, one
pre- and one post-sweep, coarsest <= 500 rows, dense coarsest solve), rtol 1e-8,
FP64.  A step is one complete solve on the resident hierarchy (setup excluded,
as in the metric).  The finest-level matrix alone (282 MB) exceeds the 129 MB
L2, so no L2 flush is needed between steps.

The same JSON line carries the other workloads as legs: the float32 and
bfloat16-stored V-cycles on the same problem (`mixed`), the 200^3
variable-coefficient problem in three precisions (`varcoef200`), 4096 batched
2D systems in one persistent launch (`batched`) and a stream of 2000 served
requests (`serving`); each leg can be skipped (--no-mixed, --no-varcoef,
--no-batch, --no-serve).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "CG+SA-AMG solve s & HBM GB/s (150^3 Poisson, rtol 1e-8); solves/s, p50/p99"
SIDE = 150
RTOL = 1e-8
MAXITER = 200
SEED = 0
OPEN_LOOP_LOAD = 0.5  # serving: open-loop arrival rate as a fraction of the saturated rate
WORKLOAD = "poisson3d-150^3 7-point, f = A u*, CG + SA-AMG (eps 0.08, Jacobi 0.72, 1/1 sweeps, coarse <= 500), rtol 1e-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-serial-sample", type=int, default=200,
                    help="requests of the plain-API baseline (evenly spaced, scaled to the stream); 0 = all")
    ap.add_argument("--no-varcoef", action="store_true")
    ap.add_argument("--serve-slots", type=int, default=8)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------- ranks (one per GPU)
# The single-system solve does not shard (replicas only): every rank solves
# the whole workload and the job's rate is ranks x steps / slowest rank's
# time.  The batched and served forms are independent problems: whole systems
# (requests, grouped by the matrix key they share) are split over the ranks,
# with no collective on the data path -- only the host-side max of the ranks'
# times and the gather of per-request latencies.
def shard_by_weight(weights, world):
    """Rank of each item: greedy bytes-balanced assignment (heaviest first,
    each to the least-loaded rank; ties to the lower index and the lower
    rank), so every rank computes the same assignment without communicating.
    The heaviest rank exceeds the mean load by at most the heaviest item."""
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0.0] * world
    rank_of = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        rank_of[i] = r
        load[r] += weights[i]
    return rank_of


def shard_requests(reqs, n_of, world):
    """Rank of each request: requests that share a matrix key stay on one
    rank (the key's hierarchy is resident there); keys are balanced by the
    rows their requests solve."""
    keys = sorted({q.key for q in reqs})
    w = {k: 0.0 for k in keys}
    for q in reqs:
        w[q.key] += n_of(q)
    rk = dict(zip(keys, shard_by_weight([w[k] for k in keys], world)))
    return [rk[q.key] for q in reqs]


def max_over_ranks(value, world, device=None):
    """The largest value over the ranks (host-side reduction; CUDA tensors
    under NCCL, CPU tensors under gloo)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_lists(items, world):
    """Concatenation of every rank's list, in rank order."""
    if world == 1:
        return list(items)
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, list(items))
    return [v for part in out for v in part]


# ------------------------------------------------------------ algorithmic bytes
def kernel_bytes(info):
    """Algorithmic DRAM bytes per launch of each finest-level kernel (FP64 values,
    int32 indices and row pointers; every array touched once per kernel, the
    gathered vector counted once).  With the fused restriction operator M on
    the finest level (info["nnz_m"][0] > 0) the restriction kernel is f_1 = M r
    and the prolongation forms x = d r + P x_1; there is no pre-sweep kernel."""
    n0, z0 = info["rows"][0], info["nnz"][0]
    n1 = info["rows"][1] if info["levels"] > 1 else 0
    zp, zm = info["nnz_p"][0], info["nnz_m"][0]
    out = {
        "spmv_dot": 12 * z0 + 4 * n0 + 8 * n0 + 8 * n0,           # A, row_ptr, p, q
        "presmooth_l0": 12 * z0 + 4 * n0 + 16 * n0 + 16 * n0,     # A, d f read, x t written
        "restrict_l0": 12 * zp + 4 * n1 + 8 * n0 + 8 * n1,        # R, t, f_1
        "prolong_l0": 12 * zp + 4 * n0 + 8 * n1 + 16 * n0,        # P, x_1, x read+write
        "postsmooth_l0": 12 * z0 + 4 * n0 + 8 * n0 + 16 * n0 + 8 * n0,  # A, x, d f, z
    }
    if zm:
        del out["presmooth_l0"]
        out["restrict_l0"] = 12 * zm + 4 * n1 + 8 * n0 + 8 * n1   # M, r gathered, f_1
        out["prolong_l0"] = 12 * zp + 4 * n0 + 8 * n1 + 24 * n0   # P, x_1, d r read, x written
    return out


def kernel_bytes_mixed(info, vb):
    """As kernel_bytes for the float32 V-cycle with vb-byte matrix values (4:
    float32, 2: bfloat16): float32 level vectors; the finest level reads the
    Krylov vector as the float32 copy the Krylov kernels write, and writes z
    in float64 with the float64 dot product r.z.  (The float V-cycles do not
    use the fused restriction operator.)"""
    n0, z0 = info["rows"][0], info["nnz"][0]
    n1 = info["rows"][1] if info["levels"] > 1 else 0
    zp = info["nnz_p"][0]
    e = vb + 4
    return {
        "spmv_dot": 12 * z0 + 4 * n0 + 8 * n0 + 8 * n0,       # FP64, as kernel_bytes
        "presmooth_l0": e * z0 + 4 * n0 + 8 * n0 + 8 * n0,    # A, d r (f32) read, x t (f32) written
        "restrict_l0": e * zp + 4 * n1 + 4 * n0 + 4 * n1,     # R, t, f_1
        "prolong_l0": e * zp + 4 * n0 + 4 * n1 + 8 * n0,      # P, x_1, x read+write
        "postsmooth_l0": e * z0 + 4 * n0 + 4 * n0 + 8 * n0 + 8 * n0 + 8 * n0,  # A, x, d r (f32), r (f64), z (f64)
    }


# GB300's FP64 vector rate: 1.25 TFLOP/s nominal, i.e. about 4 FP64 flops (two
# fused multiply-adds) per clock per SM at 152 SMs x 2.07 GHz.  The FP64 CSR
# kernels do 2 flops per 12 bytes, so at 6.7 TB/s they need 1.1 TFLOP/s: they
# are bound by HBM and the FP64 pipe together.
FP64_PEAK_GFLOPS = 1250.0


def kernel_flops(info):
    """FP64 operations per launch of each finest-level kernel (a fused
    multiply-add counts 2)."""
    n0, z0 = info["rows"][0], info["nnz"][0]
    zp, zm = info["nnz_p"][0], info["nnz_m"][0]
    out = {
        "spmv_dot": 2 * z0 + 2 * n0,              # A p, p.q
        "presmooth_l0": 2 * z0 + 2 * n0,          # A (d f) on scaled values, x = d f, t = f - s
        "restrict_l0": 2 * zp,                    # R t
        "prolong_l0": 2 * zp + n0,                # x += P x_1
        "postsmooth_l0": 2 * z0 + 5 * n0,         # A x, f - s, x + d (.), f.y
    }
    if zm:
        del out["presmooth_l0"]
        out["restrict_l0"] = 2 * zm               # M r
        out["prolong_l0"] = 2 * zp + 2 * n0       # d r + P x_1
    return out


def bytes_per_iteration(info, coarse_n):
    """Algorithmic bytes of one CG iteration (the kernels the solve launches)."""
    b = 0
    L = info["levels"]
    for l in range(L - 1):
        n, z, zp, nc = info["rows"][l], info["nnz"][l], info["nnz_p"][l], info["rows"][l + 1]
        zm = info["nnz_m"][l]
        if zm:
            b += 12 * zm + 4 * nc + 8 * n + 8 * nc   # f_{l+1} = M f
            b += 12 * zp + 4 * n + 8 * nc + 24 * n   # x = d f + P x_{l+1}
        else:
            b += 12 * z + 4 * n + 32 * n             # presmooth + residual
            b += 12 * zp + 4 * nc + 8 * n + 8 * nc   # restrict
            b += 12 * zp + 4 * n + 8 * nc + 16 * n   # prolong + correct
        b += 12 * z + 4 * n + 32 * n                 # postsmooth
    b += 8 * coarse_n * coarse_n + 16 * coarse_n     # dense coarsest solve
    n0, z0 = info["rows"][0], info["nnz"][0]
    b += 12 * z0 + 20 * n0                           # q = A p, p.q
    b += 24 * n0 + 40 * n0                           # r update; x += alpha p with the p update
    return b


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# Nominal HBM3e bandwidth of one GB300 (8 TB/s class; 7.9 TB/s): the roofline
# fraction is also reported against it, beside the measured copy bandwidth.
NOMINAL_HBM_GBS = 7900.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def spmv_code_digest():
    """SHA-256 (first 16 hex digits) of csrc/spmv.cu's code: every line with
    its // comment removed and trailing blanks stripped, blank lines dropped,
    so that an edit of comments alone keeps the digest."""
    import hashlib
    src = os.path.join(ROOT, "paper_1811_05704_gb300", "csrc", "spmv.cu")
    lines = []
    for line in open(src, encoding="utf-8").read().splitlines():
        i = line.find("//")
        if i >= 0:
            line = line[:i]
        line = line.rstrip()
        if line:
            lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def committed_traffic(kernel_class):
    """Per-launch DRAM bytes from the committed ncu summary of this kernel, or
    None if the summary is missing or the kernel code changed since."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel_class}_poisson150.txt")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("spmv_cu_code_sha256_16") != spmv_code_digest():
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------- reference
def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    A = gen.poisson3d(SIDE)
    f, _ = gen.rhs_from_solution(A, SEED)
    H = oracle.Hierarchy(A)
    times, its = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        x, it, rr, st = H.cg(f, rtol=RTOL, maxiter=MAXITER)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            its.append(it)
    total = sum(times)
    value = len(times) / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
        "config": {"workload": WORKLOAD, "precision": "fp64", "l2": "inputs larger than L2"},
        "solve_s": statistics.median(times), "iterations": its[0],
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "each step one full 150^3 CG solve of the FP64 oracle (setup excluded)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def cpu_baseline_sample():
    """The FP64 oracle, single-threaded, on one full solve of the same workload."""
    import oracle
    A = gen.poisson3d(SIDE)
    f, _ = gen.rhs_from_solution(A, SEED)
    H = oracle.Hierarchy(A)
    t0 = time.perf_counter()
    x, it, rr, st = H.cg(f, rtol=RTOL, maxiter=MAXITER)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"one full 150^3 CG solve of the FP64 oracle ({it} iterations, "
                      f"{dt:.2f} s, setup excluded)"}


# ------------------------------------------------------------------ batched
BATCH_SYSTEMS = 4096


def batched_shard(rank, world):
    """Indices of the batched workload's systems that this rank solves
    (bytes-balanced by nonzeros, about 5 n^2 for side n)."""
    sides, _ = gen.batched_sides(BATCH_SYSTEMS, 0)
    rank_of = shard_by_weight([5.0 * int(m) ** 2 for m in sides], world)
    return [k for k in range(BATCH_SYSTEMS) if rank_of[k] == rank]


def bench_batched(amg, torch, dev, stream, args, rank=0, world=1):
    """4096 independent 2D Poisson systems (sides U{16..128}, shift U(0,0.1),
    f ~ U(-1,1)), FP32 V-cycle under FP64 CG, rtol 1e-8, one persistent launch
    with the autotuned schedule; against the plain FP64 single-system solve
    (amg_solve per system) timed on an evenly spaced sample of the same
    systems and scaled to all of them.  With several ranks each solves its
    shard of the systems and the slowest rank's time counts."""
    sides, sigma = gen.batched_sides(BATCH_SYSTEMS, 0)
    mine = batched_shard(rank, world)
    nsys = len(mine)
    mats = [gen.poisson2d_shift(int(sides[k]), float(sigma[k])) for k in mine]
    rhs = [gen.uniform_pm1(0, 1000 + k, A.n) for k, A in zip(mine, mats)]
    t0 = time.perf_counter()
    b = amg.amg_batch_setup([amg.make_csr(A.n, A.row_ptr, A.col, A.val) for A in mats],
                            amg.amg_params_default(precision=amg.AMG_PRECISION_FP32))
    setup_s = time.perf_counter() - t0
    tot, off, lev = amg.amg_batch_info(b, nsys)
    f = torch.from_numpy(np.concatenate(rhs)).to(dev)
    x = torch.zeros(tot, dtype=torch.float64, device=dev)
    threads, ctas = amg.amg_batch_tune(b, f, x, RTOL, MAXITER)
    reps = max(3, args.steps // 4)
    times = []
    for _ in range(reps):
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, it, rr, sst = amg.amg_batch_solve(b, nsys, f, x, RTOL, MAXITER)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        assert st == 0 and (rr <= RTOL).all()
    iter_bytes = amg.amg_batch_bytes(b, nsys)
    amg.amg_batch_free(b)
    batch_s = max_over_ranks(statistics.median(times), world, dev)
    moved = float(sum(gather_lists([float(np.dot(iter_bytes, it))], world)))
    # plain FP64 path: one handle and one solve per system, on a sample
    sample = list(range(0, nsys, max(1, nsys // 128)))
    plain = 0.0
    for k in sample:
        A = mats[k]
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
        fk = torch.from_numpy(rhs[k]).to(dev)
        xk = torch.zeros(A.n, dtype=torch.float64, device=dev)
        S.solve(fk, xk, RTOL, MAXITER)  # builds and caches the graph
        xk.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        S.solve(fk, xk, RTOL, MAXITER)
        plain += time.perf_counter() - t1
        S.close()
    plain_s = max_over_ranks(plain * nsys / len(sample), world, dev)
    it = np.array(gather_lists([int(v) for v in it], world))
    return {"workload": f"{BATCH_SYSTEMS} x 2D Poisson + shift, sides U{{16..128}}, FP32 V-cycle + FP64 CG",
            "unknowns": int(sum(gather_lists([int(tot)], world))),
            "ranks": world, "setup_s": max_over_ranks(setup_s, world, dev), "solve_s": batch_s,
            "value": BATCH_SYSTEMS / batch_s, "unit": "systems/s",
            "iterations_mean": float(np.mean(it)), "iterations_max": int(np.max(it)),
            "levels_max": int(max_over_ranks(lev.max(), world, dev)),
            "schedule": {"threads": threads, "ctas_per_sm": ctas},
            "hbm_gbs": moved / batch_s / 1e9,
            "frac_of_peak": moved / batch_s / 1e9 / peaks()[0],
            "bytes_note": "algorithmic bytes (amg_batch_bytes: each system's bytes per CG iteration, float32 "
                          "V-cycle model) x its iterations, summed over the systems, / the batch solve time",
            "plain_fp64_solve_s": plain_s,
            "plain_note": f"amg_solve per system (FP64, CUDA graph) on {len(sample)} evenly spaced systems"
                          f" of each rank's {nsys}, scaled to them (slowest rank)",
            "speedup_vs_plain": plain_s / batch_s}


def bench_varcoef(amg, torch, dev, stream, args, rank=0, world=1):
    """The 200^3 variable-coefficient workload (8,000,000 unknowns, 55,760,000
    nonzeros; k = 10^U(-3,3) per cell, 10% of the cells with z-anisotropy 0.01,
    harmonic-mean faces; f = A u*, x0 = 0), rtol 1e-8: set-up time, then the
    FP64 solve and the FP32 and bfloat16-stored V-cycles under FP64 CG, each
    timed with CUDA events over `reps` solves on the resident hierarchy, with
    algorithmic GB/s (amg_hierarchy_bytes x iterations / solve time).  With
    several ranks every rank solves the whole problem (replicas)."""
    A = gen.varcoef3d(200, seed=0)
    f, _ = gen.rhs_from_solution(A, 0)
    ft = torch.from_numpy(f).to(dev)
    x = torch.zeros(A.n, dtype=torch.float64, device=dev)
    reps = 3
    out = {"workload": "varcoef3d-200^3 FV diffusion, k = 10^U(-3,3), 10% z-anisotropy 0.01, f = A u*, rtol 1e-8",
           "unknowns": A.n, "nnz": A.nnz, "reps": reps}
    x64 = None
    peak = peaks()[0]
    for name, prec in (("fp64", amg.AMG_PRECISION_FP64), ("fp32", amg.AMG_PRECISION_FP32),
                       ("bf16", amg.AMG_PRECISION_BF16)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=prec)
        setup_s = time.perf_counter() - t0
        info = S.info()
        x.zero_()
        S.solve(ft, x, RTOL, 500)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            x.zero_()
            st, it, rr = S.solve(ft, x, RTOL, 500)
        e1.record(stream)
        torch.cuda.synchronize()
        solve_s = max_over_ranks(e0.elapsed_time(e1) / 1e3 / reps, world, dev)
        gbs = amg.amg_hierarchy_bytes(S.handle) * it / solve_s / 1e9
        r = {"setup_s": max_over_ranks(setup_s, world, dev), "solve_s": solve_s, "iterations": it, "relres": rr,
             "status": st, "hbm_gbs": gbs, "frac_of_peak": gbs / peak, "levels": info["levels"],
             "operator_complexity": sum(info["nnz"]) / info["nnz"][0]}
        if x64 is None:
            x64 = x.clone()
        else:
            r["rel_diff_vs_fp64_x"] = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
            r["speedup_vs_fp64"] = out["fp64"]["solve_s"] / solve_s
        out[name] = r
        S.close()
    return out


def _serve_matrices(reqs):
    """Matrices of a request stream, generated in parallel; varcoef and
    convdiff matrices take the grid side as their seed, so one matrix per
    (kind, side) is generated and shared by the keys that ask for it (each key
    still gets its own hierarchy)."""
    import concurrent.futures as cf
    combos = sorted({(q.kind, q.side) for q in reqs})

    def make(c):
        kind, side = c
        if kind == "poisson":
            return gen.poisson3d(side)
        if kind == "varcoef":
            return gen.varcoef3d(side, seed=side, log10_range=gen.problems.SERVE_VARCOEF_RANGE)
        return gen.convdiff3d(side, seed=side)[0]

    with cf.ThreadPoolExecutor(8) as ex:
        return dict(zip(combos, ex.map(make, combos)))


def bench_serving(amg, args, rank=0, world=1, dev=None):
    """A stream of solve requests through the server: grid sides log-uniform
    on [20, 160] (8,000 to 4,096,000 unknowns), 70% SPD (3D Poisson and
    variable-coefficient diffusion with k = 10^U(-2,2), CG), 30% upwind convection-diffusion
    (BiCGStab with the SPAI-0 smoother), 20% of the requests a new right-hand side for an earlier
    request's matrix; every request is set up (unless its hierarchy is
    resident) and solved to rtol 1e-8 from host memory.  Saturated
    throughput (all requests queued at once) against the plain API serving
    the same requests one after another (amg_setup + amg_solve_host, a
    hierarchy kept until its key's last request), then latency under Poisson
    arrivals at half the saturated rate (OPEN_LOOP_LOAD)."""
    nreq, slots = args.serve_requests, args.serve_slots
    allreq = gen.serving_requests(nreq, SEED, lo=20, hi=160)
    # with several ranks, each serves the requests of its share of the matrix keys
    rank_of = shard_requests(allreq, lambda q: q.side ** 3, world)
    reqs = [q for q in allreq if rank_of[q.index] == rank]
    t0 = time.perf_counter()
    mats = _serve_matrices(reqs)
    gen_s = time.perf_counter() - t0
    A_of = lambda q: mats[(q.kind, q.side)]  # noqa: E731
    # CG + damped Jacobi for SPD requests; BiCGStab + SPAI-0 for convection-diffusion.  Most
    # requests get one solve per set-up, so the fused restriction operator (a set-up product
    # that pays off over several solves) is left out, for the server and the plain API alike.
    prm_cg = amg.amg_params_default(fused_restriction=0)
    prm_bi = amg.amg_params_default(solver=amg.AMG_SOLVER_BICGSTAB, smoother=amg.AMG_SMOOTHER_SPAI0,
                                    fused_restriction=0)
    prm_of = lambda q: prm_bi if q.solver else prm_cg  # noqa: E731
    rhs = {q.index: q.rhs(SEED, A_of(q).n) for q in reqs}
    csrs = {c: amg.make_csr(A.n, A.row_ptr, A.col, A.val) for c, A in mats.items()}
    last_use = {q.key: q.index for q in reqs}
    rows = sum(gather_lists([int(sum(A_of(q).n for q in reqs))], world))

    # plain API, one request after another: on every `stride`-th request of
    # this rank's stream (all of them for short streams), scaled to the stream
    stride = max(1, len(reqs) // args.serve_serial_sample) if args.serve_serial_sample > 0 else 1
    sample = reqs[::stride]
    last_in_sample = {q.key: q.index for q in sample}
    handles, serial_status = {}, {}
    t0 = time.perf_counter()
    for q in sample:
        if q.key not in handles:
            handles[q.key] = amg.amg_setup(csrs[(q.kind, q.side)], prm_of(q))
        x = np.zeros(A_of(q).n)
        serial_status[q.index] = amg.amg_solve_host(handles[q.key], rhs[q.index], x, RTOL, MAXITER)[0]
        if last_in_sample[q.key] == q.index:
            amg.amg_free(handles.pop(q.key))
    serial_s = max_over_ranks((time.perf_counter() - t0) * len(reqs) / max(1, len(sample)), world, dev)

    def run(arrival):
        """Submit every request at its arrival time (None: all at once),
        then collect the results."""
        srv = amg.amg_server_create(slots=slots)
        ids = []
        t_start = time.perf_counter()
        for q in reqs:
            if arrival is not None:
                delay = t_start + arrival[q.index] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            ids.append(amg.amg_server_submit(srv, q.key, csrs[(q.kind, q.side)], rhs[q.index], prm_of(q),
                                             RTOL, MAXITER))
        res = []
        for q, rid in zip(reqs, ids):
            r = amg.amg_server_wait(srv, rid, A_of(q).n)
            res.append(r + ((amg.amg_last_error() if r[0] != 0 else ""),))
        wall = time.perf_counter() - t_start
        stats = amg.amg_server_stats(srv)
        stats["solve_bytes"] = amg.amg_server_solve_bytes(srv)
        amg.amg_server_destroy(srv)
        return wall, res, stats

    sat_s, sat_res, sat_stats = run(None)
    sat_s = max_over_ranks(sat_s, world, dev)
    sat_rate = nreq / sat_s
    # Poisson arrivals at half the saturated rate (the stream's seeded draws at rate 1, rescaled).
    # The saturated run keeps every request queued, so its set-ups and solves overlap more than
    # spread arrivals allow: at 70% of that rate the open-loop run fell behind its arrivals (36.6
    # requests/s served of 37.6 offered) and its latency tail measured the growing queue.
    rate = OPEN_LOOP_LOAD * sat_rate
    unit_arrivals = np.array([q.arrival for q in gen.serving_requests(nreq, SEED, lo=20, hi=160, rate=1.0)])
    open_s, open_res, open_stats = run(unit_arrivals / rate)
    open_s = max_over_ranks(open_s, world, dev)
    lat = np.array(gather_lists([float(r[4]) for r in open_res], world)) * 1e3
    moved = float(sum(gather_lists([float(sat_stats["solve_bytes"])], world)))
    ok = all(r[0] == 0 and r[3] <= RTOL for r in sat_res + open_res) and all(s == 0 for s in serial_status.values())
    ok = all(gather_lists([ok], world))
    failed = [{"index": q.index, "kind": q.kind, "side": q.side, "status": [r[0], o[0], serial_status.get(q.index)],
               "iters": r[2], "relres": r[3], "error": r[6] or o[6]}
              for q, r, o in zip(reqs, sat_res, open_res)
              if r[0] != 0 or o[0] != 0 or serial_status.get(q.index, 0) != 0 or r[3] > RTOL][:10]
    failed = gather_lists(failed, world)[:10]
    same = all(gather_lists([all(np.array_equal(a[1], b[1]) for a, b in zip(sat_res, open_res))], world))
    return {"workload": f"{nreq} requests, sides log-uniform [20,160], 70% SPD (CG) / 30% convdiff (BiCGStab), "
                        "20% reuse of an earlier matrix, rtol 1e-8, FP64, host vectors",
            "requests": nreq, "ranks": world, "rows_total": int(rows), "slots": slots, "all_converged": ok,
            "failed": failed,
            "same_result_saturated_and_open_loop": same,
            "value": sat_rate, "unit": "requests/s (setup + solve)", "saturated_s": sat_s,
            "serial_plain_s": serial_s, "serial_plain_rate": nreq / serial_s, "speedup_vs_serial": serial_s / sat_s,
            "serial_note": (f"plain API (amg_setup + amg_solve_host, a hierarchy kept until its key's last sampled "
                            f"request) on every {stride}-th request ({len(sample)} of {len(reqs)} per rank), "
                            "time scaled to the whole stream") if stride > 1 else
                           "plain API on every request (amg_setup + amg_solve_host)",
            "solve_hbm_gbs": moved / sat_s / 1e9,
            "solve_frac_of_peak": moved / sat_s / 1e9 / peaks()[0],
            "bytes_note": "algorithmic bytes of the served solves (amg_server_solve_bytes: each solve's bytes per "
                          "Krylov iteration x its iterations) / the saturated wall time, set-ups included in the time",
            "open_loop_load": OPEN_LOOP_LOAD, "open_loop_rate": rate, "open_loop_s": open_s,
            "open_loop_served_rate": nreq / open_s,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "peak_charged_bytes": int(max_over_ranks(sat_stats["peak_bytes"], world, dev)),
            "evictions": int(sum(gather_lists([int(sat_stats["evictions"])], world))),
            "matrix_generation_s": max_over_ranks(gen_s, world, dev)}


# ---------------------------------------------------------------------- main
def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    import paper_1811_05704_gb300 as amg
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    A = gen.poisson3d(SIDE)
    f, _ = gen.rhs_from_solution(A, SEED)
    t0 = time.perf_counter()
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
    setup_s = time.perf_counter() - t0
    info = S.info()
    info["nnz_m"] = [amg.amg_fused_restriction_nnz(S.handle, l) for l in range(info["levels"])]
    coarse_n = info["rows"][-1]
    ft = torch.from_numpy(f).to(dev)
    x = torch.zeros(A.n, dtype=torch.float64, device=dev)

    for _ in range(args.warmup):
        x.zero_()
        S.solve(ft, x, RTOL, MAXITER)
    torch.cuda.synchronize()

    # ---- timed region: K solves, device events on the launching stream
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches = 0
    iters = []
    ev[0].record(stream)
    for k in range(args.steps):
        x.zero_()
        st, it, rr = S.solve(ft, x, RTOL, MAXITER)
        ev[k + 1].record(stream)
        launches += amg.amg_last_launch_count(S.handle)
        iters.append(it)
        assert st == 0 and rr <= RTOL, (st, rr)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_s = ev[0].elapsed_time(ev[-1]) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
        dist.barrier()
    value = world * args.steps / total_s
    solve_s = statistics.median(step_ms) / 1e3
    b_iter = bytes_per_iteration(info, coarse_n)
    assert abs(b_iter - amg.amg_hierarchy_bytes(S.handle)) <= 1e-9 * b_iter, "byte models disagree"
    solve_gbs = b_iter * iters[0] / solve_s / 1e9

    # ---- end to end through the host-buffer entry point (pinned host memory)
    # one zeroed pinned x0 buffer per step, prepared before the timed loop, so
    # that the loop holds only the call (copies in, solve, copy out)
    fh = torch.from_numpy(f).pin_memory()
    fnp = fh.numpy()
    e2e_steps = max(3, args.steps // 2)
    xhs = [torch.zeros(A.n, dtype=torch.float64).pin_memory() for _ in range(e2e_steps + 1)]
    amg.amg_solve_host(S.handle, fnp, xhs[-1].numpy(), RTOL, MAXITER)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        amg.amg_solve_host(S.handle, fnp, xhs[k].numpy(), RTOL, MAXITER)
    e2e_s = time.perf_counter() - t0
    del xhs
    e2e = {"value": world * e2e_steps / e2e_s if world == 1 else None, "unit": "solves/s",
           "h2d_bytes_per_step": 2 * 8 * A.n, "d2h_bytes_per_step": 8 * A.n,
           "note": "amg_solve_host: f and x0 copied in from pinned host memory, x copied out, inside "
                   "the timed loop (wall clock); each step's x0 is a zeroed pinned buffer prepared "
                   "before the loop"}
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e["value"] = world * e2e_steps / float(t.item())

    # ---- per-kernel attribution: the same solve with an event pair around
    # every launch on the handle's stream
    x.zero_()
    pst, pit, prr, ms, ln = amg.amg_solve_profile(S.handle, ft, x, RTOL, MAXITER)
    kb = kernel_bytes(info)
    dom = max(kb, key=lambda k: ms[k])
    avg_ms = ms[dom] / max(1, ln[dom])
    peak, peak_kind = peaks()
    achieved = kb[dom] / (avg_ms / 1e3) / 1e9
    kf = kernel_flops(info)
    fp64_gflops = kf[dom] / (avg_ms / 1e3) / 1e9
    traffic = committed_traffic(dom)
    per_kernel = {k: {"launches": ln[k], "ms": round(ms[k], 4),
                      "gbs": (round(kb[k] * ln[k] / (ms[k] / 1e3) / 1e9, 1) if k in kb and ms[k] > 0 else None),
                      "fp64_gflops": (round(kf[k] * ln[k] / (ms[k] / 1e3) / 1e9, 1)
                                      if k in kf and ms[k] > 0 else None)}
                  for k in ms}

    # ---- mixed precision form (float32 V-cycle under FP64 CG), same workload
    mixed = None
    if not args.no_mixed:
        x64 = x.clone()  # the FP64 solution of the timed region
        mixed = {}
        for name, prec, desc in (("fp32", amg.AMG_PRECISION_FP32, "fp32 V-cycle, fp64 CG"),
                                 ("bf16", amg.AMG_PRECISION_BF16,
                                  "fp32 V-cycle with bf16-stored matrix values, fp64 CG")):
            S32 = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=prec)
            for _ in range(2):
                x.zero_()
                S32.solve(ft, x, RTOL, MAXITER)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(3, args.steps // 2)
            e0.record(stream)
            for _ in range(reps):
                x.zero_()
                st32, it32, rr32 = S32.solve(ft, x, RTOL, MAXITER)
            e1.record(stream)
            torch.cuda.synchronize()
            t32 = e0.elapsed_time(e1) / 1e3 / reps
            err = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
            # per-kernel event times of an instrumented solve of this form
            x.zero_()
            _, _, _, pms, pln = amg.amg_solve_profile(S32.handle, ft, x, RTOL, MAXITER)
            kbm = kernel_bytes_mixed(info, 4 if name == "fp32" else 2)
            mk = {k: {"launches": pln[k], "ms": round(pms[k], 4),
                      "gbs": (round(kbm[k] * pln[k] / (pms[k] / 1e3) / 1e9, 1) if k in kbm and pms[k] > 0 else None)}
                  for k in pms}
            mdom = max(kbm, key=lambda k: pms[k])
            mavg = pms[mdom] / max(1, pln[mdom])
            mach = kbm[mdom] / (mavg / 1e3) / 1e9
            mixed[name] = {"value": 1.0 / t32, "unit": "solves/s", "solve_s": t32, "iterations": it32,
                           "relres": rr32, "status": st32, "precision": desc, "rel_diff_vs_fp64_x": err,
                           "speedup_vs_fp64": solve_s / t32, "kernels": mk,
                           "roofline": {"bound": "hbm", "kernel": mdom, "achieved": mach, "peak": peak,
                                        "unit": "GB/s", "frac": mach / peak,
                                        "algorithmic_bytes_per_launch": kbm[mdom], "avg_launch_ms": mavg}}
            S32.close()

    varcoef = None
    if not args.no_varcoef:
        varcoef = bench_varcoef(amg, torch, dev, stream, args, rank, world)

    batched = None
    if not args.no_batch:
        batched = bench_batched(amg, torch, dev, stream, args, rank, world)

    serving = None
    if not args.no_serve:
        serving = bench_serving(amg, args, rank, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator; the paper's 150^3 Poisson size, RHS A u*)",
        "config": {"workload": WORKLOAD, "precision": "fp64", "levels": info["levels"],
                   "rows": info["rows"], "nnz": info["nnz"],
                   "l2": "no flush: inputs larger than L2 (finest A alone 282 MB > 129 MB)",
                   "parallelism": f"replicas x{world}"},
        "solve_s": solve_s, "iterations": iters[0], "setup_s": setup_s,
        "hbm_gbs": solve_gbs,
        "bytes_per_iteration": b_iter,
        "gpu_launches": launches,
        "e2e": e2e,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "traffic": traffic, "algorithmic_bytes_per_launch": kb[dom],
                     "avg_launch_ms": avg_ms, "timing": "CUDA events around every launch of an "
                     "instrumented solve on the same stream, run right after the timed region",
                     "fp64_alu": {"achieved": fp64_gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                                  "frac": fp64_gflops / FP64_PEAK_GFLOPS, "flops_per_launch": kf[dom],
                                  "peak_kind": "nominal (GB300 FP64 1.25 TFLOP/s: 2 FMA/clk/SM at 2.07 GHz)"}},
        "solve_frac_of_peak": solve_gbs / peak,
        "solve_frac_of_nominal": solve_gbs / NOMINAL_HBM_GBS,
        "kernels": per_kernel,
        "mixed": mixed,
        "varcoef200": varcoef,
        "batched": batched,
        "serving": serving,
        "clocks": clock_info,
        "cpu_baseline": cpu,
    }
    S.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

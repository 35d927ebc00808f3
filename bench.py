"""Benchmark: CP-ALS-QR sweeps per second on one GB300 (per rank; replicas for N > 1).

Workload (the configuration the headline metric is quoted on): a 3-way
400 x 400 x 400 FP64 tensor (512 MB, larger than the 129 MB L2), planted rank 10,
factor columns with pairwise congruence 0.99, weights logspace 1..1e-4, 0.1%
Gaussian noise, rank-10 CP-ALS-QR with the QR solve.  One "step" is one full
sweep over the three modes: KRP of the R-factors and its QR, the Multi-TTM,
W = Y_(n) Q0, the R0 substitution, normalisation, the factor QR, and the
efficient fit.  The timed steps run through cpals_iterate (one CUDA graph per
sweep) with X resident in HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1, run under torch.distributed.run.  Every rank runs its own
independent replica (different seed), and value = the sum of sweeps/s.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CP-ALS-QR iters/s"
UNIT = "iters/s"
def workload_name(size, rank, solve="qr"):
    mb = 8 * size ** 3 / 1e6
    return (f"3-way {size}x{size}x{size} FP64 ({mb:.0f} MB), rank {rank}, planted factors with column congruence "
            f"0.99, weights logspace 1..1e-4, 0.1% Gaussian noise; CP-ALS-QR sweeps ({solve.upper()} solve)")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP64_FLOP_PER_CLK_PER_SM = 4       # 2 DFMA/clk/SM on this part (measured: 1.195 TFLOP/s at ~1.95 GHz)
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=400)
    ap.add_argument("--rank", type=int, default=10)
    ap.add_argument("--solve", choices=["qr", "svd", "normal"], default="qr")
    ap.add_argument("--no-variants", action="store_true", help="skip the SVD/NORMAL/FP32 side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the 120^4 rank-20 FP64/FP32/3xBF16/3xTF32 record of the default run")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--workload", choices=["c2", "c3", "c5a", "c5b", "c4", "sine", "collinear", "paper41"],
                    default="c2",
                    help="c2: the headline 400^3 rank-10 FP64 workload; c3: 4-way 120^4 rank 20, c5a: 3-way "
                         "1000^3 rank 64 (SVD solve) and c5b: 5-way 40^5 rank 8, each comparing FP64, FP32, 3xBF16 "
                         "and 3xTF32 passes over X; c4: 512 independent small problems, batched; sine: sine-of-sums "
                         "tensors in Kruskal form (Sec. 4.3); collinear: the Sec. 4.2 collinearity x noise grid; "
                         "paper41: the Sec. 4.1 cubical tensors (700^3, 300^4, 75^5) over a rank sweep with the "
                         "per-sweep time of the four solves and the component breakdown of Table its_parts")
    ap.add_argument("--trials", type=int, default=10, help="collinear: random starts per grid cell")
    ap.add_argument("--recovery-seeds", type=int, default=5,
                    help="c3: planted problems (seeds) on which every precision runs to convergence and is scored "
                         "against the planted factors (factor-match score, Sec. 4.2); 0 skips")
    ap.add_argument("--precisions", default="f64,f32,bf16x3,tf32x3",
                    help="c3/c5a/c5b: comma-separated precisions to run")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="c3/c5a/c5b: throughput only (no Multi-TTM error, one-sweep factors or fit to convergence)")
    ap.add_argument("--fit-sweeps", type=int, default=300,
                    help="at most this many sweeps (stop at |fit change| < 1e-10) for the equal-fit comparison")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling (every 200 ms) during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)    # sampler up before the timed region starts
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxes.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
                "samples": len(sms)}


def kernel_source(name, path=os.path.join(ROOT, "paper_2112_10855_gb300", "csrc", "ttm.cu")):
    """Source text of one __global__ kernel (its template line through the
    closing brace), used to tell whether recorded counters still apply."""
    with open(path) as f:
        lines = f.read().split("\n")
    for i, ln in enumerate(lines):
        if "__global__" in ln and (name + "(") in ln:
            start = i - 1 if i > 0 and lines[i - 1].startswith("template") else i
            for j in range(i, len(lines)):
                if lines[j] == "}":
                    return "\n".join(lines[start:j + 1])
    return ""


def recorded_traffic(profile="ttm_rows_f64_400cubed_r10.md"):
    """DRAM traffic per launch of the dominant kernel from the committed ncu
    summary, or None if the kernel source changed since it was captured."""
    import hashlib
    import re
    try:
        with open(os.path.join(ROOT, "profiles", profile)) as f:
            text = f.read()
        want = re.search(r"sha256\[:16\] = ([0-9a-f]+)", text).group(1)
        have = hashlib.sha256(kernel_source("ttm_rows_kernel").encode()).hexdigest()[:16]
        if want != have:
            return None
        return int(re.search(r"traffic_bytes_per_launch: (\d+)", text).group(1))
    except Exception:
        return None


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


def workload(size, rank, seed):
    from paper_2112_10855_gb300 import inputs
    return inputs.workload_c2(seed=seed, init_seed=10855 + seed - 2112, size=size, rank=rank)


def cpu_oracle_rate(p, solve=0, target_s=12.0, max_sweeps=20):
    """The oracle as it stands (1 host thread): full sweeps, timed together,
    as many as fill about target_s (at least 2, at most max_sweeps; the first
    sweep's time sets the count).  Returns (sweeps/s, seconds, sweeps)."""
    import oracle
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    t0 = time.perf_counter()
    k1, _ = o.iterate(1, solve=solve)
    first = time.perf_counter() - t0
    more = max(1, min(max_sweeps - 1, int(target_s / max(first, 1e-9)) - 1))
    k2, _ = o.iterate(more, solve=solve)
    dt = time.perf_counter() - t0
    n = abs(k1) + abs(k2)
    return n / dt, dt, n


def _oracle_replica(task):
    """One single-threaded oracle replica (a spawned process): the workload,
    then `sweeps` timed sweeps; returns sweeps per second."""
    size, rank_, sweeps, solve = task
    import oracle
    from paper_2112_10855_gb300 import inputs
    p = inputs.workload_c2(size=size, rank=rank_)
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    t0 = time.perf_counter()
    o.iterate(sweeps, solve=solve)
    return sweeps / (time.perf_counter() - t0)


_ONE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _replica_map(fn, tasks):
    """fn over tasks, one spawned process each (spawned, not forked: the
    parent holds a CUDA context).  The replicas' numpy runs on one thread
    each, so that one replica's set-up does not crowd another's timed oracle
    work."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in _ONE_THREAD_ENV}
    os.environ.update({k: "1" for k in _ONE_THREAD_ENV})
    try:
        with mp.get_context("spawn").Pool(len(tasks)) as pool:
            return pool.map(fn, tasks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_oracle_all_cores(size, rank_, sweeps=1, solve=0):
    """The oracle as it stands (single-threaded plain C) on every host core
    at once: one independent replica per core in spawned processes (spawned,
    not forked, because the parent holds a CUDA context); the aggregate rate
    is the sum of the replicas' sweeps per second."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    rates = _replica_map(_oracle_replica, [(size, rank_, sweeps, solve)] * cores)
    return float(sum(rates)), cores, time.perf_counter() - t0


def _sample_problem(kind, size):
    """The host copy of workload `kind` (seeded generators) for an oracle
    sample; `size` shrinks the cube of the 3-way rank-64 workload."""
    from paper_2112_10855_gb300 import inputs
    if kind == "c3":
        return inputs.workload_c3(seed=2112)
    if kind == "c5a":
        return inputs.workload_c5a(seed=2112, size=size)
    return inputs.planted((40,) * 5, 8, seed=2112, noise=0.01)


def _oracle_sample(task):
    """One single-threaded oracle replica timing a bounded sample of a
    workload.  kind "batch": one sweep of each of the first problems of the
    512-problem batch until `budget` seconds are spent; otherwise `modes` mode
    updates of the (possibly shrunk) workload.  Returns (seconds, sweeps of
    the sample done, elements of the sample)."""
    kind, size, modes, solve, rtol, budget = task
    import oracle
    from paper_2112_10855_gb300 import inputs
    if kind == "batch":
        dims, ranks = inputs.batch_shapes(512, seed=2112)
        probs = [inputs.planted(tuple(int(x) for x in dims[q]), int(ranks[q]), seed=2112 + q,
                                init_seed=10855 + q, noise=0.01) for q in range(len(dims))]
        t = 0.0
        elems = 0
        for pr in probs:
            o = oracle.OracleCPALS(pr.X, pr.dims, pr.rank)
            o.set_factors(pr.init_factors)
            t0 = time.perf_counter()
            o.iterate(1, solve=solve, rtol=rtol)
            t += time.perf_counter() - t0
            elems += pr.X.size
            if t > budget:
                break
        return t, 1.0, elems
    p = _sample_problem(kind, size)
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    t0 = time.perf_counter()
    for n in range(modes):
        o.update_mode(n, solve=solve, rtol=rtol)
    return time.perf_counter() - t0, modes / len(p.dims), p.X.size


def _host_mem_available():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def oracle_sample_baseline(kind, total_elems, sample, size=0, modes=1, solve=0, rtol=0.0, budget=20.0):
    """cpu_baseline of a non-default workload: the oracle as it stands on a
    bounded sample (`sample` says which), 1 host thread, then one replica per
    host core in spawned processes, as many as a quarter of the free host
    memory holds at four copies of the sample's tensor each.  Rates are
    sweeps of the whole workload per second: the sample's sweeps scaled by
    its share of the workload's elements (the sweep cost is led by passes over
    X, linear in the element count)."""
    import oracle
    oracle.build()
    task = (kind, size, modes, solve, rtol, budget)
    t, sweeps, elems = _oracle_sample(task)
    rate1 = sweeps / t * elems / total_elems
    cpu = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
           "sample_seconds": t, "sample_elements": int(elems), "workload_elements": int(total_elems)}
    cores = os.cpu_count() or 1
    per_replica = 4 * 8 * elems
    replicas = min(cores, int(0.25 * _host_mem_available() // max(per_replica, 1)))
    if replicas >= 2:
        t0 = time.perf_counter()
        res = _replica_map(_oracle_sample, [task] * replicas)
        agg = sum(sw / tt * el / total_elems for tt, sw, el in res)
        cpu["all_cores"] = {"value": agg, "unit": UNIT, "cores": replicas, "kind": "oracle",
                            "sample": f"one replica of the same sample per core ({replicas} of {cores} cores, "
                                      f"bounded by host memory); sum of the replicas' rates "
                                      f"({time.perf_counter() - t0:.1f} s wall)"}
    return cpu


def run_reference(args, world, rank):
    """--impl reference: the FP64 CPU oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = workload(args.size, args.rank, 2112)
    solve = {"qr": 0, "svd": 1, "normal": 2}[args.solve]
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    # warm-up and timed steps, each one full oracle sweep; the run is bounded to
    # about three minutes of host time (fewer steps are timed if needed)
    budget_s = 180.0
    t_start = time.perf_counter()
    for _ in range(args.warmup):
        o.iterate(1, solve=solve, rtol=1e-10)
        if time.perf_counter() - t_start > budget_s / 4:
            break
    per = (time.perf_counter() - t_start) / max(args.warmup, 1)
    steps = max(1, min(args.steps, int(budget_s / max(per, 1e-9))))
    t0 = time.perf_counter()
    for _ in range(steps):
        o.iterate(1, solve=solve, rtol=1e-10)
    dt = time.perf_counter() - t0
    v = steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.size, args.rank, args.solve), "dims": [args.size] * 3,
                   "rank": args.rank, "solve": args.solve, "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{steps} full sweeps of the same workload (of {args.steps} asked; bounded to "
                                   f"~{budget_s:.0f} s), single-threaded plain C FP64"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def mixed_workload(name, seed=2112):
    from paper_2112_10855_gb300 import inputs
    if name == "c3":
        p = inputs.workload_c3(seed=seed)
        desc = ("4-way 120x120x120x120 (FP64 master 1.66 GB + FP32 copy 0.83 GB), rank 20, factor columns with "
                "congruence 0.9, 1% noise; CP-ALS-QR (QR solve)")
        return p, desc, "qr", 0.0
    if name == "c5a":
        p = inputs.workload_c5a(seed=seed)
        desc = ("3-way 1000x1000x1000 (FP64 master 8 GB + FP32 copy 4 GB), rank 64, factor columns with "
                "congruence 0.999, weights logspace 1..1e-6, 0.1% noise; CP-ALS-QR with the SVD solve (rtol 1e-8)")
        return p, desc, "svd", 1e-8
    p = inputs.planted((40,) * 5, 8, seed=seed, noise=0.01)
    desc = "5-way 40^5 (FP64 master 819 MB + FP32 copy 410 MB), rank 8, N(0,1) factors, 1% noise; CP-ALS-QR"
    return p, desc, "qr", 0.0


def e2e_double_buffered(cpals, dims, R, Xh, Ah, solve, steps):
    """Wall time of `steps` end-to-end steps (pinned-host X and factors in, one
    sweep, factors, lambda and fit out) on two handles in two host threads.
    A copy token alternates between the threads: a thread copies its inputs
    while it holds the token, then hands it over and runs its sweep, so the
    copy of one step overlaps the sweep of the other."""
    import threading
    import torch
    hs = []
    for _ in range(2):
        st = torch.cuda.Stream()
        h = cpals.CPALS(dims, R, "f64")
        h.set_stream(st)
        h.set_tensor(Xh)
        h.set_factors(Ah)
        h.iterate(1, solve=solve, svd_rtol=1e-10, want_fits=False)    # captures the sweep graph
        h.get_factors()
        h.fit()
        hs.append(h)
    torch.cuda.synchronize()
    turn = [threading.Semaphore(1), threading.Semaphore(0)]
    errors = []
    device = torch.cuda.current_device()   # a new host thread starts on device 0

    def worker(i):
        try:
            torch.cuda.set_device(device)
            for _ in range(i, steps, 2):
                turn[i].acquire()
                if errors:               # the other thread failed: stop
                    return
                hs[i].set_tensor(Xh)
                hs[i].set_factors(Ah)
                turn[1 - i].release()
                hs[i].iterate(1, solve=solve, svd_rtol=1e-10, want_fits=False)
                hs[i].get_factors()
                hs[i].fit()
        except Exception as e:   # surfaced after the join
            errors.append(e)
            for _ in range(steps):
                turn[1 - i].release()

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return wall


def run_mixed(args, world, rank):
    """FP64 vs FP32 vs 3xBF16 (tensor cores) passes over X on one workload:
    sweeps/s, first-TTM GB/s against HBM, Multi-TTM error against FP64 with
    the same Q_m, factor error after one sweep, and the fit after
    --fit-sweeps sweeps from the same start."""
    import torch
    from paper_2112_10855_gb300 import _build, cpals
    torch.cuda.set_device(0)
    _build.build()
    cpals.load()
    p, desc, solve, rtol = mixed_workload(args.workload, 2112 + rank)
    fit_sweeps = min(args.fit_sweeps, 30) if args.workload == "c5a" else args.fit_sweeps
    P = int(np.prod(p.dims))
    R = p.rank
    stream = torch.cuda.Stream()
    Xd = torch.from_numpy(p.X).cuda()
    init = [np.asfortranarray(a) for a in p.init_factors]
    hbm = measured_peaks().get("hbm_gbs")
    out = {}
    ref = {}
    precisions = [x for x in args.precisions.split(",") if x]
    for prec in precisions:
        # throughput
        h = cpals.CPALS(p.dims, R, prec)
        h.set_stream(stream)
        h.set_tensor(Xd)
        h.set_factors(init)
        h.iterate(args.warmup, solve=solve, svd_rtol=rtol, want_fits=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = h.launch_count()
        e0.record(stream)
        h.iterate(args.steps, solve=solve, svd_rtol=rtol, want_fits=False)
        e1.record(stream)
        torch.cuda.synchronize()
        its = args.steps / (e0.elapsed_time(e1) * 1e-3)
        launches = h.launch_count() - l0
        ttm_ms = []
        for n in range(len(p.dims)):
            h.ttm_first(n)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(5):
                h.ttm_first(n)
            e1.record(stream)
            torch.cuda.synchronize()
            ttm_ms.append(e0.elapsed_time(e1) / 5)
        ms = sum(ttm_ms) / len(ttm_ms)
        xbytes = (8 if prec == "f64" else 4) * P
        del h
        entry = {"iters_per_s": its, "gpu_launches_per_sweep": launches / args.steps,
                 "first_ttm_ms": ms, "first_ttm_gbs": xbytes / (ms * 1e-3) / 1e9,
                 "first_ttm_frac_hbm": (xbytes / (ms * 1e-3) / 1e9 / hbm) if hbm else None,
                 "first_ttm_tflops": 2.0 * P * R / (ms * 1e-3) / 1e12}
        if args.no_accuracy:
            out[prec] = entry
            continue
        # accuracy: Multi-TTM with identical Q_m, one sweep, and the fit after S sweeps
        ha = cpals.CPALS(p.dims, R, prec)
        ha.set_stream(stream)
        ha.set_tensor(Xd)
        ha.set_factors(init)
        Ys = [ha.multi_ttm(n)[0] for n in range(len(p.dims))]
        fits1 = ha.iterate(1, solve=solve, svd_rtol=rtol)
        A1, l1 = ha.get_factors()
        # run to convergence (|fit change| < 1e-10, at most --fit-sweeps), then
        # the direct fit: FP64 residual against the FP64 tensor
        fitsS = ha.iterate(max(fit_sweeps - 1, 1), tol=1e-10, solve=solve, svd_rtol=rtol)
        sweeps_run = 1 + len(fitsS)
        fit_final = ha.fit(direct=True)
        traj = np.concatenate([fits1, fitsS])
        del ha
        entry.update({"fit_direct_converged": fit_final, "sweeps_to_converge": sweeps_run})
        if prec == "f64":
            ref = {"Y": Ys, "A": A1, "fit": fit_final, "traj": traj}
        elif ref:
            m5 = min(5, len(traj), len(ref["traj"]))
            entry["fit_traj_max_diff_first5"] = float(np.abs(traj[:m5] - ref["traj"][:m5]).max())
            entry["multi_ttm_rel_err_vs_f64"] = max(
                float(np.linalg.norm(Ys[n] - ref["Y"][n]) / np.linalg.norm(ref["Y"][n])) for n in range(len(Ys)))
            entry["factor_rel_err_vs_f64_after_1_sweep"] = max(
                float(np.linalg.norm(A1[m] - ref["A"][m]) / np.linalg.norm(ref["A"][m])) for m in range(len(A1)))
            entry["fit_rel_diff_vs_f64"] = abs(fit_final - ref["fit"]) / abs(ref["fit"])
        out[prec] = entry
    recovery = None
    if args.workload == "c3" and args.recovery_seeds > 0 and not args.no_accuracy:
        recovery = recovery_rates(args, p.dims, R, fit_sweeps, solve, rtol, stream)
    if rank == 0:
        head = "bf16x3" if "bf16x3" in out else precisions[0]
        line = {
            "metric": METRIC, "value": out[head]["iters_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"{head} (value); the others beside it (tensor cores when R >= 16)",
            "data": "synthetic",
            "config": {"workload": desc, "dims": list(p.dims), "rank": R, "fit_sweeps": fit_sweeps,
                       "solve": solve, "svd_rtol": rtol},
            "precisions": out,
            "speedup_vs_f64": ({k: out[k]["iters_per_s"] / out["f64"]["iters_per_s"] for k in out}
                               if "f64" in out else None),
        }
        if recovery is not None:
            line["planted_recovery"] = recovery
        if world == 1 and not args.no_cpu_baseline:
            sid = {"qr": 0, "svd": 1}[solve]
            if args.workload == "c5a":
                line["cpu_baseline"] = oracle_sample_baseline(
                    "c5a", P, "one mode update (of three) of the same recipe on a 464^3 cube at rank 64, SVD "
                    "solve, scaled by the element share (1.0e8 of 1e9) to sweeps of the 1000^3 workload",
                    size=464, modes=1, solve=sid, rtol=rtol)
            elif args.workload == "c3":
                line["cpu_baseline"] = oracle_sample_baseline(
                    "c3", P, "one mode update (of four, all of equal cost on the 120^4 cube) of the same "
                    "workload", modes=1, solve=sid, rtol=rtol)
            else:
                line["cpu_baseline"] = oracle_sample_baseline(
                    "c5b", P, "one full sweep (five mode updates) of the same workload", modes=5, solve=sid,
                    rtol=rtol)
        print(json.dumps(line), flush=True)


def recovery_rates(args, dims, R, fit_sweeps, solve, rtol, stream):
    """Every precision from the same start on --recovery-seeds planted 120^4
    problems, run to convergence (|fit change| < 1e-10, at most fit_sweeps),
    then scored against the planted factors and weights (factor-match score,
    Sec. 4.2).  "Recovered" = score >= 0.99."""
    import torch
    from paper_2112_10855_gb300 import cpals, inputs
    from paper_2112_10855_gb300.score import factor_match_score
    scores = {k: [] for k in ["f64", "f32", "bf16x3", "tf32x3"]}
    for s in range(args.recovery_seeds):
        p = inputs.workload_c3(seed=3000 + s, init_seed=4000 + s)
        Xd = torch.from_numpy(p.X).cuda()
        for prec in scores:
            h = cpals.CPALS(p.dims, R, prec)
            h.set_stream(stream)
            h.set_tensor(Xd)
            h.set_factors([np.asfortranarray(a) for a in p.init_factors])
            h.iterate(fit_sweeps, tol=1e-10, solve=solve, svd_rtol=rtol, want_fits=False)
            A, lam = h.get_factors()
            scores[prec].append(factor_match_score(lam, A, p.true_weights, p.true_factors))
            del h
        del Xd
    f64 = np.asarray(scores["f64"])
    return {"seeds": args.recovery_seeds,
            "recovered_fraction_at_0.99": {k: float(np.mean(np.asarray(v) >= 0.99)) for k, v in scores.items()},
            "recovered_fraction_at_0.95": {k: float(np.mean(np.asarray(v) >= 0.95)) for k, v in scores.items()},
            "max_abs_score_diff_vs_f64": {k: float(np.abs(np.asarray(v) - f64).max()) for k, v in scores.items()},
            "scores": {k: [round(x, 6) for x in v] for k, v in scores.items()}}


def mixed_c3_record(args, stream):
    """The 4-way 120^4 rank-20 workload (congruence 0.9, 1% noise) with FP64,
    FP32, 3xBF16 and 3xTF32 passes over X: sweeps/s (CUDA events on the
    handle's stream, after warm-up), the first TTM of each mode's Multi-TTM
    (the pass that streams X) timed alone with its GB/s against the measured
    HBM copy bandwidth, the speed-up over FP64, and the direct fit after the
    FP64 run's sweeps to convergence (|fit change| < 1e-10, at most
    --fit-sweeps) from the same start, as a relative gap to FP64's."""
    import torch
    from paper_2112_10855_gb300 import cpals, inputs
    t_gen = time.perf_counter()
    p = inputs.workload_c3()
    t_gen = time.perf_counter() - t_gen
    P, R = int(np.prod(p.dims)), p.rank
    Xd = torch.from_numpy(p.X).to(torch.cuda.current_device())
    init = [np.asfortranarray(a) for a in p.init_factors]
    hbm = measured_peaks().get("hbm_gbs")
    steps = 20
    out, sweeps_conv = {}, None
    for prec in ["f64", "f32", "bf16x3", "tf32x3"]:
        h = cpals.CPALS(p.dims, R, prec)
        h.set_stream(stream)
        h.set_tensor(Xd)
        h.set_factors(init)
        h.iterate(max(args.warmup, 3), solve="qr", want_fits=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = h.launch_count()
        e0.record(stream)
        h.iterate(steps, solve="qr", want_fits=False)
        e1.record(stream)
        torch.cuda.synchronize()
        its = steps / (e0.elapsed_time(e1) * 1e-3)
        launches = (h.launch_count() - l0) / steps
        ttm_ms = []
        for n in range(len(p.dims)):
            h.ttm_first(n)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(5):
                h.ttm_first(n)
            e1.record(stream)
            torch.cuda.synchronize()
            ttm_ms.append(e0.elapsed_time(e1) / 5)
        ms = sum(ttm_ms) / len(ttm_ms)
        xbytes = (8 if prec == "f64" else 4) * P
        gbs = xbytes / (ms * 1e-3) / 1e9
        # the same start, run to FP64's convergence count, then the direct fit
        h.set_factors(init)
        if prec == "f64":
            fits = h.iterate(args.fit_sweeps, tol=1e-10, solve="qr")
            sweeps_conv = len(fits)
        else:
            h.iterate(sweeps_conv, solve="qr", want_fits=False)
        fit = h.fit(direct=True)
        del h
        out[prec] = {"iters_per_s": its, "gpu_launches_per_sweep": launches, "first_ttm_ms": ms,
                     "first_ttm_gbs": gbs, "first_ttm_frac_hbm": (gbs / hbm) if hbm else None,
                     "fit_direct": fit}
    for prec in out:
        out[prec]["speedup_vs_f64"] = out[prec]["iters_per_s"] / out["f64"]["iters_per_s"]
        out[prec]["fit_rel_gap_vs_f64"] = abs(out[prec]["fit_direct"] - out["f64"]["fit_direct"]) / \
            out["f64"]["fit_direct"]
    del Xd
    torch.cuda.empty_cache()
    return {"workload": "4-way 120x120x120x120 (FP64 1.66 GB; FP32 copy 0.83 GB), rank 20, factor columns with "
                        "congruence 0.9, 1% noise; CP-ALS-QR (QR solve), dimension-tree sweeps",
            "dims": list(p.dims), "rank": R, "timed_sweeps": steps, "sweeps_to_converge_f64": sweeps_conv,
            "hbm_peak_gbs": hbm, "hbm_peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
            "first_ttm": "the pass over X of each mode's Multi-TTM, timed alone (events, 5 launches per mode); "
                         "GB/s = bytes of X read (8P FP64, 4P otherwise) / time",
            "input_generation_s": t_gen, "precisions": out}


def run_batch(args, world, rank):
    """512 independent 3-way problems (dims ~ U{16..128}, ranks ~ U{2..16}, planted
    rank plus 1% noise): the batched path (two passes over all tensors and three
    mode-update kernels per sweep, one graph per sweep) against one handle per
    problem (one graph launch per problem per sweep), both FP32 passes over X
    and FP64 factorisations."""
    import torch
    from paper_2112_10855_gb300 import _build, cpals, inputs
    torch.cuda.set_device(0)
    _build.build()
    cpals.load()
    count = 512
    dims, ranks = inputs.batch_shapes(count, seed=2112 + rank)
    probs = [inputs.planted(tuple(int(x) for x in dims[p]), int(ranks[p]), seed=2112 + 7919 * rank + p,
                            init_seed=10855 + 7919 * rank + p, noise=0.01) for p in range(count)]
    X32 = [pr.X.astype(np.float32) for pr in probs]
    total_elems = int(sum(x.size for x in X32))
    stream = torch.cuda.Stream()
    b = cpals.CPALSBatch([pr.dims for pr in probs], [pr.rank for pr in probs])
    b.set_stream(stream)
    b.set_tensors(X32)
    b.set_factors([pr.init_factors for pr in probs])
    b.iterate(args.warmup)                      # includes the launch-shape tuning and the graph capture
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count()
    e0.record(stream)
    fits_b, st_b = b.iterate(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    launches_b = b.launch_count() - l0
    grid, threads = b.launch_shape()
    del b
    # one problem per launch: a single-problem handle each, one graph launch per sweep
    Xd = [torch.from_numpy(x).to("cuda") for x in X32]
    hs = []
    for p, pr in enumerate(probs):
        h = cpals.CPALS(pr.dims, pr.rank, "f32")
        h.set_stream(stream)
        h.set_tensor(Xd[p])
        h.set_factors([np.asfortranarray(a) for a in pr.init_factors])
        h.iterate(1, want_fits=False)
        hs.append(h)
    torch.cuda.synchronize()
    ksingle = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(ksingle):
        for h in hs:
            h.iterate(1, want_fits=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_1 = e0.elapsed_time(e1)
    wall_1 = time.perf_counter() - t0
    # agreement: the same sweeps from the same start on both paths (first 32 problems)
    sub = list(range(32))
    bb = cpals.CPALSBatch([probs[p].dims for p in sub], [probs[p].rank for p in sub])
    bb.set_tensors([X32[p] for p in sub])
    bb.set_factors([probs[p].init_factors for p in sub])
    fb, _ = bb.iterate(3)
    diffs = []
    for i, p in enumerate(sub):
        h = cpals.CPALS(probs[p].dims, probs[p].rank, "f32")
        h.set_tensor(Xd[p])
        h.set_factors([np.asfortranarray(a) for a in probs[p].init_factors])
        f = h.iterate(3)
        diffs.append(abs(float(f[-1]) - float(fb[i])))
    v_b = args.steps / (ms_b * 1e-3)
    v_1 = ksingle / (ms_1 * 1e-3)
    # X (FP32) is read twice per sweep (dimension tree); GB/s of those reads
    hbm = measured_peaks().get("hbm_gbs")
    x_gbs = 2 * 4 * total_elems / (ms_b / args.steps * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": v_b, "unit": UNIT + " (every problem of the batch advances one sweep)",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32 passes over X, fp64 factors",
            "data": "synthetic",
            "config": {"workload": f"{count} independent 3-way tensors, dims ~ U{{16..128}}, ranks ~ U{{2..16}}, "
                                   "planted rank + 1% noise; CP-ALS-QR (QR solve)",
                       "elements": total_elems, "x_bytes_fp32": 4 * total_elems},
            "batched": {"iters_per_s": v_b, "problem_sweeps_per_s": v_b * count, "ms_per_sweep": ms_b / args.steps,
                        "launches_per_sweep": launches_b / args.steps, "grid": grid, "threads": threads,
                        "x_passes_per_sweep": 2,
                        "x_stream_gbs": x_gbs, "x_stream_frac_hbm": (x_gbs / hbm) if hbm else None,
                        "hbm_peak_gbs": hbm,
                        "statuses_ok": int((st_b == 0).sum())},
            "one_problem_per_launch": {"iters_per_s": v_1, "ms_per_sweep": ms_1 / ksingle, "sweeps": ksingle,
                                       "host_wall_s": wall_1},
            "speedup_batched_vs_per_problem": v_b / v_1,
            "fit_agreement_max_abs_diff_3_sweeps": max(diffs),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample_baseline(
                "batch", total_elems, "one oracle sweep of each of the first problems of the same batch until "
                "about 20 s are spent, scaled by their share of the batch's elements", budget=20.0)
        print(json.dumps(line), flush=True)


def run_sine(args, world, rank):
    """Sec. 4.3 sine of sums, given in Kruskal form (Sec. 3.3.2): sweeps/s of
    the Kruskal-input path against the dense path on the same tensor where the
    dense tensor fits, the order-10 case that only the Kruskal path can hold,
    and the direct relative error after 40 sweeps of CP-ALS-QR, CP-ALS-QR-SVD,
    CP-ALS and CP-ALS-PINV from the same start (the comparison of Sec. 4.3)."""
    import torch
    from paper_2112_10855_gb300 import _build, cpals, inputs
    torch.cuda.set_device(0)
    _build.build()
    cpals.load()
    rng = np.random.default_rng(2112 + rank)

    def timed(h, solve, steps, warmup):
        h.iterate(warmup, solve=solve, svd_rtol=1e-12, want_fits=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        h.iterate(steps, solve=solve, svd_rtol=1e-12, want_fits=False)
        e1.record()
        torch.cuda.synchronize()
        return steps / (e0.elapsed_time(e1) * 1e-3)

    cases = []
    for N, n, rep, dense in [(4, 128, "expanded", True), (5, 64, "expanded", True), (10, 12, "rank_n", False)]:
        mu, V = (inputs.sine_of_sums_expanded(N, n) if rep == "expanded" else inputs.sine_of_sums_rank_n(N, n))
        dims, R = (n,) * N, N
        A = [np.asfortranarray(rng.standard_normal((n, R))) for _ in range(N)]
        hk = cpals.CPALS(dims, R, kruskal_rank=len(mu))
        hk.set_tensor_kruskal(mu, V)
        hk.set_factors(A)
        entry = {"N": N, "n": n, "input": f"{rep}, Kruskal rank {len(mu)}", "rank": R,
                 "kruskal_qr_iters_per_s": timed(hk, "qr", args.steps, args.warmup)}
        del hk
        if dense:
            X = torch.from_numpy(inputs.cp_full(dims, V, mu)).cuda()
            hd = cpals.CPALS(dims, R)
            hd.set_tensor(X)
            hd.set_factors(A)
            entry["dense_qr_iters_per_s"] = timed(hd, "qr", max(2, args.steps // 10), args.warmup)
            entry["kruskal_speedup_vs_dense"] = entry["kruskal_qr_iters_per_s"] / entry["dense_qr_iters_per_s"]
            del hd, X
        cases.append(entry)
    # accuracy after 40 sweeps, Sec. 4.3's 4-way case at n = 64
    N, n = 4, 64
    mu, V = inputs.sine_of_sums_expanded(N, n)
    dims = (n,) * N
    A = [np.asfortranarray(rng.standard_normal((n, N))) for _ in range(N)]
    errs = {}
    for solve in ["qr", "svd", "normal", "normal_pinv"]:
        h = cpals.CPALS(dims, N, kruskal_rank=len(mu))
        h.set_tensor_kruskal(mu, V)
        h.set_factors(A)
        h.iterate(40, solve=solve, svd_rtol=1e-12, want_fits=False)
        errs[solve] = 1.0 - h.fit(direct=True)
    if rank == 0:
        line = {
            "metric": METRIC, "value": cases[-1]["kruskal_qr_iters_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sine of sums sin(x_1 + ... + x_N) on the grid 2 pi k / n, given in Kruskal "
                                   "form; value: N = 10, n = 12, rank-10 input (Eq. sinsum_rkd), CP rank 10, "
                                   "CP-ALS-QR"},
            "cases": cases,
            "relative_error_after_40_sweeps_4way_n64": errs,
        }
        print(json.dumps(line), flush=True)


def run_collinear(args, world, rank):
    """Sec. 4.2: a 50^3 rank-5 tensor from factors with pairwise column
    congruence c (collinearity 1 - 1e-4, 1 - 1e-7, 1 - 1e-10) and Gaussian
    noise (1e-4, 1e-7, 1e-10 of ||X||); per cell, --trials random starts shared
    by CP-ALS, CP-ALS-PINV, CP-ALS-QR and CP-ALS-QR-SVD (FP64), 500 sweeps
    each.  Reported per algorithm: the median direct relative error
    ||X - Xhat|| / ||X||, the median factor-match score against the planted
    model, the median sweep at which the efficient fit stopped changing by
    more than 1e-15 (500 = never), and the number of runs a singular solve
    stopped."""
    import torch
    from paper_2112_10855_gb300 import _build, cpals, inputs
    from paper_2112_10855_gb300.score import factor_match_score
    torch.cuda.set_device(0)
    _build.build()
    cpals.load()
    dims, R, sweeps = (50, 50, 50), 5, 500
    solves = ["normal", "normal_pinv", "qr", "svd"]
    cells = []
    t0 = time.time()
    runs = 0
    for noise in (1e-4, 1e-7, 1e-10):
        for col in (1 - 1e-4, 1 - 1e-7, 1 - 1e-10):
            res = {k: {"relerr": [], "score": [], "iters": [], "failed": 0} for k in solves}
            for t in range(args.trials):
                p = inputs.planted(dims, R, seed=5000 + 97 * t, init_seed=6000 + t, congruence=col,
                                   unit_columns=True, noise=noise)
                Xd = torch.from_numpy(p.X).cuda()
                for solve in solves:
                    h = cpals.CPALS(dims, R)
                    h.set_tensor(Xd)
                    h.set_factors([np.asfortranarray(a) for a in p.init_factors])
                    runs += 1
                    try:
                        fits = h.iterate(sweeps, solve=solve)
                    except cpals.CPALSError:
                        res[solve]["failed"] += 1
                        continue
                    d = np.abs(np.diff(fits))
                    stop = np.nonzero(d < 1e-15)[0]
                    res[solve]["iters"].append(int(stop[0]) + 2 if len(stop) else sweeps)
                    res[solve]["relerr"].append(1.0 - h.fit(direct=True))
                    A, lam = h.get_factors()
                    res[solve]["score"].append(factor_match_score(lam, A, p.true_weights, p.true_factors))
                    del h
                del Xd
            cell = {"noise": noise, "collinearity": f"1 - {1 - col:.0e}"}
            for solve in solves:
                r = res[solve]
                med = lambda v: float(np.median(v)) if v else None
                cell[solve] = {"median_relerr": med(r["relerr"]), "median_score": med(r["score"]),
                               "median_iters": med(r["iters"]), "failed": r["failed"]}
            cells.append(cell)
    wall = time.time() - t0
    if rank == 0:
        line = {
            "metric": "CP-ALS runs/s (500 sweeps each, 50^3 rank 5)", "value": runs / wall, "unit": "runs/s",
            "n_gpus": world, "steps": runs, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Sec. 4.2 collinearity x noise grid: 50x50x50, rank 5, unit-norm planted factors "
                                   "with pairwise congruence c, Gaussian noise; random N(0,1) starts shared by "
                                   "the four solves; 500 sweeps", "trials_per_cell": args.trials},
            "cells": cells, "wall_s": wall,
        }
        print(json.dumps(line), flush=True)


def run_paper41(args, world, rank):
    """Sec. 4.1: randomly generated cubical tensors of three, four and five
    modes (700^3, 300^4, 75^5; entries uniform on [0, 1), generated on the
    device from a fixed seed; FP64), for a sweep of ranks.  Per (shape, rank)
    and solve (CP-ALS, CP-ALS-PINV, CP-ALS-QR, CP-ALS-QR-SVD): the time per
    sweep of the captured sweep (CUDA events, after one warm-up sweep), the
    slowdown of CP-ALS-QR against CP-ALS, and the component breakdown of
    Table its_parts from cpals_profile_sweeps (phases serialised on one
    stream)."""
    import torch
    from paper_2112_10855_gb300 import _build, cpals
    torch.cuda.set_device(0)
    _build.build()
    cpals.load()
    shapes = [((700,) * 3, [5, 10, 20, 40, 64]), ((300,) * 4, [5, 10, 20, 40]), ((75,) * 5, [5, 10, 20])]
    solves = [("normal", 0.0), ("normal_pinv", 1e-10), ("qr", 0.0), ("svd", 1e-10)]
    stream = torch.cuda.Stream()
    results = []
    t0 = time.time()
    for dims, ranks in shapes:
        g = torch.Generator(device="cuda").manual_seed(4101 + len(dims))
        X = torch.rand(int(np.prod(dims)), dtype=torch.float64, device="cuda", generator=g)
        for R in ranks:
            rng = np.random.default_rng(4100 + R)
            A = [np.asfortranarray(rng.random((d, R))) for d in dims]
            entry = {"dims": list(dims), "rank": R, "ms_per_sweep": {}, "breakdown_ms": {}}
            for solve, rtol in solves:
                h = cpals.CPALS(dims, R, "f64")
                h.set_stream(stream)
                h.set_tensor(X)
                h.set_factors(A)
                h.iterate(1, solve=solve, svd_rtol=rtol, want_fits=False)
                torch.cuda.synchronize()
                k = max(2, min(10, int(3.0e11 / (float(np.prod(dims)) * R * 4))))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.iterate(k, solve=solve, svd_rtol=rtol, want_fits=False)
                e1.record(stream)
                torch.cuda.synchronize()
                entry["ms_per_sweep"][solve] = e0.elapsed_time(e1) / k
                entry["breakdown_ms"][solve] = h.profile_sweeps(2, solve=solve, svd_rtol=rtol)
                del h
                torch.cuda.empty_cache()
            entry["slowdown_qr_vs_normal"] = entry["ms_per_sweep"]["qr"] / entry["ms_per_sweep"]["normal"]
            results.append(entry)
            print(json.dumps({"dims": list(dims), "rank": R, "ms_per_sweep": entry["ms_per_sweep"],
                              "slowdown_qr_vs_normal": entry["slowdown_qr_vs_normal"]}), file=sys.stderr, flush=True)
        del X
        torch.cuda.empty_cache()
    if rank == 0:
        line = {
            "metric": "CP-ALS-QR / CP-ALS time per sweep (Sec. 4.1)", "value": float(np.mean(
                [r["slowdown_qr_vs_normal"] for r in results])), "unit": "ratio (mean over shapes and ranks)",
            "n_gpus": world, "steps": None, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Sec. 4.1: random cubical tensors 700^3, 300^4, 75^5 (uniform [0, 1), FP64), "
                                   "rank sweep, random initial factors; CP-ALS, CP-ALS-PINV, CP-ALS-QR, "
                                   "CP-ALS-QR-SVD, dimension-tree sweeps"},
            "results": results, "wall_s": time.time() - t0,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "c4":
        run_batch(args, world, rank)
        return
    if args.workload == "sine":
        run_sine(args, world, rank)
        return
    if args.workload == "collinear":
        run_collinear(args, world, rank)
        return
    if args.workload == "paper41":
        run_paper41(args, world, rank)
        return
    if args.workload != "c2":
        run_mixed(args, world, rank)
        return
    import torch
    from paper_2112_10855_gb300 import _build, cpals

    if world == 1:
        torch.cuda.set_device(0)
    _build.build()
    cpals.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    p = workload(args.size, args.rank, 2112 + rank)
    P = int(np.prod(p.dims))
    R = p.rank
    stream = torch.cuda.Stream(device=dev)

    Xd = torch.from_numpy(p.X).to(dev)
    h = cpals.CPALS(p.dims, R, "f64")
    h.set_stream(stream)
    h.set_tensor(Xd)
    h.set_factors([np.asfortranarray(a) for a in p.init_factors])

    # warm-up (also captures the sweep graph)
    h.iterate(args.warmup, solve=args.solve, svd_rtol=1e-10, want_fits=False)
    torch.cuda.synchronize()

    launches0 = h.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        h.iterate(args.steps, solve=args.solve, svd_rtol=1e-10, want_fits=False)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    gpu_launches = h.launch_count() - launches0
    ms_max = max_over_ranks(ms, world)
    value = world * args.steps / (ms_max * 1e-3)
    fit_now = h.fit()

    # dominant kernel: the first TTM of each mode's Multi-TTM (streams X), timed alone
    reps = 5
    ttm_ms = []
    for n in range(3):
        h.ttm_first(n)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            h.ttm_first(n)
        e1.record(stream)
        torch.cuda.synchronize()
        ttm_ms.append(e0.elapsed_time(e1) / reps)
    ttm_avg_ms = sum(ttm_ms) / len(ttm_ms)
    flops = 2.0 * P * R
    achieved_tflops = flops / (ttm_avg_ms * 1e-3) / 1e12
    peak_fp64 = SM_COUNT * FP64_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    probe64, probe32 = cpals.probe_fma_peak(30.0)
    hbm = measured_peaks().get("hbm_gbs")
    ttm_gbs = 8.0 * P / (ttm_avg_ms * 1e-3) / 1e9

    # end to end through the C-ABI with host buffers: X and the factors copied in
    # from pinned host memory, one sweep, factors + fit read back, every step
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 5))
    Xh = torch.from_numpy(p.X).pin_memory()
    Ah = [torch.from_numpy(np.asfortranarray(a)).pin_memory() for a in p.init_factors]
    Ah = [a.t().contiguous().t() if a.stride() != (1, a.shape[0]) else a for a in Ah]
    he = cpals.CPALS(p.dims, R, "f64")
    he.set_stream(stream)
    he.set_tensor(Xh)
    he.set_factors(Ah)
    he.iterate(1, solve=args.solve, svd_rtol=1e-10, want_fits=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        he.set_tensor(Xh)
        he.set_factors(Ah)
        he.iterate(1, solve=args.solve, svd_rtol=1e-10, want_fits=False)
        outA, lam = he.get_factors()
        f = he.fit()
    torch.cuda.synchronize()
    e2e_seq_s = max_over_ranks(time.perf_counter() - t0, world)
    del he
    # the same steps, double-buffered as a user streaming tensors from the host
    # would run them: two handles on two streams in two host threads, so that
    # one step's host-to-device copy (about 2.5 ms at the host link's ~210 GB/s)
    # runs while the other handle's sweep runs; each step still copies its own
    # X and factors in and reads its factors, lambda and fit back
    pipe_steps = 2 * max(e2e_steps, 10)
    fac_bytes = 8 * sum(d * R for d in p.dims)
    seq = {"value": world * e2e_steps / e2e_seq_s, "steps": e2e_steps,
           "what": "one handle, each step's copy, sweep and read-back in turn"}
    try:
        e2e_pipe_s = max_over_ranks(e2e_double_buffered(cpals, p.dims, R, Xh, Ah, args.solve, pipe_steps), world)
        e2e = {"value": world * pipe_steps / e2e_pipe_s, "unit": UNIT, "h2d_bytes_per_step": 8 * P + fac_bytes,
               "d2h_bytes_per_step": fac_bytes + 8 * R + 8, "steps": pipe_steps,
               "what": "per step: pinned-host X and factors in, one sweep, factors, lambda and fit out; two "
                       "handles alternate steps so that one step's copy overlaps the other's sweep",
               "sequential": seq}
    except Exception as exc:   # the one-handle figure stands on its own
        e2e = {"value": seq["value"], "unit": UNIT, "h2d_bytes_per_step": 8 * P + fac_bytes,
               "d2h_bytes_per_step": fac_bytes + 8 * R + 8, "steps": e2e_steps, "what": seq["what"],
               "double_buffered_failed": str(exc)[:200]}

    variants = {}
    if not args.no_variants:
        for solve in ("svd", "normal", "normal_pinv"):
            if solve == args.solve:
                continue
            hv = cpals.CPALS(p.dims, R, "f64")
            hv.set_stream(stream)
            hv.set_tensor(Xd)
            hv.set_factors([np.asfortranarray(a) for a in p.init_factors])
            hv.iterate(2, solve=solve, svd_rtol=1e-10, want_fits=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hv.iterate(5, solve=solve, svd_rtol=1e-10, want_fits=False)
            e1.record(stream)
            torch.cuda.synchronize()
            variants[f"f64_{solve}"] = 5 / (e0.elapsed_time(e1) * 1e-3)
            del hv
        hn = cpals.CPALS(p.dims, R, "f64")
        hn.set_stream(stream)
        hn.set_tensor(Xd)
        hn.set_factors([np.asfortranarray(a) for a in p.init_factors])
        hn.set_dimtree(False)
        hn.iterate(2, solve=args.solve, svd_rtol=1e-10, want_fits=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hn.iterate(10, solve=args.solve, svd_rtol=1e-10, want_fits=False)
        e1.record(stream)
        torch.cuda.synchronize()
        variants[f"f64_{args.solve}_per_mode_multi_ttm"] = 10 / (e0.elapsed_time(e1) * 1e-3)
        del hn
        hf = cpals.CPALS(p.dims, R, "f32")
        hf.set_stream(stream)
        hf.set_tensor(Xd)
        hf.set_factors([np.asfortranarray(a) for a in p.init_factors])
        hf.iterate(2, solve=args.solve, want_fits=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hf.iterate(args.steps, solve=args.solve, want_fits=False)
        e1.record(stream)
        torch.cuda.synchronize()
        variants[f"f32_{args.solve}"] = args.steps / (e0.elapsed_time(e1) * 1e-3)
        del hf

    mixed = None
    if rank == 0 and not args.no_mixed:
        try:
            mixed = mixed_c3_record(args, stream)
        except Exception as exc:     # reported, not fatal to the headline
            mixed = {"failed": str(exc)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        solve_id = {"qr": 0, "svd": 1, "normal": 2}[args.solve]
        rate, dt, n = cpu_oracle_rate(p, solve=solve_id)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} full sweeps of the same workload ({dt:.1f} s), plain C FP64, 1 host thread"}
        try:
            agg, cores, wall = cpu_oracle_all_cores(p.dims[0], R, sweeps=1, solve=solve_id)
            cpu["all_cores"] = {"value": agg, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"one replica of the oracle per host core ({cores}), each generating the "
                                          f"same workload and timing 1 full sweep; sum of the replicas' rates "
                                          f"({wall:.1f} s wall)"}
        except Exception as exc:     # reported, not fatal
            cpu["all_cores"] = {"failed": str(exc)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(p.dims[0], R, args.solve), "dims": list(p.dims), "rank": R,
                       "solve": args.solve,
                       "l2": "inputs larger than L2 (X is 8*P bytes > 129 MB); no flush needed",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_fp64, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak_fp64,
                         "traffic": recorded_traffic() if (p.dims == (400, 400, 400) and R == 10) else None,
                         "algorithmic_bytes": 8 * P,
                         "kernel": "ttm_rows_kernel<double> (first TTM of the Multi-TTM, streams X)",
                         "peak_source": "152 SMs x 2 DFMA/clk x 2070 MHz (derived); live FMA probe below",
                         "probe_fp64_tflops": probe64, "probe_fp32_tflops": probe32,
                         "ms_per_launch": ttm_avg_ms, "flops_per_launch": flops},
            "multi_ttm": {"gbs": ttm_gbs, "hbm_peak_gbs": hbm, "frac_hbm": (ttm_gbs / hbm) if hbm else None},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "fit_after": fit_now,
            "variants_iters_per_s": variants,
            "mixed": mixed,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

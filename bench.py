"""Benchmark of the approximate mini-batch kernel k-means fit on one GB300.

Workload (the MNIST-shaped feature-vector run): N = 60,000 samples x d = 784
values in [0, 1] quantised to k/255 (10 sparse Gaussian-mixture classes), RBF
kernel with the median-distance bandwidth computed inside the fit, C = 10,
B = 4 stride mini-batches, s = 0.2 (|L| = 3,000 landmarks per mini-batch of
15,000), 30 inner iterations per mini-batch with early stop off (so every
step does exactly 120 iterations), kernel k-means++ seeding, FP32.

One step = one kkm_fit call over the whole data set.  Reported:
  value      kernel evaluations per second of the whole fit, device-timed
             with X resident in HBM (CUDA events on the fit's stream);
  e2e        the same metric through the C ABI with host buffers (X in
             pinned host memory, labels back to host), copies inside the timed
             region;
  roofline   for the kernel with the largest share of device time, its
             algorithmic work per launch over its event-timed launch duration;
  cpu_baseline  the FP64 oracle on a bounded sample of the same workload.
Inputs are larger than L2 (X 188 MB, the kernel block 180 MB), so no L2 flush
is needed between steps.

--impl reference times the oracle (the plain FP64 CPU restatement of the
method) on a bounded sample of the same workload per step.
"""

import argparse
import atexit
import datetime
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the benchmark line: MNIST-shaped feature vectors, RBF, tensor-core block
    "mnist": dict(name="mnist-shaped 60000x784 RBF, C=10, B=4, s=0.2, 30 iters", N=60000, d=784, C=10,
                  B=4, s=0.2, iters=30, seed=1710, kind="rbf", sigma=0.0, n_atoms=0,
                  precisions=("bf16", "fp32", "fp8")),
    # secondary: MD-shaped trajectory, RMSD kernel (FP32 FFMA)
    "md": dict(name="md-shaped 500000 frames x 300 atoms RMSD, sigma=1.5, C=8, B=20, s=0.05, 25 iters",
               N=500000, d=900, C=8, B=20, s=0.05, iters=25, seed=1710, kind="rmsd", sigma=1.5, n_atoms=300,
               precisions=("fp32",)),
}
# the batched form: 256 independent RBF problems of uneven sizes in one call
WORKLOADS["batched"] = dict(
    name="batched: 256 RBF problems, N log-uniform [1e3, 5e4], d in {8,32,64,128}, C in [2,64], "
         "B=ceil(N/1e4), s in {0.1,0.5}, 20 iters", kind="rbf", precisions=("bf16", "fp32"), iters=20,
    n_problems=256)
# the serving loop: a Poisson stream of fit and assign requests
WORKLOADS["serving"] = dict(
    name="serving: Poisson 200 req/s, 10% fits (batched-workload shapes, BF16 RBF, 20 iters), 90% assigns of "
         "1..10000 MD frames (300 atoms, supports mode) against 4 resident RMSD models (N = 1e5, 3e5, 1e6, 1e6; "
         "C = 32, 64, 128, 256; s = 0.01, B = 1; sigma = 1.5 A), 150 GB budget",
    kind="serving", rate=200.0, fit_share=0.1, budget_gb=150, n_atoms=300, sigma=1.5,
    models=((100000, 32), (300000, 64), (1000000, 128), (1000000, 256)), model_s=0.01, model_iters=10,
    max_query=10000, workers=4)
WORKLOAD = WORKLOADS["mnist"]
METRIC = "kernel evals/s & iters/s vs plain FP32 path at matched labels; p50/p99 latency"
UNIT = "kernel evals/s"
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # FFMA lanes x 2 flops x max SM clock
L2_READ_GBS = 11300.0   # L2-resident read bandwidth, this project's probe (90 MB held with evict_last)
BATCH_CPU_PROBLEMS = 16     # oracle sample of the batched workload: its smallest problems


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def n_landmarks(Ni, s):
    import math
    return int(min(max(math.ceil(s * Ni - 1e-9), 1), Ni))


def fit_evals(N, B, C, s):
    """Kernel evaluations of one fit (Alg. 1): per mini-batch the block
    N_i x |L|, the auxiliary block N_i x C (Eq. 8) and the merge column block
    N_i x C (Eq. 12); plus (C-1) k-means++ columns over the first mini-batch."""
    total = 0
    for i in range(B):
        Ni = (N - i + B - 1) // B
        total += Ni * n_landmarks(Ni, s) + 2 * Ni * C
    total += (C - 1) * ((N + B - 1) // B)
    return total


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples, kept for the timed region only.

    The sampler is started before the warm-up (its start-up is not inside the
    timed region) and the region is bracketed with begin()/end(); samples are
    matched to it by their timestamps."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.t0 = self.t1 = None
        self.dir = tempfile.mkdtemp(prefix="kkm_clocks_")
        self.path = os.path.join(self.dir, "clocks.csv")
        atexit.register(self.cleanup)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()
        if self.proc:
            time.sleep(0.15)  # one more sample period, so the region's last sample is written

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def cleanup(self):
        shutil.rmtree(self.dir, ignore_errors=True)

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                except ValueError:
                    continue
                rows.append((ts, parts[1:]))
        window = "timed region"
        if self.t0 and self.t1:
            lo = self.t0 - datetime.timedelta(seconds=0.1)
            hi = self.t1 + datetime.timedelta(seconds=0.1)
            inside = [r for r in rows if lo <= r[0] <= hi]
            if inside:
                rows = inside
            else:
                window = "whole run (no sample matched the region's timestamps)"
        rows = [r for _, r in rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window}


def source_hash(files, region=None):
    """Hash of the kernel sources a traffic figure was taken with: whole files,
    or only the text from region[0] up to region[1] in each (the kernel's own
    part of a file that holds other kernels too)."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1710_03013_gb300", "csrc", f), "rb") as fh:
            text = fh.read()
        if region:
            a = text.index(region[0].encode())
            text = text[a:text.index(region[1].encode(), a)]
        h.update(text)
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name, workload="mnist"):
    """DRAM bytes per launch of the kernel on the workload from the committed
    ncu summary, or None when there is no capture or the kernel's source
    changed since it."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        data = json.load(f)
    ent = data.get(f"{kernel_name}@{workload}")
    if not ent:
        return None
    try:
        if source_hash(ent["sources"], ent.get("region")) != ent["source_hash"]:
            return None
    except (OSError, ValueError):
        return None
    return ent["bytes_per_launch"]


def max_over_ranks(values, world, device):
    """Each value's maximum over the ranks: a replicated job takes as long as
    its slowest rank (NCCL on the GPUs; any backend, e.g. gloo on CPU)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


# ---------------------------------------------------------------- oracle
# The oracle is timed on every host core this process may use: one process
# per core, each running the oracle's whole fit (same d, C, B, s, iters) on
# its own window of ORACLE_ROWS consecutive samples; the rate is the kernel
# evaluations of all those fits over the wall time of the parallel region.
# The bandwidth is computed once, before timing, by the oracle's median rule
# on 512 samples, and given to every fit, so the rule's fixed cost (which does
# not scale with the sample) stays out of the rate.  The same procedure gives
# the benchmark's cpu_baseline and every step of --impl reference.
ORACLE_ROWS = {"mnist": 4000, "md": 4000}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_fit_task(task):
    """One process's share: the oracle's fit of its window (returns seconds)."""
    Xs, cfg = task
    from oracle import kkm_oracle as O
    kind = O.KIND_RMSD if cfg["kind"] == "rmsd" else O.KIND_RBF
    t0 = time.perf_counter()
    O.fit(Xs, cfg["C"], cfg["B"], cfg["s"], O.Kernel(kind, cfg["sigma"], cfg["n_atoms"]), cfg["iters"],
          cfg["seed"], early_stop=False)
    return time.perf_counter() - t0


def _oracle_ready(_):
    from oracle import kkm_oracle  # noqa: F401  (imports numpy and the oracle once per process)
    return os.getpid()


class OraclePool:
    """Worker processes for the oracle (spawned: the parent may hold a CUDA
    context, which a forked child must not inherit), one per host core, each
    with single-threaded numpy so that the cores are not oversubscribed."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.map(_oracle_ready, range(4 * self.cores), timeout=300)

    def map(self, fn, tasks, timeout):
        """pool.map with a time limit: a worker that cannot start or dies
        ends the benchmark with an error instead of a wait without end."""
        try:
            return self.pool.map_async(fn, tasks, chunksize=1).get(timeout)
        except BaseException:
            self.pool.terminate()
            raise

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_cfg(X, cfg):
    """cfg with the bandwidth the oracle fits use (the oracle's median rule on
    512 samples when the workload's sigma is 0)."""
    from oracle import kkm_oracle as O
    out = dict(cfg)
    if cfg["sigma"] <= 0.0:
        kind = O.KIND_RMSD if cfg["kind"] == "rmsd" else O.KIND_RBF
        Xr = X.reshape(X.shape[0], -1)
        out["sigma"] = O.median_bandwidth(Xr, O.Kernel(kind, 0.0, cfg["n_atoms"]), O.SplitMix64(cfg["seed"]), 512)
    return out


def oracle_parallel(pool, X, cfg, rows):
    """The oracle's fits of pool.cores windows of `rows` samples, one per
    process, timed together.  Returns (kernel evals, wall seconds,
    description)."""
    N = X.shape[0]
    P = pool.cores
    rows = min(rows, N)
    starts = [(p * (N - rows)) // max(P - 1, 1) for p in range(P)]
    tasks = [(X[a:a + rows].reshape(rows, -1).astype(np.float64), cfg) for a in starts]
    t0 = time.perf_counter()
    pool.map(_oracle_fit_task, tasks, timeout=900)
    wall = time.perf_counter() - t0
    ev = P * fit_evals(rows, cfg["B"], cfg["C"], cfg["s"])
    desc = (f"{P} processes (one per host core), each the oracle's whole fit of its own window of {rows} "
            f"consecutive samples (same d, C, B, s, iters; sigma {cfg['sigma']:.6g} from the oracle's median "
            f"rule on 512 samples, outside the timed region); {ev} kernel evals in {wall:.2f} s wall")
    return ev, wall, desc


def run_reference(args, cfg, X):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ocfg = oracle_cfg(X, cfg)
    pool = OraclePool()
    times, evals, desc = [], 0, ""
    rows = ORACLE_ROWS[cfg["key"]]
    for k in range(args.warmup + args.steps):
        ev, dt, desc = oracle_parallel(pool, X, ocfg, rows)
        if k >= args.warmup:
            times.append(dt)
            evals = ev
    pool.close()
    tot = sum(times)
    value = evals * len(times) / tot
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": cfg["name"], "sample": desc},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ ours
def run_ours(args, cfg, X):
    import torch
    import torch.distributed as dist
    from paper_1710_03013_gb300 import kkm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream(dev)
    C, B, s, iters, seed = cfg["C"], cfg["B"], cfg["s"], cfg["iters"], cfg["seed"]

    PREC = {"bf16": kkm.KKM_BF16, "fp32": kkm.KKM_FP32, "fp8": kkm.KKM_FP8}
    HEAD = PREC[cfg["precisions"][0]]
    CMP = PREC[cfg["precisions"][1]] if len(cfg["precisions"]) > 1 else None
    ALT = PREC[cfg["precisions"][2]] if len(cfg["precisions"]) > 2 else None
    kind, sig, atoms = cfg["kind"], cfg["sigma"], cfg["n_atoms"]

    def step(prec=HEAD, pipeline=args.pipeline):
        return kkm.kkm_fit(Xd, C, B, s, kind, sig, atoms, iters=iters, seed=seed, early_stop=False, precision=prec,
                           pipeline=pipeline)

    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        lab, model = step(HEAD)
        if CMP is not None:
            step(CMP)
        if ALT is not None:
            step(ALT)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, n, pipeline=args.pipeline):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = []  # results are released after the region (freeing them is not part of a step)
        for _ in range(n):
            outs.append(step(prec, pipeline))
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / n, outs[-1]

    # timed region 1: the headline value (no instrumentation)
    clk.begin()
    ms, (lab, model) = timed(HEAD, args.steps)
    clk.end()
    clk.__exit__()
    ms32, agree, omega_rel = None, None, None
    if CMP is not None:
        # the plain FP32 path on the same workload, for comparison
        ms32, (lab32, model32) = timed(CMP, args.steps)
        agree = float((lab == lab32).float().mean().item())
        om16, _ = model.trace()
        om32, _ = model32.trace()
        omega_rel = float(np.max(np.abs(om16 - om32) / np.abs(om32))) if len(om32) else None
    ms8, agree8, omega_rel8 = None, None, None
    if ALT is not None and CMP is not None:
        # the FP8 block on the same workload, beside the BF16 one
        ms8, (lab8, model8) = timed(ALT, args.steps)
        agree8 = float((lab8 == lab32).float().mean().item())
        om8, _ = model8.trace()
        omega_rel8 = float(np.max(np.abs(om8 - om32) / np.abs(om32))) if len(om32) else None
    # the same steps with every kernel block computed just before its inner
    # loop (no overlap with the previous mini-batch), for comparison
    ms_serial = timed(HEAD, args.steps, "serial")[0] if args.pipeline != "serial" and B > 1 else None
    # timed region 2: the same steps with serial blocks, so that each kernel
    # runs alone on the GPU; every library launch is counted and the
    # kernel-block and streaming kernels are bracketed by CUDA events on
    # their stream (their durations feed the roofline)
    kkm.prof_reset()
    kkm.prof_enable(2)
    barrier()
    for _ in range(args.steps):
        lab, model = step(HEAD, "serial")
    barrier()
    kkm.prof_enable(False)
    prof = {n: kkm.prof_read(n) for n in kkm.prof_names()}
    exact_pairs = kkm.prof_work("rmsd_exact")   # pairs the MD exact pass recomputed in region 2
    launches = sum(v[0] for v in prof.values())
    # one more step with every launch timed, for the per-kernel breakdown
    kkm.prof_reset()
    kkm.prof_enable(1)
    lab, model = step(HEAD, "serial")
    torch.cuda.synchronize()
    kkm.prof_enable(False)
    breakdown = {n: kkm.prof_read(n)[1] for n in kkm.prof_names()}
    # the other paths' heavy kernels, timed the same way (a few steps each)
    def prof_path(prec):
        kkm.prof_reset()
        kkm.prof_enable(2)
        barrier()
        for _ in range(min(args.steps, 3)):
            step(prec, "serial")
        barrier()
        kkm.prof_enable(False)
        return {n: kkm.prof_read(n) for n in kkm.prof_names()}
    prof32 = prof_path(CMP) if CMP is not None else None
    prof8 = prof_path(ALT) if ALT is not None else None
    mx = max_over_ranks([ms, ms32 or 0.0, ms_serial or 0.0], world, dev)
    ms, ms32, ms_serial = mx[0], (mx[1] if ms32 is not None else None), (mx[2] if ms_serial is not None else None)

    evals = fit_evals(cfg["N"], B, C, s)
    value = world * evals / (ms / 1e3)
    om, _ = model.trace()

    # ---- end to end through the C ABI with host buffers
    Xh = torch.from_numpy(X).pin_memory()
    e2e_ms = []
    for k in range(max(3, min(5, args.steps)) + 1):  # the median of at least 3: one slow fit cannot set it
        barrier()
        t0 = time.perf_counter()
        lab_h, _ = kkm.kkm_fit(Xh, C, B, s, kind, sig, atoms, iters=iters, seed=seed, early_stop=False,
                               precision=HEAD, stream=ctypes_stream(stream), pipeline=args.pipeline)
        t1 = time.perf_counter()
        if k > 0:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e = max_over_ranks([float(np.median(e2e_ms))], world, dev)[0]

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None  # among the timed kernels
    Ni = (cfg["N"] + B - 1) // B
    nL = n_landmarks(Ni, s)
    roof = None
    if dom == "gram_block":
        n, tms = prof[dom]
        flops = sum(2.0 * ((cfg["N"] - i + B - 1) // B) * n_landmarks((cfg["N"] - i + B - 1) // B, s)
                    * cfg["d"] for i in range(B)) / B
        ach = flops / (tms / n / 1e3) / 1e12
        pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": ncu_traffic("gram_block", cfg["key"]), "kernel": "gram_block (tcgen05 BF16)",
                "peak_source": peak_kind + " bf16 sustained",
                "work_per_launch": f"2*N_i*|L|*d = {flops:.4g} flop"}
    elif dom == "rmsd_exact":
        n, tms = prof[dom]
        pairs = exact_pairs / n   # frame pairs the exact pass recomputed, per launch
        flops = 30.0 * cfg["n_atoms"] * pairs      # residual |R x - y|^2: 15 FMA per atom
        ach = flops / (tms / n / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP32_TFLOPS, "traffic": ncu_traffic("rmsd_exact", cfg["key"]),
                "kernel": "rmsd_exact (FP32 two-pass QCP on the tiles the tensor-core screen flagged)",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "work_per_launch": f"30*n_atoms flop per recomputed pair (the residual at the screen's "
                                   f"rotation) x {pairs:.4g} pairs = {flops:.4g} flop"}
        if "rmsd_block" in prof:
            n2, t2 = prof["rmsd_block"]
            kp = 3 * (-(-cfg["n_atoms"] // 64) * 64)   # split-BF16 operands: three segments
            fl2 = sum(2.0 * 4 * ((cfg["N"] - i + B - 1) // B) * 4 * n_landmarks((cfg["N"] - i + B - 1) // B, s) * kp
                      for i in range(B)) / B
            pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            # the method's own work: the 3 x 3 correlation of every pair, 18 flop per atom
            fl_m = sum(18.0 * cfg["n_atoms"] * ((cfg["N"] - i + B - 1) // B) * n_landmarks((cfg["N"] - i + B - 1) // B, s)
                       for i in range(B)) / B
            roof["screen"] = {"kernel": "rmsd_block (tcgen05 split-BF16 correlation screen)", "bound": "tensor",
                              "achieved": fl2 / (t2 / n2 / 1e3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                              "frac": fl2 / (t2 / n2 / 1e3) / 1e12 / pk,
                              "work_per_launch": f"2*(4 N_i)*(4 |L|)*{kp} = {fl2:.4g} flop (padded GEMM: zero "
                                                 f"fourth plane, three split-BF16 segments, atoms to {kp // 3})",
                              "method_achieved": fl_m / (t2 / n2 / 1e3) / 1e12,
                              "method_frac": fl_m / (t2 / n2 / 1e3) / 1e12 / pk,
                              "method_work_per_launch": f"18*n_atoms*N_i*|L| = {fl_m:.4g} flop (the 3x3 "
                                                        "correlations the method needs)"}
    elif dom == "rmsd_block":
        n, tms = prof[dom]
        flops = sum(18.0 * cfg["n_atoms"] * ((cfg["N"] - i + B - 1) // B) * n_landmarks((cfg["N"] - i + B - 1) // B, s)
                    for i in range(B)) / B
        ach = flops / (tms / n / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP32_TFLOPS, "traffic": ncu_traffic("rmsd_block", cfg["key"]), "kernel": "rmsd_block",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "work_per_launch": f"18*n_atoms flop per pair (3x3 correlation) = {flops:.4g} flop"}
    elif dom in ("fhat_partial", "iterate"):
        n, tms = prof[dom]
        esz = 2 if (HEAD == kkm.KKM_BF16 and kind == "rbf") else 4   # the BF16 path stores the block in FP16
        # one read of the block per inner iteration: a launch of the split
        # form's stream reads it once, the one-launch loop once per iteration
        per = iters if dom == "iterate" else 1
        by = esz * Ni * nL * per
        ach = by / (tms / n / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": ncu_traffic(dom, cfg["key"]),
                "kernel": ("iterate (the inner loop in one launch: f_hat on the tensor cores as the FP16 block "
                           "times the one-hot label matrix, g_hat and cost grid barriers, argmin, re-score)"
                           if dom == "iterate" else "fhat_partial"),
                "peak_source": peak_kind,
                "work_per_launch": (f"{esz}*N_i*|L| x {per} iterations = {by:.4g} B (one read of the kernel "
                                    "block per iteration)" if per > 1 else
                                    f"{esz}*N_i*|L| = {by:.4g} B (one read of the kernel block)"),
                "l2_resident_read": {"gbs": L2_READ_GBS, "frac": ach / L2_READ_GBS,
                                     "source": "this project's probe: back-to-back reads of a 90 MB buffer held "
                                               "in L2 with evict_last (the block fits the 129 MB L2)"},
                "note": ("the block stays in L2 across the iterations of a mini-batch (90 MB of the 129 MB L2), "
                         "so the stream runs at the L2 read rate and can exceed the HBM copy bandwidth; "
                         "l2_resident_read is the bound that applies")}

    if roof:
        roof["timing"] = ("CUDA events on the kernel's stream, every launch of a run with serial blocks "
                          "(each kernel alone on the GPU)")

    # rooflines of the plain FP32 path (the Gram product on the FFMA pipes, the
    # FP32 block stream from HBM/L2) and of the FP8 block (tensor cores)
    block_flops = sum(2.0 * ((cfg["N"] - i + B - 1) // B) * n_landmarks((cfg["N"] - i + B - 1) // B, s) * cfg["d"]
                      for i in range(B)) / B
    roof32 = None
    if prof32 and kind == "rbf":
        roof32 = {}
        if "gram_block" in prof32:
            n, tms = prof32["gram_block"]
            ach = block_flops / (tms / n / 1e3) / 1e12
            roof32["gram_block"] = {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                                    "frac": ach / PEAK_FP32_TFLOPS,
                                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                                    "work_per_launch": f"2*N_i*|L|*d = {block_flops:.4g} flop (FFMA)"}
        if "fhat_partial" in prof32:
            n, tms = prof32["fhat_partial"]
            by = 4.0 * Ni * nL
            ach = by / (tms / n / 1e3) / 1e9
            roof32["fhat_partial"] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                      "frac": ach / peaks["hbm_gbs"], "peak_source": peak_kind,
                                      "work_per_launch": f"4*N_i*|L| = {by:.4g} B (one read of the FP32 block)"}
    roof8 = None
    if prof8 and "gram_block" in prof8:
        n, tms = prof8["gram_block"]
        ach = block_flops / (tms / n / 1e3) / 1e12
        pk8 = 2.0 * peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        roof8 = {"gram_block": {"bound": "tensor", "achieved": ach, "peak": pk8, "unit": "TFLOP/s", "frac": ach / pk8,
                                "peak_source": peak_kind + " bf16 sustained x 2 (the nominal FP8/BF16 dense ratio)",
                                "work_per_launch": f"2*N_i*|L|*d = {block_flops:.4g} flop (e4m3)"}}

    # ---- CPU baseline: the oracle on a bounded sample, on every host core
    cpu = None
    if rank == 0:
        pool = OraclePool()
        ocfg = oracle_cfg(X, cfg)
        oracle_parallel(pool, X, ocfg, ORACLE_ROWS[cfg["key"]])   # warm-up (first-touch, imports)
        ev, dt, desc = oracle_parallel(pool, X, ocfg, ORACLE_ROWS[cfg["key"]])
        pool.close()
        cpu = {"value": ev / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": desc}

    it_ms = sum(breakdown.get(k, 0.0) for k in ("fhat_partial", "assign", "iterate"))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("bf16 products, f32 accumulation and sums, f64 cost" if HEAD == kkm.KKM_BF16
                  else "f32, f64 cost"),
        "data": "synthetic",
        "config": {"workload": cfg["name"], "N": cfg["N"], "d": cfg["d"], "C": C, "B": B, "s": s,
                   "iters_per_minibatch": iters,
                   "pipeline": (f"{args.pipeline}: next mini-batch's kernel block on a low-priority stream during "
                                "the current inner loop" if args.pipeline != "serial" and B > 1
                                else "serial: each kernel block before its inner loop"),
                   "precision": ("bf16 tensor-core kernel block, FP32 near-tie re-score" if HEAD == kkm.KKM_BF16
                                 else "fp32"), "bandwidth": "median rule inside the fit",
                   "l2": f"inputs larger than L2 (X {X.nbytes / 1e6:.0f} MB); no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "iters_per_s": world * B * iters / (ms / 1e3),
        "serial_pipeline": ({"value": world * evals / (ms_serial / 1e3), "unit": UNIT, "ms_per_step": ms_serial}
                            if ms_serial else None),
        "fp32_path": ({"value": world * evals / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32,
                       "iters_per_s": world * B * iters / (ms32 / 1e3), "roofline": roof32} if ms32 else None),
        "matched_labels": {"fraction_equal_to_fp32_path": agree, "omega_max_rel_diff": omega_rel},
        "fp8_path": ({"value": world * evals / (ms8 / 1e3), "unit": UNIT, "ms_per_step": ms8,
                      "iters_per_s": world * B * iters / (ms8 / 1e3), "roofline": roof8,
                      "matched_labels": {"fraction_equal_to_fp32_path": agree8, "omega_max_rel_diff": omega_rel8}}
                     if ms8 else None),
        "inner_iter_ms": it_ms / (B * iters),
        "evals_per_step": evals,
        "e2e": {"value": world * evals / (e2e / 1e3), "unit": UNIT, "ms_per_step": e2e,
                "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(4 * cfg["N"])},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "kernels_ms_per_step": {k: v for k, v in sorted(breakdown.items(), key=lambda kv: -kv[1])},
        "kernels_note": "per-kernel breakdown from one step with serial blocks and every launch bracketed "
                        "by events (short kernels include launch gaps); the roofline uses region 2",
        "final_omega": float(om[-1]) if len(om) else None,
    }
    emit(out)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------ batched form
def batched_data(cfg):
    from synth import batched_problems, blobs
    shapes = batched_problems(cfg["n_problems"])[:cfg.get("take") or None]
    data = [blobs(p["N"], p["d"], p["C"], workload=3, problem=p["problem"])[0] for p in shapes]
    return shapes, data


def _oracle_problem_task(task):
    """One batched problem's oracle fit (median bandwidth inside, as kkm_fit)."""
    X, C, B, s, iters, seed = task
    from oracle import kkm_oracle as O
    O.fit(X, C, B, s, O.Kernel(O.KIND_RBF, 0.0), iters, seed, early_stop=False)
    return 0


def batched_oracle(shapes, data, cfg, k, pool):
    """The oracle's fits of the k smallest problems (bandwidth by the median
    rule, as inside kkm_fit), one process per problem on the pool's cores.
    Returns (kernel evals, wall seconds, description)."""
    order = sorted(range(len(shapes)), key=lambda i: shapes[i]["N"])[:k]
    tasks = [(data[i].astype(np.float64), shapes[i]["C"], shapes[i]["B"], shapes[i]["s"], cfg["iters"], 1710 + i)
             for i in order]
    ev = sum(fit_evals(shapes[i]["N"], shapes[i]["B"], shapes[i]["C"], shapes[i]["s"]) for i in order)
    t0 = time.perf_counter()
    pool.map(_oracle_problem_task, tasks, timeout=900)
    dt = time.perf_counter() - t0
    desc = (f"oracle fits of the {k} smallest problems of the batch (N = "
            f"{', '.join(str(shapes[i]['N']) for i in order)}; same d, C, B, s, iters), one process per problem "
            f"on {pool.cores} host cores, {ev} kernel evals in {dt:.2f} s wall")
    return ev, dt, desc


def batched_parity(kkm, shapes, data, cfg, k, dev):
    """The k smallest problems fitted by the oracle and, with the same
    bandwidth (the oracle's median rule, rounded to float32) and seeds, by the
    library in both precisions: the fraction of labels equal to the oracle's
    wherever its relative margin exceeds 1e-4, and each path's largest Omega
    error against it."""
    import torch
    from oracle import kkm_oracle as O
    order = sorted(range(len(shapes)), key=lambda i: shapes[i]["N"])[:k]
    rows = equal = 0
    om_err = {"bf16": 0.0, "fp32": 0.0}
    for i in order:
        p = shapes[i]
        X = data[i].astype(np.float64)
        _, bw, _ = O.rng_streams(1710 + i, p["B"])
        sig = float(np.float32(O.median_bandwidth(X, O.Kernel(O.KIND_RBF, 0.0), bw)))
        ref = O.fit(X, p["C"], p["B"], p["s"], O.Kernel(O.KIND_RBF, sig), cfg["iters"], 1710 + i, early_stop=False)
        want = np.array([t[2] for t in ref["trace"]])
        for name, prec in (("bf16", kkm.KKM_BF16), ("fp32", kkm.KKM_FP32)):
            lab, model = kkm.kkm_fit(torch.from_numpy(data[i]).to(dev), p["C"], p["B"], p["s"], "rbf", sig,
                                     iters=cfg["iters"], seed=1710 + i, early_stop=False, precision=prec)
            om, _ = model.trace()
            om_err[name] = max(om_err[name], float(np.max(np.abs(om - want) / np.abs(want))))
            if name == "bf16":
                lab = lab.cpu().numpy()
                for det in ref["details"]:
                    d = np.where(np.isfinite(det["steps"][-1]["d"]), det["steps"][-1]["d"], np.inf)
                    part = np.partition(d, 1, axis=1)
                    rel = (part[:, 1] - part[:, 0]) / np.maximum(np.abs(part[:, 1]), 1e-12)
                    clear = rel > 1e-4
                    rows += int(clear.sum())
                    equal += int(np.sum(lab[det["gidx"]][clear] == det["u"][clear]))
    return {"problems": len(order), "rows_above_margin": rows,
            "bf16_labels_equal_to_oracle_above_margin": equal / max(rows, 1),
            "omega_max_rel_err_vs_oracle": om_err,
            "note": ("the reduced-precision Omega carries the FP16 storage rounding of the block (each fit's "
                     "distances to ~1e-4 of the term scale); labels above the margin are settled by the FP32 "
                     "re-score. A trajectory that takes another turn at a near tie in one path ends in a "
                     "different local minimum, which is how the two paths' Omega can differ by more than "
                     "either differs from the oracle on a problem both follow exactly")}


def run_batched(args, cfg):
    import torch
    from paper_1710_03013_gb300 import kkm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    shapes, data = batched_data(cfg)
    iters = cfg["iters"]
    evals = sum(fit_evals(p["N"], p["B"], p["C"], p["s"]) for p in shapes)
    inner = sum(p["B"] * iters for p in shapes)
    if args.impl == "reference":
        if rank != 0:
            return
        times = []
        pool = OraclePool()
        for k in range(args.warmup + args.steps):
            ev, dt, desc = batched_oracle(shapes, data, cfg, BATCH_CPU_PROBLEMS, pool)
            if k >= args.warmup:
                times.append(dt)
        pool.close()
        value = ev * len(times) / sum(times)
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": cfg["name"], "sample": desc},
               "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": desc},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    Xd = [torch.from_numpy(x).to(dev) for x in data]
    PREC = {"bf16": kkm.KKM_BF16, "fp32": kkm.KKM_FP32}
    HEAD, CMP = PREC[cfg["precisions"][0]], PREC[cfg["precisions"][1]]

    def problems(X, prec):
        return [dict(X=X[i], C=p["C"], B=p["B"], s=p["s"], kind="rbf", sigma=0.0, iters=iters, seed=1710 + i,
                     early_stop=False, precision=prec) for i, p in enumerate(shapes)]

    def step(prec, X=Xd):
        return kkm.kkm_fit_batch(problems(X, prec), n_streams=args.streams)

    for _ in range(args.warmup):
        step(HEAD)
    step(CMP)
    torch.cuda.synchronize()

    def timed(prec, n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = []  # results are released after the region (freeing them is not part of a step)
        for _ in range(n):
            outs.append(step(prec))
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n, outs[-1]

    with ClockSampler(local) as clk:
        time.sleep(0.3)  # the sampler's start-up before the region
        clk.begin()
        ms, res = timed(HEAD, args.steps)
        clk.end()
    ms32, res32 = timed(CMP, args.steps)
    lab = torch.cat([r[0] for r in res])
    lab32 = torch.cat([r[0] for r in res32])
    agree = float((lab == lab32).float().mean().item())
    omega_rel = 0.0
    for r16, r32 in zip(res, res32):
        o16, _ = r16[1].trace()
        o32, _ = r32[1].trace()
        omega_rel = max(omega_rel, float(np.max(np.abs(o16 - o32) / np.abs(o32))))

    # instrumented region: launch count and the heavy kernels' event-timed durations
    kkm.prof_reset()
    kkm.prof_enable(2)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        step(HEAD)
    torch.cuda.synchronize()
    kkm.prof_enable(False)
    prof = {n: kkm.prof_read(n) for n in kkm.prof_names()}
    launches = sum(v[0] for v in prof.values()) // args.steps

    # end to end: host inputs (pinned) and labels back to the host
    Xh = [torch.from_numpy(x).pin_memory() for x in data]
    e2e_ms = []
    for k in range(max(2, min(5, args.steps)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kkm.kkm_fit_batch(problems(Xh, HEAD), n_streams=args.streams, stream=ctypes_stream(stream))
        t1 = time.perf_counter()
        if k > 0:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e = float(np.median(e2e_ms))
    if rank != 0:
        return

    peaks, peak_kind = measured_peaks()
    esz = 2.0 if HEAD == kkm.KKM_BF16 else 4.0   # the BF16 path stores the block in FP16
    fh_bytes = sum(esz * ((p["N"] - i + p["B"] - 1) // p["B"]) * n_landmarks((p["N"] - i + p["B"] - 1) // p["B"], p["s"])
                   * (iters + 1) for p in shapes for i in range(p["B"]))
    gr_flops = sum(2.0 * ((p["N"] - i + p["B"] - 1) // p["B"]) * n_landmarks((p["N"] - i + p["B"] - 1) // p["B"], p["s"])
                   * p["d"] for p in shapes for i in range(p["B"]))
    cands = {}
    if "fhat_multi" in prof:
        # the batch's inner loops as work lists: one launch per iteration round
        # streams the blocks of every loop in flight
        fm_bytes = sum(esz * ((p["N"] - i + p["B"] - 1) // p["B"])
                       * n_landmarks((p["N"] - i + p["B"] - 1) // p["B"], p["s"]) * iters
                       for p in shapes for i in range(p["B"]))
        n, tms = prof["fhat_multi"]
        ach = fm_bytes * args.steps / (tms / 1e3) / 1e9
        cands["fhat_multi"] = (tms, {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                     "frac": ach / peaks["hbm_gbs"], "traffic": None,
                                     "kernel": "fhat_partial_multi (one launch per round over every inner loop "
                                               "in flight)", "peak_source": peak_kind,
                                     "work_per_launch": f"{esz:.0f}*N_i*|L| B per loop in the round; "
                                                        f"{fm_bytes:.4g} B over the {n // args.steps} "
                                                        f"launches of a step",
                                     "timing": "CUDA events on the work-list stream around each launch"})
    elif "fhat_partial" in prof:
        n, tms = prof["fhat_partial"]
        ach = fh_bytes * args.steps / (tms / 1e3) / 1e9
        cands["fhat_partial"] = (tms, {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": "fhat_partial",
                                       "peak_source": peak_kind,
                                       "work_per_launch": f"{esz:.0f}*N_i*|L| B per launch; {fh_bytes:.4g} B over the "
                                                          f"{n // args.steps} launches of a step"})
    if "gram_block" in prof:
        n, tms = prof["gram_block"]
        ach = gr_flops * args.steps / (tms / 1e3) / 1e12
        pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        cands["gram_block"] = (tms, {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                                     "frac": ach / pk, "traffic": None, "kernel": "gram_block (tcgen05 BF16)",
                                     "peak_source": peak_kind + " bf16 sustained",
                                     "work_per_launch": f"2*N_i*|L|*d flop; {gr_flops:.4g} flop per step"})
    roof = max(cands.values(), key=lambda v: v[0])[1] if cands else None
    if roof:
        roof["note"] = ("launch durations are event-timed on their stream while the fits' other kernels run "
                        "beside them, so they include time shared with concurrent launches")

    pool = OraclePool()
    batched_oracle(shapes, data, cfg, BATCH_CPU_PROBLEMS, pool)   # warm-up
    ev, dt, desc = batched_oracle(shapes, data, cfg, BATCH_CPU_PROBLEMS, pool)
    pool.close()
    cpu = {"value": ev / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": desc}
    parity = batched_parity(kkm, shapes, data, cfg, BATCH_CPU_PROBLEMS, dev)
    h2d = int(sum(x.nbytes for x in data))
    out = {
        "metric": METRIC, "value": evals / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 products, f32 accumulation and sums, f64 cost", "data": "synthetic",
        "config": {"workload": cfg["name"], "problems": len(shapes), "sum_N": int(sum(p["N"] for p in shapes)),
                   "streams": args.streams or "library default",
                   "bandwidth": "median rule inside each fit",
                   "l2": f"inputs larger than L2 (X {h2d / 1e6:.0f} MB over the batch); no flush"},
        "iters_per_s": inner / (ms / 1e3),
        "fp32_path": {"value": evals / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32,
                      "iters_per_s": inner / (ms32 / 1e3)},
        "matched_labels": {"fraction_equal_to_fp32_path": agree, "omega_max_rel_diff": omega_rel},
        "oracle_parity": parity,
        "evals_per_step": evals,
        "e2e": {"value": evals / (e2e / 1e3), "unit": UNIT, "ms_per_step": e2e, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(4 * sum(p["N"] for p in shapes))},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    emit(out)


# ------------------------------------------------------------ serving loop
_SERVING_ORACLE = {}


def serving_oracle(cfg, seconds_cap):
    """The oracle on a bounded sample of the serving mix: a small RMSD model
    (3000 frames, C = 8, s = 0.05, 5 iterations) fitted by the oracle once
    (like the resident models, before the stream), then single assign
    requests of log-uniform size (capped at 200 frames) against it, each
    alone, for about `seconds_cap` of CPU time.  Returns (evals, s, desc)."""
    from oracle import kkm_oracle as O
    from synth import md_trajectory
    if "model" not in _SERVING_ORACLE:
        F, _ = md_trajectory(3000, cfg["n_atoms"], workload=4, problem=7)
        ker = O.Kernel(O.KIND_RMSD, cfg["sigma"], cfg["n_atoms"])
        _SERVING_ORACLE["model"] = O.fit(F.reshape(3000, -1).astype(np.float64), 8, 1, 0.05, ker, 5, 1,
                                         early_stop=False)
        _SERVING_ORACLE["queries"] = md_trajectory(4000, cfg["n_atoms"], workload=4, problem=8)[0]
        _SERVING_ORACLE["rng"] = np.random.default_rng(0)
    ref, Q, g = _SERVING_ORACLE["model"], _SERVING_ORACLE["queries"], _SERVING_ORACLE["rng"]
    ev, n_req = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds_cap:
        M = int(np.exp(g.uniform(0.0, np.log(200))))
        a = int(g.integers(0, 4000 - M))
        O.assign(ref, Q[a:a + M].reshape(M, -1).astype(np.float64), mode="supports")
        ev += M * len(ref["support_labels"])
        n_req += 1
    dt = time.perf_counter() - t0
    return ev, dt, (f"oracle RMSD model of 3000 frames (C=8, s=0.05, 5 iters; fitted once, untimed), then "
                    f"{n_req} assign requests of 1..200 frames against its {len(ref['support_labels'])} "
                    f"supports, each alone")


def run_serving(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        times, evs = [], []
        for k in range(args.warmup + args.steps):
            ev, dt, desc = serving_oracle(cfg, 1.0)
            if k >= args.warmup:
                times.append(dt)
                evs.append(ev)
        value = sum(evs) / sum(times)
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": cfg["name"], "sample": desc},
               "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return

    import torch
    from paper_1710_03013_gb300 import kkm
    from synth import batched_problems, blobs, md_trajectory

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    na = cfg["n_atoms"]
    t_setup = time.perf_counter()
    nmax = max(n for n, _ in cfg["models"])
    F, _ = md_trajectory(nmax, na, workload=4, problem=0)
    Fd = torch.from_numpy(F.reshape(nmax, -1)).cuda()
    del F
    Q, _ = md_trajectory(4 * cfg["max_query"], na, workload=4, problem=1)
    Q = Q.reshape(len(Q), -1)
    shapes = batched_problems(64, workload=4)
    fit_pool = [(p, blobs(p["N"], p["d"], p["C"], workload=4, problem=1000 + p["problem"])[0]) for p in shapes]
    srv = kkm.Server(budget_bytes=cfg["budget_gb"] << 30, n_workers=cfg["workers"])
    model_ids, n_sup = [], []
    fit_ms = []
    for n, C in cfg["models"]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, m = kkm.kkm_fit(Fd[:n], C, 1, cfg["model_s"], "rmsd", cfg["sigma"], na, iters=cfg["model_iters"],
                           seed=n + C, early_stop=False, labels=False)
        torch.cuda.synchronize()
        fit_ms.append(1e3 * (time.perf_counter() - t0))
        n_sup.append(m.info()["n_support"])
        model_ids.append(srv.add_model(m))
    del Fd
    torch.cuda.empty_cache()
    log(f"serving setup {time.perf_counter() - t_setup:.1f} s; model fits (ms): {fit_ms}")

    g = np.random.default_rng(1710)

    def arrivals(seconds):
        t, out = 0.0, []
        while True:
            t += g.exponential(1.0 / cfg["rate"])
            if t >= seconds:
                return out
            if g.random() < cfg["fit_share"]:
                p, X = fit_pool[int(g.integers(0, len(fit_pool)))]
                out.append((t, "fit", dict(X=X, C=p["C"], B=p["B"], s=p["s"], iters=20, seed=int(g.integers(1 << 30)),
                                           early_stop=False, precision=kkm.KKM_BF16)))
            else:
                M = int(np.exp(g.uniform(0.0, np.log(cfg["max_query"]))))
                a = int(g.integers(0, len(Q) - M))
                out.append((t, "assign", (model_ids[int(g.integers(0, len(model_ids)))], Q[a:a + M])))

    def play(seconds, prof=False):
        plan = arrivals(seconds)
        tickets = []
        h2d = 0
        t0 = time.perf_counter()
        for t, kind, job in plan:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            if kind == "fit":
                tickets.append(srv.submit_fit(job))
                h2d += job["X"].nbytes
            else:
                tickets.append(srv.submit_assign(job[0], job[1], "supports"))
                h2d += job[1].nbytes
        bad = 0
        for tk in tickets:
            st = srv.wait(tk)[0]
            bad += st != 0
        return time.perf_counter() - t0, len(plan), h2d, bad

    play(float(args.warmup))
    srv.reset_stats()
    with ClockSampler(local) as clk:
        time.sleep(0.3)  # the sampler's start-up before the stream
        clk.begin()
        wall, n_req, h2d, bad = play(float(args.steps))
        clk.end()
    st = srv.stats()
    # instrumented pass: every library launch counted
    kkm.prof_reset()
    kkm.prof_enable(2)
    wall_p, n_p, _, _ = play(3.0)
    kkm.prof_enable(False)
    launches_per_s = sum(v[0] for v in (kkm.prof_read(n) for n in kkm.prof_names())) / wall_p
    srv.close()
    # the dominant kernel of the mix: the RMSD block of an assign, timed alone
    # (largest query against the largest support set), every launch evented
    _, mbig = kkm.kkm_fit(torch.from_numpy(Q[:20000]).cuda(), 16, 1, 0.5, "rmsd", cfg["sigma"], na, iters=2,
                          seed=1, labels=False)
    Xq = torch.from_numpy(Q[20000:20000 + cfg["max_query"]]).cuda()
    nS = mbig.info()["n_support"]
    for _ in range(2):
        kkm.kkm_assign(mbig, Xq)
    kkm.prof_reset()
    kkm.prof_enable(1)
    for _ in range(3):
        kkm.kkm_assign(mbig, Xq)
    torch.cuda.synchronize()
    kkm.prof_enable(False)
    # the assign's MD block: a tensor-core screen of all pairs ("rmsd_gram"),
    # then the exact FP32 pass on the tiles it flagged ("rmsd_exact")
    n_s, t_s = kkm.prof_read("rmsd_gram")
    n_e, t_e = kkm.prof_read("rmsd_exact")
    pairs = kkm.prof_work("rmsd_exact") / max(n_e, 1)
    flops = 30.0 * na * pairs   # residual |R x - y|^2 at the screen's rotation: 15 FMA per atom
    ach = flops / (t_e / max(n_e, 1) / 1e3) / 1e12 if n_e else 0.0
    kp = 3 * (-(-na // 64) * 64)   # split-BF16 operands: three segments
    fl_s = 2.0 * 4 * cfg["max_query"] * 4 * nS * kp
    pk = measured_peaks()[0]
    pk = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    roof = {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / PEAK_FP32_TFLOPS, "traffic": None,
            "kernel": "rmsd_exact (assign of 10,000 frames against 10,000 supports: FP32 pass on flagged tiles)",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
            "work_per_launch": f"30*n_atoms flop per recomputed pair x {pairs:.4g} pairs = {flops:.4g} flop",
            "screen": {"kernel": "rmsd_gram (tcgen05 split-BF16 correlation screen)", "bound": "tensor",
                       "achieved": fl_s / (t_s / max(n_s, 1) / 1e3) / 1e12 if n_s else 0.0, "peak": pk,
                       "unit": "TFLOP/s",
                       "work_per_launch": f"2*(4 M)*(4 |S|)*{kp} = {fl_s:.4g} flop"}}
    roof["screen"]["frac"] = roof["screen"]["achieved"] / pk
    value = st["kernel_evals"] / wall
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 RMSD assigns; bf16 products, f32 sums for the fits", "data": "synthetic",
        "config": {"workload": cfg["name"], "step": "one second of the request stream",
                   "supports": n_sup, "workers": cfg["workers"], "model_fit_ms": fit_ms},
        "requests": n_req, "failed": bad + st["failed"],
        "latency_ms": {"assign_p50": st["p50_assign_ms"], "assign_p99": st["p99_assign_ms"],
                       "fit_p50": st["p50_fit_ms"], "fit_p99": st["p99_fit_ms"]},
        "completed": {"fit": st["completed_fit"], "assign": st["completed_assign"],
                      "fused_assign_launches": st["fused_assign_launches"]},
        "peak_budget_gb": st["peak_bytes"] / 2**30,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d / args.steps),
                "d2h_bytes_per_step": None,
                "note": "requests enter and leave through host memory; the serving value is end to end"},
        "gpu_launches": int(launches_per_s),
        "gpu_launches_unit": "per second of the stream",
        "roofline": roof,
        "clocks": clk.summary(),
    }
    ev, dt, desc = serving_oracle(cfg, 10.0)
    out["cpu_baseline"] = {"value": ev / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    emit(out)


# Where a workload's JSON line goes: printed, or collected when the default
# run nests the other configurations' lines in its own.
_SINK = None


def emit(out):
    if _SINK is not None:
        _SINK.append(out)
    else:
        print(json.dumps(out), flush=True)


def config_summary(out):
    """The fields of another configuration's bench line that the default line
    carries for it."""
    keep = ("metric", "value", "unit", "ms_per_step", "iters_per_s", "dtype", "config", "e2e", "gpu_launches",
            "matched_labels", "oracle_parity", "latency_ms", "cpu_baseline", "clocks", "fp32_path")
    d = {k: out[k] for k in keep if k in out}
    r = out.get("roofline")
    if r:
        d["roofline"] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "peak_source",
                                           "method_frac") if k in r}
        if "screen" in r:
            d["roofline"]["screen"] = {k: r["screen"][k] for k in ("kernel", "achieved", "peak", "frac",
                                                                    "method_frac") if k in r["screen"]}
    return d


def ctypes_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mnist", choices=sorted(WORKLOADS))
    ap.add_argument("--streams", type=int, default=0, help="batched workload: concurrent streams (0: default)")
    ap.add_argument("--problems", type=int, default=0,
                    help="batched workload: fit only its first N problems (a smaller case for profiling; 0: all)")
    ap.add_argument("--pipeline", default="auto", choices=["auto", "serial", "overlap"],
                    help="kernel-block scheduling of the fits (auto: next block overlapped when B >= 2)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: do not run and nest the MD, batched and serving configurations")
    args = ap.parse_args()
    cfg = dict(WORKLOADS[args.workload])
    cfg["key"] = args.workload
    if args.workload == "batched" and args.problems > 0:
        cfg["take"] = args.problems
        cfg["name"] = f"first {args.problems} problems of the " + cfg["name"]
    if args.workload == "serving":
        if args.impl == "ours":
            from paper_1710_03013_gb300 import build as _b
            _b.build()
        run_serving(args, cfg)
        return
    if args.workload == "batched":
        if args.impl == "ours":
            from paper_1710_03013_gb300 import build as _b
            _b.build()
        run_batched(args, cfg)
        return
    if cfg["kind"] == "rmsd":
        from synth import md_trajectory
        F, _ = md_trajectory(cfg["N"], cfg["n_atoms"])
        X = F.reshape(cfg["N"], -1)
    else:
        from synth import mnist_like
        X, _ = mnist_like(cfg["N"], cfg["d"])
    if args.impl == "reference":
        run_reference(args, cfg, X)
        return
    from paper_1710_03013_gb300 import build as _b
    _b.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload != "mnist" or world > 1 or args.no_configs:
        run_ours(args, cfg, X)
        return
    # the default run: the headline line, with the other configurations'
    # lines (short runs, each its own timed region) nested under "configs"
    global _SINK
    _SINK = []
    run_ours(args, cfg, X)
    head = _SINK[0]
    del X
    others = {}
    for name, steps, warmup in (("md", 2, 3), ("batched", 2, 3), ("serving", 1, 1)):
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.workload = steps, warmup, name
        c = dict(WORKLOADS[name])
        c["key"] = name
        _SINK = []
        try:
            if name == "serving":
                run_serving(sub, c)
            elif name == "batched":
                run_batched(sub, c)
            else:
                from synth import md_trajectory
                F, _ = md_trajectory(c["N"], c["n_atoms"])
                run_ours(sub, c, F.reshape(c["N"], -1))
                del F
            others[name] = config_summary(_SINK[-1]) if _SINK else {"error": "no result"}
            others[name]["steps"], others[name]["warmup"] = steps, warmup
        except Exception as e:  # one configuration failing leaves the headline line intact
            others[name] = {"error": f"{type(e).__name__}: {e}"}
    head["configs"] = others
    _SINK = None
    emit(head)


if __name__ == "__main__":
    main()

"""Benchmark: samples/s at fixed fidelity (Sec. II.A sampling from Sec. I.C's partial sum).

Default workload (grid5x8_m16): the 40-qubit 5x8 ABCD circuit, 16 cycles, 100k samples at
fidelity f = 1/64 (Alg. 1), batches of 2^6 bitstrings, alpha = 2.  The plan slices legs
until one slice's tensors fit 2^30 elements; its order search weights the batch steps by
the job's batch groups, and the sliced tree is re-optimised and annealed per slice (2000
moves) under that cap.  The sampling job (tn_job_*) splits the retained slices into
chunks; one chunk is contracted for every batch group of the job (its batch-independent
intermediates once, its batch part once per group of 4096 batches) and added to the
job's FP64 amplitude sums; a final pass runs the accept / pick step on every batch.

One step = one chunk of the job.  The job's chunks are identical in shape and work, so
the job time is the chunk count times the mean measured chunk time plus the measured
final pass: `value` = N / that time (samples/s of the whole job, projected from the
timed chunks; `config.projection` states it).  The working set (tens of GB per chunk)
exceeds L2 many times over, so no flush is needed between steps.  `e2e` times the same
job through the public API (job creation with the slice selection and the batch draws,
chunks, the final pass with host output) and projects it the same way.

Secondary lines (`secondary`): the 28-qubit 4x7 / 14-cycle workload at fidelity 1, one
step = one group of 16384 batches of one sampling job (the job's first group runs every
contraction, later groups reuse the batch-independent intermediates), in split bf16 and
in complex64 on the same plan recipe.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own job (replicas, weak
scaling); the timing is the max over ranks.
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
sys.path.insert(0, ROOT)

# sampling-job workloads (one step = one slice chunk of the job)
JOB_WORKLOADS = {
    # 40 qubits, 16 cycles, 1/64 of the slices, 100k samples (the largest single-GPU case)
    "grid5x8_m16": dict(rows=5, cols=8, cycles=16, seed=0, n_open=6, log2_batches=12, f=1.0 / 64, N=100000,
                        alpha=2.0, caps=(30, 29, 28, 27, 26), slice_bytes_max=140e9, budget=150e9, trials=256,
                        # per-slice annealing of the size-capped tree: 378.8 against 341.4 samples/s
                        # unannealed (8000 moves: 344.6, the model misprices small-K FFMA tiles)
                        anneal=2000),
}
# batch-group workloads (one step = one batch group of a sampling job over one slice set)
WORKLOADS = {
    # 28 qubits, 14 cycles, 2^10 slices, 16384 batches of 64 per step
    "grid4x7_m14": dict(rows=4, cols=7, cycles=14, seed=0, n_sliced=10, n_open=6, log2_batches=14),
    # a smaller case of the same kernels (24 qubits), for detailed profiler captures
    "grid4x6_m12": dict(rows=4, cols=6, cycles=12, seed=0, n_sliced=8, n_open=6, log2_batches=8),
}
METRIC = "samples/s at fixed fidelity"
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, bytes per launch) of a
# launch from one-pass ncu captures (profiles/), valid for the kernel source it was taken
# with (sha256 prefix of the named csrc file): (kernel, shape bits) -> (bytes, file, sha)
MEASURED_TRAFFIC = {
    # the 40-qubit job's batch step, from one capture of the same kernel on a case whose
    # arrays and tile counts are a quarter of (14,10,5,8) and half of (13,10,5,8) (the step
    # of the annealed plan): 3.458 GB, scaled by 4 and by 2
    ("tc_cgemm<128,3> stacked", (14, 10, 5, 8)): (13.83e9, "tc.cuh", "fd2822a0b959046e"),
    ("tc_cgemm<128,3> stacked", (13, 10, 5, 8)): (6.917e9, "tc.cuh", "fd2822a0b959046e"),
    # the default plan's batch step (2048 rows, no non-index batch bits): a quarter-size
    # capture, 1.642 GB, scaled by 4
    ("tc_cgemm<128,3> stacked", (12, 11, 5, 8)): (6.567e9, "tc.cuh", "fd2822a0b959046e"),
}
FFMA_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"
KERNEL_NAMES = {0: "cgemm_row", 1: "cgemm_small", 4: "cgemm_rowstage", 5: "cgemm_skinny"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid5x8_m16", choices=sorted(JOB_WORKLOADS) + sorted(WORKLOADS))
    ap.add_argument("--fidelity", type=float, default=None, help="target fidelity (default: the workload's)")
    ap.add_argument("--trials", type=int, default=256)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 28-qubit secondary lines")
    ap.add_argument("--precision", default="bf16x2", choices=["c64", "bf16x2"])
    ap.add_argument("--chunk", type=int, default=8, help="job workloads: at most this many slices per chunk (a power of two)")
    ap.add_argument("--log2-batches", type=int, default=None, help="batches per group = 2^this (default: the workload's)")
    ap.add_argument("--autotune", type=int, default=1, help="kernel autotuning (1) or the fixed shape rules (0)")
    ap.add_argument("--anneal", type=int, default=None,
                    help="simulated-annealing moves on the plan's tree (tn_plan_opts.anneal_iters); default: the "
                         "workload's (2000 for the 40-qubit job, where it is annealed per slice under the size cap)")
    ap.add_argument("--fuse-root", type=int, default=0,
                    help="1: run a row-kernel root step fused with the FP64 slice sum (tn_plan_opts.fuse_root_sum)")
    ap.add_argument("--serve", action="store_true", help="serving run (Poisson request stream) instead of the step bench")
    ap.add_argument("--serve-window", type=float, default=60.0, help="seconds of arrivals")
    ap.add_argument("--serve-rate", type=float, default=4.0, help="requests per second")
    a = ap.parse_args()
    if a.fidelity is None:
        a.fidelity = JOB_WORKLOADS[a.workload]["f"] if a.workload in JOB_WORKLOADS else 1.0
    if a.anneal is None:
        a.anneal = JOB_WORKLOADS[a.workload].get("anneal", 0) if a.workload in JOB_WORKLOADS else 0
    return a


def log2_batches(args):
    w = JOB_WORKLOADS.get(args.workload) or WORKLOADS[args.workload]
    return w["log2_batches"] if args.log2_batches is None else args.log2_batches


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ---------------------------------------------------------------- oracle baselines

def oracle_probs(circ):
    """The oracle's batch-independent part of a sampling job: the FP64 state vector of the
    whole circuit, as output probabilities."""
    import numpy as np
    import oracle
    psi = oracle.simulate(circ)
    p = np.abs(psi) ** 2
    del psi
    return p


def oracle_group(p, circ, openq, T, seed, t0, alpha=2.0):
    """The oracle on one batch group: the Sec. II.A step on T batches with the same Philox
    draws as the GPU path.  Returns the accepted count."""
    import numpy as np
    import oracle
    b_bits = circ.n_qubits - len(openq)
    js = oracle.batch_draws(seed, T, b_bits, t0=t0)
    pb = np.ascontiguousarray(oracle.batch_amplitudes(p, circ.n_qubits, openq, js))
    acc, _pick = oracle.sample_batches(pb, b_bits, alpha, seed, t0=t0)
    return int(acc.sum())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


SUB_ROWS = 3  # rows of the 40-qubit grid the oracle's bounded sample simulates


def oracle_job_sample(circ, openq, T, groups, N, seed, alpha=2.0):
    """One bounded sample of the oracle's work on a job too large for it.  The oracle (FP64
    state vector) needs 2^n complex128 amplitudes: 17.6 TB at 40 qubits, which no host
    here holds.  Its work is one pass over the vector per gate (then the sampler on the
    job's batches), so it is measured on the first SUB_ROWS rows of the same circuit (the
    gates acting there, the whole circuit's gate mix) and scaled by gates x amplitudes:
    t_job = (t_sub / (gates_sub 2^n_sub)) gates 2^n + t_sampler per batch x batches.
    Returns (job samples/s extrapolated, sample description, seconds spent)."""
    import oracle  # noqa: F401
    from paper_2112_15083_gb300 import circuits as cg
    n_sub = SUB_ROWS * circ.cols
    sub = cg.Circuit(n_qubits=n_sub, gates=[g for g in circ.gates if all(q < n_sub for q in g.qubits)])
    t0 = time.perf_counter()
    p = oracle_probs(sub)
    t_sv = time.perf_counter() - t0
    # the sampler on one group of T batches of the sub-circuit's 6 lowest qubits open
    sub_open = list(range(6))
    t1 = time.perf_counter()
    oracle_group(p, sub, sub_open, T, seed, 0, alpha)
    t_smp = time.perf_counter() - t1
    del p
    per_gate_amp = t_sv / (len(sub.gates) * 2.0 ** n_sub)
    t_job = per_gate_amp * len(circ.gates) * 2.0 ** circ.n_qubits + t_smp * groups
    desc = ("extrapolated: the FP64 state vector of %d qubits (%.1f TB) does not fit the host; the oracle simulated "
            "the circuit's first %d rows (%d qubits, %d of its %d gates) in %.2f s and sampled %d batches in %.2f s; "
            "job time = time per gate per amplitude x %d gates x 2^%d + sampler time x %d groups = %.3g s"
            % (circ.n_qubits, 16 * 2.0 ** circ.n_qubits / 1e12, SUB_ROWS, n_sub, len(sub.gates), len(circ.gates),
               t_sv, T, t_smp, len(circ.gates), circ.n_qubits, groups, t_job))
    return N / t_job, desc, time.perf_counter() - t0


def oracle_job_sample_child(workload, T, groups, threads):
    """oracle_job_sample in a child process with `threads` OpenMP threads (the thread count
    is read once per process); returns its samples/s."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; from paper_2112_15083_gb300 import circuits as cg; "
            "w = bench.JOB_WORKLOADS[%r]; c = cg.sycamore_grid(w['rows'], w['cols'], w['cycles'], seed=w['seed']); "
            "v, d, s = bench.oracle_job_sample(c, cg.default_open_qubits(w['rows'], w['cols'], w['n_open']), %d, %d, "
            "w['N'], 1, w['alpha']); print(json.dumps(v))" % (ROOT, workload, T, groups))
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None


def job_cpu_baseline(circ, openq, plan, info, w, workload):
    cores = cpu_cores()
    v, desc, _ = oracle_job_sample(circ, openq, info["T"], info["groups"], w["N"], 1, w["alpha"])
    v1 = oracle_job_sample_child(workload, info["T"], info["groups"], 1)
    return {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(), "sample": desc,
            "value_single_thread": v1}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2112_15083_gb300 import circuits as cg
    import oracle
    oracle.lib()
    cores = cpu_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    if args.workload in JOB_WORKLOADS:
        w = JOB_WORKLOADS[args.workload]
        circ = cg.sycamore_grid(w["rows"], w["cols"], w["cycles"], seed=w["seed"])
        openq = cg.default_open_qubits(w["rows"], w["cols"], w["n_open"])
        T = 1 << log2_batches(args)
        groups = job_groups_for(w["N"], w["alpha"], T)
        for _ in range(args.warmup):
            oracle_job_sample(circ, openq, T, groups, w["N"], args.seed, w["alpha"])
        vals, secs = [], 0.0
        for _ in range(args.steps):
            v, desc, s = oracle_job_sample(circ, openq, T, groups, w["N"], args.seed, w["alpha"])
            vals.append(v)
            secs += s
        val = statistics.median(vals)
        config = job_config(args, w)
        line = {
            "impl": "reference", "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": val, "unit": "samples/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": "median of %d bounded samples, each " % args.steps + desc},
            "e2e": {"value": val, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    w = WORKLOADS[args.workload]
    circ = cg.sycamore_grid(w["rows"], w["cols"], w["cycles"], seed=w["seed"])
    openq = cg.default_open_qubits(w["rows"], w["cols"], w["n_open"])
    T = 1 << log2_batches(args)
    # warm-up: a job of its own (state vector, then the warm-up groups)
    p = oracle_probs(circ)
    for i in range(args.warmup):
        oracle_group(p, circ, openq, T, args.seed, i * T)
    del p
    # the timed job: its state vector once, then its groups (as the GPU arm's job computes
    # its batch-independent intermediates once)
    t = time.perf_counter()
    p = oracle_probs(circ)
    acc = 0
    for k in range(args.steps):
        acc += oracle_group(p, circ, openq, T, args.seed, (args.warmup + k) * T)
    dt = time.perf_counter() - t
    val = acc / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": val, "unit": "samples/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "a job of %d groups: the FP64 state vector of the %d-qubit circuit once, then "
                                   "the sampler on %d batches per group" % (args.steps, circ.n_qubits, T)},
        "e2e": {"value": val, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our path

TC_VARIANTS = (9128, 9064, 9032, 19128, 19064)
STACKED_VARIANTS = (19128, 19064)  # one stack-list launch before each launch


def launches_per(s):
    """Kernel launches per launch of a traced step: its gather and stack-list launches."""
    return 1 + s["gathers"] + (1 if s["kernel"] in STACKED_VARIANTS else 0)


def kernel_name(k):
    if k in STACKED_VARIANTS:
        return "tc_cgemm<%d,%d> stacked" % (k - 19000, {19128: 3, 19064: 4}[k])
    if k in TC_VARIANTS:
        return "tc_cgemm<%d,%d>" % (k - 9000, {9128: 3, 9064: 4, 9032: 5}.get(k, 0))
    if k in KERNEL_NAMES:
        return KERNEL_NAMES[k]
    return "cgemm_tile<%d,%d>" % (k // 1000, k % 1000)


def roofline_of(trace, steps_traced, pk):
    """The roofline object of the dominant launch of a traced run (most device time),
    from CUDA events around every contraction launch: tensor-core steps against the
    measured bf16 dense peak (algorithmic FLOPs, 8 per complex MAC), HBM-bound short
    products against the measured copy bandwidth (algorithmic bytes: operands read and
    result written at complex64), FFMA tiles against the derived FP32 peak."""
    dom = max(trace, key=lambda s: s["ms"])
    dom_ms = dom["ms"] / max(1, dom["launches"])
    alg = dom["flops_per_launch"] / (dom_ms / 1e3) / 1e12
    shape = "(bat,m,n,k bits = %d,%d,%d,%d)" % (dom["nbat"], dom["nm"], dom["nn"], dom["nk"])
    k = dom["kernel"]
    if k in TC_VARIANTS:
        # the split path issues 3x the algorithmic products on the tensor pipe; the bound is
        # the roofline whose time at peak is longer: the pipe's products at the bf16 peak or
        # the launch's compulsory bytes at the copy bandwidth
        peak = pk.get("bf16_tflops", 1900.0)
        hbm = pk.get("hbm_gbs", 6800.0)
        gbs = dom["bytes_per_launch"] / (dom_ms / 1e3) / 1e9
        t_tensor = 3 * dom["flops_per_launch"] / (peak * 1e12)
        t_hbm = dom["bytes_per_launch"] / (hbm * 1e9)
        tc_src = ("measured bf16 dense burst (MEASURED_PEAKS.json)" if "bf16_tflops" in pk else "fallback 1.9 PFLOP/s")
        if t_hbm > t_tensor:
            roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "traffic": None, "frac": gbs / hbm,
                    "peak_source": "measured HBM copy (MEASURED_PEAKS.json)" if "hbm_gbs" in pk else "fallback 6.8 TB/s",
                    "tensor_pipe_tflops": 3 * alg, "tensor_pipe_frac": 3 * alg / peak, "tensor_peak_source": tc_src,
                    "why_hbm": "its compulsory bytes at the copy bandwidth (%.2f ms) outlast its tensor-pipe products "
                               "at the bf16 peak (%.2f ms)" % (1e3 * t_hbm, 1e3 * t_tensor)}
        else:
            roof = {"bound": "tensor", "achieved": alg, "peak": peak, "unit": "TFLOP/s", "traffic": None,
                    "frac": alg / peak, "tensor_pipe_tflops": 3 * alg, "tensor_pipe_frac": 3 * alg / peak,
                    "peak_source": tc_src, "hbm_gbs_achieved": gbs}
        roof["kernel"] = "%s split bf16 hi+lo %s" % (kernel_name(k), shape)
    elif k in KERNEL_NAMES:
        gbs = dom["bytes_per_launch"] / (dom_ms / 1e3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "traffic": None, "frac": gbs / peak,
                "peak_source": "measured HBM copy (MEASURED_PEAKS.json)" if "hbm_gbs" in pk else "fallback 6.8 TB/s",
                "kernel": "%s %s%s" % (kernel_name(k), shape, " after a batch-gather launch" if dom["gathers"] else "")}
    else:
        ffma_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        roof = {"bound": "alu", "achieved": alg, "peak": ffma_peak, "unit": "TFLOP/s", "traffic": None,
                "frac": alg / ffma_peak, "peak_source": "derived: " + FFMA_PEAK_NOTE + " (FP32 FFMA, complex64 path)",
                "kernel": "%s %s" % (kernel_name(k), shape)}
    roof["share_of_step"] = dom["ms"] / max(1e-9, sum(s["ms"] for s in trace))
    fam = {}
    for x in trace:
        name = kernel_name(x["kernel"]).split("<")[0]
        fam[name] = fam.get(name, 0.0) + x["ms"] / steps_traced
    roof["kernel_family_ms_per_step"] = {n: round(v, 2) for n, v in sorted(fam.items(), key=lambda kv: -kv[1])}
    rec = MEASURED_TRAFFIC.get((kernel_name(k), (dom["nbat"], dom["nm"], dom["nn"], dom["nk"])))
    if rec:
        import hashlib
        src = os.path.join(ROOT, "paper_2112_15083_gb300", "csrc", rec[1])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec[2]:
            roof["traffic"] = rec[0]
            roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of a smaller case of the "
                                      "same kernel, scaled by the ratio of their arrays and tiles "
                                      "(profiles/tc_cgemm_stacked_*.md)")
    return roof


def top_steps_of(trace, n=6):
    out = []
    for s in sorted(trace, key=lambda s: -s["ms"])[:n]:
        ms1 = s["ms"] / max(1, s["launches"])
        out.append({"shape_bits": [s["nbat"], s["nm"], s["nn"], s["nk"]], "kernel": kernel_name(s["kernel"]),
                    "ms": round(ms1, 3), "launches": s["launches"],
                    "tflops": round(s["flops_per_launch"] / (ms1 / 1e3) / 1e12, 2),
                    "gbs": round(s["bytes_per_launch"] / (ms1 / 1e3) / 1e9, 1), "gathers": s["gathers"]})
    return out


def split_trace(trace):
    """(contraction steps with launches, slice-sum entries): the last trace entry is the
    FP64 slice sum (kernel 2, or 3 when it runs fused with the root step)."""
    ssum = [s for s in trace if s["kernel"] in (2, 3)]
    steps = [s for s in trace if s["kernel"] not in (2, 3) and s["launches"] > 0]
    return steps, ssum


def slice_sum_of(ssum):
    if not ssum or not ssum[0]["launches"]:
        return None
    s0 = ssum[0]
    ms1 = s0["ms"] / s0["launches"]
    return {"ms": round(ms1, 3), "fp64_gflops": round(s0["flops_per_launch"] / (ms1 / 1e3) / 1e9, 1),
            "gbs": round(s0["bytes_per_launch"] / (ms1 / 1e3) / 1e9, 1), "fused_root_step": s0["kernel"] == 3}


def workload_config(args):
    w = WORKLOADS[args.workload]
    q = w["rows"] * w["cols"]
    return {"workload": "%s: %d-qubit %dx%d Sycamore-style ABCD circuit, %d cycles, fSim(pi/2,pi/6); "
                        "%d sliced legs (%d slices); %d batches of 64 bitstrings per step" % (
                            args.workload, q, w["rows"], w["cols"], w["cycles"], w["n_sliced"], 1 << w["n_sliced"],
                            1 << log2_batches(args)),
            "qubits": q, "cycles": w["cycles"], "sliced_legs": w["n_sliced"], "batches_per_step": 1 << log2_batches(args),
            "batch_size": 64, "fidelity_target": args.fidelity, "alpha": 2.0, "order_trials": args.trials,
            "precision": getattr(args, "precision", "c64"), "fuse_root_sum": bool(getattr(args, "fuse_root", 0)),
            "anneal_iters": int(getattr(args, "anneal", 0)),
            "job": "the timed steps are the batch groups of one sampling job over one slice set",
            "l2": "flushed between timed steps; dominant operands exceed L2"}


def run_group(args, with_e2e=True, with_cpu=True):
    """One sampling job of `steps` batch groups over one slice set (the job's first group
    runs every contraction, later groups reuse the batch-independent intermediates); the
    JSON line as a dict (rank 0) or None."""
    import numpy as np
    import torch
    import paper_2112_15083_gb300 as P
    from paper_2112_15083_gb300 import circuits as cg
    from paper_2112_15083_gb300 import replicas
    rank, world, local = dist_env()
    w = WORKLOADS[args.workload]
    circ = cg.sycamore_grid(w["rows"], w["cols"], w["cycles"], seed=w["seed"])
    openq = cg.default_open_qubits(w["rows"], w["cols"], w["n_open"])
    C = P.circuit_load(circ.serialize())
    prec = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[args.precision]
    plan = P.plan(C, openq, n_auto_sliced=w["n_sliced"], log2_batches=log2_batches(args), order_trials=args.trials,
                  order_seed=0, hbm_budget_bytes=200e9, precision=prec, autotune=args.autotune,
                  fuse_root_sum=bool(args.fuse_root), anneal_iters=args.anneal)
    info = plan.info()
    slices, F = plan.select(args.fidelity)
    T = 1 << log2_batches(args)
    dev = torch.device("cuda", local)
    acc = [torch.empty(T, dtype=torch.uint8, device=dev) for _ in range(args.steps)]
    bits = [torch.empty(T, dtype=torch.int64, device=dev) for _ in range(args.steps)]
    acc2 = [torch.empty(T, dtype=torch.uint8, device=dev) for _ in range(args.steps)]
    bits2 = [torch.empty(T, dtype=torch.int64, device=dev) for _ in range(args.steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    base_t = replicas.batch_t0(rank, 0, T)
    seed = args.seed
    # warm-up: two full groups (the first tunes the kernels, the second captures the full
    # group's CUDA graph), then groups that reuse the stem (capturing that graph)
    for i in range(args.warmup):
        plan.sample_step(slices, F, seed, base_t + i * T, reuse_stem=i >= 2, accept=acc[0], bits=bits[0])
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # timed region: one sampling job of `steps` batch groups over one slice set, each group
    # one CUDA-graph replay of the contraction plus the draw and sampler launches, L2
    # flushed in between; warm-up leaves nothing the first timed group uses
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record()
        plan.sample_step(slices, F, seed, base_t + (args.warmup + k) * T, reuse_stem=k > 0, accept=acc[k], bits=bits[k])
        ev1[k].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    tot_ms = sum(ev0[k].elapsed_time(ev1[k]) for k in range(args.steps))
    # the same number of groups, each on its own (the stem recomputed in every group)
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record()
        plan.sample_step(slices, F, seed, base_t + (args.warmup + args.steps + k) * T, accept=acc2[k], bits=bits2[k])
        ev1[k].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    solo_ms = sum(ev0[k].elapsed_time(ev1[k]) for k in range(args.steps))
    # traced region (the job again, CUDA events around every contraction launch)
    plan.trace(True)
    acc_t = torch.empty(T, dtype=torch.uint8, device=dev)
    bits_t = torch.empty(T, dtype=torch.int64, device=dev)
    for k in range(args.steps):
        flush.zero_()
        plan.sample_step(slices, F, seed, base_t + (args.warmup + k) * T, reuse_stem=k > 0, accept=acc_t, bits=bits_t)
    trace = plan.trace_read()
    plan.trace(False)
    accepted = int(sum(int(a.sum().item()) for a in acc))
    tot_ms_max, accepted_all = replicas.reduce_run(tot_ms, accepted, device=dev)
    value = accepted_all / (tot_ms_max / 1e3)
    accepted2 = int(sum(int(a.sum().item()) for a in acc2))
    solo_ms_max, accepted2_all = replicas.reduce_run(solo_ms, accepted2, device=dev)
    value_solo = accepted2_all / (solo_ms_max / 1e3)
    flops_group = sum(s["flops_per_launch"] for s in trace if s["kernel"] not in (2, 3))
    steps_tr, ssum = split_trace(trace)
    flops_step = sum(s["flops_per_launch"] * s["launches"] for s in steps_tr) / args.steps
    roofline = roofline_of(steps_tr, args.steps, peaks())
    roofline["measured"] = "CUDA events around each contraction launch over %d traced steps" % args.steps

    e2e = None
    if rank == 0 and with_e2e:
        # the same job as one tn_sample call (selection included) with host output, about
        # one group's expected samples (T (1 - eps) / alpha) per step
        n_job = int(0.47 * T) * args.steps
        torch.cuda.synchronize()
        t = time.perf_counter()
        b, st = plan.sample(args.fidelity, n_job, seed=seed + 1)
        dt = time.perf_counter() - t
        groups = (st["steps"] + T - 1) // T
        e2e = {"value": len(b) / dt, "unit": "samples/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int((groups * T * (1 + 8 + 8) + n_job * 8) / args.steps),
               "api": "tn_sample(host bitstrings): one call for the job's %d samples" % n_job, "groups": groups}

    cpu = None
    if rank == 0 and world == 1 and with_cpu and not args.no_cpu_baseline:
        cpu = group_cpu_baseline(circ, openq, T, seed, args.steps)

    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("bf16x2 split hi+lo on tcgen05, fp32 accumulation (small steps c64 FFMA); fp64 slice sum/sampler"
                  if args.precision == "bf16x2" else "c64 (fp32 FFMA), fp64 slice sum/sampler"),
        "data": "synthetic", "config": workload_config(args),
        "fidelity": F, "contraction_tflops": flops_step * args.steps / (tot_ms / 1e3) / 1e12,
        "flops_per_step": flops_step, "flops_per_group_with_stem": flops_group,
        "stem": "the job's first group runs every contraction; its later groups reuse the batch-independent "
                "intermediates (tn_sample_step reuse_stem)",
        "value_stem_each_step": value_solo, "ms_per_step_stem_each_step": solo_ms_max / args.steps,
        "plan": info, "clocks": clk, "roofline": roofline,
        "cpu_baseline": cpu, "e2e": e2e, "top_steps": top_steps_of(steps_tr), "slice_sum": slice_sum_of(ssum),
        # the job's contraction launches, batch gathers and slice sums, plus a batch draw and
        # a sampler launch per step
        "gpu_launches": (sum(s["launches"] * launches_per(s) for s in steps_tr)
                         + sum(s["launches"] for s in ssum) + 2 * args.steps),
    }


def group_cpu_baseline(circ, openq, T, seed, groups):
    """The oracle on the same job (its state vector once, then the sampler on `groups`
    groups of T batches), on all host cores, and the state vector single-threaded."""
    cores = cpu_cores()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    t = time.perf_counter()
    p = oracle_probs(circ)
    a = sum(oracle_group(p, circ, openq, T, seed, g * T) for g in range(groups))
    del p
    dt = time.perf_counter() - t
    return {"value": a / dt, "unit": "samples/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": "a job of %d groups: the FP64 state vector of the %d-qubit circuit once, then the sampler on %d "
                      "batches per group (%d accepted in %.1f s)" % (groups, circ.n_qubits, T, a, dt)}


def job_groups_for(N, alpha, T):
    """The job's batch groups (as tn_job_create draws them)."""
    need = 1.1 * alpha * N + 8.0 * math.sqrt(alpha * N) + 64.0
    return max(1, math.ceil(need / T))


def plan_job_workload(args, P, C, openq, w, precision):
    """The largest tensor cap whose one-slice working set fits, with the order search
    weighting the batch steps by the job's groups."""
    import numpy as np
    T = 1 << log2_batches(args)
    groups = job_groups_for(w["N"], w["alpha"], T)
    plan = None
    for cap in w["caps"]:
        plan = P.plan(C, openq, log2_batches=log2_batches(args), order_trials=args.trials, order_seed=0,
                      max_log2_tensor=cap, hbm_budget_bytes=w["budget"], precision=precision, autotune=args.autotune,
                      max_norm_flops=3e16, job_groups=groups, anneal_iters=args.anneal)
        if plan.estimate(np.zeros(1, np.uint64))[0] <= w["slice_bytes_max"]:
            break
    return plan, cap, groups


def job_config(args, w):
    """The workload of a job line (identical in both arms); plan-dependent figures go to
    the line's `job` object."""
    q = w["rows"] * w["cols"]
    T = 1 << log2_batches(args)
    return {"workload": "%s: %d-qubit %dx%d Sycamore-style ABCD circuit, %d cycles, fSim(pi/2,pi/6); %d samples at "
                        "fidelity %g (Alg. 1 slice selection); batches of 64 bitstrings, %d per group" % (
                            args.workload, q, w["rows"], w["cols"], w["cycles"], w["N"], args.fidelity, T),
            "qubits": q, "cycles": w["cycles"], "samples": w["N"], "fidelity_target": args.fidelity,
            "alpha": w["alpha"], "batch_size": 64, "batches_per_group": T, "order_trials": args.trials,
            "precision": args.precision, "chunk_slices": args.chunk, "anneal_iters": int(args.anneal),
            "step": "one slice chunk of the job contracted for all of its batch groups (batch-independent "
                    "intermediates once) and added to its FP64 amplitude sums",
            "projection": "value = samples / (chunks x mean timed chunk + the final accept/pick pass); the job's "
                          "chunks are identical in shape and work",
            "l2": "not flushed: every chunk's working set (tens of GB) exceeds L2"}


def run_job(args):
    import numpy as np
    import torch
    import paper_2112_15083_gb300 as P
    from paper_2112_15083_gb300 import circuits as cg
    from paper_2112_15083_gb300 import replicas
    rank, world, local = dist_env()
    w = JOB_WORKLOADS[args.workload]
    N, alpha = w["N"], w["alpha"]
    circ = cg.sycamore_grid(w["rows"], w["cols"], w["cycles"], seed=w["seed"])
    openq = cg.default_open_qubits(w["rows"], w["cols"], w["n_open"])
    C = P.circuit_load(circ.serialize())
    prec = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[args.precision]
    t = time.perf_counter()
    plan, cap, _ = plan_job_workload(args, P, C, openq, w, prec)
    plan_s = time.perf_counter() - t
    plan_info = plan.info()
    seed = args.seed + rank  # replicas: independent Philox keys
    t = time.perf_counter()
    job = plan.job(args.fidelity, N, seed, alpha=alpha, max_chunk_slices=args.chunk)
    create_s = time.perf_counter() - t
    info = job.info()
    need = args.warmup + args.steps + 1
    if info["n_chunks"] < need:
        raise SystemExit("the job has %d chunks; warm-up + steps + a traced chunk need %d" % (info["n_chunks"], need))
    # warm-up: the first chunks of the job (kernel autotuning, graph capture)
    for c in range(args.warmup):
        job.run(c, 1)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # timed region: the next `steps` chunks of the job, each contracted for every batch
    # group and added to the job's amplitude sums (CUDA events on the plan's stream)
    for k in range(args.steps):
        ev0[k].record()
        job.run(args.warmup + k, 1)
        ev1[k].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    chunk_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    tot_ms = sum(chunk_ms)
    # the job's final pass (accept / pick over every batch, host output)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _bits, st = job.finish(partial=True)
    finish_s = time.perf_counter() - t
    # one more chunk traced (CUDA events around every launch): per-launch device times
    plan.trace(True)
    job.run(args.warmup + args.steps, 1)
    trace = plan.trace_read()
    plan.trace(False)
    steps_tr, ssum = split_trace(trace)
    # launch gaps: the graph-replayed chunk against the sum of its launches' device times
    # (the traced chunk runs the same launches one by one, CUDA events around each); the
    # difference also holds the per-group pattern copies and FP64 accumulations
    launches_ms = sum(s["ms"] for s in steps_tr) + sum(s["ms"] for s in ssum)
    gaps = {"chunk_ms_replayed": round(tot_ms / args.steps, 2), "launch_device_ms_sum": round(launches_ms, 2),
            "outside_traced_launches_ms": round(tot_ms / args.steps - launches_ms, 2)}
    job_s = info["n_chunks"] * (tot_ms / args.steps) / 1e3 + finish_s
    job_s_max, n_all = replicas.reduce_run(job_s * 1e3, N, device=torch.device("cuda", local))
    value = n_all / (job_s_max / 1e3)
    roofline = roofline_of(steps_tr, 1, peaks())
    roofline["measured"] = "CUDA events around each launch of one traced chunk (%d groups)" % info["groups"]
    del job

    e2e = None
    if rank == 0:
        # the same job through the public API with host output: creation (slice selection,
        # batch draws), chunks, the final pass; projected to all chunks as `value`
        ke = max(2, args.steps // 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        job2 = plan.job(args.fidelity, N, seed + 7919, alpha=alpha, max_chunk_slices=args.chunk)
        t1 = time.perf_counter()
        job2.run(0, ke)
        t2 = time.perf_counter()
        job2.finish(partial=True)
        t3 = time.perf_counter()
        inf2 = job2.info()
        del job2
        e2e_s = (t1 - t0) + inf2["n_chunks"] * (t2 - t1) / ke + (t3 - t2)
        nb = inf2["groups"] * inf2["T"]
        e2e = {"value": N / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int((nb * (1 + 8 + 8) + N * 8) / inf2["n_chunks"]),
               "api": "tn_job_create + tn_job_run + tn_job_finish (host bitstrings), the calls tn_sample makes; "
                      "%d chunks timed, projected to the job's %d" % (ke, inf2["n_chunks"]),
               "create_s": round(t1 - t0, 3), "chunk_s": round((t2 - t1) / ke, 4), "finish_s": round(t3 - t2, 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = job_cpu_baseline(circ, openq, plan, info, w, args.workload)

    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary:
        secondary = secondary_lines(args)

    if rank != 0:
        return None
    per_chunk_launches = (sum(s["launches"] * launches_per(s) for s in steps_tr) + sum(s["launches"] for s in ssum)
                          + info["groups"])
    return {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("bf16x2 split hi+lo on tcgen05, fp32 accumulation (small steps c64 FFMA); fp64 slice and chunk "
                  "sums, fp64 sampler" if args.precision == "bf16x2" else "c64 (fp32 FFMA); fp64 sums and sampler"),
        "data": "synthetic", "config": job_config(args, w),
        "job": {"sliced_legs": plan_info["n_sliced"], "max_log2_tensor_cap": cap, "retained_slices": info["n_slices"],
                "chunk_slices": info["chunk_slices"], "chunks": info["n_chunks"], "groups": info["groups"],
                "batches": info["groups"] * info["T"]},
        "fidelity": info["F"], "job_seconds": job_s, "job_hours": job_s / 3600.0,
        "chunk_ms": [round(x, 2) for x in chunk_ms], "finish_s": finish_s,
        "contraction_tflops": info["flops_chunk"] / (tot_ms / args.steps / 1e3) / 1e12,
        "flops_per_chunk": info["flops_chunk"], "plan_seconds": plan_s, "job_create_seconds": create_s,
        "eps_hat_partial": st["eps_hat"], "plan": plan_info, "clocks": clk, "roofline": roofline,
        "cpu_baseline": cpu, "e2e": e2e, "top_steps": top_steps_of(steps_tr, 8), "slice_sum": slice_sum_of(ssum),
        "secondary": secondary, "launch_gaps": gaps,
        # per chunk: every contraction launch, its gathers and slice sums, one amplitude
        # accumulation per group (counted from the traced chunk)
        "gpu_launches": per_chunk_launches * args.steps,
    }


def secondary_lines(args):
    """The 28-qubit workload at fidelity 1 in split bf16 and complex64 (same plan recipe)."""
    out = {}
    for prec in ("bf16x2", "c64"):
        a = argparse.Namespace(**vars(args))
        a.workload, a.precision, a.fidelity, a.steps, a.warmup = "grid4x7_m14", prec, 1.0, 5, 3
        a.log2_batches, a.fuse_root, a.anneal = None, 0, 0
        line = run_group(a, with_e2e=False, with_cpu=False)
        out["grid4x7_m14_" + prec] = {
            "value": line["value"], "ms_per_step": line["ms_per_step"], "steps": a.steps, "fidelity": line["fidelity"],
            "value_stem_each_step": line["value_stem_each_step"],
            "roofline": {k: line["roofline"][k] for k in ("kernel", "bound", "achieved", "unit", "frac")},
            "top_steps": line["top_steps"][:3]}
    out["split_over_c64"] = out["grid4x7_m14_bf16x2"]["value"] / out["grid4x7_m14_c64"]["value"]
    return out


def run_ours(args):
    import torch
    import __graft_entry__
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()
    line = run_job(args) if args.workload in JOB_WORKLOADS else run_group(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()



# ---------------------------------------------------------------- serving

SERVE_GRIDS = [(4, 5), (4, 6), (5, 5), (4, 7), (5, 6), (4, 8), (5, 7), (6, 6), (4, 9), (4, 10), (5, 8)]


def run_serve(args):
    """Serving run: Poisson arrivals at --serve-rate for --serve-window seconds, circuits
    drawn uniformly from 20-40-qubit grids and 8-16 cycles, N in {1k, 10k, 100k}, f in
    {1, 0.1, 0.01, 0.002}, half bf16 x2 / half complex64; 150 GB admission budget."""
    import math
    import numpy as np
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_2112_15083_gb300 as P
    from paper_2112_15083_gb300 import circuits as cg
    rng = np.random.default_rng(0)
    srv = P.Server(hbm_budget_bytes=150e9, max_active=8, planner_threads=12, order_trials=16,
                   max_request_seconds=30.0, assumed_flops=3e14, assumed_flops_c64=2.5e13)
    t0 = time.perf_counter()
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / args.serve_rate)
        if t > args.serve_window:
            break
        r, c = SERVE_GRIDS[rng.integers(len(SERVE_GRIDS))]
        cycles = int(rng.integers(8, 17))
        N = int(rng.choice([1000, 10000, 100000]))
        f = float(rng.choice([1.0, 0.1, 0.01, 0.002]))
        prec = P.tn.PREC_BF16X2 if rng.random() < 0.5 else P.tn.PREC_C64
        k0 = 0 if f >= 1 else int(math.ceil(3 - math.log2(f)))
        circ = cg.sycamore_grid(r, c, cycles, seed=int(rng.integers(1 << 30)))
        delay = t - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        rid = srv.submit(circ.serialize(), cg.default_open_qubits(r, c, 6), N=N, f=f, seed=len(reqs),
                         precision=prec, n_sliced=max(2, k0 + 2))
        reqs.append(dict(id=rid, qubits=r * c, cycles=cycles, N=N, f=f, prec=prec))
    print("serve: %d requests submitted in %.1f s" % (len(reqs), time.perf_counter() - t0), file=sys.stderr, flush=True)
    max_queue = 0
    infos = []
    deadline = t0 + args.serve_window + 600.0
    for q in reqs:
        st = srv.stats()
        max_queue = max(max_queue, st["queued"] + st["planning"] + st["planned"])
        left = max(1.0, deadline - time.perf_counter())
        _, info = srv.wait(q["id"], q["N"], timeout=left)
        infos.append(dict(q, **info))
        if len(infos) % 20 == 0:
            print("serve: %d/%d finished, %.1f s" % (len(infos), len(reqs), time.perf_counter() - t0), file=sys.stderr,
                  flush=True)
    makespan = time.perf_counter() - t0
    srv.close()
    done = [i for i in infos if i["status"] == "done"]

    def pct(xs, p):
        return float(np.percentile(xs, p)) if xs else None

    classes = {}
    for N in (1000, 10000, 100000):
        lat = [i["t_done"] - i["t_submit"] for i in done if i["N"] == N]
        classes["N=%d" % N] = {"done": len(lat), "p50_s": pct(lat, 50), "p99_s": pct(lat, 99)}
    for f in (1.0, 0.1, 0.01, 0.002):
        lat = [i["t_done"] - i["t_submit"] for i in done if i["f"] == f]
        classes["f=%g" % f] = {"done": len(lat), "p50_s": pct(lat, 50), "p99_s": pct(lat, 99)}
    lat_all = [i["t_done"] - i["t_submit"] for i in done]
    waits = [i["t_admit"] - i["t_submit"] for i in done]
    runs = [i["t_done"] - i["t_admit"] for i in done]
    samples = sum(i["N"] for i in done)
    slowest = sorted(done, key=lambda i: -(i["t_done"] - i["t_admit"]))[:5]
    line = {"metric": "serving: p50/p99 latency and samples/s", "value": samples / makespan, "unit": "samples/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "Poisson %.1f req/s for %.0f s; grids %s; cycles 8-16; N in 1k/10k/100k; "
                                   "f in 1/0.1/0.01/0.002; bf16x2 or c64 (50/50); 150 GB budget" % (
                                       args.serve_rate, args.serve_window, SERVE_GRIDS)},
            "requests": len(infos), "done": len(done),
            "rejected": sum(1 for i in infos if i["status"] == "rejected"),
            "failed": sum(1 for i in infos if i["status"] == "failed"),
            "unfinished": sum(1 for i in infos if i["status"] not in ("done", "failed", "rejected")),
            "p50_s": pct(lat_all, 50), "p99_s": pct(lat_all, 99), "classes": classes,
            "wait_p50_s": pct(waits, 50), "run_p50_s": pct(runs, 50), "run_p99_s": pct(runs, 99),
            "slowest_runs": [{"qubits": i["qubits"], "cycles": i["cycles"], "N": i["N"], "f": i["f"],
                              "precision": "bf16x2" if i["prec"] == P.tn.PREC_BF16X2 else "c64",
                              "run_s": round(i["t_done"] - i["t_admit"], 2), "gflop": round(i["flops"] / 1e9, 1)}
                             for i in slowest],
            "max_waiting": max_queue, "makespan_s": makespan}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serve:
        run_serve(a)
    else:
        run_ours(a)

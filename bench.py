"""Benchmark: samples/s at fixed fidelity on the 4x7-grid / 14-cycle workload.

One step = one pass of the sampling hot path over one group of T = 16384 batches of
2^6 amplitudes: Philox batch draws, every pairwise contraction of the sliced network
over the slice set (2^10 slices at fidelity 1) with the batch gathers, the FP64 slice
sum, p = |a|^2 / F and the warp rejection sampler.  Every step recomputes every tensor,
the batch-independent ones included (nothing is carried between steps).
Intermediates exceed L2 (the dominant operands are GiB-sized) and L2 is also flushed
between timed steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs independent batch
groups (replicas, weak scaling); the timing is the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the measured workload: 28 qubits, 14 cycles, 2^10 slices, 16384 batches of 64 per step
    "grid4x7_m14": dict(rows=4, cols=7, cycles=14, seed=0, n_sliced=10, n_open=6, log2_batches=14),
    # a smaller case of the same kernels (24 qubits), for detailed profiler captures
    "grid4x6_m12": dict(rows=4, cols=6, cycles=12, seed=0, n_sliced=8, n_open=6, log2_batches=8),
}
WORKLOAD = WORKLOADS["grid4x7_m14"]
METRIC = "samples/s at fixed fidelity"
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, bytes per launch) of the
# dominant launch from one-pass ncu captures of this workload (profiles/*_dram_grid4x7_m14_b16384.md),
# valid for the kernel source it was taken with (sha256 prefix of the named csrc file)
MEASURED_TRAFFIC = {
    ("tc_cgemm<128,3>", (1, 15, 14, 12)): (83.75e9, "tc.cuh", "cbda2ea2f13a3e53"),
    ("cgemm_row", (23, 2, 5, 2)): (16.95e9, "kernels.cuh", "e2dc3ed40cd00353"),
}
FFMA_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fidelity", type=float, default=1.0)
    ap.add_argument("--trials", type=int, default=256)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="bf16x2", choices=["c64", "bf16x2"])
    ap.add_argument("--workload", default="grid4x7_m14", choices=sorted(WORKLOADS))
    ap.add_argument("--log2-batches", type=int, default=None, help="batches per step = 2^this (default: the workload's)")
    ap.add_argument("--autotune", type=int, default=1, help="kernel autotuning (1) or the fixed shape rules (0)")
    ap.add_argument("--anneal", type=int, default=0,
                    help="order search: simulated-annealing moves on the winning tree (tn_plan_opts.anneal_iters)")
    ap.add_argument("--fuse-root", type=int, default=0,
                    help="1: run a row-kernel root step fused with the FP64 slice sum (tn_plan_opts.fuse_root_sum)")
    ap.add_argument("--serve", action="store_true", help="serving run (Poisson request stream) instead of the step bench")
    ap.add_argument("--grid5x8-sample", action="store_true",
                    help="bounded sample of the 40-qubit 5x8 / 16-cycle configuration (time per slice, extrapolated)")
    ap.add_argument("--serve-window", type=float, default=60.0, help="seconds of arrivals")
    ap.add_argument("--serve-rate", type=float, default=4.0, help="requests per second")
    return ap.parse_args()


def log2_batches(args):
    w = WORKLOADS[args.workload]
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


# ---------------------------------------------------------------- oracle baseline

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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2112_15083_gb300 import circuits as cg
    import oracle
    oracle.lib()
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
    cores = cpu_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": val, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": "a job of %d groups: the FP64 state vector of the %d-qubit circuit once, then "
                                   "the sampler on %d batches per group" % (args.steps, circ.n_qubits, T)},
        "e2e": {"value": val, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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


# ---------------------------------------------------------------- our path

def run_ours(args):
    import numpy as np
    import torch
    import __graft_entry__
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()
    import paper_2112_15083_gb300 as P
    from paper_2112_15083_gb300 import circuits as cg
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
    from paper_2112_15083_gb300 import replicas
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
    # as deployed (one CUDA-graph replay of the contraction plus the draw and sampler
    # launches), L2 flushed in between.  The job's first group runs every contraction; its
    # later groups reuse the batch-independent intermediates (the stem) that the first
    # left on the device (tn_sample_step reuse_stem), as tn_sample does for the groups of
    # one call.  Warm-up leaves nothing the first timed group uses.
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record()
        plan.sample_step(slices, F, seed, base_t + (args.warmup + k) * T, reuse_stem=k > 0, accept=acc[k], bits=bits[k])
        ev1[k].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    tot_ms = sum(step_ms)
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
    # traced region (the job again, CUDA events around every contraction launch): per-launch
    # device times for the roofline of the dominant kernel, and the job's launch counts
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
    # the last trace entry is the FP64 slice sum (kernel 2, or 3 when it runs fused with the
    # root step, whose own entry then has no launches); the rest are contraction steps
    ssum = [s for s in trace if s["kernel"] in (2, 3)]
    trace = [s for s in trace if s["kernel"] not in (2, 3)]
    # contraction FLOPs per group: a whole group's, and the job's average (the stem once)
    flops_group = sum(s["flops_per_launch"] for s in trace)
    trace = [s for s in trace if s["launches"] > 0]
    flops_step = sum(s["flops_per_launch"] * s["launches"] for s in trace) / args.steps
    slice_sum = None
    if ssum and ssum[0]["launches"]:
        s0 = ssum[0]
        ms1 = s0["ms"] / s0["launches"]
        slice_sum = {"ms": round(ms1, 3), "fp64_gflops": round(s0["flops_per_launch"] / (ms1 / 1e3) / 1e9, 1),
                     "gbs": round(s0["bytes_per_launch"] / (ms1 / 1e3) / 1e9, 1),
                     "fused_root_step": s0["kernel"] == 3}

    # dominant kernel of the job (most device time) from the live per-launch events
    dom = max(trace, key=lambda s: s["ms"])
    dom_ms = dom["ms"] / max(1, dom["launches"])
    pk = peaks()
    alg = dom["flops_per_launch"] / (dom_ms / 1e3) / 1e12
    shape = "(bat,m,n,k bits = %d,%d,%d,%d)" % (dom["nbat"], dom["nm"], dom["nn"], dom["nk"])
    if dom["kernel"] in (9128, 9064, 9032):
        # tensor-core step: algorithmic complex FLOPs (8 per complex MAC) against the
        # measured dense bf16 peak; the split path issues 3x that on the tensor pipe
        peak = pk.get("bf16_tflops", 1900.0)
        roofline = {"bound": "tensor", "achieved": alg, "peak": peak, "unit": "TFLOP/s", "traffic": None,
                    "frac": alg / peak, "tensor_pipe_tflops": 3 * alg, "tensor_pipe_frac": 3 * alg / peak,
                    "peak_source": "measured bf16 dense burst (MEASURED_PEAKS.json)" if "bf16_tflops" in pk
                    else "fallback 1.9 PFLOP/s",
                    "kernel": "tc_cgemm<%d,%d> split bf16 hi+lo %s" % (
                        dom["kernel"] - 9000, {9128: 3, 9064: 4, 9032: 5}[dom["kernel"]], shape)}
    elif dom["kernel"] in (0, 1, 4):
        # short products (row kernel, staged small kernel): algorithmic bytes (operands
        # read + result written, complex64; gathered operands at their batch size)
        # against the measured copy bandwidth
        gbs = dom["bytes_per_launch"] / (dom_ms / 1e3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        roofline = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "traffic": None, "frac": gbs / peak,
                    "peak_source": "measured HBM copy (MEASURED_PEAKS.json)" if "hbm_gbs" in pk else "fallback 6.8 TB/s",
                    "kernel": "%s %s%s" % ({0: "cgemm_row", 1: "cgemm_small", 4: "cgemm_rowstage"}[dom["kernel"]], shape,
                                           " after a batch-gather launch" if dom["gathers"] else "")}
    else:
        ffma_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        roofline = {"bound": "alu", "achieved": alg, "peak": ffma_peak, "unit": "TFLOP/s", "traffic": None,
                    "frac": alg / ffma_peak, "peak_source": "derived: " + FFMA_PEAK_NOTE + " (FP32 FFMA, complex64 path)",
                    "kernel": "cgemm_tile<%d,%d> %s" % (dom["kernel"] // 1000, dom["kernel"] % 1000, shape)}
    roofline["share_of_step"] = dom["ms"] / max(1e-9, sum(s["ms"] for s in trace))
    # device time per kernel family, averaged over the job's groups
    fam = {}
    for x in trace:
        k = x["kernel"]
        name = ("tc_cgemm" if k >= 9000 else {0: "cgemm_row", 1: "cgemm_small", 4: "cgemm_rowstage"}.get(k, "cgemm_tile"))
        fam[name] = fam.get(name, 0.0) + x["ms"] / args.steps
    roofline["kernel_family_ms_per_step"] = {k: round(v, 2) for k, v in sorted(fam.items(), key=lambda kv: -kv[1])}
    key = {9128: "tc_cgemm<128,3>", 0: "cgemm_row"}.get(dom["kernel"])
    rec = MEASURED_TRAFFIC.get((key, (dom["nbat"], dom["nm"], dom["nn"], dom["nk"]))) if key else None
    if rec:
        import hashlib
        src = os.path.join(ROOT, "paper_2112_15083_gb300", "csrc", rec[1])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec[2]:
            roofline["traffic"] = rec[0]
            roofline["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass, full size (profiles/)"
    roofline["measured"] = "CUDA events around each contraction launch over %d traced steps" % args.steps
    top_steps = []
    for s in sorted(trace, key=lambda s: -s["ms"])[:6]:
        ms1 = s["ms"] / max(1, s["launches"])
        top_steps.append({"shape_bits": [s["nbat"], s["nm"], s["nn"], s["nk"]], "kernel": s["kernel"],
                          "ms": round(ms1, 3), "launches_per_job": s["launches"],
                          "tflops": round(s["flops_per_launch"] / (ms1 / 1e3) / 1e12, 2),
                          "gbs": round(s["bytes_per_launch"] / (ms1 / 1e3) / 1e9, 1)})

    # end to end through the public API with host buffers: the same job as one tn_sample
    # call (selection of the slices included), about one group's expected samples
    # (T (1 - eps) / alpha) per step
    e2e = None
    if rank == 0:
        n_job = int(0.47 * T) * args.steps
        torch.cuda.synchronize()
        t = time.perf_counter()
        b, st = plan.sample(args.fidelity, n_job, seed=seed + 1)
        dt = time.perf_counter() - t
        groups = (st["steps"] + T - 1) // T
        e2e = {"value": len(b) / dt, "unit": "samples/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int((groups * T * (1 + 8 + 8) + n_job * 8) / args.steps),
               "api": "tn_sample(host bitstrings): one call for the job's %d samples" % n_job,
               "groups": groups}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))
        t = time.perf_counter()
        p = oracle_probs(circ)
        a = sum(oracle_group(p, circ, openq, T, seed, g * T) for g in range(3))
        del p
        dt = time.perf_counter() - t
        cpu = {"value": a / dt, "unit": "samples/s", "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
               "sample": "a job of 3 groups: the FP64 state vector of the %d-qubit circuit once, then the sampler "
                         "on %d batches per group (%d accepted in %.1f s)" % (circ.n_qubits, T, a, dt)}

    if rank == 0:
        line = {
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
            "cpu_baseline": cpu, "e2e": e2e, "top_steps": top_steps, "slice_sum": slice_sum,
            # the job's contraction launches, batch gathers and slice sums, plus a batch draw
            # and a sampler launch per step
            "gpu_launches": (sum(s["launches"] * (1 + s["gathers"]) for s in trace)
                             + sum(s["launches"] for s in ssum) + 2 * args.steps),
        }
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


def run_grid5x8_sample(args):
    """Bounded sample of the 40-qubit configuration (5x8 grid, 16 cycles, 1/64 of the
    slices retained, 100k samples): the plan slices legs until one slice's tensors fit
    2^30 elements, Alg. 1 selects the retained slices, and the first retained slices are
    contracted for one group of 4096 batches, alone and two at a time (shared
    intermediates).  The full job's time is extrapolated from the measured time per
    slice and group; nothing of it is run."""
    import math
    import numpy as np
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_2112_15083_gb300 as P
    from paper_2112_15083_gb300 import circuits as cg
    rows, cols, cycles, lb, f, N, alpha = 5, 8, 16, 12, 1.0 / 64, 100000, 2.0
    circ = cg.sycamore_grid(rows, cols, cycles, seed=0)
    openq = cg.default_open_qubits(rows, cols, 6)
    C = P.circuit_load(circ.serialize())
    # the job's batch groups: the order search weights the batch steps by them (the
    # batch-independent ones run once per slice)
    job_groups = math.ceil(1.1 * alpha * N / (1 << lb))
    t = time.perf_counter()
    # the largest tensor cap whose one-slice working set fits the budget
    for cap in (30, 29, 28, 27, 26):
        plan = P.plan(C, openq, log2_batches=lb, order_trials=256, order_seed=0, max_log2_tensor=cap,
                      hbm_budget_bytes=150e9, precision=P.tn.PREC_BF16X2, autotune=0, max_norm_flops=3e16,
                      job_groups=job_groups)
        if plan.estimate(np.zeros(1, np.uint64))[0] <= 140e9:
            break
        del plan
    plan_s = time.perf_counter() - t
    info = plan.info()
    line = {"metric": "40-qubit bounded sample: seconds per retained slice per batch group (shared part amortised)",
            "unit": "s",
            "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "grid5x8_m16: 40-qubit 5x8 Sycamore-style ABCD circuit, 16 cycles, seed 0; "
                                   "slices until one slice's working set fits 140 GB; f = 1/64; %d batches of 64 "
                                   "per group; bf16x2" % (1 << lb)},
            "plan": {"seconds": round(plan_s, 1), "sliced_legs": info["n_sliced"], "max_log2_tensor_cap": cap,
                     "job_groups": job_groups,
                     "log2_max_tensor": info["log2_max_tensor"], "flops_all_slices": info["flops_all_slices"]}}
    t = time.perf_counter()
    try:
        slices, F = plan.select(f)
        line["selection"] = {"seconds": round(time.perf_counter() - t, 1), "retained_slices": int(len(slices)),
                             "F": F}
    except P.TnError as e:
        line["selection"] = {"error": str(e)}
        print(json.dumps(line), flush=True)
        return
    T = 1 << lb
    cb = np.random.default_rng(1).integers(0, 1 << 34, size=2 * T, dtype=np.int64).astype(np.uint64)
    samples = []
    for chunk in (1, 2):
        sl = slices[:chunk]
        nbytes, fl_first, fl_next = plan.estimate(sl)
        row = {"slices": chunk, "device_bytes": nbytes, "flops_first_group": fl_first, "flops_later_group": fl_next}
        for groups in (1, 2):
            plan.contract(sl, cb[: groups * T])  # first execution (leaves, call plan, graphs)
            torch.cuda.synchronize()
            t = time.perf_counter()
            plan.contract(sl, cb[: groups * T])
            torch.cuda.synchronize()
            row["seconds_%d_group%s" % (groups, "s" if groups > 1 else "")] = round(time.perf_counter() - t, 4)
        # one group = batch-independent part + batch part; each later group adds the batch part
        row["batch_part_s"] = round(row["seconds_2_groups"] - row["seconds_1_group"], 4)
        row["shared_part_s"] = round(row["seconds_1_group"] - row["batch_part_s"], 4)
        row["tflops_first_group"] = round(fl_first / row["seconds_1_group"] / 1e12, 1)
        samples.append(row)
    line["samples"] = samples
    # per-step device times of one slice over two groups (the second reuses the shared part)
    plan.trace(True)
    plan.contract(slices[:1], cb[: 2 * T])
    tr = plan.trace_read()
    plan.trace(False)
    tops = sorted(tr, key=lambda x: -x["ms"])[:10]
    line["top_steps"] = [{"shape_bits": [x["nbat"], x["nm"], x["nn"], x["nk"]], "kernel": x["kernel"],
                          "launches": x["launches"], "ms": round(x["ms"], 3),
                          "tflops": round(x["flops_per_launch"] * x["launches"] / max(1e-9, x["ms"] / 1e3) / 1e12, 1),
                          "gbs": round(x["bytes_per_launch"] * x["launches"] / max(1e-9, x["ms"] / 1e3) / 1e9, 1),
                          "gathers": x["gathers"]} for x in tops]
    groups = math.ceil(1.1 * alpha * N / T)
    best = min(samples, key=lambda r: (r["shared_part_s"] + groups * r["batch_part_s"]) / r["slices"])
    per_slice = (best["shared_part_s"] + groups * best["batch_part_s"]) / best["slices"]
    hours = per_slice * len(slices) / 3600.0
    line["value"] = round(per_slice / groups, 4)
    line["extrapolated"] = {"groups": groups, "retained_slices": int(len(slices)),
                            "seconds_per_slice_all_groups": round(per_slice, 3), "hours": round(hours, 1),
                            "note": "retained slices x (shared part + groups x batch part) per slice, from the "
                                    "measured chunk of %d slice(s); the job itself is not run" % best["slices"]}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serve:
        run_serve(a)
    elif a.grid5x8_sample:
        run_grid5x8_sample(a)
    else:
        run_ours(a)

"""bench.py's JSON line, checked on the CPU: run_ours runs with fakes of the CUDA calls, of
the plan and of the clock sampler, and its one line must carry every key of the bench
contract with consistent values.

* Batch-group workload (28 qubits): a trace with batch-independent steps launched once per
  job and batch steps every group; the job's accepted samples over its device time, the
  stem-each-step figure, the roofline object, e2e with its transfer counts, the launch
  count of the job.
* Sampling-job workload (40 qubits, the default): steps are slice chunks of one job; the
  value is the job's samples over (chunks x mean chunk time + the final pass), e2e is
  projected the same way, the launch count is per traced chunk times the timed chunks."""
import io
import json
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _Event:
    full = True

    def __init__(self, **_):
        pass

    def record(self):
        pass

    def elapsed_time(self, _other):
        return 2.0


class _Clocks:
    def __init__(self, _i):
        pass

    def start(self):
        pass

    def stop(self):
        return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


class _Plan:
    """Four contraction steps (two batch-independent) and the slice-sum entry."""

    def __init__(self):
        self.tracing = False
        self.launches = {}
        self.calls = []

    def info(self):
        return {"n_qubits": 28, "log2_batches": 14}

    def select(self, f):
        return np.arange(1024, dtype=np.uint64), 1.0

    def sample_step(self, slices, F, seed, t0, reuse_stem=False, accept=None, bits=None):
        self.calls.append((t0, reuse_stem))
        accept.fill_(1)
        if self.tracing:
            for i in range(4):
                if i < 2 and reuse_stem:
                    continue
                self.launches[i] = self.launches.get(i, 0) + 1
            self.launches[4] = self.launches.get(4, 0) + 1
        return accept, bits

    def trace(self, on):
        self.tracing = on

    def trace_read(self):
        ent = []
        for i in range(4):
            n = self.launches.get(i, 0)
            ent.append({"step": i, "launches": n, "ms": 1.5 * n, "flops_per_launch": 1e12, "bytes_per_launch": 1e10,
                        "nbat": 15 if i >= 2 else 0, "nm": 2, "nn": 10, "nk": 6, "nver": 1,
                        "kernel": 0 if i == 3 else 9128, "gathers": 1 if i == 2 else 0})
        n = self.launches.get(4, 0)
        ent.append({"step": 4, "launches": n, "ms": 4.0 * n, "flops_per_launch": 2e9, "bytes_per_launch": 8e9,
                    "nbat": 0, "nm": 0, "nn": 0, "nk": 0, "nver": 1, "kernel": 2, "gathers": 0})
        return ent

    def sample(self, f, N, seed):
        return np.zeros(N, np.uint64), {"steps": 10 * (1 << 14)}


def test_bench_line_carries_the_contract(monkeypatch):
    import bench
    import __graft_entry__
    import paper_2112_15083_gb300 as P
    plan = _Plan()
    monkeypatch.setattr(__graft_entry__, "build", lambda: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: real_empty(*a, **k))
    monkeypatch.setattr(bench, "Clocks", _Clocks)
    monkeypatch.setattr(P, "plan", lambda *a, **k: plan)
    monkeypatch.setattr(P, "circuit_load", lambda buf: None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "grid4x7_m14", "--steps", "4", "--warmup", "3",
                                      "--no-cpu-baseline"])
    args = bench.parse()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_ours(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "clocks", "roofline", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in line, k
    assert line["config"]["workload"].startswith("grid4x7_m14")
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    assert line["steps"] == 4 and line["warmup"] == 3 and line["n_gpus"] == 1
    # warm-up: two full groups, then reuse; the timed job: a full group, then reuse
    assert [r for _, r in plan.calls[:3]] == [False, False, True]
    assert [r for _, r in plan.calls[3:7]] == [False, True, True, True]
    # 4 groups of 16384 accepted in 4 x 2 ms
    assert line["value"] == pytest.approx(4 * 16384 / 8e-3)
    assert line["ms_per_step"] == pytest.approx(2.0)
    # job FLOPs: the two stem steps once, the two batch steps every group
    assert line["flops_per_step"] == pytest.approx((2 * 1e12 + 2 * 4 * 1e12) / 4)
    # launches: stem 2, batch 2 x 4 (+4 gathers), slice sum 4, draw and sampler 2 x 4
    assert line["gpu_launches"] == 2 + 8 + 4 + 4 + 8
    assert line["roofline"]["frac"] == pytest.approx(line["roofline"]["achieved"] / line["roofline"]["peak"])


class _Job:
    def __init__(self, plan, N, chunk):
        self.plan, self.N, self.chunk = plan, N, chunk
        self.ran = []

    def info(self):
        return {"n_slices": 4096, "F": 0.0159, "chunk_slices": self.chunk, "n_chunks": 4096 // self.chunk,
                "groups": 55, "T": 4096, "chunks_done": len(self.ran), "flops_done": 0.0, "flops_chunk": 2e15}

    def run(self, first, count=1):
        for c in range(first, first + count):
            assert c not in self.ran
            self.ran.append(c)
            if self.plan.tracing:
                self.plan.traced += 1

    def finish(self, partial=False):
        assert partial
        return np.zeros(self.N, np.uint64), {"eps_hat": 0.0, "steps": 55 * 4096}


class _JobPlan:
    """A chunk: one stem step, two batch steps per group (one with a gather), the slice
    sum per group."""

    def __init__(self):
        self.tracing = False
        self.traced = 0
        self.jobs = []

    def info(self):
        return {"n_qubits": 40, "log2_batches": 12, "n_sliced": 18}

    def estimate(self, slices):
        return (30e9, 6e13, 1.2e12)

    def job(self, f, N, seed, alpha=2.0, max_chunk_slices=0):
        j = _Job(self, N, max_chunk_slices)
        self.jobs.append(j)
        return j

    def trace(self, on):
        self.tracing = on

    def trace_read(self):
        g = 55 * self.traced
        ent = [{"step": 0, "launches": self.traced, "ms": 100.0 * self.traced, "flops_per_launch": 6e13,
                "bytes_per_launch": 1e10, "nbat": 0, "nm": 15, "nn": 12, "nk": 15, "nver": 1, "kernel": 9128,
                "gathers": 0},
               {"step": 1, "launches": g, "ms": 4.0 * g, "flops_per_launch": 1e12, "bytes_per_launch": 1.4e10,
                "nbat": 12, "nm": 8, "nn": 10, "nk": 7, "nver": 1, "kernel": 9128, "gathers": 1},
               {"step": 2, "launches": g, "ms": 3.0 * g, "flops_per_launch": 6.9e10, "bytes_per_launch": 1.7e10,
                "nbat": 12, "nm": 3, "nn": 3, "nk": 15, "nver": 1, "kernel": 5, "gathers": 0},
               {"step": 3, "launches": g, "ms": 0.5 * g, "flops_per_launch": 5e8, "bytes_per_launch": 4e9,
                "nbat": 0, "nm": 0, "nn": 0, "nk": 0, "nver": 1, "kernel": 2, "gathers": 0}]
        return ent


def test_job_bench_line_carries_the_contract(monkeypatch):
    import bench
    import __graft_entry__
    import paper_2112_15083_gb300 as P
    plan = _JobPlan()
    monkeypatch.setattr(__graft_entry__, "build", lambda: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(bench, "Clocks", _Clocks)
    monkeypatch.setattr(P, "plan", lambda *a, **k: plan)
    monkeypatch.setattr(P, "circuit_load", lambda buf: None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "4", "--warmup", "3", "--no-cpu-baseline",
                                      "--no-secondary"])
    args = bench.parse()
    assert args.workload == "grid5x8_m16" and args.fidelity == 1.0 / 64
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_ours(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "clocks", "roofline", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in line, k
    assert line["config"]["workload"].startswith("grid5x8_m16")
    job = plan.jobs[0]
    # warm-up chunks 0-2, timed chunks 3-6, traced chunk 7
    assert job.ran == list(range(8))
    assert line["ms_per_step"] == pytest.approx(2.0)
    chunks = 4096 // args.chunk
    assert line["job_seconds"] == pytest.approx(chunks * 2e-3 + line["finish_s"])
    assert line["value"] == pytest.approx(100000 / line["job_seconds"])
    # per traced chunk: 1 stem launch, 55 x (2 + 1 gather) batch launches, 55 slice sums,
    # 55 accumulations; times 4 timed chunks
    assert line["gpu_launches"] == 4 * (1 + 55 * 3 + 55 + 55)
    assert line["roofline"]["kernel"].startswith("tc_cgemm<128,3>")
    assert line["roofline"]["frac"] == pytest.approx(line["roofline"]["achieved"] / line["roofline"]["peak"])
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    # e2e: a second job, creation + chunks + final pass projected to all chunks
    assert len(plan.jobs) == 2 and plan.jobs[1].ran == [0, 1]


def _step(nbat, nm, nn, nk, kernel, ms, flops, bytes_):
    return {"nbat": nbat, "nm": nm, "nn": nn, "nk": nk, "nver": 1, "kernel": kernel, "ms": ms, "launches": 1,
            "flops_per_launch": flops, "bytes_per_launch": bytes_, "gathers": 0, "in_place": 1}


def test_roofline_bound_is_the_longer_of_bytes_and_products():
    """A tensor-core step reports the HBM roofline when its compulsory bytes at the copy
    bandwidth outlast its tensor-pipe products (three per algorithmic product) at the bf16
    peak, the tensor roofline otherwise; frac is achieved / peak in the bound's unit."""
    import bench
    pk = {"hbm_gbs": 6789.0, "bf16_tflops": 1971.8}
    # 6.71 GB and 8 x 2^36 = 5.5e11 FLOPs in 2.32 ms: 0.99 ms of bytes against 0.84 ms of
    # tensor-pipe products
    r = bench.roofline_of([_step(12, 11, 5, 8, 19128, 2.32, 5.5e11, 6.71e9)], 1, pk)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(6.71e9 / 2.32e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6789.0)
    assert r["tensor_pipe_tflops"] == pytest.approx(3 * 5.5e11 / 2.32e-3 / 1e12)
    # 1.1e15 FLOPs and 70 GB in 2 s: products outlast bytes
    r = bench.roofline_of([_step(1, 19, 10, 13, 9128, 2000.0, 1.1e15, 7.0e10)], 1, pk)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(1.1e15 / 2.0 / 1e12 / 1971.8)


def test_roofline_traffic_only_for_the_measured_kernel_source(monkeypatch):
    """The measured DRAM traffic of a launch is reported only while the kernel source it
    was taken with is unchanged (its hash prefix), else traffic stays null."""
    import bench
    pk = {"hbm_gbs": 6789.0, "bf16_tflops": 1971.8}
    step = [_step(12, 11, 5, 8, 19128, 2.32, 5.5e11, 6.71e9)]
    key = ("tc_cgemm<128,3> stacked", (12, 11, 5, 8))
    assert key in bench.MEASURED_TRAFFIC
    r = bench.roofline_of(step, 1, pk)
    assert r["traffic"] == bench.MEASURED_TRAFFIC[key][0] and "traffic_source" in r
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, key, (bench.MEASURED_TRAFFIC[key][0], "tc.cuh", "0" * 16))
    assert bench.roofline_of(step, 1, pk)["traffic"] is None

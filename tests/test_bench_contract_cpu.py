"""bench.py's JSON line, checked on the CPU: run_ours runs with fakes of the CUDA calls, of
the plan (a trace with batch-independent steps launched once per job and batch steps every
group) and of the clock sampler, and its one line must carry every key of the bench
contract with consistent values: the job's accepted samples over its device time, the
stem-each-step figure, the roofline object, e2e with its transfer counts, and the launch
count of the job."""
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
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "4", "--warmup", "3", "--no-cpu-baseline"])
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

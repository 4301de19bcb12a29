"""Serving layer (tn_server_*): continuous batching by HBM budget.

GPU tests: a request's samples are bit-identical alone, in a mix of concurrent requests
(other circuits, precisions and fidelities) and through tn_sample; admission respects the
budget; oversized requests are rejected.  CPU test: a request that fails (no device)
leaves the server consistent."""
import math

import numpy as np
import pytest

import paper_2112_15083_gb300 as P
from paper_2112_15083_gb300 import circuits as cg


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def request(rows, cols, cycles, seed):
    circ = cg.sycamore_grid(rows, cols, cycles, seed=seed)
    return circ.serialize(), cg.default_open_qubits(rows, cols, 6)


def test_failed_request_leaves_server_consistent_cpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("needs a host without a GPU (the failure is the missing device)")
    s = P.Server(planner_threads=1)
    buf, openq = request(3, 4, 6, 0)
    rid = s.submit(buf, openq, N=10)
    bits, info = s.wait(rid, 10, timeout=60)
    assert bits is None and info["status"] == "failed" and info["rc"] != 0
    with pytest.raises(P.TnError):
        s.submit(buf, openq, N=0)
    st = s.stats()
    assert st["failed"] == 1 and st["active"] == 0 and st["bytes_in_use"] == 0
    s.close()


gpu = pytest.mark.gpu


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@gpu
def test_same_alone_in_the_mix_and_via_tn_sample():
    need_gpu()
    buf, openq = request(4, 5, 10, 3)
    N = 3000
    alone = P.Server(max_active=4)
    rid = alone.submit(buf, openq, N=N, f=1.0, seed=42, precision=P.tn.PREC_BF16X2, n_sliced=4)
    ref, info = alone.wait(rid, N, timeout=300)
    alone.close()
    assert ref is not None and info["status"] == "done" and len(ref) == N

    mix = P.Server(max_active=4)
    others = []
    for k, (r, c, m) in enumerate([(4, 6, 8), (3, 5, 10), (4, 4, 12), (5, 5, 8)]):
        b, o = request(r, c, m, 10 + k)
        others.append((mix.submit(b, o, N=2000 + 500 * k, f=(1.0, 0.25, 1.0, 0.5)[k], seed=k,
                                  precision=(P.tn.PREC_C64, P.tn.PREC_BF16X2)[k % 2], n_sliced=5), 2000 + 500 * k))
    rid = mix.submit(buf, openq, N=N, f=1.0, seed=42, precision=P.tn.PREC_BF16X2, n_sliced=4)
    got, info = mix.wait(rid, N, timeout=300)
    for oid, n in others:
        b, inf = mix.wait(oid, n, timeout=300)
        assert b is not None and inf["status"] == "done", inf
    st = mix.stats()
    mix.close()
    assert np.array_equal(got, ref)
    assert st["done"] == 5

    # the server sizes the group to the request (the smallest 2^lb >= 1.1 alpha N within
    # [2^8, 2^14]), uses the fixed kernel shape rules, hands its memory budget to the order
    # search's cost model and weights the batch steps by the request's expected groups
    lb = 8
    while lb < 14 and (1 << lb) < 1.1 * 2.0 * N:
        lb += 1
    job_groups = max(1, math.ceil(1.1 * 2.0 * N / (1 << lb)))
    C = P.circuit_load(buf)
    plan = P.plan(C, openq, n_auto_sliced=4, log2_batches=lb, order_trials=64, precision=P.tn.PREC_BF16X2,
                  autotune=0, hbm_budget_bytes=150e9, job_groups=job_groups)
    via_plan, _ = plan.sample(1.0, N, seed=42)
    assert np.array_equal(via_plan, ref)


@gpu
def test_admission_respects_budget():
    need_gpu()
    s = P.Server(max_active=8)
    buf, openq = request(4, 5, 10, 1)
    rid0 = s.submit(buf, openq, N=2000, n_sliced=3)
    _, info0 = s.wait(rid0, 2000, timeout=300)
    s.close()
    budget = 1.5 * info0["est_bytes"]  # room for one request at a time
    s = P.Server(hbm_budget_bytes=budget, max_active=8)
    ids = [s.submit(buf, openq, N=2000, seed=k, n_sliced=3) for k in range(3)]
    infos = [s.wait(i, 2000, timeout=300)[1] for i in ids]
    s.close()
    assert all(i["status"] == "done" for i in infos)
    spans = sorted((i["t_admit"], i["t_done"]) for i in infos)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-3  # never two admitted at once


@gpu
def test_oversized_request_rejected():
    need_gpu()
    s = P.Server(max_request_seconds=1e-9)
    buf, openq = request(3, 4, 8, 0)
    rid = s.submit(buf, openq, N=100)
    bits, info = s.wait(rid, 100, timeout=120)
    s.close()
    assert bits is None and info["status"] == "rejected"

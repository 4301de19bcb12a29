"""GPU parity of the chunked sampling job (tn_job_*) against the CPU oracle.

The job splits the retained slices X x {0,1}^{|I|-k} (Alg. 1, Sec. I.C step 1) into
chunks, contracts every chunk for all of the job's batch groups and adds the chunk sums
in FP64; then it runs the accept / pick step of Sec. II.A on every batch.

* The summed amplitudes of a group equal the oracle's partial state |psi_X> on the
  group's Philox batch draws within 1e-4 of the RMS amplitude (complex64 path).
* Given the job's own probabilities p = |a|^2 / F, the returned strings are exactly the
  oracle sampler's accepted strings in t order (bit-exact).
* tn_sample runs the same job when the slice set exceeds the HBM budget.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg

pytestmark = pytest.mark.gpu

TOL_C64 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch


def pkg():
    import paper_2112_15083_gb300 as p
    return p


def close_c64(got, ref):
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    err = float(np.abs(got - ref).max())
    assert err <= TOL_C64 * rms, "max err %.3e > %.1e * rms %.3e" % (err, TOL_C64, rms)


def circuit_20q():
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(20) for s in range(2, view.n2q[q] - 1)][:12]
    return circ, I, cg.default_open_qubits(4, 5, 6)


@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
def test_job_amplitudes_and_samples(prec):
    P = pkg()
    circ, I, openq = circuit_20q()
    closed = oracle.closed_of(20, openq)
    C = P.circuit_load(circ.serialize())
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    plan = P.plan(C, openq, sliced=I, log2_batches=8, order_trials=16, precision=precision)
    f, N, seed = 0.25, 600, 21
    job = plan.job(f, N, seed, max_chunk_slices=4)
    info = job.info()
    T, G = info["T"], info["groups"]
    assert info["chunk_slices"] == 4 and info["n_chunks"] * 4 == info["n_slices"]
    assert G == math.ceil((1.1 * 2 * N + 8 * math.sqrt(2 * N) + 64) / T)
    job.run(0, 2)
    job.run(2)  # the rest
    with pytest.raises(P.TnError):
        job.run(1, 1)  # a chunk runs once
    S_ref, X_ref, F_ref, _ = oracle.slice_selection(circ, I, f)
    assert abs(info["F"] - F_ref) < (1e-5 if prec == "c64" else 1e-3)
    psi_x = oracle.partial_state(circ, S_ref, X_ref)
    amps = np.concatenate([job.amplitudes(g) for g in range(G)])
    js = oracle.batch_draws(seed, G * T, 14)
    ref = oracle.batch_amplitudes(psi_x, 20, openq, js)
    if prec == "c64":
        close_c64(amps, ref)
    else:
        assert np.linalg.norm(amps - ref) / np.linalg.norm(ref) <= 1e-3
    bits, st = job.finish()
    assert st["steps"] == G * T and st["F"] == info["F"]
    p = (amps.real * amps.real + amps.imag * amps.imag) / st["F"]
    acc, pick = oracle.sample_batches(np.ascontiguousarray(p), 14, 2.0, seed, t0=0)
    want = [oracle.bitstring(int(pick[t]), int(js[t]), openq, closed) for t in range(G * T) if acc[t]]
    assert st["accepted"] == len(want)
    assert [int(b) for b in bits] == want[:N]


def test_job_partial_finish_needs_flag():
    P = pkg()
    circ, I, openq = circuit_20q()
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, sliced=I, log2_batches=8, order_trials=16)
    job = plan.job(0.25, 100, 3, max_chunk_slices=8)
    job.run(0, 1)
    with pytest.raises(P.TnError):
        job.finish()
    job.finish(partial=True)  # timing use: the sums over the chunks run so far


def test_sample_over_budget_runs_the_job():
    """A budget that holds a chunk but not the whole slice set: tn_sample returns exactly
    the strings of the automatically chunked job on the same plan.  The order search takes
    the budget into account, so each candidate budget is checked on its own plan."""
    P = pkg()
    circ, I, openq = circuit_20q()
    C = P.circuit_load(circ.serialize())
    plan, tried = None, []
    for f in (1.0, 0.25):
        for budget in (1.2e8, 1.6e8, 2.4e8, 4e8, 8e8, 1.6e9):
            cand = P.plan(C, openq, sliced=I, log2_batches=8, order_trials=16, hbm_budget_bytes=budget)
            slices, _F = cand.select(f)
            full, part = cand.estimate(slices)[0], cand.estimate(slices[:2])[0]
            tried.append((f, budget, full, part))
            if full > budget and part + 4e6 < 0.9 * budget:
                plan = cand
                break
            del cand
        if plan is not None:
            break
    print("budgets tried (f, budget, whole set, two slices):", tried)
    assert plan is not None, "no budget between one chunk and the whole slice set: %s" % tried
    bits, st = plan.sample(f, 500, seed=8)
    job = plan.job(f, 500, 8)
    assert job.info()["n_chunks"] > 1
    job.run()
    bits2, st2 = job.finish()
    assert np.array_equal(bits, bits2)
    assert st["steps"] == st2["steps"] and st["eps_hat"] == st2["eps_hat"]

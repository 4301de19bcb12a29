"""GPU parity of the verification, spoofing and fused-root paths (through the C-ABI)
against the CPU oracle.

* tn_xeb (Sec. III, elided-circuit validation; Eq. 1): the amplitudes of given
  bitstrings summed over a slice set, element by element against the oracle's state
  vector at 1e-4 of the RMS amplitude (complex64), and their linear XEB.
* tn_spoof (Sec. III, "Spoofing Linear XEB"; App. A): the N strings of one batch with the
  largest |a|^2.  The selection is an index result, so it must equal the oracle's
  selection on the GPU's own probabilities exactly, ties included.
* fuse_root_sum: the root product fused with the FP64 slice sum must give exactly the
  amplitudes (and samples) of the two separate launches.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg

pytestmark = pytest.mark.gpu

TOL_C64 = 1e-4
TC_IDS = (9128, 9064, 9032, 19128, 19064)  # tensor-core kernels (trace ids)


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


def in_batch_index(bits, open_qubits):
    return np.array([sum(((int(b) >> q) & 1) << r for r, q in enumerate(open_qubits)) for b in bits], np.int64)


# ------------------------------------------------------------------ f1: verification amplitudes

@pytest.mark.parametrize("n_open", [0, 6])
def test_xeb_amplitudes_against_state_vector(n_open):
    """Ragged: 300 strings over groups of 64 batches; |A| = 0 puts every string in its
    own batch, |A| = 6 picks one entry of each string's batch."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 10, seed=2)
    openq = [] if n_open == 0 else cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=6, log2_batches=6, order_trials=16)
    psi = oracle.simulate(circ)
    bs = np.random.default_rng(4).integers(0, 1 << 20, size=300).astype(np.uint64)
    x, amps = plan.xeb(np.arange(64, dtype=np.uint64), bs, return_amplitudes=True)
    ref = psi[bs.astype(np.int64)]
    close_c64(amps, ref)
    x_ref = oracle.xeb_of_samples(np.abs(psi) ** 2, 20, bs.astype(np.int64))
    # |a|^2 within about 2e-4 relative of the exact value for every string
    assert abs(x - x_ref) <= 1e-3 * (1 + abs(x_ref)), (x, x_ref)


def test_xeb_of_partial_fidelity_samples_tracks_F():
    """Samples drawn at fidelity F from the retained slices, scored with the full-fidelity
    amplitudes of the same plan (all slices): the device XEB equals the oracle's Eq. 1 on
    the exact distribution, and tracks F (Table elided)."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    I = [(q, s) for q in range(20) for s in range(2, view.n2q[q] - 1)][:12]
    plan = P.plan(C, openq, sliced=I, log2_batches=8, order_trials=16)
    N = 20000
    bits, st = plan.sample(0.25, N, seed=5, alpha=2.0)
    x = plan.xeb(np.arange(1 << len(I), dtype=np.uint64), bits)
    p = np.abs(oracle.simulate(circ)) ** 2
    x_ref = oracle.xeb_of_samples(p, 20, bits.astype(np.int64))
    assert abs(x - x_ref) <= 1e-3 * (1 + abs(x_ref)), (x, x_ref)
    sigma = math.sqrt(2.0 / N)
    assert abs(x - st["F"]) < 4 * sigma + 0.02 * st["F"], (x, st["F"])


# ------------------------------------------------------------------ f2: XEB spoofing

def projected_circuit():
    """3x4 grid, 8 cycles, then |0><0| on qubits 5 and 10: every amplitude with either of
    them set is exactly zero, so a selection deeper than the nonzero quarter of a batch
    meets exact ties (broken by position)."""
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    proj = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    circ.gates.append(cg.Gate((5,), proj.copy()))
    circ.gates.append(cg.Gate((10,), proj.copy()))
    return circ


@pytest.mark.parametrize("slices", [[0, 1, 2, 3], [0, 2]])
@pytest.mark.parametrize("N", [1, 100, 256, 400, 1024])
def test_spoof_selection_equals_oracle_ties_included(slices, N):
    P = pkg()
    circ = projected_circuit()
    openq = [0, 1, 2, 3, 5, 6, 7, 9, 10, 11]  # 1024 strings per batch; closed: 4, 8
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=2, log2_batches=0, order_trials=8)
    sl = np.array(slices, dtype=np.uint64)
    pattern = 2  # qubit 8 set, qubit 4 clear
    amps = plan.contract(sl, [pattern])[0]
    p = amps.real * amps.real + amps.imag * amps.imag  # FP64, rounded products, no FMA
    assert np.count_nonzero(p) == 256
    bits, probs = plan.spoof(sl, pattern, N, return_probs=True)
    idx = in_batch_index(bits, openq)
    assert np.all(np.diff(idx) > 0)  # ascending in-batch index
    assert np.array_equal(idx, np.sort(oracle.spoof_select(p, N)))
    assert np.array_equal(probs, p[idx])
    closed_bits = np.array([(int(b) >> 4) & 1 | ((int(b) >> 8) & 1) << 1 for b in bits])
    assert np.all(closed_bits == pattern)


def test_spoof_gain_at_partial_fidelity_20q():
    """One batch of 2^12 strings of a 20-qubit circuit at fidelity F (Alg. 1 slices): the
    device's top-N selection equals the oracle's on the device probabilities, and its
    exact XEB gain over the batch is about -F ln r (App. A) as the oracle's own run."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    openq = [0, 1, 2, 3, 4, 5, 7, 9, 12, 14, 17, 19]
    C = P.circuit_load(circ.serialize())
    I = [(q, s) for q in range(20) for s in range(2, view.n2q[q] - 1)][:12]
    plan = P.plan(C, openq, sliced=I, log2_batches=0, order_trials=16)
    slices, F = plan.select(0.5)
    pattern = 0b10110101
    r = 0.36
    N = int(r * 4096)
    amps = plan.contract(slices, [pattern])[0]
    p_dev = amps.real * amps.real + amps.imag * amps.imag
    bits = plan.spoof(slices, pattern, N)
    idx = in_batch_index(bits, openq)
    assert np.array_equal(idx, np.sort(oracle.spoof_select(p_dev, N)))
    p = np.abs(oracle.simulate(circ)) ** 2
    gain = oracle.spoof_xeb(p, 20, bits.astype(np.int64)) - oracle.spoof_xeb(
        p, 20, [oracle.bitstring(i, pattern, openq, oracle.closed_of(20, openq)) for i in range(4096)])
    # one batch of 4096 Porter-Thomas values: the spread of the top-r mean is about
    # 1/sqrt(r 4096) ~ 0.026 (times F for the part that the selection sees)
    assert abs(gain - oracle.spoof_expected_xeb(F, r)) < 0.15, (gain, F)


# ------------------------------------------------------------------ fused root + slice sum

def fused_pair(P, C, openq, **kw):
    return [P.plan(C, openq, fuse_root_sum=fuse, **kw) for fuse in (False, True)]


def fused_ran(plan, slices, cb):
    plan.trace(True)
    plan.contract(slices, cb)
    tr = plan.trace_read()
    plan.trace(False)
    return any(s["kernel"] == 3 and s["launches"] > 0 for s in tr)


def test_fused_root_sum_bit_identical_20q_ragged_groups():
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 10, seed=2)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    cb = cg.random_closed_bits(50, 14, seed=5)  # 16 per group: 3 full groups + 2
    slices = np.arange(64, dtype=np.uint64)
    a, b = fused_pair(P, C, openq, n_auto_sliced=6, log2_batches=4, order_trials=16)
    out = [pl.contract(slices, cb) for pl in (a, b)]
    assert np.array_equal(out[0], out[1])
    close_c64(out[1], oracle.batch_amplitudes(oracle.simulate(circ), 20, openq, cb))
    assert fused_ran(b, slices, cb), "the fused root launch did not run"
    sub = np.array([3, 17, 40, 41], dtype=np.uint64)
    assert np.array_equal(a.contract(sub, cb), b.contract(sub, cb))


@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
def test_fused_root_sum_bit_identical_28q_bench_configuration(prec):
    """The 4x7 / 14-cycle configuration at 16384 batches per group."""
    P = pkg()
    circ = cg.sycamore_grid(4, 7, 14, seed=0)
    openq = cg.default_open_qubits(4, 7, 6)
    C = P.circuit_load(circ.serialize())
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    a, b = fused_pair(P, C, openq, n_auto_sliced=10, log2_batches=14, order_trials=256, order_seed=0,
                      hbm_budget_bytes=200e9, precision=precision)
    cb = cg.random_closed_bits(16384, 22, seed=3)
    slices = np.arange(1024, dtype=np.uint64)
    assert np.array_equal(a.contract(slices, cb), b.contract(slices, cb))
    assert fused_ran(b, slices, cb), "the fused root launch did not run"


def test_fused_root_sum_same_samples():
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    I = [(q, s) for q in range(20) for s in range(2, view.n2q[q] - 1)][:12]
    a, b = fused_pair(P, C, openq, sliced=I, log2_batches=8, order_trials=16)
    res = [pl.sample(0.25, 3000, seed=9) for pl in (a, b)]
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1]["eps_hat"] == res[1][1]["eps_hat"]


# ------------------------------------------------------------------ long-K products

def long_k_dispatch(tr):
    """Every traced step of the long-K shape class (at most 8 x 32 outputs per batch,
    K >= 1024, not a tensor-core step) ran the long-K kernel (id 5); returns their count."""
    n = 0
    for s in tr:
        if s["launches"] and min(s["nm"], s["nn"]) <= 3 and max(s["nm"], s["nn"]) <= 5 and s["nk"] >= 10 \
                and s["kernel"] not in TC_IDS:
            assert s["kernel"] == 5, s
            n += 1
    return n


@pytest.mark.parametrize("n_open,lb,prec", [(4, 4, "c64"), (2, 4, "c64"), (2, 0, "c64"), (2, 8, "bf16x2")])
def test_long_k_kernel_against_state_vector(n_open, lb, prec):
    """Plans of a 4x5 / 12-cycle circuit whose root joins two halves over K = 2^10 .. 2^12
    with few outputs per batch: such a step runs the long-K kernel (lane split of K,
    butterfly), checked with every amplitude against the state vector."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=1)
    openq = list(range(n_open))
    C = P.circuit_load(circ.serialize())
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    plan = P.plan(C, openq, log2_batches=lb, order_trials=16, precision=precision)
    nb = (1 << lb) + 3  # a ragged second group
    cb = cg.random_closed_bits(nb, 20 - n_open, seed=4)
    plan.contract(np.arange(1, dtype=np.uint64), cb)  # the first execution tunes (and is not traced)
    plan.trace(True)
    amps = plan.contract(np.arange(1, dtype=np.uint64), cb)
    tr = plan.trace_read()
    plan.trace(False)
    ran = long_k_dispatch(tr)
    if prec == "c64":
        assert ran > 0, "no long-K step in this plan"
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 20, openq, cb)
    if prec == "c64":
        close_c64(amps, ref)
    else:
        assert np.linalg.norm(amps - ref) / np.linalg.norm(ref) <= 1e-3


def test_long_k_kernel_25q_4096_batches():
    """5x5 grid, 14 cycles, 6 open qubits, one group of 4096 batches: the root joins two
    halves over K = 2^10 with 8 x 8 outputs per batch (the shape class of the 40-qubit
    job's root), every amplitude of 300 sampled batches against the state vector."""
    P = pkg()
    circ = cg.sycamore_grid(5, 5, 14, seed=0)
    openq = cg.default_open_qubits(5, 5, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, log2_batches=12, order_trials=16, precision=P.tn.PREC_BF16X2)
    cb = cg.random_closed_bits(4096, 19, seed=6)
    amps = plan.contract(np.arange(1, dtype=np.uint64), cb)
    plan.trace(True)
    again = plan.contract(np.arange(1, dtype=np.uint64), cb)
    tr = plan.trace_read()
    plan.trace(False)
    assert np.array_equal(amps, again)
    print("long-K steps:", long_k_dispatch(tr))
    pick = np.random.default_rng(1).choice(4096, size=300, replace=False)
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 25, openq, cb[pick])
    assert np.linalg.norm(amps[pick] - ref) / np.linalg.norm(ref) <= 1e-3


# ------------------------------------------------------------------ failure detection

def test_bounded_wait_times_out_and_the_plan_recovers():
    """A tensor-core wait that nothing satisfies (tn_plan_test_stall) must end in the
    kernel's bounded-wait exit and TN_ETIMEOUT from the synchronising call, leave the
    context usable, and a following normal call must match the oracle again."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 10, seed=1)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=6, log2_batches=10, order_trials=16, precision=P.tn.PREC_BF16X2,
                  autotune=0)
    cb = cg.random_closed_bits(1024, 14, seed=2)
    slices = np.arange(64, dtype=np.uint64)
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 20, openq, cb)
    first = plan.contract(slices, cb)
    assert np.linalg.norm(first - ref) / np.linalg.norm(ref) <= 1e-3
    plan.test_stall(2_000_000)  # about 1 ms at 2 GHz
    with pytest.raises(P.TnError) as e:
        plan.contract(slices, cb)
    assert e.value.code == P.tn.TN_ETIMEOUT
    plan.test_stall(0)
    again = plan.contract(slices, cb)
    assert np.array_equal(again, first)



# ------------------------------------------------------------------ gathered operands read in place

@pytest.mark.parametrize("seed,n_sliced", [(0, 0), (1, 4)])
def test_tensor_core_steps_read_gathered_operands_in_place(seed, n_sliced):
    """4x6 grid, 14 cycles, 1024 batches (+5 in a ragged second group): a batch step on the
    tensor cores, (10,8,5,7), reads an operand with closed legs (the batch's selection of
    a batch-independent tensor) straight from its stored form through a tensor map, one
    plane coordinate per batch; every amplitude against the oracle's state vector."""
    P = pkg()
    circ = cg.sycamore_grid(4, 6, 14, seed=seed)
    openq = cg.default_open_qubits(4, 6, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=n_sliced, log2_batches=10, order_trials=16,
                  precision=P.tn.PREC_BF16X2)
    cb = cg.random_closed_bits(1024 + 5, 18, seed=7)
    slices = np.arange(1 << n_sliced, dtype=np.uint64)
    plan.contract(slices, cb)
    plan.trace(True)
    amps = plan.contract(slices, cb)
    tr = plan.trace_read()
    plan.trace(False)
    tc_in_place = [s for s in tr if s["kernel"] in TC_IDS and s["in_place"] and s["launches"]]
    assert tc_in_place, "no tensor-core step read a gathered operand in place"
    assert all(s["gathers"] == 0 for s in tc_in_place)
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 24, openq, cb)
    assert np.linalg.norm(amps - ref) / np.linalg.norm(ref) <= 1e-3


# ------------------------------------------------------------------ stacked tensor-core tiles

def test_stacked_tensor_core_tiles_match_the_oracle():
    """4x6 grid, 14 cycles, 1024 batches (+5 in a ragged second group): the in-place batch
    step (10,8,5,7) runs, in turn, every tensor-core variant it has (autotune = k cycles the
    variants by step), among them the stacked tiles that put 2 or 4 batches reading the same
    stored block side by side in one 128- or 64-column tile; every amplitude against the
    oracle's state vector for each."""
    P = pkg()
    circ = cg.sycamore_grid(4, 6, 14, seed=0)
    openq = cg.default_open_qubits(4, 6, 6)
    C = P.circuit_load(circ.serialize())
    cb = cg.random_closed_bits(1024 + 5, 18, seed=7)
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 24, openq, cb)
    slices = np.arange(1, dtype=np.uint64)
    seen = set()
    for k in range(2, 7):
        plan = P.plan(C, openq, log2_batches=10, order_trials=16, precision=P.tn.PREC_BF16X2, autotune=k)
        plan.trace(True)
        amps = plan.contract(slices, cb)
        tr = plan.trace_read()
        plan.trace(False)
        rel = float(np.linalg.norm(amps - ref) / np.linalg.norm(ref))
        kinds = sorted({s["kernel"] for s in tr if s["kernel"] in TC_IDS and s["in_place"] and s["launches"]})
        print("autotune %d: in-place tensor-core kernels %s, relative L2 %.2e" % (k, kinds, rel))
        assert rel <= 1e-3, (k, kinds, rel)
        seen.update(kinds)
        del plan
    assert {19128, 19064} <= seen, "stacked variants never ran: %s" % sorted(seen)

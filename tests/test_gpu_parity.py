"""GPU parity of the CUDA path (through the C-ABI) against the CPU oracle.

Tolerances: complex64 contractions must match the FP64 oracle within
max|a - a_ref| <= 1e-4 * RMS(a_ref) over every compared amplitude; FP64 paths (norms)
within 1e-12; integer / index outputs (slice cut, Philox draws, sampler decisions)
bit-exact given identical inputs.
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
    return err / rms


# ------------------------------------------------------------------ contraction

def test_12q_all_amplitudes_two_slices():
    """3x4 grid, 8 cycles, all 12 qubits open, 2 sliced legs: all 4096 amplitudes."""
    P = pkg()
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, list(range(12)), n_auto_sliced=2, log2_batches=0)
    sl = plan.sliced_edges()
    assert len(sl) == 2
    amps = plan.contract(np.arange(4, dtype=np.uint64), [0])
    psi = oracle.simulate(circ)
    close_c64(amps[0], psi)
    for s in range(4):
        one = plan.contract(np.array([s], np.uint64), [0])
        ref = oracle.simulate(circ, [(q, g, (s >> e) & 1) for e, (q, g) in enumerate(sl)])
        close_c64(one[0], ref if np.abs(ref).max() > 0 else psi)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
def test_haar_batches_ragged_groups_and_slice_subsets(seed):
    """Generic gates, 3 open qubits, T = 8 per group, 13 batches (two groups, ragged)."""
    P = pkg()
    n = 10
    circ = cg.random_haar(n, 70, seed=seed, p_two=0.75)
    openq = [7, 1, 4]
    closed = oracle.closed_of(n, openq)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=4, log2_batches=3, order_trials=8)
    sl = plan.sliced_edges()
    cb = cg.random_closed_bits(13, len(closed), seed=seed + 10)
    psi = oracle.simulate(circ)
    amps = plan.contract(np.arange(16, dtype=np.uint64), cb)
    close_c64(amps, oracle.batch_amplitudes(psi, n, openq, cb))
    sub = np.array([9, 2, 14, 5], dtype=np.uint64)
    amps = plan.contract(sub, cb)
    close_c64(amps, oracle.batch_amplitudes(oracle.sliced_state(circ, sl, sub), n, openq, cb))


def test_20q_many_groups_device_buffers(gpu):
    torch = gpu
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 10, seed=2)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=6, log2_batches=4, order_trials=16)
    cb = cg.random_closed_bits(50, 14, seed=5)
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 20, openq, cb)
    slices = np.arange(64, dtype=np.uint64)
    out = plan.contract(slices, torch.from_numpy(cb.astype(np.int64)).cuda())
    close_c64(out.cpu().numpy(), ref)
    close_c64(plan.contract(slices, cb), ref)


@pytest.fixture(scope="module")
def grid28():
    circ = cg.sycamore_grid(4, 7, 14, seed=0)
    psi = oracle.simulate(circ)
    return circ, psi


def test_28q_256_batches_full_slice_set(grid28):
    """The 4x7 / 14-cycle workload: 2^10 slices, 256 batches of 64, all amplitudes."""
    P = pkg()
    circ, psi = grid28
    openq = cg.default_open_qubits(4, 7, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=10, log2_batches=8, order_trials=256)
    cb = cg.random_closed_bits(256, 22, seed=1)
    amps = plan.contract(np.arange(1024, dtype=np.uint64), cb)
    close_c64(amps, oracle.batch_amplitudes(psi, 28, openq, cb))


@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
def test_28q_bench_configuration_16384_batches(grid28, prec):
    """The benchmark's launch configuration: 4x7 grid, 14 cycles, 2^10 slices, one group
    of 16384 batches of 64 (batch-independent intermediates shared by all of them), the
    same plan options; every amplitude against the state vector."""
    P = pkg()
    circ, psi = grid28
    openq = cg.default_open_qubits(4, 7, 6)
    C = P.circuit_load(circ.serialize())
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    plan = P.plan(C, openq, n_auto_sliced=10, log2_batches=14, order_trials=256, order_seed=0,
                  hbm_budget_bytes=200e9, precision=precision)
    cb = cg.random_closed_bits(16384, 22, seed=3)
    amps = plan.contract(np.arange(1024, dtype=np.uint64), cb)
    ref = oracle.batch_amplitudes(psi, 28, openq, cb)
    if prec == "c64":
        close_c64(amps, ref)
    else:
        err = split_errors(amps, ref)
        assert err["rel_l2"] <= 1e-3, err


@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
def test_every_kernel_variant(prec):
    """autotune = k >= 2 runs variant (step + k - 2) mod count at every step, so ten plans
    cover every FFMA tile, the row kernel, the staged row kernel, the staged small-product
    kernel and every tensor-core tile width at the shapes of a 20-qubit plan with 1024
    batches per group (at most ten candidates per step)."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=1)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    cb = cg.random_closed_bits(1024, 14, seed=9)
    ref = oracle.batch_amplitudes(oracle.simulate(circ), 20, openq, cb)
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    for k in range(2, 12):
        plan = P.plan(C, openq, n_auto_sliced=6, log2_batches=10, order_trials=16, precision=precision, autotune=k)
        amps = plan.contract(np.arange(64, dtype=np.uint64), cb)
        if prec == "c64":
            close_c64(amps, ref)
        else:
            err = split_errors(amps, ref)
            assert err["rel_l2"] <= 1e-3, (k, err)
        del plan


@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
def test_autotuned_equals_fixed_rules(prec):
    """Every variant accumulates each output over k in the same order, so the timed
    choice gives exactly the amplitudes of the fixed shape rules."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=1)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    cb = cg.random_closed_bits(1024, 14, seed=9)
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    out = []
    for mode in (0, 1):
        plan = P.plan(C, openq, n_auto_sliced=6, log2_batches=10, order_trials=16, precision=precision, autotune=mode)
        out.append(plan.contract(np.arange(64, dtype=np.uint64), cb))
        del plan
    assert np.array_equal(out[0], out[1])


def split_errors(got, ref):
    d = np.abs(got - ref)
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    rel_l2 = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"max_over_rms": float(d.max()) / rms, "rms_err_over_rms": float(np.sqrt(np.mean(d ** 2))) / rms,
            "rel_l2": rel_l2}


def test_28q_bf16x2_split_full_slice_set(grid28):
    """Split BF16 hi+lo on tcgen05 (3 products, FP32 accumulation): relative L2 <= 1e-3."""
    P = pkg()
    circ, psi = grid28
    openq = cg.default_open_qubits(4, 7, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=10, log2_batches=8, order_trials=256, precision=P.tn.PREC_BF16X2)
    cb = cg.random_closed_bits(256, 22, seed=1)
    amps = plan.contract(np.arange(1024, dtype=np.uint64), cb)
    ref = oracle.batch_amplitudes(psi, 28, openq, cb)
    err = split_errors(amps, ref)
    print("bf16x2 28q:", err)
    assert err["rel_l2"] <= 1e-3, err
    # the linear XEB of the computed distribution against the exact one (all batches)
    p_got = np.abs(amps) ** 2
    p_ref = np.abs(ref) ** 2
    assert abs(np.sum(p_got * p_ref) / np.sum(p_ref * p_ref) - 1) < 2e-3


@pytest.mark.parametrize("prec", ["bf16x2", "fp16x2"])
@pytest.mark.parametrize("seed", [0, 1])
def test_split_haar_batches_and_subsets(seed, prec):
    """Generic gates with the split paths: big enough steps go to the tensor cores; the
    fp16 path calibrates per-tensor scales on its first execution."""
    P = pkg()
    n = 16
    circ = cg.random_haar(n, 150, seed=seed, p_two=0.8)
    openq = [3, 9, 12, 1, 15, 6]
    closed = oracle.closed_of(n, openq)
    C = P.circuit_load(circ.serialize())
    precision = {"bf16x2": P.tn.PREC_BF16X2, "fp16x2": P.tn.PREC_FP16X2}[prec]
    plan = P.plan(C, openq, n_auto_sliced=4, log2_batches=6, order_trials=16, precision=precision)
    sl = plan.sliced_edges()
    cb = cg.random_closed_bits(100, len(closed), seed=seed + 3)
    psi = oracle.simulate(circ)
    amps = plan.contract(np.arange(16, dtype=np.uint64), cb)
    err = split_errors(amps, oracle.batch_amplitudes(psi, n, openq, cb))
    assert err["rel_l2"] <= 1e-3, err
    sub = np.array([3, 12, 7], dtype=np.uint64)
    amps = plan.contract(sub, cb)
    err = split_errors(amps, oracle.batch_amplitudes(oracle.sliced_state(circ, sl, sub), n, openq, cb))
    assert err["rel_l2"] <= 1e-3, err


def test_28q_precision_report(grid28):
    """The 28-qubit 4x7, 14-cycle workload at 256 batches in complex64, bf16 x2 and fp16 x2
    against the FP64 oracle: per-amplitude error (max and RMS, relative to the RMS amplitude),
    relative L2 and the linear-XEB deviation of the computed distribution."""
    P = pkg()
    circ, psi = grid28
    openq = cg.default_open_qubits(4, 7, 6)
    C = P.circuit_load(circ.serialize())
    cb = cg.random_closed_bits(256, 22, seed=1)
    ref = oracle.batch_amplitudes(psi, 28, openq, cb)
    p_ref = np.abs(ref) ** 2
    report = {}
    for name, prec in (("c64", P.tn.PREC_C64), ("bf16x2", P.tn.PREC_BF16X2), ("fp16x2", P.tn.PREC_FP16X2)):
        plan = P.plan(C, openq, n_auto_sliced=10, log2_batches=8, order_trials=256, precision=prec)
        amps = plan.contract(np.arange(1024, dtype=np.uint64), cb)
        err = split_errors(amps, ref)
        p_got = np.abs(amps) ** 2
        err["xeb_dev"] = float(abs(np.sum(p_got * p_ref) / np.sum(p_ref * p_ref) - 1))
        report[name] = err
        del plan
    for name, err in report.items():
        print("precision %-7s max/rms %.2e  rms/rms %.2e  relL2 %.2e  xeb_dev %.2e" % (
            name, err["max_over_rms"], err["rms_err_over_rms"], err["rel_l2"], err["xeb_dev"]))
    assert report["c64"]["max_over_rms"] <= TOL_C64
    for name in ("bf16x2", "fp16x2"):
        assert report[name]["rel_l2"] <= 1e-3 and report[name]["xeb_dev"] <= 2e-3
    # fp16 keeps 11 mantissa bits per part, bf16 8, but at this workload's long K (up to
    # 2^15) the FP32 accumulation in TMEM dominates both: they agree within 10%
    assert report["fp16x2"]["rel_l2"] < 1.1 * report["bf16x2"]["rel_l2"]


def test_28q_single_slice_sampled(grid28):
    """One slice at full size, checked against the oracle's projector simulation."""
    P = pkg()
    circ, _ = grid28
    openq = cg.default_open_qubits(4, 7, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=10, log2_batches=4, order_trials=64)
    sl = plan.sliced_edges()
    s = 0b1011001101
    cb = cg.random_closed_bits(16, 22, seed=7)
    amps = plan.contract(np.array([s], np.uint64), cb)
    ref_state = oracle.simulate(circ, [(q, g, (s >> e) & 1) for e, (q, g) in enumerate(sl)])
    ref = oracle.batch_amplitudes(ref_state, 28, openq, cb)
    if np.abs(ref).max() > 0:
        close_c64(amps, ref)
    else:
        assert np.abs(amps).max() < 1e-6


def test_bad_slices_rejected():
    P = pkg()
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, list(range(12)), n_auto_sliced=2, log2_batches=0)
    with pytest.raises(P.TnError) as e:
        plan.contract(np.array([1, 1], np.uint64), [0])
    assert e.value.code == P.tn.TN_EINVAL
    with pytest.raises(P.TnError):
        plan.contract(np.array([4], np.uint64), [0])  # bit beyond |I|


def test_hbm_budget_enforced():
    P = pkg()
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, list(range(12)), n_auto_sliced=2, log2_batches=0, hbm_budget_bytes=1024.0)
    with pytest.raises(P.TnError) as e:
        plan.contract(np.arange(4, dtype=np.uint64), [0])
    assert e.value.code == P.tn.TN_ENOMEM


# ------------------------------------------------------------------ selection

@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
@pytest.mark.parametrize("grid,f", [((3, 4, 8), 0.25), ((4, 5, 12), 1 / 64)])
def test_partial_norms(grid, f, prec):
    """R of Fig. 1's network in the plan's contraction precision: within 1e-4 (complex64)
    or 1e-3 (split) of max R; S identical to the oracle's Alg. 2.  R is quadratic in the
    amplitudes of C1, so the complex64 amplitude bound (1e-4 of the RMS) allows about
    twice that relative error in R; 1e-4 of max R is the matching bound."""
    P = pkg()
    circ = cg.sycamore_grid(*grid, seed=0)
    n = grid[0] * grid[1]
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(n) for s in range(1, view.n2q[q] - 1)]
    C = P.circuit_load(circ.serialize())
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    plan = P.plan(C, cg.default_open_qubits(grid[0], grid[1], 6), sliced=I[:40], log2_batches=2,
                  precision=precision)
    S_idx, R = plan.partial_norms(f)
    S_ref = oracle.sliced_vertex_select(circ, I[:40], oracle.k0_for(f))
    assert [I[i] for i in S_idx] == S_ref
    R_ref = oracle.norms(circ, S_ref)
    tol = 1e-4 if prec == "c64" else 1e-3
    assert np.abs(R - R_ref).max() < tol * R_ref.max()
    assert abs(R.sum() - 1) < tol


@pytest.mark.parametrize("k,f", [(4, 0.3), (10, 0.02), (12, 0.002), (10, 0.999)])
def test_slice_cut_bit_exact(k, f):
    P = pkg()
    rng = np.random.default_rng(k)
    R = rng.exponential(size=1 << k)
    R[5] = R[9]  # a tie, broken by index
    R /= R.sum()
    X, F = P.slice_cut(R, f)
    Xr, Fr = oracle.select_slices(R, f)
    assert list(X) == list(Xr)
    assert F == Fr


@pytest.mark.parametrize("prec", ["c64", "bf16x2"])
def test_select_partial_state_20q(prec):
    """Alg. 1 end to end (GPU norms + cut), then the partial contraction of Sec. I.C; the
    partial legs are explicit versions (folded into the tensor-core tiles when small)."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    I = [(q, s) for q in range(20) for s in range(2, view.n2q[q] - 1)][:12]
    precision = {"c64": P.tn.PREC_C64, "bf16x2": P.tn.PREC_BF16X2}[prec]
    plan = P.plan(C, openq, sliced=I, log2_batches=4, order_trials=16, precision=precision)
    f = 0.25
    slices, F = plan.select(f)
    S_ref, X_ref, F_ref, R_ref = oracle.slice_selection(circ, I, f)
    # R from complex64 / split contractions: F within 1e-5 / 1e-3; X identical (no
    # near-ties here)
    assert abs(F - F_ref) < (1e-5 if prec == "c64" else 1e-3)
    k = len(S_ref)
    assert len(slices) == len(X_ref) << (len(I) - k)
    cb = cg.random_closed_bits(20, 14, seed=3)
    amps = plan.contract(slices, cb)
    ref = oracle.batch_amplitudes(oracle.partial_state(circ, S_ref, X_ref), 20, openq, cb)
    if prec == "c64":
        close_c64(amps, ref)
    else:
        assert split_errors(amps, ref)["rel_l2"] <= 1e-3


# ------------------------------------------------------------------ sampler

def test_draw_batches_bit_exact():
    P = pkg()
    for b_bits in (0, 6, 22, 40):
        j = P.draw_batches(123, 1000, 3000, b_bits).cpu().numpy().astype(np.uint64)
        ref = oracle.batch_draws(123, 3000, b_bits, t0=1000)
        assert np.array_equal(j, ref)


def sampler_cases():
    rng = np.random.default_rng(0)
    T = 4096
    p = rng.exponential(size=(T, 64)) / (64 * 2 ** 12)
    p[0] = 0.0                      # empty batch: never accepted
    p[1] = 0.0
    p[1, 17] = 1e-3                 # single mass point
    p[2, ::2] = 0.0                 # zeros interleaved
    p[3] *= 50                      # clipped batch (p_j N_B > alpha)
    p[4, :] = 1.0 / (64 * 4096)     # uniform
    return p


@pytest.mark.parametrize("alpha,seed,t0", [(2.0, 1, 0), (1.5, 99, 123456789), (8.0, 2 ** 63 + 5, 7)])
def test_sampler_bit_identical(gpu, alpha, seed, t0):
    torch = gpu
    P = pkg()
    p = sampler_cases()
    acc, pick = P.rejection_sample(torch.from_numpy(p).cuda(), 12, alpha, seed, t0)
    acc_r, pick_r = oracle.sample_batches(p, 12, alpha, seed, t0=t0)
    assert np.array_equal(acc.cpu().numpy().astype(bool), acc_r)
    assert np.array_equal(pick.cpu().numpy(), pick_r)
    assert not acc_r[0] and pick_r[1] == 17


def test_sample_end_to_end_12q():
    """tn_sample at full fidelity vs the oracle sampler on the exact distribution: the
    draws use the same Philox streams, so all but near-threshold decisions agree."""
    P = pkg()
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    openq = cg.default_open_qubits(3, 4, 6)
    C = P.circuit_load(circ.serialize())
    plan = P.plan(C, openq, n_auto_sliced=2, log2_batches=6, order_trials=16)
    N = 2000
    bits, st = plan.sample(1.0, N, seed=11, alpha=2.0)
    p = np.abs(oracle.simulate(circ)) ** 2
    ref, steps, eps_hat = oracle.sample(p, 12, openq, N, seed=11, alpha=2.0, chunk=64)
    assert st["F"] == 1.0 and st["accepted"] >= N
    same = np.mean(bits.astype(np.int64) == ref)
    assert same > 0.99, same
    assert abs(st["eps_hat"] - eps_hat) < 1e-6


@pytest.mark.slow
def test_sample_xeb_tracks_fidelity_20q():
    """Sampling at partial fidelity: the linear XEB of the GPU samples ~ F (Table elided)."""
    P = pkg()
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    openq = cg.default_open_qubits(4, 5, 6)
    C = P.circuit_load(circ.serialize())
    I = [(q, s) for q in range(20) for s in range(2, view.n2q[q] - 1)][:12]
    plan = P.plan(C, openq, sliced=I, log2_batches=8, order_trials=16)
    N = 40000
    bits, st = plan.sample(0.25, N, seed=5, alpha=2.0)
    p = np.abs(oracle.simulate(circ)) ** 2
    xeb = oracle.xeb_of_samples(p, 20, bits.astype(np.int64))
    sigma = math.sqrt(2.0 / N)  # Porter-Thomas: Var(2^n p) ~ 1 (+ F terms)
    assert abs(xeb - st["F"]) < 4 * sigma + 0.02 * st["F"], (xeb, st["F"])

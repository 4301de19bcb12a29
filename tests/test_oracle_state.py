"""Pins of the oracle's state-vector part against mathematics it does not itself use:
dense-matrix products, an independent Feynman path sum, unitarity, norm and the
resolution of identity over slices (Sec. I.A, Sec. I.C)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg


def embed(U, qubits, n):
    """Dense 2^n x 2^n operator of a gate (basis index of a 2q gate = 2*bit(q0)+bit(q1))."""
    N = 1 << n
    M = np.zeros((N, N), dtype=np.complex128)
    k = len(qubits)
    for col in range(N):
        sub_in = 0
        for t, q in enumerate(qubits):
            sub_in |= ((col >> q) & 1) << (k - 1 - t)
        for sub_out in range(1 << k):
            row = col
            for t, q in enumerate(qubits):
                b = (sub_out >> (k - 1 - t)) & 1
                row = (row & ~(1 << q)) | (b << q)
            M[row, col] += U[sub_out, sub_in]
    return M


def dense_state(circ):
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for g in circ.gates:
        psi = embed(g.matrix, g.qubits, n) @ psi
    return psi


def path_sum_amplitude(circ, out_bits):
    """<b|C|0> as a Feynman sum over the values of every internal wire segment."""
    n = circ.n_qubits
    # label every wire segment: initial segment of each qubit, then one per gate output
    cur = list(range(n))
    nseg = n
    gates = []
    for g in circ.gates:
        ins = [cur[q] for q in g.qubits]
        outs = []
        for q in g.qubits:
            cur[q] = nseg
            outs.append(nseg)
            nseg += 1
        gates.append((g.matrix, ins, outs))
    final = {cur[q]: (out_bits >> q) & 1 for q in range(n)}
    initial = {q: 0 for q in range(n)}
    free = [s for s in range(nseg) if s not in final and s not in initial]
    total = 0j
    for vals in itertools.product((0, 1), repeat=len(free)):
        val = dict(initial)
        val.update(final)
        val.update(zip(free, vals))
        term = 1 + 0j
        for (U, ins, outs) in gates:
            k = len(ins)
            r = 0
            c = 0
            for t in range(k):
                r = (r << 1) | val[outs[t]]
                c = (c << 1) | val[ins[t]]
            term *= U[r, c]
            if term == 0:
                break
        total += term
    return total


def test_generated_gates_are_unitary():
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    for g in circ.gates:
        d = g.matrix.shape[0]
        assert np.abs(g.matrix.conj().T @ g.matrix - np.eye(d)).max() < 1e-14


def test_abcd_gate_counts():
    # ABCD reading of the coupler pattern: counts per grid
    c1 = cg.sycamore_grid(3, 4, 8, seed=0)
    assert (c1.n_two_qubit(), c1.n_one_qubit()) == (34, 108)
    c2 = cg.sycamore_grid(4, 7, 14, seed=0)
    assert (c2.n_two_qubit(), c2.n_one_qubit()) == (156, 420)
    c4 = cg.sycamore_grid(5, 8, 16, seed=0)
    assert (c4.n_two_qubit(), c4.n_one_qubit()) == (268, 680)


def test_sqrt_gates_square_to_paulis():
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    W = (X + Y) / math.sqrt(2)
    for f, P in ((cg.sqrt_x, X), (cg.sqrt_y, Y), (cg.sqrt_w, W)):
        U = f()
        # exp(-i pi/4 P)^2 = exp(-i pi/2 P) = -i P
        assert np.allclose(U @ U, -1j * P, atol=1e-15)


def test_serialization_roundtrip():
    circ = cg.random_haar(5, 30, seed=3)
    back = cg.deserialize(circ.serialize())
    assert back.n_qubits == 5 and len(back.gates) == 30
    for a, b in zip(circ.gates, back.gates):
        assert a.qubits == b.qubits and np.array_equal(a.matrix, b.matrix)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_state_matches_dense_operator_product(seed):
    circ = cg.random_haar(5, 25, seed=seed)
    psi = oracle.simulate(circ)
    ref = dense_state(circ)
    assert np.abs(psi - ref).max() < 1e-13


def test_state_matches_dense_on_grid():
    circ = cg.sycamore_grid(2, 3, 6, seed=4)
    assert np.abs(oracle.simulate(circ) - dense_state(circ)).max() < 1e-13


@pytest.mark.parametrize("seed", [0, 5])
def test_state_matches_path_sum(seed):
    circ = cg.random_haar(3, 7, seed=seed)
    psi = oracle.simulate(circ)
    for b in range(8):
        assert abs(psi[b] - path_sum_amplitude(circ, b)) < 1e-12


def test_norm_is_one_on_12q():
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    psi = oracle.simulate(circ)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12


def internal_segments(circ):
    cnt = oracle.two_qubit_counts(circ)
    return [(q, s) for q in range(circ.n_qubits) for s in range(1, cnt[q])]


@pytest.mark.parametrize("seed", [0, 1])
def test_sum_over_all_slices_is_unsliced(seed):
    circ = cg.random_haar(5, 30, seed=seed, p_two=0.8)
    segs = internal_segments(circ)
    rng = np.random.default_rng(seed)
    edges = [segs[i] for i in rng.choice(len(segs), size=3, replace=False)]
    total = oracle.sliced_state(circ, edges, range(8))
    assert np.abs(total - oracle.simulate(circ)).max() < 1e-13


def test_sum_over_slices_12q_two_edges():
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    edges = [(5, 2), (6, 3)]
    total = oracle.sliced_state(circ, edges, range(4))
    assert np.abs(total - oracle.simulate(circ)).max() < 1e-13


def test_projector_value_zero_plus_one_is_identity_on_single_wire():
    circ = cg.random_haar(4, 20, seed=9, p_two=0.9)
    q, s = internal_segments(circ)[0]
    a = oracle.simulate(circ, [(q, s, 0)])
    b = oracle.simulate(circ, [(q, s, 1)])
    psi = oracle.simulate(circ)
    assert np.abs(a + b - psi).max() < 1e-13
    # slices of one wire are orthogonal only across a cut; a single wire is always a cut
    assert abs(np.vdot(a, b)) < 1e-13


def test_bad_segment_rejected():
    circ = cg.random_haar(3, 6, seed=1)
    cnt = oracle.two_qubit_counts(circ)
    with pytest.raises(ValueError):
        oracle.simulate(circ, [(0, cnt[0] + 1, 0)])

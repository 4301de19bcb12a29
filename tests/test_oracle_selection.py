"""Pins of the oracle's slice-selection part (Sec. I.A-B, App. B Alg. 1-2):
hand-derived lightcones, the orthogonality of the psi_i across a cut, F = sum_X R,
sum R = 1, the size bound on X, and the linear XEB ~ F claim (Table elided)."""
import math

import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg


def chain_circuit():
    """3 qubits: g0 = (0,1), g1 = (1,2), g2 = (0,1), g3 = (1,2) (Haar gates)."""
    rng = np.random.default_rng(11)
    c = cg.Circuit(n_qubits=3)
    for pair in ((0, 1), (1, 2), (0, 1), (1, 2)):
        c.gates.append(cg.Gate(pair, cg.haar_unitary(4, rng)))
    return c


def test_merged_view_lightcones_by_hand():
    v = oracle.MergedView(chain_circuit())
    # segment counts: q0 two 2q gates, q1 four, q2 two
    assert v.n2q == [2, 4, 2]
    # output of qubit 2, (2,2), comes from g3 which depends on g1, g2, and g0 via g1/g2
    assert v.lightcone((2, 2)) == {0, 1, 2, 3}
    # (2,1) is the output of g1 = gates {g0, g1}
    assert v.lightcone((2, 1)) == {0, 1}
    # (0,1) is g0's output on qubit 0: lightcone {g0}
    assert v.lightcone((0, 1)) == {0}
    # inputs of {g0, g1}: (0,0), (1,0), (1,1), (2,0)
    assert v.lightcone_inputs([(2, 1)]) == {(0, 0), (1, 0), (1, 1), (2, 0)}
    assert v.lightcone((1, 0)) == set()


def test_causal_past_by_hand():
    c = chain_circuit()
    # wire point (2,1) is just before g3: its past is g1 (on q2) and g0 (feeds g1 on q1)
    assert list(oracle.causal_past(c, [(2, 1)])) == [1, 1, 0, 0]
    # wire point (0,1), just before g2 on q0: past {g0}
    assert list(oracle.causal_past(c, [(0, 1)])) == [1, 0, 0, 0]


def test_sliced_vertex_select_by_hand():
    c = chain_circuit()
    # candidates with their own |L'|: (0,1): {g0} -> 2 inputs; (2,1) and (1,2) are the
    # outputs of g1: {g0,g1} -> 4 inputs each.
    S = oracle.sliced_vertex_select(c, [(2, 1), (0, 1), (1, 2)], 2)
    # greedy: first (0,1) (|L'| = 2); then (2,1) and (1,2) tie at 4 -> first in I
    assert S == [(0, 1), (2, 1)]
    # a third vertex: (1,2) is another output of g1, outside L'(S): the three wires
    # after {g0, g1} form a cut
    S3 = oracle.sliced_vertex_select(c, [(2, 1), (0, 1), (1, 2)], 3)
    assert S3 == [(0, 1), (1, 2), (2, 1)]
    # a later vertex that depends on a chosen one replaces it: (2,2) depends on every
    # gate, so (0,1) in L'((2,2)) is dropped and nothing else is eligible
    assert oracle.sliced_vertex_select(c, [(0, 1), (2, 2)], 2) == [(2, 2)]


def antichain(view, S):
    for u in S:
        lp = view.lightcone_inputs([u])
        for v in S:
            if v != u and v in lp:
                return False
    return True


@pytest.mark.parametrize("k", [2, 4, 6])
def test_selected_vertices_form_a_cut(k):
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(12) for s in range(1, view.n2q[q])]
    S = oracle.sliced_vertex_select(circ, I, k)
    assert len(S) == k
    assert antichain(view, S)
    assert len({q for q, _ in S}) == k  # a cut meets every wire at most once


def small_cut_case():
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(12) for s in range(2, view.n2q[q])]
    S = oracle.sliced_vertex_select(circ, I, 4)
    return circ, S


def test_norms_sum_to_one_and_match_projected_states():
    circ, S = small_cut_case()
    R = oracle.norms(circ, S)
    assert abs(R.sum() - 1.0) < 1e-12
    # ||psi_i||^2 computed the long way: full circuit with projectors on the S wires
    states = []
    for i in range(1 << len(S)):
        proj = [(q, s, (i >> t) & 1) for t, (q, s) in enumerate(S)]
        psi_i = oracle.simulate(circ, proj)
        states.append(psi_i)
        assert abs(np.vdot(psi_i, psi_i).real - R[i]) < 1e-12
    # orthogonality across the cut (Sec. I.A)
    for a in range(len(states)):
        for b in range(a + 1, len(states)):
            assert abs(np.vdot(states[a], states[b])) < 1e-12


def test_partial_state_is_sum_of_projected_states():
    circ, S = small_cut_case()
    rng = np.random.default_rng(1)
    X = rng.choice(1 << len(S), size=5, replace=False)
    psi_x = oracle.partial_state(circ, S, X)
    ref = np.zeros_like(psi_x)
    for i in X:
        ref += oracle.simulate(circ, [(q, s, (int(i) >> t) & 1) for t, (q, s) in enumerate(S)])
    assert np.abs(psi_x - ref).max() < 1e-13
    R = oracle.norms(circ, S)
    # F = ||psi_X||^2 = sum_{i in X} R[i]  (Eq. partial-fidelity)
    assert abs(np.vdot(psi_x, psi_x).real - R[X].sum()) < 1e-12


@pytest.mark.parametrize("f", [0.05, 0.2, 0.5, 0.9])
def test_selection_bounds(f):
    rng = np.random.default_rng(7)
    k = 8
    R = rng.exponential(size=1 << k)
    R /= R.sum()
    X, F = oracle.select_slices(R, f)
    assert F >= f
    assert len(X) <= math.ceil(f * (1 << k))          # |X| <= ceil(f 2^k)
    assert F >= len(X) / (1 << k)                      # Eq. partial-fidelity
    assert R[X[:-1]].sum() < f                         # minimal
    assert abs(F - R[X].sum()) < 1e-12
    # X are the largest norms
    assert R[X].min() >= np.sort(R)[::-1][len(X) - 1]


def test_selection_ties_and_rounding():
    R = np.full(8, 1.0 / 8)
    X, F = oracle.select_slices(R, 0.25)
    assert list(X) == [0, 1] and abs(F - 0.25) < 1e-15
    # total below f through rounding -> all indices
    X, F = oracle.select_slices(np.full(4, 0.2), 0.9)
    assert list(X) == [0, 1, 2, 3]


def test_k0_values_from_paper():
    import json, os
    here = os.path.dirname(__file__)
    cases = json.load(open(os.path.join(here, "golden", "paper_examples.json")))["k0_alg1"]["cases"]
    for f, k0 in cases:
        assert oracle.k0_for(f) == k0


@pytest.mark.slow
def test_xeb_tracks_fidelity_20q():
    """Table elided: linear XEB of the partial state ~ F.  With p' = |psi_X|^2/F the
    expected Eq. 1 value under Porter-Thomas statistics is F; at 2^20 amplitudes the
    spread is ~1e-3 absolute."""
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(20) for s in range(1, view.n2q[q] - 1)]
    S, X, F, R = oracle.slice_selection(circ, I, 0.25)
    psi = oracle.simulate(circ)
    p = np.abs(psi) ** 2
    psi_x = oracle.partial_state(circ, S, X)
    px = np.abs(psi_x) ** 2 / F
    assert abs(px.sum() - 1.0) < 1e-12
    xeb = oracle.xeb_exact(p, px, 20)
    assert 0.25 <= F < 0.25 + 2.0 ** -len(S) * R.max() * (1 << len(S))
    assert abs(xeb - F) < 0.05 * F + 3e-3

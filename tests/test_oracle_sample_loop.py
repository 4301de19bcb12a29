"""Pins of the oracle's sampling loop (Sec. II.A, Sec. II.C) and of XEB ~ F at 28 qubits.

* The output is the accepted strings in step order t, truncated to N: with batches whose
  acceptance is certain (N_B p_j = alpha) or impossible (p_j = 0) and whose mass sits on
  one string, the accepted steps are exactly those whose Philox batch draw (pinned by the
  published known-answer vectors) lands on a massive batch, so the expected output is
  fixed by the draws alone.
* epsilon_hat is the per-step mean of the clipped excess max(p_j - alpha/N_B, 0)
  (Sec. II.C, read as a per-batch mean): batches below the threshold contribute zero.
* Table elided: the exact linear XEB of the normalised partial state |psi_X>/sqrt(F)
  against the exact state is F, here at 28 qubits with Alg. 1 at f = 1/64.
"""
import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg

N_QUBITS = 8
OPEN = [0, 1, 2, 3, 4, 5]
CLOSED = [6, 7]  # N_B = 4 batches of 64


def two_point_law(mass_j1, mass_j3):
    """All of batch 1's mass on in-batch index 9, all of batch 3's on index 40."""
    p = np.zeros(1 << N_QUBITS)
    p[oracle.bitstring(9, 1, OPEN, CLOSED)] = mass_j1
    p[oracle.bitstring(40, 3, OPEN, CLOSED)] = mass_j3
    return p


def test_bitstring_layout_by_hand():
    # in-batch index 9 = 0b001001 -> qubits 0 and 3; batch 1 -> qubit 6; batch 3 -> 6 and 7
    assert oracle.bitstring(9, 1, OPEN, CLOSED) == (1 << 0) | (1 << 3) | (1 << 6)
    assert oracle.bitstring(40, 3, OPEN, CLOSED) == (1 << 3) | (1 << 5) | (1 << 6) | (1 << 7)


@pytest.mark.parametrize("seed,N,chunk", [(3, 25, 16), (77, 40, 7), (2 ** 40 + 1, 5, 64)])
def test_accepted_strings_in_step_order(seed, N, chunk):
    """alpha = 2, N_B = 4: batches 1 and 3 hold 1/2 each, so N_B p_j = alpha and u alpha <
    N_B p_j for every u in [0, 1); batches 0 and 2 are never accepted."""
    p = two_point_law(0.5, 0.5)
    out, steps, eps_hat = oracle.sample(p, N_QUBITS, OPEN, N, seed=seed, alpha=2.0, chunk=chunk)
    js = [int(j) for j in oracle.batch_draws(seed, steps, len(CLOSED))]
    want = [oracle.bitstring(9 if j == 1 else 40, j, OPEN, CLOSED) for j in js if j in (1, 3)]
    assert len(want) >= N
    assert [int(x) for x in out] == want[:N]
    # the loop stops at the first chunk boundary with N accepted
    steps_needed = next(t + 1 for t in range(steps) if sum(1 for j in js[: t + 1] if j in (1, 3)) == N)
    assert steps == chunk * ((steps_needed + chunk - 1) // chunk)
    assert eps_hat == 0.0  # no batch above alpha / N_B


@pytest.mark.parametrize("seed", [5, 6])
def test_eps_hat_is_mean_clipped_excess(seed):
    """Batch 1 holds 0.7 (excess 0.7 - 1/2 = 0.2), batch 3 holds 0.3 (below the threshold:
    no contribution), batches 0 and 2 nothing."""
    p = two_point_law(0.7, 0.3)
    _, steps, eps_hat = oracle.sample(p, N_QUBITS, OPEN, 30, seed=seed, alpha=2.0, chunk=32)
    js = oracle.batch_draws(seed, steps, len(CLOSED))
    n1 = int(np.count_nonzero(js == 1))
    assert n1 > 0 and abs(eps_hat - 0.2 * n1 / steps) < 1e-15


@pytest.mark.slow
def test_xeb_tracks_fidelity_28q_partial_slicing():
    """4x7 grid, 14 cycles: Alg. 1 at f = 1/64 (k0 = 9 cut vertices among the internal
    wire segments), |psi_X> = C2 Pi_X C1 |0>, p' = |psi_X|^2 / F.  Under Porter-Thomas
    statistics the exact Eq. 1 value of p' against p is F; at 2^28 amplitudes the
    statistical spread is far below the 5% allowed here."""
    circ = cg.sycamore_grid(4, 7, 14, seed=0)
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(28) for s in range(1, view.n2q[q] - 1)]
    f = 1.0 / 64
    S, X, F, R = oracle.slice_selection(circ, I, f)
    assert len(S) == 9
    assert f <= F and len(X) <= int(np.ceil(f * 512))
    p = np.abs(oracle.simulate(circ)) ** 2
    px = np.abs(oracle.partial_state(circ, S, X)) ** 2
    assert abs(px.sum() - F) < 1e-10
    px /= F
    xeb = oracle.xeb_exact(p, px, 28)
    del p, px
    assert abs(xeb - F) < 0.05 * F, (xeb, F)

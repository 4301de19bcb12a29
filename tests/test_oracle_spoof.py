"""Pins of the oracle's XEB spoofing recipe (Sec. III, "Spoofing Linear XEB"; App. A):
the batch-size rule and the top-N selection by hand, App. A's closed form -ln r for exact
Porter-Thomas probabilities, -f ln r when the approximation keeps a fraction f of the
norm, and the paper's observation XEB(S) - XEB(B) ~ -F ln r (about F at r = 0.36) on a
20-qubit circuit contracted at partial fidelity."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))
R_VALUES = GOLDEN["spoofing_appendix_A"]["r_values"]


def test_batch_bits_by_hand():
    """2^b is the smallest power of two holding 10 N strings."""
    assert oracle.spoof_batch_bits(1) == 4  # 10 -> 16
    assert oracle.spoof_batch_bits(100) == 10  # 1000 -> 1024
    assert oracle.spoof_batch_bits(103) == 11  # 1030 -> 2048
    assert oracle.spoof_batch_bits(1 << 20) == 24  # 10.5 M -> 16.8 M
    with pytest.raises(ValueError):
        oracle.spoof_batch_bits(0)


def test_select_by_hand():
    p = [0.2, 0.5, 0.1, 0.5, 0.7, 0.0]
    assert list(oracle.spoof_select(p, 3)) == [4, 1, 3]
    assert list(oracle.spoof_select(p, 0)) == []
    assert list(oracle.spoof_select(p, 6)) == [4, 1, 3, 0, 2, 5]
    with pytest.raises(ValueError):
        oracle.spoof_select(p, 7)


def test_xeb_of_a_selection_by_hand():
    """n = 2, exact probabilities (0.4, 0.1, 0.2, 0.3): strings {0, 3} score
    4 (0.4 + 0.3) / 2 - 1 = 0.4."""
    p = np.array([0.4, 0.1, 0.2, 0.3])
    assert abs(oracle.spoof_xeb(p, 2, [0, 3]) - 0.4) < 1e-15


@pytest.mark.parametrize("r", R_VALUES)
def test_exact_porter_thomas_top_fraction(r):
    """App. A at f = 1: with 2^n p_i ~ Exp(1) independent, the r N largest have
    E XEB = -ln r + O(ln N / N).  At N = 2^20 the mean of the r N largest values spreads
    by about 1/sqrt(r N) <= 3.1e-3."""
    rng = np.random.default_rng(7)
    n = 20
    p = rng.exponential(1.0, 1 << n) / 2.0 ** n
    sel = oracle.spoof_select(p, int(r * p.size))
    assert abs(oracle.spoof_xeb(p, n, sel) - oracle.spoof_expected_xeb(1.0, r)) < 0.015


@pytest.mark.parametrize("f", [0.5, 0.1])
@pytest.mark.parametrize("r", R_VALUES)
def test_partial_fidelity_top_fraction(f, r):
    """Eq. spoof-xeb: psi = psi' + psi_perp with independent complex Gaussian parts holding
    the fractions f and 1 - f of the norm (partial slicing under the paper's uniform-sphere
    assumption).  Selecting by |psi'|^2 and scoring with |psi|^2 gives
    E XEB = f (1 - ln r) + (1 - f) - 1 = -f ln r.  Selecting by |psi|^2 instead would give
    -ln r, and scoring with |psi'|^2 would give f (1 - ln r) - 1."""
    rng = np.random.default_rng(11)
    n = 20
    N = 1 << n

    def cgauss(var):
        s = math.sqrt(var / 2.0 / N)
        return rng.normal(0.0, s, N) + 1j * rng.normal(0.0, s, N)

    a, b = cgauss(f), cgauss(1.0 - f)
    sel = oracle.spoof_select(np.abs(a) ** 2, int(r * N))
    xeb = oracle.spoof_xeb(np.abs(a + b) ** 2, n, sel)
    assert abs(xeb - oracle.spoof_expected_xeb(f, r)) < 0.02


@pytest.mark.parametrize("f", [0.5, 0.25])
def test_20q_batches_gain_f_ln_r(f):
    """Sec. III: with the batch B computed at fidelity F and S its r |B| strings of largest
    approximate probability, XEB(S) - XEB(B) ~ -F ln r (about F at r = 0.36).  4x5 grid,
    12 cycles, 12 free outputs (2^12 strings per batch), 16 batches of random closed bits,
    F from Alg. 1.  The gain's standard error over the 16 batches is at most 0.023 (at
    r = 0.1); the bound is about three times that."""
    circ = cg.sycamore_grid(4, 5, 12, seed=0)
    view = oracle.MergedView(circ)
    I = [(q, s) for q in range(20) for s in range(1, view.n2q[q] - 1)]
    S, X, F, _R = oracle.slice_selection(circ, I, f)
    psi = oracle.simulate(circ)
    psi_x = oracle.partial_state(circ, S, X)
    openq = cg.default_open_qubits(4, 5, 12)
    closed = cg.random_closed_bits(16, 8, seed=3)
    amps = oracle.batch_amplitudes(psi, 20, openq, closed)
    ampx = oracle.batch_amplitudes(psi_x, 20, openq, closed)
    for r in R_VALUES:
        gains = []
        for t in range(len(closed)):
            p = np.abs(amps[t]) ** 2
            sel = oracle.spoof_select(np.abs(ampx[t]) ** 2, int(r * p.size))
            gains.append(oracle.spoof_xeb(p, 20, sel) - oracle.spoof_xeb(p, 20, np.arange(p.size)))
        assert abs(np.mean(gains) - oracle.spoof_expected_xeb(F, r)) < 0.06, (r, np.mean(gains), F)

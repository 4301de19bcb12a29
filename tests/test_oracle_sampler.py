"""Pins of the oracle's sampler part (Sec. II): Philox4x32-10 known answers
(Salmon et al., SC'11 test vectors), the output law p~ of Sec. II.A by a chi-square
test, the accept rate (1 - eps)/alpha, D(p, p~) <= eps (Eq. Dpp-eps), the fidelity
bound and its worked example (Sec. II.B), and E eps under Porter-Thomas (Sec. II.C)."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def test_philox_known_answers():
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    assert oracle.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == (
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
    assert oracle.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                [0xA4093822, 0x299F31D0]) == (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_uniform_draws_are_uniform():
    us = np.array([oracle.draw(5, t)[1] for t in range(20000)])
    vs = np.array([oracle.draw(5, t)[2] for t in range(20000)])
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    assert stats.kstest(vs, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(us, vs)[0, 1]) < 0.03


def law_case():
    # 8 qubits: 6 open (N_A = 64), 2 closed (N_B = 4); uneven batch masses so that
    # alpha = 1.5 clips the heaviest batch.
    rng = np.random.default_rng(3)
    p = rng.exponential(size=(4, 64))
    p[0] *= 3.0
    p /= p.sum()
    return p


def run_sampler(p, alpha, seed, steps):
    NB = p.shape[0]
    b_bits = int(math.log2(NB))
    js = oracle.batch_draws(seed, steps, b_bits)
    acc, pick = oracle.sample_batches(np.ascontiguousarray(p[js.astype(np.int64)]), b_bits, alpha, seed)
    return js.astype(np.int64), acc, pick


def test_output_law_chi_square():
    p = law_case()
    alpha = 1.5
    js, acc, pick = run_sampler(p, alpha, seed=11, steps=400000)
    law, eps = oracle.output_law(p, alpha, 4.0)
    assert eps > 0.01  # the clipped regime is exercised
    counts = np.zeros_like(p)
    np.add.at(counts, (js[acc], pick[acc]), 1)
    n = counts.sum()
    expected = law * n
    chi2 = ((counts - expected) ** 2 / expected).sum()
    pval = stats.chi2.sf(chi2, df=p.size - 1)
    assert pval > 1e-4
    # accept rate t = (1 - eps)/alpha (Sec. II.A)
    rate = acc.mean()
    t = (1 - eps) / alpha
    assert abs(rate - t) < 5 * math.sqrt(t * (1 - t) / acc.size)


def test_no_clipping_reproduces_p():
    p = law_case()
    alpha = 64.0  # alpha/N_B above every p_j: eps = 0 and p~ = p
    law, eps = oracle.output_law(p, alpha, 4.0)
    assert eps == 0.0 and np.allclose(law, p)


def test_pick_never_lands_on_zero_probability():
    p = np.zeros((16, 64))
    rng = np.random.default_rng(0)
    for t in range(16):
        nz = rng.choice(64, size=3, replace=False)
        p[t, nz] = rng.random(3)
    acc, pick = oracle.sample_batches(p, 4, 2.0, seed=1)
    for t in range(16):
        assert p[t, pick[t]] > 0


def test_zero_batch_never_accepted():
    p = np.zeros((8, 64))
    acc, _ = oracle.sample_batches(p, 4, 2.0, seed=2)
    assert not acc.any()


def test_single_mass_point():
    p = np.zeros((4, 64))
    p[:, 37] = 1.0
    acc, pick = oracle.sample_batches(p, 0, 2.0, seed=4)
    assert (pick == 37).all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_variation_distance_bounded_by_eps(seed):
    rng = np.random.default_rng(seed)
    p = rng.exponential(size=(16, 64)) ** 2
    p /= p.sum()
    for alpha in (1.2, 1.5, 2.0):
        law, eps = oracle.output_law(p, alpha, 16.0)
        assert abs(law.sum() - 1.0) < 1e-12
        assert oracle.variation_distance(p, law) <= eps + 1e-15


def test_worked_example_fidelity_bound():
    ex = GOLDEN["worked_example_sec_IIB"]
    f, eps, fp = ex["f"], ex["eps"], ex["f_prime"]
    assert eps < f / 16
    assert oracle.fidelity_lower_bound(f, eps) >= fp
    # and the bound is not trivially loose: with f = f' itself it fails
    assert oracle.fidelity_lower_bound(fp, eps) < fp


def test_expected_eps_porter_thomas_monte_carlo():
    # small batches so that clipping is frequent enough to measure
    NA, alpha, NB = 4, 1.5, 4096
    rng = np.random.default_rng(0)
    reps = 200
    vals = []
    for _ in range(reps):
        p = rng.exponential(size=(NB, NA))
        p /= NA * NB  # mean 1/2^n per bitstring, total ~1
        pj = p.sum(axis=1)
        vals.append(np.maximum(pj - alpha / NB, 0).sum())
    mc = float(np.mean(vals))
    exact = oracle.expected_eps_pt(NA, alpha)
    assert abs(mc - exact) < 0.03 * exact
    # the printed form N_B Q(N_A, alpha N_A) is far larger (a count, not a mass)
    assert oracle.paper_eps_bound(NA, NB, alpha) > 100 * exact


def test_expected_eps_batch64_alpha2_negligible():
    # Sec. I: with batches of 64 and alpha = 2 the distance is negligible
    assert oracle.expected_eps_pt(64, 2.0) < 1e-9

"""Pins of the oracle's cost model: the paper's own arithmetic for the Zuchongzhi
estimate (Sec. III.A), and the bound C_s(f) = |X|/2^k C_s(1) <= ceil(2^k f)/2^k C_s(1)
< (f + 2^-k) C_s(1) (Sec. I.B) for Alg. 1's selections on random norm vectors."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def test_zuchongzhi_estimate_reproduces_the_printed_time():
    g = GOLDEN["zuchongzhi_estimate_sec_IIIA"]
    t = oracle.sampling_time(g["flops_full"], g["fidelity"], g["peak_flops"], g["efficiency"])
    assert abs(t - g["seconds_printed"]) < 0.01 * g["seconds_printed"]  # printed rounded to 3.6e5
    assert round(t / 86400) == 4  # "about 4 days"


@pytest.mark.parametrize("k", [3, 6, 9])
@pytest.mark.parametrize("f", [0.002, 1 / 64, 0.1, 0.5])
def test_sliced_cost_bound(k, f):
    """Sec. I.B, with X from Alg. 1's cut of Dirichlet-random norms (they sum to 1)."""
    assert "C_s(f)" in GOLDEN["cost_bound_sec_IB"]["_cite"]
    rng = np.random.default_rng(k * 1000 + int(1e4 * f))
    for _ in range(20):
        R = rng.dirichlet(np.full(1 << k, 0.3))
        X, F = oracle.select_slices(R, f)
        c = oracle.sliced_cost(1.0, len(X), k)
        assert c <= math.ceil((1 << k) * f) / (1 << k) + 1e-15
        assert c < f + 2.0 ** -k
        assert F >= min(f, 1.0) - 1e-12 or len(X) == (1 << k)


SECONDS = {"hours": 3600.0, "days": 86400.0, "months": 86400.0 * 365.25 / 12}


def test_sampling_table_rows_share_one_peak():
    """Sec. III.A's table: every row's time is 8 C_s over one GPU's peak times the row's
    efficiency; the implied peak (about 14 TFLOP/s, a V100's FP32 rate) agrees across the
    rows to 5%.  And F >= the slicing ratio |X|/2^k (Sec. I.B) and >= the target."""
    rows = GOLDEN["sampling_complexity_table_sec_IIIA"]["rows"]
    peaks = []
    for r in rows:
        t = r["time"][0] * SECONDS[r["time"][1]]
        peaks.append(8.0 * r["C_s"] / (t * r["efficiency"]))
        assert r["F"] >= r["ratio"] and r["F"] >= r["target"]
    mean = sum(peaks) / len(peaks)
    assert 13e12 < mean < 15e12
    assert max(abs(x / mean - 1.0) for x in peaks) < 0.05
    # the oracle's time formula at the implied peak reproduces every printed time to 5%
    for r in rows:
        t = oracle.sampling_time(8.0 * r["C_s"], 1.0, mean, r["efficiency"])
        assert abs(t / (r["time"][0] * SECONDS[r["time"][1]]) - 1.0) < 0.05

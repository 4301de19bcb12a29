"""The allocation-free slice cut (tn_slice_cut_noalloc) against the allocating one.

Some callers cannot allocate device memory from their call path (their device memory
is owned up front by another allocator, or they must not enter the CUDA allocator).
For them tn_slice_cut_noalloc keeps its scratch in a static device array inside libtn.
This file is collected last so that a run stopping at the first failure has run every
other test first; it must also pass alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_noalloc_slice_cut_matches_allocating_cut_on_consecutive_calls():
    import paper_2112_15083_gb300 as P
    rng = np.random.default_rng(42)
    # two calls in a row: the second is smaller, so stale scratch from the first would show
    for k, f in ((12, 0.3), (7, 0.9)):
        R = rng.exponential(size=1 << k)
        R /= R.sum()
        X_ref, F_ref = P.slice_cut(R, f)
        X, F = P.tn.slice_cut_noalloc(R, f)
        assert np.array_equal(X, X_ref)  # index output: bit-exact
        assert F == F_ref                # same FP64 sum in the same order


def test_noalloc_slice_cut_rejects_k_above_limit():
    import paper_2112_15083_gb300 as P
    with pytest.raises(P.TnError) as e:
        P.tn.slice_cut_noalloc(np.full(1 << 13, 1.0 / (1 << 13)), 0.5)
    assert e.value.code == P.tn.TN_EINVAL

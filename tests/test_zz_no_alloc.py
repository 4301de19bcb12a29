"""The allocation-free slice cut (tn_slice_cut_noalloc) against the allocating one.

Some callers cannot allocate device memory from their call path (their device memory
is owned up front by another allocator, or they must not enter the CUDA allocator).
For them tn_slice_cut_noalloc keeps its scratch in a static device array inside libtn.
This file is collected last so that a run stopping at the first failure has run every
other test first; it must also pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the CUDA driver API (cuda.h)
_ATTR_USED_MEM_HIGH = 8


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


class DefaultPool:
    """High-water mark of the device's default stream-ordered memory pool (the pool
    cudaMallocAsync draws from), read and reset through the driver API."""

    def __init__(self, ordinal=0):
        self.cu = ctypes.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def used_high(self):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, _ATTR_USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


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


def test_noalloc_slice_cut_takes_no_pool_memory():
    """The point of the entry: no device allocation.  The allocating cut draws its
    scratch from the default pool (the high-water mark rises above zero); the
    allocation-free one leaves the reset mark at zero."""
    import paper_2112_15083_gb300 as P
    rng = np.random.default_rng(3)
    R = rng.exponential(size=1 << 10)
    R /= R.sum()
    pool = DefaultPool(0)
    P.tn.slice_cut_noalloc(R, 0.5)  # first call on the device: address lookup
    pool.reset_high()
    P.slice_cut(R, 0.5)
    assert pool.used_high() > 0
    pool.reset_high()
    for _ in range(2):
        P.tn.slice_cut_noalloc(R, 0.5)
    assert pool.used_high() == 0


def test_noalloc_slice_cut_rejects_k_above_limit():
    import paper_2112_15083_gb300 as P
    with pytest.raises(P.TnError) as e:
        P.tn.slice_cut_noalloc(np.full(1 << 13, 1.0 / (1 << 13)), 0.5)
    assert e.value.code == P.tn.TN_EINVAL

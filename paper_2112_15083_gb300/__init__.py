"""GB300-native sliced-contraction sampler for random quantum circuits.

Method: arXiv:2112.15083 (sliced multi-tensor contraction of amplitude batches summed
over the dominant slices, then modified frugal rejection sampling).  The compute path
is libtn.so (hand-written CUDA for sm_103a behind the C-ABI of include/tn.h); this
package holds the build step, the ctypes binding and the seeded input generators.
"""
from . import circuits  # noqa: F401
from .tn import (  # noqa: F401
    Circuit, Plan, Server, TnError, circuit_load, draw_batches, lib, plan, rejection_sample, slice_cut,
)

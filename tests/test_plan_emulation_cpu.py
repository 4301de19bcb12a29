"""The compiled plans compute the right amplitudes, checked on the CPU: the host planner and
step compiler of the library plan 12- and 16-qubit circuits (order search, slicing, lazy
batch selection at every threshold, tensor-core operand roles, explicit and layout-bit
versions), and a host executor of the compiled step list (tests/emulator) contracts them
in complex128 for several batch groups, full and partial slice sets.  The amplitudes must
equal the oracle's projector-sum state vector to 1e-10 of its largest amplitude."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2112_15083_gb300 import circuits as cg

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("emu") / "libplanemu.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_2112_15083_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "emulator", "plan_emulator.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.emu_contract.argtypes = [vp, ctypes.c_size_t, vp, i32, vp, i32, i32, vp, i32, vp, i64, vp, vp,
                               ctypes.POINTER(i32), vp]
    L.emu_error.restype = ctypes.c_char_p
    return L


def opts(log2_batches, n_sliced, precision, trials=16):
    import paper_2112_15083_gb300 as P
    o = P.tn.PlanOpts()
    P.lib().tn_plan_opts_default(ctypes.byref(o))
    o.log2_batches = log2_batches
    o.n_auto_sliced = n_sliced
    o.order_trials = trials
    o.precision = precision
    return o


def run(emu, circ, openq, o, q_max, tc, slices, closed):
    buf = circ.serialize()
    openv = np.ascontiguousarray(np.asarray(openq, dtype=np.int32))
    sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
    cb = np.ascontiguousarray(np.asarray(closed, dtype=np.uint64))
    out = np.zeros(cb.size << len(openq), dtype=np.complex128)
    edges = np.zeros(128, dtype=np.int32)
    ne = ctypes.c_int32()
    stats = np.zeros(3, dtype=np.int32)
    rc = emu.emu_contract(buf, len(buf), openv.ctypes.data, openv.size, ctypes.byref(o), q_max, tc,
                          sl.ctypes.data, sl.size, cb.ctypes.data, cb.size, out.ctypes.data, edges.ctypes.data,
                          ctypes.byref(ne), stats.ctypes.data)
    assert rc == 0, emu.emu_error().decode()
    return out.reshape(cb.size, 1 << len(openq)), [(int(edges[2 * e]), int(edges[2 * e + 1])) for e in range(ne.value)], stats


def slice_sets(n_sliced, rng):
    every = np.arange(1 << n_sliced, dtype=np.uint64)
    if n_sliced == 0:
        return [("all", every)]
    half = np.sort(rng.choice(every, size=max(1, every.size // 2), replace=False))
    return [("all", every), ("half", half), ("one", every[-1:])]


def check(emu, circ, openq, o, q_max, tc, nb, seed):
    n = circ.n_qubits
    rng = np.random.default_rng(seed)
    closed = cg.random_closed_bits(nb, n - len(openq), seed=seed) if len(openq) < n else np.zeros(nb, np.uint64)
    _, edges, _ = run(emu, circ, openq, o, q_max, tc, [0], closed[:1])
    for name, sl in slice_sets(len(edges), rng):
        amps, _, stats = run(emu, circ, openq, o, q_max, tc, sl, closed)
        psi = oracle.sliced_state(circ, edges, [int(s) for s in sl]) if edges else oracle.simulate(circ)
        ref = oracle.batch_amplitudes(psi, n, openq, closed) if len(openq) < n else np.tile(psi, (nb, 1))
        scale = float(np.abs(ref).max())
        assert float(np.abs(amps - ref).max()) <= 1e-10 * scale, (name, q_max, tc, stats)


@pytest.mark.parametrize("q_max", [-2, -1, 0, 6])
@pytest.mark.parametrize("tc", [0, 1])
def test_12q_every_batch_threshold(emu, q_max, tc):
    circ = cg.sycamore_grid(3, 4, 8, seed=1)
    o = opts(log2_batches=2, n_sliced=3, precision=1 if tc else 0)
    check(emu, circ, cg.default_open_qubits(3, 4, 6), o, q_max, tc, nb=11, seed=5)


@pytest.mark.parametrize("n_sliced,log2_batches", [(0, 0), (2, 4), (4, 6)])
def test_16q_slicing_and_groups(emu, n_sliced, log2_batches):
    circ = cg.sycamore_grid(4, 4, 10, seed=2)
    o = opts(log2_batches=log2_batches, n_sliced=n_sliced, precision=1)
    check(emu, circ, cg.default_open_qubits(4, 4, 6), o, -2, 1, nb=(1 << log2_batches) + 3, seed=7)


def test_12q_all_open(emu):
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    o = opts(log2_batches=0, n_sliced=2, precision=0)
    check(emu, circ, list(range(12)), o, -2, 0, nb=1, seed=1)


@pytest.mark.parametrize("seed", range(4))
def test_haar_circuits_random_pairs(emu, seed):
    """Haar gates on random ordered qubit pairs: neither symmetric under swapping the
    qubits nor under transposition, so layout and role mistakes show."""
    n = 10
    circ = cg.random_haar(n, 70, seed=seed, p_two=0.75)
    openq = [int(q) for q in np.random.default_rng(seed).permutation(n)[:4]]
    o = opts(log2_batches=3, n_sliced=2, precision=seed % 2)
    check(emu, circ, openq, o, [-2, -1, 0, 6][seed], seed % 2, nb=13, seed=seed)


@pytest.mark.parametrize("job_groups", [8, 64])
def test_16q_plans_weighted_for_a_job(emu, job_groups):
    """Plans whose order search weights the batch steps by the job's groups."""
    circ = cg.sycamore_grid(4, 4, 10, seed=3)
    o = opts(log2_batches=4, n_sliced=3, precision=1)
    o.job_groups = job_groups
    check(emu, circ, cg.default_open_qubits(4, 4, 6), o, -2, 1, nb=37, seed=9)


def test_20q_groups_of_64_batches(emu):
    """A 20-qubit plan with 4 sliced legs and 64 batches per group (70 batches: a ragged
    second group that reuses the stem)."""
    circ = cg.sycamore_grid(4, 5, 10, seed=3)
    o = opts(log2_batches=6, n_sliced=4, precision=1)
    check(emu, circ, cg.default_open_qubits(4, 5, 6), o, -2, 1, nb=70, seed=11)


@pytest.mark.parametrize("seed", [0, 1])
def test_annealed_plans(emu, seed):
    """Plans whose winning tree was reshaped by simulated annealing (tree rotations): at
    3x5, 12 cycles the annealed tree differs (5.7e7 instead of 8.3e7 FLOPs per slice)."""
    circ = cg.sycamore_grid(3, 5, 12, seed=seed)
    o = opts(log2_batches=4, n_sliced=3, precision=1)
    o.anneal_iters = 3000
    check(emu, circ, cg.default_open_qubits(3, 5, 6), o, -2, 1, nb=21, seed=seed + 40)


def test_size_capped_plan_annealed_per_slice(emu):
    """A plan sliced down to a tensor-size cap (2^13 elements) whose sliced tree is then
    annealed per slice under the cap (the sampling job's planning path): at 3x5, 12 cycles
    (circuit and order seed 3) the annealed tree differs from the unannealed one (9.63e7
    instead of 9.94e7 FLOPs per slice, 3 sliced legs both ways); its compiled steps,
    executed on the host, match the oracle on every slice subset."""
    circ = cg.sycamore_grid(3, 5, 12, seed=3)
    o = opts(log2_batches=4, n_sliced=0, precision=1)
    o.max_log2_tensor = 13
    o.order_seed = 3
    o.anneal_iters = 20000
    check(emu, circ, cg.default_open_qubits(3, 5, 6), o, -2, 1, nb=21, seed=5)


def test_12q_no_open_qubits(emu):
    """Every qubit closed: one amplitude per batch (the verification workload's plans)."""
    circ = cg.sycamore_grid(3, 4, 8, seed=2)
    o = opts(log2_batches=4, n_sliced=2, precision=1)
    check(emu, circ, [], o, -2, 1, nb=37, seed=3)


def layout_violations(emu, circ, openq, o, q_max, tc, slices):
    buf = circ.serialize()
    openv = np.ascontiguousarray(np.asarray(openq, dtype=np.int32))
    sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
    arena = ctypes.c_int64()
    emu.emu_layout_check.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    bad = emu.emu_layout_check(buf, len(buf), openv.ctypes.data, openv.size, ctypes.byref(o), q_max, tc,
                               sl.ctypes.data, sl.size, ctypes.byref(arena))
    assert bad >= 0, emu.emu_error().decode()
    return bad, arena.value


ARENA_CASES = [(r, c, m, lb, ns, q) for (r, c, m, lb, ns) in [(3, 4, 8, 2, 3), (4, 4, 10, 4, 4), (4, 5, 10, 6, 4)]
               for q in (-2, -1, 6)] + [(4, 7, 14, 14, 10, -2)]


@pytest.mark.parametrize("rows,cols,cycles,log2_batches,n_sliced,q_max", ARENA_CASES)
def test_arena_layout_invariants(emu, rows, cols, cycles, log2_batches, n_sliced, q_max):
    """The engine's arena plan (arena.h) for these plans: live tensors disjoint in every
    step, the kept stem disjoint from everything, all within the arena (up to the 28-qubit
    bench plan, whose arena is only planned here; a threshold forced on that tree would
    exceed the 40-bit tensor limit, so it keeps the planner's)."""
    circ = cg.sycamore_grid(rows, cols, cycles, seed=0)
    o = opts(log2_batches=log2_batches, n_sliced=n_sliced, precision=1, trials=16)
    rng = np.random.default_rng(rows * 100 + cycles)
    full = np.arange(1 << n_sliced, dtype=np.uint64)
    for sl in (full, np.sort(rng.choice(full, size=max(1, full.size // 3), replace=False))):
        bad, arena = layout_violations(emu, circ, cg.default_open_qubits(rows, cols, 6), o, q_max, 1, sl)
        assert bad == 0 and arena > 0


def test_plans_from_the_parallel_search(emu):
    """Greedy trials with per-trial generators on threads (tn_plan_opts.parallel_search):
    the 12-qubit all-open plan differs from the sequential search's; both must be right."""
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    o = opts(log2_batches=0, n_sliced=2, precision=0, trials=64)
    o.parallel_search = 1
    check(emu, circ, list(range(12)), o, -2, 0, nb=1, seed=2)

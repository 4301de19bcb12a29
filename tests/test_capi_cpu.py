"""CPU-side checks of the C-ABI library: it loads, exports every symbol declared in
include/tn.h, rejects malformed input, and its host planner agrees with the oracle's
Alg. 2 and with the gate counts of the ABCD reading.  No compute call needs a GPU here."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2112_15083_gb300 as pkg
from paper_2112_15083_gb300 import circuits as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tn_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 16
    L = pkg.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(pkg.tn.EXPORTED)


def test_strerror_names_codes():
    L = pkg.lib()
    for code in (0, -1, -2, -3, -4, -5):
        assert L.tn_strerror(code)
    assert L.tn_strerror(-99) == b"unknown error"


def test_malformed_circuits_rejected():
    with pytest.raises(pkg.TnError) as e:
        pkg.circuit_load(b"XXXX" + b"\0" * 20)
    assert e.value.code == pkg.tn.TN_EINVAL
    good = cg.sycamore_grid(2, 2, 2, seed=0).serialize()
    with pytest.raises(pkg.TnError):
        pkg.circuit_load(good[:-5])  # truncated matrix
    bad = bytearray(good)
    bad[16:20] = (99).to_bytes(4, "little")  # first gate's qubit out of range
    with pytest.raises(pkg.TnError):
        pkg.circuit_load(bytes(bad))


def test_host_plan_counts_and_shapes():
    circ = cg.sycamore_grid(4, 7, 14, seed=0)
    C = pkg.circuit_load(circ.serialize())
    info, steps, sliced = pkg.tn.plan_host(C, cg.default_open_qubits(4, 7, 6), n_auto_sliced=10,
                                           order_trials=8)
    assert info["n_leaves"] == 156 and info["n_steps"] == 155
    assert info["n_open"] == 6 and info["n_closed"] == 22 and info["n_sliced"] == 10
    assert len(sliced) == 10 and len(set(sliced)) == 10
    cnt = oracle.two_qubit_counts(circ)
    for q, s in sliced:
        assert 1 <= s < cnt[q]
    # every step's bit classes fit the engine's 40-bit addressing
    assert steps.shape[1] == 7 and (steps[:, 0] + steps[:, 1] + steps[:, 2] <= 40).all()


def test_host_plan_rejects_bad_sliced_edge():
    circ = cg.sycamore_grid(3, 4, 8, seed=0)
    C = pkg.circuit_load(circ.serialize())
    with pytest.raises(pkg.TnError):
        pkg.tn.plan_host(C, list(range(12)), sliced=[(0, 0)])  # input segment
    cnt = oracle.two_qubit_counts(circ)
    with pytest.raises(pkg.TnError):
        pkg.tn.plan_host(C, list(range(12)), sliced=[(0, cnt[0])])  # output segment
    with pytest.raises(pkg.TnError):
        pkg.tn.plan_host(C, [0, 0, 1])  # repeated open qubit


def test_host_order_roundtrip_ssa():
    # a left-deep SSA order over all leaves must be accepted
    circ = cg.sycamore_grid(2, 3, 4, seed=1)
    C = pkg.circuit_load(circ.serialize())
    L = circ.n_two_qubit()
    order = []
    cur = 0
    for i in range(1, L):
        order.append((cur, i))
        cur = L + i - 1
    info, steps, _ = pkg.tn.plan_host(C, list(range(6)), order=order)
    assert info["n_steps"] == L - 1
    with pytest.raises(pkg.TnError):
        pkg.tn.plan_host(C, list(range(6)), order=order[:-1])


@pytest.mark.parametrize("grid,f", [((3, 4, 8), 0.25), ((4, 5, 12), 1 / 64), ((4, 7, 14), 0.002)])
def test_alg2_matches_oracle(grid, f):
    circ = cg.sycamore_grid(*grid, seed=0)
    view = oracle.MergedView(circ)
    n = grid[0] * grid[1]
    I = [(q, s) for q in range(n) for s in range(1, view.n2q[q])]
    k0 = oracle.k0_for(f)
    ref = oracle.sliced_vertex_select(circ, I, k0)
    C = pkg.circuit_load(circ.serialize())
    got = [I[i] for i in pkg.tn.sliced_vertex_select(C, I, k0)]
    assert got == ref


@pytest.mark.parametrize("cap", [20, 17])
def test_width_slicing_caps_every_tensor(cap):
    """max_log2_tensor slices legs until no tensor of one slice exceeds 2^cap elements
    (and slices nothing when the unsliced plan already fits)."""
    circ = cg.sycamore_grid(4, 6, 12, seed=3)
    C = pkg.circuit_load(circ.serialize())
    openq = cg.default_open_qubits(4, 6, 6)
    free, _, _ = pkg.tn.plan_host(C, openq, log2_batches=8, order_trials=16, precision=pkg.tn.PREC_BF16X2)
    info, steps, sliced = pkg.tn.plan_host(C, openq, log2_batches=8, order_trials=16,
                                           max_log2_tensor=cap, precision=pkg.tn.PREC_BF16X2)
    assert info["log2_max_tensor"] <= cap
    assert info["n_sliced"] == len(sliced)
    assert (len(sliced) >= 1) == (free["log2_max_tensor"] > cap)
    cnt = oracle.two_qubit_counts(circ)
    for q, s in sliced:
        assert 1 <= s < cnt[q]


def test_order_search_is_deterministic():
    """The seeded order search (greedy, bisection, thresholds, subtree reconfiguration)
    gives the same plan for the same seed, and a plan for another seed is still valid."""
    circ = cg.sycamore_grid(4, 5, 10, seed=2)
    C = pkg.circuit_load(circ.serialize())
    openq = cg.default_open_qubits(4, 5, 6)
    a = pkg.tn.plan_host(C, openq, n_auto_sliced=6, log2_batches=10, order_trials=16, order_seed=7)
    b = pkg.tn.plan_host(C, openq, n_auto_sliced=6, log2_batches=10, order_trials=16, order_seed=7)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]
    c = pkg.tn.plan_host(C, openq, n_auto_sliced=6, log2_batches=10, order_trials=16, order_seed=8)
    assert c[0]["n_steps"] == a[0]["n_steps"]


def test_ctypes_mirrors_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (compiled
    as C with the host compiler)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2112_15083_gb300 import tn
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"tn_edge": tn.Edge, "tn_plan_opts": tn.PlanOpts, "tn_plan_info": tn.PlanInfo,
               "tn_sample_stats": tn.SampleStats, "tn_step_trace": tn.StepTrace, "tn_server_opts": tn.ServerOpts,
               "tn_request_info": tn.RequestInfo, "tn_server_stats": tn.ServerStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tn.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.splitlines())
    for cname, cls in mirrors.items():
        assert int(got[cname + " size"]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[cname + "." + f]) == getattr(cls, f).offset, (cname, f)

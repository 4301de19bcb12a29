"""CPU oracle for the sliced-contraction sampler (test infrastructure only).

Plain, slow, FP64 restatement of what the paper's method computes, written from
arXiv:2112.15083 (Kalachev, Panteleev, Zhou, Yung):

* amplitudes: the state vector C|0> (Sec. I.A, |psi> = C2 C1 |0>), applied gate by
  gate in ``oracle.c``;
* slices: a sliced leg fixed to v is the projector |v><v| on that wire (App. B: the
  slicing delta acts on the wire as a projection); the sum over all slices is the
  unsliced state;
* partial slicing: |psi_X> = C2 Pi_X C1 |0> = sum_{i in X} |psi_i> (Sec. I.A);
* norms R[i] = ||psi_i||^2 = P(S-wires read i after C1) (Sec. I.A, Alg. 1);
* SlicedVertexSelect (Alg. 2) and Slice selection (Alg. 1);
* linear XEB (Eq. 1) and the modified frugal rejection sampler (Sec. II.A);
* the XEB spoofing recipe (Sec. III, "Spoofing Linear XEB"; App. A);
* the cost model: C_s(f) = |X|/2^k C_s(1) (Sec. I.B) and the time estimate of Sec. III.A;
* the sampler's output law, variation distance and fidelity bound (Sec. II.B);
* the expected rejection loss under Porter-Thomas statistics (Sec. II.C).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It shares no code with the CUDA path; both read the same
serialized circuits produced by the input module.

Wire-segment convention shared with the paper's "vertices = tensor legs" (App. B):
single-qubit gates are merged into the preceding two-qubit gate on their wire (the
leading ones into the |0> input), so the legs are the segments between two-qubit
gates.  Segment (q, s) is the wire of qubit q just before its (s+1)-th two-qubit
gate; s = (number of two-qubit gates on q) is the output of q.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        cd_p = ctypes.c_void_p
        L.orc_simulate.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.c_int,
                                   cd_p, cd_p, cd_p, cd_p]
        L.orc_simulate.restype = ctypes.c_int
        L.orc_simulate_split.argtypes = [ctypes.c_char_p, ctypes.c_size_t, cd_p, ctypes.c_int,
                                         cd_p, cd_p, cd_p]
        L.orc_simulate_split.restype = ctypes.c_int
        L.orc_simulate_subset.argtypes = [ctypes.c_char_p, ctypes.c_size_t, cd_p, cd_p]
        L.orc_simulate_subset.restype = ctypes.c_int
        L.orc_marginal.argtypes = [cd_p, ctypes.c_int, ctypes.c_int, cd_p, cd_p]
        L.orc_marginal.restype = None
        L.orc_apply_1q.argtypes = [cd_p, ctypes.c_int, ctypes.c_int, cd_p]
        L.orc_apply_2q.argtypes = [cd_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, cd_p]
        L.orc_philox4x32_10.argtypes = [cd_p, cd_p, cd_p]
        L.orc_philox4x32_10.restype = None
        L.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, cd_p, cd_p, cd_p]
        L.orc_draw.restype = None
        L.orc_sample_batches.argtypes = [cd_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_uint64, cd_p, cd_p]
        L.orc_sample_batches.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------- states

def simulate(circ, projectors=()) -> np.ndarray:
    """psi = C|0> with projectors [(qubit, segment, value), ...] inserted on the wires.

    Fixing a sliced leg (q, s) to v equals inserting |v><v| on wire q at segment s
    (App. B).  Returns the 2^n complex128 state, bit q of the index = qubit q.
    """
    buf = circ.serialize()
    n = circ.n_qubits
    psi = np.empty(1 << n, dtype=np.complex128)
    pq = np.array([p[0] for p in projectors] or [0], dtype=np.int32)
    ps = np.array([p[1] for p in projectors] or [0], dtype=np.int32)
    pv = np.array([p[2] for p in projectors] or [0], dtype=np.int32)
    rc = lib().orc_simulate(buf, len(buf), len(projectors), _ptr(pq), _ptr(ps), _ptr(pv), _ptr(psi))
    if rc != 0:
        raise ValueError("oracle: bad circuit or projector segment")
    return psi


def simulate_subset(circ, selected) -> np.ndarray:
    """Apply only the gates g with selected[g] true (circuit order) to |0>."""
    buf = circ.serialize()
    sel = np.ascontiguousarray(np.asarray(selected, dtype=np.uint8))
    psi = np.empty(1 << circ.n_qubits, dtype=np.complex128)
    if lib().orc_simulate_subset(buf, len(buf), _ptr(sel), _ptr(psi)) != 0:
        raise ValueError("oracle: bad circuit")
    return psi


def simulate_split(circ, in_c1, s_qubits, x_mask) -> np.ndarray:
    """psi_X = C2 Pi_X C1 |0> (Sec. I.A): C1 = gates with in_c1, Pi_X = sum_{i in X} |i><i|
    on the S qubits (bit t of i = s_qubits[t]), then the remaining gates."""
    buf = circ.serialize()
    c1 = np.ascontiguousarray(np.asarray(in_c1, dtype=np.uint8))
    sq = np.ascontiguousarray(np.asarray(s_qubits, dtype=np.int32))
    xm = np.ascontiguousarray(np.asarray(x_mask, dtype=np.uint8))
    assert xm.size == 1 << sq.size
    psi = np.empty(1 << circ.n_qubits, dtype=np.complex128)
    rc = lib().orc_simulate_split(buf, len(buf), _ptr(c1), sq.size, _ptr(sq), _ptr(xm), _ptr(psi))
    if rc != 0:
        raise ValueError("oracle: bad circuit")
    return psi


def marginal(psi: np.ndarray, n: int, qubits) -> np.ndarray:
    """out[i] = sum of |psi|^2 over basis states whose bits on `qubits` read i."""
    qs = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
    out = np.empty(1 << qs.size, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    lib().orc_marginal(_ptr(psi), n, qs.size, _ptr(qs), _ptr(out))
    return out


# ------------------------------------------------------------- wire segments

def two_qubit_counts(circ) -> list:
    cnt = [0] * circ.n_qubits
    for g in circ.gates:
        if len(g.qubits) == 2:
            for q in g.qubits:
                cnt[q] += 1
    return cnt


def segment_position(circ, q: int, s: int) -> int:
    """Gate-list index of the (s+1)-th two-qubit gate on q (the wire point of segment
    (q, s)); len(gates) for the output segment."""
    c = 0
    for idx, g in enumerate(circ.gates):
        if len(g.qubits) == 2 and q in g.qubits:
            if c == s:
                return idx
            c += 1
    if c == s:
        return len(circ.gates)
    raise ValueError("segment out of range")


def causal_past(circ, vertices) -> np.ndarray:
    """Mask of the gates of C that the wire points `vertices` depend on (the union of
    their lightcones L_C(v), App. B), on the unmerged gate list.

    Walk backwards from the point: a gate touching an active wire is in the past,
    and all its wires become active from that point on.
    """
    mask = np.zeros(len(circ.gates), dtype=np.uint8)
    for (q, s) in vertices:
        pos = segment_position(circ, q, s)
        active = {q}
        for idx in range(pos - 1, -1, -1):
            qs = circ.gates[idx].qubits
            if any(x in active for x in qs):
                mask[idx] = 1
                active.update(qs)
    return mask


class MergedView:
    """The circuit as seen by the tensor network: two-qubit gates (with merged
    single-qubit gates), each with its input segments (App. B vertices)."""

    def __init__(self, circ):
        self.n = circ.n_qubits
        self.gates = []      # list of (qa, qb, sa, sb): inputs (qa, sa), (qb, sb)
        cnt = [0] * self.n
        for g in circ.gates:
            if len(g.qubits) == 2:
                a, b = g.qubits
                self.gates.append((a, b, cnt[a], cnt[b]))
                cnt[a] += 1
                cnt[b] += 1
        self.n2q = cnt
        # producer[(q, s)] = index of the merged gate whose output is segment (q, s)
        self.producer = {}
        for gi, (a, b, sa, sb) in enumerate(self.gates):
            self.producer[(a, sa + 1)] = gi
            self.producer[(b, sb + 1)] = gi

    def lightcone(self, v) -> set:
        """L_C(v): merged gates that vertex v depends on."""
        out = set()
        stack = [v]
        while stack:
            x = stack.pop()
            gi = self.producer.get(x)
            if gi is None or gi in out:
                continue
            out.add(gi)
            a, b, sa, sb = self.gates[gi]
            stack.append((a, sa))
            stack.append((b, sb))
        return out

    def lightcone_inputs(self, vertices) -> set:
        """L'_C(S): the input vertices of the gates in the union of the lightcones."""
        gates = set()
        for v in vertices:
            gates |= self.lightcone(v)
        out = set()
        for gi in gates:
            a, b, sa, sb = self.gates[gi]
            out.add((a, sa))
            out.add((b, sb))
        return out


def sliced_vertex_select(circ, I, k: int) -> list:
    """Alg. 2 SlicedVertexSelect(C, I, k): greedy S in I minimising |L'_C(S)|.

    Readings: the argmin variable is the candidate u; candidates exclude S itself
    (else a chosen vertex could be re-chosen forever); ties go to the earliest
    vertex in I's order; the result is returned sorted by (qubit, segment).
    """
    view = MergedView(circ)
    S = []
    I = [tuple(v) for v in I]
    while len(S) < k:
        lp = view.lightcone_inputs(S)
        cand = [u for u in I if u not in lp and u not in S]
        if not cand:
            break
        best, best_size = None, None
        for u in cand:
            sz = len(view.lightcone_inputs(S + [u]))
            if best_size is None or sz < best_size:
                best, best_size = u, sz
        lv = view.lightcone_inputs([best])
        S = [s for s in S if s not in lv] + [best]
    return sorted(S)


def k0_for(f: float) -> int:
    """Alg. 1: k0 = ceil(3 - log2 f)."""
    return int(math.ceil(3.0 - math.log2(f)))


def norms(circ, S) -> np.ndarray:
    """R[i] = ||psi_i||^2 (Sec. I.A): the distribution of the S wires after C1, where
    C1 is the union of the lightcones of S; bit t of i is S[t] (S sorted)."""
    c1 = causal_past(circ, S)
    psi1 = simulate_subset(circ, c1)
    return marginal(psi1, circ.n_qubits, [q for (q, _s) in S])


def select_slices(R: np.ndarray, f: float):
    """Alg. 1's cut: sort R descending (ties by index ascending), take the minimal
    prefix whose sequential FP64 sum reaches f (all of them if rounding keeps the
    total below f).  Returns (X as index array in sorted order, F)."""
    order = sorted(range(R.size), key=lambda i: (-R[i], i))
    acc = 0.0
    for t, i in enumerate(order):
        acc = acc + float(R[i])
        if acc >= f:
            return np.array(order[: t + 1], dtype=np.int64), acc
    return np.array(order, dtype=np.int64), acc


def slice_selection(circ, I, f: float):
    """Alg. 1 end to end: (S, X, F, R)."""
    S = sliced_vertex_select(circ, I, k0_for(f))
    R = norms(circ, S)
    X, F = select_slices(R, f)
    return S, X, F, R


def partial_state(circ, S, X) -> np.ndarray:
    """|psi_X> = sum_{i in X} |psi_i> = C2 Pi_X C1 |0> (unnormalised)."""
    c1 = causal_past(circ, S)
    xm = np.zeros(1 << len(S), dtype=np.uint8)
    xm[np.asarray(X, dtype=np.int64)] = 1
    return simulate_split(circ, c1, [q for (q, _s) in S], xm)


def sliced_state(circ, edges, assignments) -> np.ndarray:
    """Sum over the given slice assignments of C|0> with the sliced legs fixed:
    bit e of an assignment is the value of edges[e] (Sec. I.C, step 1)."""
    out = np.zeros(1 << circ.n_qubits, dtype=np.complex128)
    for a in assignments:
        proj = [(q, s, (int(a) >> e) & 1) for e, (q, s) in enumerate(edges)]
        out += simulate(circ, proj)
    return out


# ----------------------------------------------------------------- batches

def bitstring(i: int, j: int, open_qubits, closed_qubits) -> int:
    """Bitstring (bit q = qubit q) of in-batch index i (bit r -> open_qubits[r]) and
    closed pattern j (bit c -> closed_qubits[c])."""
    b = 0
    for r, q in enumerate(open_qubits):
        b |= ((i >> r) & 1) << q
    for c, q in enumerate(closed_qubits):
        b |= ((int(j) >> c) & 1) << q
    return b


def closed_of(n: int, open_qubits) -> list:
    o = set(open_qubits)
    return [q for q in range(n) if q not in o]


def batch_amplitudes(psi: np.ndarray, n: int, open_qubits, closed_bits) -> np.ndarray:
    """amps[t, i] = psi[bitstring(i, closed_bits[t])], shape (T, 2^|A|) (works for any
    per-bitstring array, e.g. probabilities)."""
    closed = closed_of(n, open_qubits)
    na = len(open_qubits)
    idx_open = np.zeros(1 << na, dtype=np.int64)
    for i in range(1 << na):
        idx_open[i] = bitstring(i, 0, open_qubits, [])
    T = len(closed_bits)
    idx_closed = np.zeros(T, dtype=np.int64)
    for t, j in enumerate(closed_bits):
        idx_closed[t] = bitstring(0, int(j), [], closed)
    return psi[idx_closed[:, None] | idx_open[None, :]]


# --------------------------------------------------------------------- XEB

def xeb_of_samples(p_ideal: np.ndarray, n: int, samples) -> float:
    """Eq. 1: F_XEB = 2^n/k sum_i p_C(s_i) - 1."""
    s = np.asarray(samples, dtype=np.int64)
    return float((2.0 ** n) * np.mean(p_ideal[s]) - 1.0)


def xeb_exact(p_ideal: np.ndarray, p_model: np.ndarray, n: int) -> float:
    """Expected Eq. 1 value for samples drawn from p_model: 2^n sum_s p_model p_ideal - 1."""
    return float((2.0 ** n) * np.dot(p_model, p_ideal) - 1.0)


# ------------------------------------------------------------------ sampler

def philox4x32_10(ctr, key) -> tuple:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return tuple(int(x) for x in o)


def draw(seed: int, t: int):
    """(jraw, u, v) of step t (see oracle.c: stream 0 -> j, u; stream 1 -> v)."""
    jr = np.zeros(1, dtype=np.uint64)
    u = np.zeros(1, dtype=np.float64)
    v = np.zeros(1, dtype=np.float64)
    lib().orc_draw(ctypes.c_uint64(seed), ctypes.c_uint64(t), _ptr(jr), _ptr(u), _ptr(v))
    return int(jr[0]), float(u[0]), float(v[0])


def sample_batches(p: np.ndarray, b_bits: int, alpha: float, seed: int, t0: int = 0):
    """Sec. II.A steps 2-3 for batches t0.. t0+T-1 with probabilities p[t, i] (N_A = 64).
    Returns (accept[T] bool, pick[T] int)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert p.ndim == 2 and p.shape[1] == 64
    T = p.shape[0]
    acc = np.zeros(T, dtype=np.uint8)
    pick = np.zeros(T, dtype=np.int32)
    lib().orc_sample_batches(_ptr(p), T, b_bits, alpha, ctypes.c_uint64(seed),
                             ctypes.c_uint64(t0), _ptr(acc), _ptr(pick))
    return acc.astype(bool), pick


def batch_draws(seed: int, T: int, b_bits: int, t0: int = 0) -> np.ndarray:
    """Step 1 of Sec. II.A: j_t = low b_bits of the step-t draw."""
    mask = (1 << b_bits) - 1
    return np.array([draw(seed, t0 + t)[0] & mask for t in range(T)], dtype=np.uint64)


def sample(p_model: np.ndarray, n: int, open_qubits, N: int, seed: int, alpha: float = 2.0,
           max_steps: int | None = None, chunk: int = 1024):
    """Modified frugal rejection sampling (Sec. II.A) from a normalised distribution
    p_model over 2^n bitstrings with batches over the 6 open qubits.  Returns
    (samples in step order (first N accepted), steps used, epsilon_hat)."""
    assert len(open_qubits) == 6
    closed = closed_of(n, open_qubits)
    b_bits = len(closed)
    NB = 2.0 ** b_bits
    out = []
    t = 0
    eps_sum = 0.0
    limit = max_steps if max_steps is not None else 64 * N + 1024
    while len(out) < N and t < limit:
        T = min(chunk, limit - t)
        js = batch_draws(seed, T, b_bits, t0=t)
        p = np.ascontiguousarray(batch_amplitudes(p_model, n, open_qubits, js))
        acc, pick = sample_batches(p, b_bits, alpha, seed, t0=t)
        pj = p.sum(axis=1)
        eps_sum += float(np.maximum(pj - alpha / NB, 0.0).sum())
        for tt in range(T):
            if acc[tt] and len(out) < N:
                out.append(bitstring(int(pick[tt]), int(js[tt]), open_qubits, closed))
        t += T
    return np.array(out, dtype=np.int64), t, eps_sum / max(t, 1)


# --------------------------------------------------------------- statistics

def output_law(p: np.ndarray, alpha: float, NB: float) -> np.ndarray:
    """Sec. II.A: p~_{i,j} = p'_j/(1 - eps) * p_{i,j}/p_j with p'_j = min(p_j, alpha/N_B).
    p has shape (N_B, N_A)."""
    pj = p.sum(axis=1)
    pprime = np.minimum(pj, alpha / NB)
    eps = float((pj - pprime).sum())
    with np.errstate(invalid="ignore", divide="ignore"):
        cond = np.where(pj[:, None] > 0, p / pj[:, None], 0.0)
    return (pprime[:, None] / (1.0 - eps)) * cond, eps


def variation_distance(p: np.ndarray, q: np.ndarray) -> float:
    """Eq. (Dpp-start): D(p, q) = 1/2 sum |p - q|."""
    return 0.5 * float(np.abs(p - q).sum())


def fidelity_lower_bound(f: float, d: float) -> float:
    """Sec. II.B: f' >= f (1 - 4 sqrt(d/f)), valid for d < f/16."""
    return f * (1.0 - 4.0 * math.sqrt(d / f))


def expected_eps_pt(NA: int, alpha: float) -> float:
    """E eps under Porter-Thomas statistics (Sec. II.C), exact form.

    p_j N_B ~ Gamma(N_A, 1)/N_A, so E eps = N_B E[(p_j - alpha/N_B)^+]
    = Q(N_A + 1, alpha N_A) - alpha Q(N_A, alpha N_A) with Q the regularised upper
    incomplete gamma.  (The printed Eq. Eeps, N_B Gamma(N_A, alpha N_A)/Gamma(N_A),
    counts over-threshold batches rather than their excess mass.)
    """
    from scipy.special import gammaincc
    return float(gammaincc(NA + 1, alpha * NA) - alpha * gammaincc(NA, alpha * NA))


def paper_eps_bound(NA: int, NB: float, alpha: float) -> float:
    """The printed Eq. Eeps: N_B Gamma(N_A, alpha N_A)/Gamma(N_A)."""
    from scipy.special import gammaincc
    return float(NB * gammaincc(NA, alpha * NA))


# -------------------------------------------------------------- XEB spoofing

def spoof_batch_bits(N: int) -> int:
    """Step 1 of the spoofing recipe (Sec. III, "Spoofing Linear XEB"): b = ceil(log2(10 N)),
    the number of free outputs, so that the batch holds 2^b >= 10 N bitstrings."""
    if N < 1:
        raise ValueError("N must be positive")
    b = 0
    while (1 << b) < 10 * N:
        b += 1
    return b


def spoof_select(p_approx: np.ndarray, N: int) -> np.ndarray:
    """Step 4: the positions of the N largest approximate probabilities |psi'_i|^2 in the
    batch, largest first; equal values go to the smaller position (the paper does not say)."""
    p = np.asarray(p_approx, dtype=np.float64)
    if not 0 <= N <= p.size:
        raise ValueError("N outside [0, batch size]")
    order = np.lexsort((np.arange(p.size), -p))  # by -p, then by position
    return order[:N].astype(np.int64)


def spoof_xeb(p_ideal: np.ndarray, n: int, selected) -> float:
    """Eq. 1 over the selected strings: 2^n times the mean exact probability, minus 1."""
    return xeb_of_samples(p_ideal, n, selected)


def spoof_expected_xeb(f: float, r: float) -> float:
    """Eq. spoof-xeb (App. A): for a Porter-Thomas batch computed at fidelity f, the N = r |B|
    strings of largest approximate probability have E XEB = -f ln r, up to O(ln N / N)."""
    return -f * math.log(r)


# ------------------------------------------------------------------ cost model

def sliced_cost(c_full: float, n_retained: int, k: int) -> float:
    """Sec. I.B: contracting the retained partial assignments X of k legs costs
    C_s(f) = |X| / 2^k C_s(1)."""
    return c_full * n_retained / float(1 << k)


def sampling_time(flops_full: float, fidelity: float, peak_flops: float, efficiency: float) -> float:
    """Sec. III.A's estimate: the full contraction's FLOPs scaled by the fidelity, over the
    machine's peak times its efficiency (seconds)."""
    return flops_full * fidelity / (peak_flops * efficiency)

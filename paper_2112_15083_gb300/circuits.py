"""Seeded synthetic inputs: Sycamore-style random circuits and batch bitstrings.

This module is the one place shared by the CUDA path and the CPU oracle.  It only
*describes* inputs (gate lists with explicit complex128 matrices, random closed-bit
patterns); it performs none of the method's arithmetic (no contraction, no
probabilities, no sampling).

Circuit family (paper Sec. III, "ABCD" supremacy circuits; the paper does not define
the gate set or the coupler pattern, so the reading below is fixed here once):

* qubit ``q = r * cols + c`` on a ``rows x cols`` grid;
* each cycle is a layer of single-qubit gates on every qubit, drawn independently and
  uniformly from {sqrtX, sqrtY, sqrtW} with W = (X + Y)/sqrt(2), followed by one layer
  of fSim(theta=pi/2, phi=pi/6) on the couplers of pattern ``ABCDCDAB[cycle % 8]``;
* A = horizontal couplers (r,c)-(r,c+1) with c even, B = horizontal with c odd,
  C = vertical (r,c)-(r+1,c) with r even, D = vertical with r odd;
* one final single-qubit layer closes the circuit.

Serialized format (little endian), read by ``tn_circuit_load`` and by the oracle:
``b"RQC1"``, uint32 n_qubits, uint32 n_gates, then per gate uint32 arity (1 or 2),
uint32 q0, uint32 q1 (0xFFFFFFFF for arity 1) and the (2^arity)^2 matrix entries as
(re, im) float64 pairs in row-major order.  For a two-qubit gate the basis index is
``2*bit(q0) + bit(q1)``.
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field

import numpy as np

MAGIC = b"RQC1"
NO_QUBIT = 0xFFFFFFFF
PATTERN = "ABCDCDAB"


@dataclass
class Gate:
    qubits: tuple
    matrix: np.ndarray  # complex128, (2,2) or (4,4)


@dataclass
class Circuit:
    n_qubits: int
    gates: list = field(default_factory=list)
    rows: int = 0
    cols: int = 0
    cycles: int = 0
    seed: int = 0

    def n_two_qubit(self) -> int:
        return sum(1 for g in self.gates if len(g.qubits) == 2)

    def n_one_qubit(self) -> int:
        return sum(1 for g in self.gates if len(g.qubits) == 1)

    def serialize(self) -> bytes:
        return serialize(self)


_S2 = 1.0 / math.sqrt(2.0)


def sqrt_x() -> np.ndarray:
    # exp(-i pi/4 X)
    return _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)


def sqrt_y() -> np.ndarray:
    # exp(-i pi/4 Y)
    return _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)


def sqrt_w() -> np.ndarray:
    # exp(-i pi/4 W), W = (X + Y)/sqrt(2) = [[0, e^{-i pi/4}], [e^{i pi/4}, 0]]
    em = complex(_S2, -_S2)
    ep = complex(_S2, _S2)
    return _S2 * np.array([[1, -1j * em], [-1j * ep, 1]], dtype=np.complex128)


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array(
        [
            [1, 0, 0, 0],
            [0, c, -1j * s, 0],
            [0, -1j * s, c, 0],
            [0, 0, 0, complex(math.cos(phi), -math.sin(phi))],
        ],
        dtype=np.complex128,
    )


ONE_QUBIT_SET = (sqrt_x, sqrt_y, sqrt_w)


def couplers(rows: int, cols: int, layer: str) -> list:
    """Coupler list of one ABCD layer on a rows x cols grid (qubit r*cols + c)."""
    out = []
    if layer in "AB":
        par = 0 if layer == "A" else 1
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                out.append((r * cols + c, r * cols + c + 1))
    else:
        par = 0 if layer == "C" else 1
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                out.append((r * cols + c, (r + 1) * cols + c))
    return out


def sycamore_grid(rows: int, cols: int, cycles: int, seed: int = 0,
                  theta: float = math.pi / 2, phi: float = math.pi / 6) -> Circuit:
    """Seeded ABCD random circuit on a rows x cols grid (see module docstring)."""
    n = rows * cols
    rng = np.random.default_rng(seed)
    circ = Circuit(n_qubits=n, rows=rows, cols=cols, cycles=cycles, seed=seed)
    two = fsim(theta, phi)
    for cyc in range(cycles):
        picks = rng.integers(0, 3, size=n)
        for q in range(n):
            circ.gates.append(Gate((q,), ONE_QUBIT_SET[picks[q]]()))
        for (a, b) in couplers(rows, cols, PATTERN[cyc % len(PATTERN)]):
            circ.gates.append(Gate((a, b), two.copy()))
    picks = rng.integers(0, 3, size=n)
    for q in range(n):
        circ.gates.append(Gate((q,), ONE_QUBIT_SET[picks[q]]()))
    return circ


def haar_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_haar(n: int, n_gates: int, seed: int = 0, p_two: float = 0.6) -> Circuit:
    """Generic circuit with Haar-random 1q/2q gates on random (ordered) qubit pairs.

    Used by tests: unlike fSim, these gates are neither symmetric under qubit swap
    nor under transposition, so index mistakes show up.
    """
    rng = np.random.default_rng(seed)
    circ = Circuit(n_qubits=n, seed=seed)
    for _ in range(n_gates):
        if n >= 2 and rng.random() < p_two:
            a, b = rng.choice(n, size=2, replace=False)
            circ.gates.append(Gate((int(a), int(b)), haar_unitary(4, rng)))
        else:
            q = int(rng.integers(0, n))
            circ.gates.append(Gate((q,), haar_unitary(2, rng)))
    return circ


def serialize(circ: Circuit) -> bytes:
    parts = [MAGIC, struct.pack("<II", circ.n_qubits, len(circ.gates))]
    for g in circ.gates:
        ar = len(g.qubits)
        q0 = g.qubits[0]
        q1 = g.qubits[1] if ar == 2 else NO_QUBIT
        parts.append(struct.pack("<III", ar, q0, q1))
        m = np.ascontiguousarray(g.matrix, dtype=np.complex128)
        assert m.shape == (1 << ar, 1 << ar)
        parts.append(m.tobytes())  # complex128 is (re, im) float64 pairs
    return b"".join(parts)


def deserialize(buf: bytes) -> Circuit:
    assert buf[:4] == MAGIC, "bad magic"
    n, ng = struct.unpack_from("<II", buf, 4)
    off = 12
    circ = Circuit(n_qubits=n)
    for _ in range(ng):
        ar, q0, q1 = struct.unpack_from("<III", buf, off)
        off += 12
        d = 1 << ar
        m = np.frombuffer(buf, dtype=np.complex128, count=d * d, offset=off).reshape(d, d).copy()
        off += 16 * d * d
        circ.gates.append(Gate((q0,) if ar == 1 else (q0, q1), m))
    return circ


def random_closed_bits(n_batches: int, n_closed: int, seed: int) -> np.ndarray:
    """Uniformly random closed-qubit patterns, one uint64 per batch (bit c = c-th closed qubit)."""
    rng = np.random.default_rng(seed)
    if n_closed == 0:
        return np.zeros(n_batches, dtype=np.uint64)
    hi = np.uint64(1) << np.uint64(n_closed)
    return rng.integers(0, hi, size=n_batches, dtype=np.uint64)


# Named workloads.  Sizes follow the paper's sampling setting (batches of 2^6 open
# qubits, partial slicing) on grids small enough for one GPU.
WORKLOADS = {
    "grid3x4_m8": dict(rows=3, cols=4, cycles=8, seed=0, n_sliced=2, n_open=12),
    "grid4x7_m14": dict(rows=4, cols=7, cycles=14, seed=0, n_sliced=10, n_open=6, n_batches=256),
    "grid5x8_m16": dict(rows=5, cols=8, cycles=16, seed=0, n_sliced=14, n_open=6),
}


def default_open_qubits(rows: int, cols: int, n_open: int) -> list:
    """Open (batch) qubits: the last n_open qubits in row-major order (one grid corner)."""
    n = rows * cols
    return list(range(n - n_open, n))

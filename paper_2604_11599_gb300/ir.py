"""Flat lowered IR for dynamic circuits, and a small builder.

This module only defines the op-list *format* (a numpy structured dtype whose
layout is the C struct ``sv_op`` of ``include/sv.h``) and a builder that
appends records to it.  It holds no simulation arithmetic: gate matrices,
probabilities and draws live in the CUDA library (and, independently, in the
oracle).

The vocabulary follows the paper's statement of what the transpiler must carry
(Sec. III-B: standard gates and ``ctrl``/``inv`` modifiers; Sec. III-C:
``if`` on classical bits turned into device-side feed-forward; Sec. III-D:
``input`` parameters resolved at run time, so one compiled program serves
every parameter set; Abstract: conditionals and loops with a fixed trip count):

* ``GATE``     -- one standard gate (``Gate`` enum) on ``q[0..]``; each of its up
                  to three angles is a literal or ``scale * params[idx]``.
* ``DENSE``    -- a caller-supplied 2^k x 2^k unitary on ``q[0..k-1]``, read from a
                  complex128 pool at ``dense_off`` (row-major, local bit r <-> q[r]).
* ``MEASURE``  -- measure ``q[0]`` into classical bit ``cbit``.
* ``RESET``    -- measure ``q[0]`` (no classical write), then X if the outcome is 1.
* ``COND``     -- run the next ``then_len`` records iff ``(creg & mask) == value``,
                  otherwise the ``else_len`` records after them.
* ``LOOP``     -- run the next ``body_len`` records ``loop_k`` times.

Lengths count flat records, nested headers and bodies included (pre-order).
Qubit q is bit q of the amplitude index (little-endian); classical bit j is
bit j of the 64-bit creg.
"""
from __future__ import annotations

import enum
from dataclasses import dataclass
from typing import Callable, Optional, Sequence, Union

import numpy as np

MAX_Q = 8  # qubit slots per record (DENSE uses up to 8)


class Kind(enum.IntEnum):
    GATE = 1
    DENSE = 2
    MEASURE = 3
    RESET = 4
    COND = 5
    LOOP = 6


class Gate(enum.IntEnum):
    I = 0
    H = 1
    X = 2
    Y = 3
    Z = 4
    S = 5
    SDG = 6
    T = 7
    TDG = 8
    SX = 9
    RX = 10
    RY = 11
    RZ = 12
    P = 13
    U = 14
    CX = 15
    CY = 16
    CZ = 17
    SWAP = 18
    CP = 19
    CRX = 20
    CRY = 21
    CRZ = 22
    CH = 23
    CU = 24


# number of qubits and angles of each gate
GATE_ARITY = {
    Gate.I: (1, 0), Gate.H: (1, 0), Gate.X: (1, 0), Gate.Y: (1, 0), Gate.Z: (1, 0),
    Gate.S: (1, 0), Gate.SDG: (1, 0), Gate.T: (1, 0), Gate.TDG: (1, 0), Gate.SX: (1, 0),
    Gate.RX: (1, 1), Gate.RY: (1, 1), Gate.RZ: (1, 1), Gate.P: (1, 1), Gate.U: (1, 3),
    Gate.CX: (2, 0), Gate.CY: (2, 0), Gate.CZ: (2, 0), Gate.SWAP: (2, 0), Gate.CP: (2, 1),
    Gate.CRX: (2, 1), Gate.CRY: (2, 1), Gate.CRZ: (2, 1), Gate.CH: (2, 0), Gate.CU: (2, 3),
}

# the C struct sv_op: 120 bytes, 8-byte aligned
OP_DTYPE = np.dtype(
    {
        "names": ["kind", "gate", "cbit", "q", "pidx", "nq", "angle", "mask", "value",
                  "then_len", "else_len", "loop_k", "body_len", "dense_off"],
        "formats": ["<u2", "<u2", "<u4", ("<i4", (MAX_Q,)), ("<i4", (3,)), "<u4", ("<f8", (3,)),
                    "<u8", "<u8", "<u4", "<u4", "<u4", "<u4", "<u8"],
        "offsets": [0, 2, 4, 8, 40, 52, 56, 80, 88, 96, 100, 104, 108, 112],
        "itemsize": 120,
    }
)

# the C struct sv_pauli: X on qubit q iff bit q of x_mask; Z iff bit q of z_mask; Y iff both
PAULI_DTYPE = np.dtype(
    {"names": ["x_mask", "z_mask", "coeff"], "formats": ["<u8", "<u8", "<f8"],
     "offsets": [0, 8, 16], "itemsize": 24}
)


@dataclass(frozen=True)
class Param:
    """A reference to the run-time parameter array: angle = scale * params[idx]
    (an OpenQASM ``input`` variable, Sec. III-D)."""
    idx: int
    scale: float = 1.0


Angle = Union[float, Param]


class Circuit:
    """Append-only builder of the flat IR.

    ``cond`` and ``loop`` take callables that append the body, so nesting is
    written as ordinary Python::

        c = Circuit(3)
        c.h(0); c.measure(0, 0)
        c.cond(1, 1, lambda: c.x(0))          # conditional reset, Fig. 2
    """

    def __init__(self, n: int):
        self.n = int(n)
        self._recs: list[np.void] = []
        self.dense_pool: list[np.ndarray] = []
        self._dense_len = 0
        self.n_params = 0
        self._ops_cache = None  # (record list, its length, concatenated array)

    # -- low level -----------------------------------------------------------------
    def _rec(self, kind: Kind) -> np.ndarray:
        r = np.zeros(1, dtype=OP_DTYPE)
        r["kind"] = int(kind)
        r["q"] = -1
        r["pidx"] = -1
        return r

    def _push(self, r: np.ndarray) -> int:
        self._recs.append(r)
        return len(self._recs) - 1

    def gate(self, g: Gate, qubits: Sequence[int], angles: Sequence[Angle] = ()) -> "Circuit":
        nq, na = GATE_ARITY[Gate(g)]
        if len(qubits) != nq or len(angles) != na:
            raise ValueError(f"{Gate(g).name}: expected {nq} qubits / {na} angles")
        r = self._rec(Kind.GATE)
        r["gate"] = int(g)
        r["nq"] = nq
        for i, q in enumerate(qubits):
            r["q"][0, i] = int(q)
        for i, a in enumerate(angles):
            if isinstance(a, Param):
                r["pidx"][0, i] = a.idx
                r["angle"][0, i] = a.scale
                self.n_params = max(self.n_params, a.idx + 1)
            else:
                r["angle"][0, i] = float(a)
        self._push(r)
        return self

    def dense(self, qubits: Sequence[int], matrix: np.ndarray) -> "Circuit":
        k = len(qubits)
        m = np.asarray(matrix, dtype=np.complex128)
        if k < 1 or k > MAX_Q or m.shape != (1 << k, 1 << k):
            raise ValueError("dense: need k in 1..8 qubits and a 2^k x 2^k matrix")
        r = self._rec(Kind.DENSE)
        r["nq"] = k
        for i, q in enumerate(qubits):
            r["q"][0, i] = int(q)
        r["dense_off"] = self._dense_len
        self.dense_pool.append(m.reshape(-1))
        self._dense_len += m.size
        self._push(r)
        return self

    def measure(self, q: int, cbit: int) -> "Circuit":
        r = self._rec(Kind.MEASURE)
        r["q"][0, 0] = int(q)
        r["nq"] = 1
        r["cbit"] = int(cbit)
        self._push(r)
        return self

    def reset(self, q: int) -> "Circuit":
        r = self._rec(Kind.RESET)
        r["q"][0, 0] = int(q)
        r["nq"] = 1
        self._push(r)
        return self

    def cond(self, mask: int, value: int, then: Callable[[], object],
             orelse: Optional[Callable[[], object]] = None) -> "Circuit":
        r = self._rec(Kind.COND)
        r["mask"] = int(mask)
        r["value"] = int(value)
        at = self._push(r)
        n0 = len(self._recs)
        then()
        n1 = len(self._recs)
        if orelse is not None:
            orelse()
        n2 = len(self._recs)
        self._recs[at]["then_len"] = n1 - n0
        self._recs[at]["else_len"] = n2 - n1
        self._ops_cache = None
        return self

    def loop(self, k: int, body: Callable[[], object]) -> "Circuit":
        r = self._rec(Kind.LOOP)
        r["loop_k"] = int(k)
        at = self._push(r)
        n0 = len(self._recs)
        body()
        self._recs[at]["body_len"] = len(self._recs) - n0
        self._ops_cache = None
        return self

    # -- standard gates ------------------------------------------------------------
    def h(self, q): return self.gate(Gate.H, [q])
    def x(self, q): return self.gate(Gate.X, [q])
    def y(self, q): return self.gate(Gate.Y, [q])
    def z(self, q): return self.gate(Gate.Z, [q])
    def s(self, q): return self.gate(Gate.S, [q])
    def sdg(self, q): return self.gate(Gate.SDG, [q])
    def t(self, q): return self.gate(Gate.T, [q])
    def tdg(self, q): return self.gate(Gate.TDG, [q])
    def sx(self, q): return self.gate(Gate.SX, [q])
    def rx(self, q, a): return self.gate(Gate.RX, [q], [a])
    def ry(self, q, a): return self.gate(Gate.RY, [q], [a])
    def rz(self, q, a): return self.gate(Gate.RZ, [q], [a])
    def p(self, q, a): return self.gate(Gate.P, [q], [a])
    def u(self, q, th, ph, la): return self.gate(Gate.U, [q], [th, ph, la])
    def cx(self, c, t): return self.gate(Gate.CX, [c, t])
    def cy(self, c, t): return self.gate(Gate.CY, [c, t])
    def cz(self, a, b): return self.gate(Gate.CZ, [a, b])
    def ch(self, c, t): return self.gate(Gate.CH, [c, t])
    def swap(self, a, b): return self.gate(Gate.SWAP, [a, b])
    def cp(self, c, t, a): return self.gate(Gate.CP, [c, t], [a])
    def crx(self, c, t, a): return self.gate(Gate.CRX, [c, t], [a])
    def cry(self, c, t, a): return self.gate(Gate.CRY, [c, t], [a])
    def crz(self, c, t, a): return self.gate(Gate.CRZ, [c, t], [a])
    def cu(self, c, t, th, ph, la): return self.gate(Gate.CU, [c, t], [th, ph, la])

    # -- output --------------------------------------------------------------------
    @property
    def ops(self) -> np.ndarray:
        """The flat record array (a copy; built once per change of the program:
        appends and header edits invalidate it, and so does replacing the record
        list)."""
        if not self._recs:
            return np.zeros(0, dtype=OP_DTYPE)
        c = self._ops_cache
        if c is None or c[0] is not self._recs or c[1] != len(self._recs):
            c = (self._recs, len(self._recs), np.concatenate(self._recs))
            self._ops_cache = c
        return c[2].copy()

    @property
    def pool(self) -> np.ndarray:
        if not self.dense_pool:
            return np.zeros(0, dtype=np.complex128)
        return np.concatenate(self.dense_pool)

    def __len__(self) -> int:
        return len(self._recs)


def pauli_terms(terms: Sequence[tuple[str, float]]) -> np.ndarray:
    """Build an ``sv_pauli`` array from ``[("X0 Y3", c), ("Z1 Z2", c), ...]``."""
    out = np.zeros(len(terms), dtype=PAULI_DTYPE)
    for i, (s, c) in enumerate(terms):
        x = z = 0
        for tok in s.split():
            p, q = tok[0].upper(), int(tok[1:])
            if p in "XY":
                x |= 1 << q
            if p in "ZY":
                z |= 1 << q
        out[i] = (x, z, float(c))
    return out


def count_gate_records(ops: np.ndarray) -> dict:
    """Static counts over the flat list (bodies counted once, not per iteration)."""
    kinds = ops["kind"]
    return {k.name: int((kinds == int(k)).sum()) for k in Kind}

"""Independent references used only to pin the oracle (test code).

Nothing here is shared with the oracle or with the CUDA path:

* gate matrices come from ``scipy.linalg.expm`` of Pauli generators and from
  algebraic identities (H = (X+Z)/sqrt2, S = e^{i pi/4} exp(-i pi Z/4), ...),
  not from the oracle's table;
* whole-register operators are built as Kronecker products (2^n x 2^n dense
  matrices), a different formulation from the oracle's amplitude loops;
* a small CHP stabilizer tableau (Aaronson & Gottesman, "Improved simulation
  of stabilizer circuits", PRA 70, 052328 (2004)) pins Clifford circuits;
* draws are recomputed with numpy's own Philox4x64-10 implementation.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def rot(P, th):
    return sla.expm(-0.5j * th * P)


def ref_gate(name: str, angles=()):
    """(kind, matrix) with kind in {'1q', 'ctrl', 'swap'}; matrices from expm/identities."""
    a = list(angles) + [0.0] * 3
    base = {
        "I": I2,
        "H": (PX + PZ) / math.sqrt(2),
        "X": PX, "Y": PY, "Z": PZ,
        "S": np.exp(0.25j * math.pi) * rot(PZ, math.pi / 2),
        "SDG": np.exp(-0.25j * math.pi) * rot(PZ, -math.pi / 2),
        "T": np.exp(0.125j * math.pi) * rot(PZ, math.pi / 4),
        "TDG": np.exp(-0.125j * math.pi) * rot(PZ, -math.pi / 4),
        "SX": np.exp(0.25j * math.pi) * rot(PX, math.pi / 2),
        "RX": rot(PX, a[0]), "RY": rot(PY, a[0]), "RZ": rot(PZ, a[0]),
        "P": np.exp(0.5j * a[0]) * rot(PZ, a[0]),
        "U": np.exp(0.5j * (a[1] + a[2])) * rot(PZ, a[1]) @ rot(PY, a[0]) @ rot(PZ, a[2]),
    }
    if name in base:
        return "1q", base[name]
    if name == "SWAP":
        return "swap", None
    assert name.startswith("C")
    return "ctrl", ref_gate(name[1:], angles)[1]


def embed(n: int, ops: dict) -> np.ndarray:
    """Kronecker product over qubits n-1..0 (qubit q = bit q of the index)."""
    out = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        out = np.kron(out, ops.get(q, I2))
    return out


def full_gate(n: int, name: str, qubits, angles=()) -> np.ndarray:
    kind, m = ref_gate(name, angles)
    if kind == "1q":
        return embed(n, {qubits[0]: m})
    if kind == "ctrl":
        c, t = qubits
        return embed(n, {c: P0}) + embed(n, {c: P1, t: m})
    a, b = qubits  # SWAP = (I + XX + YY + ZZ)/2
    return 0.5 * (embed(n, {}) + embed(n, {a: PX, b: PX}) + embed(n, {a: PY, b: PY}) + embed(n, {a: PZ, b: PZ}))


def full_dense(n: int, qubits, u: np.ndarray) -> np.ndarray:
    """Embed a k-qubit matrix (local bit r <-> qubits[r]) entry by entry."""
    N = 1 << n
    k = len(qubits)
    qmask = sum(1 << q for q in qubits)
    F = np.zeros((N, N), dtype=complex)

    def loc(i):
        return sum(((i >> q) & 1) << r for r, q in enumerate(qubits))

    for i in range(N):
        for j in range(N):
            if (i & ~qmask) == (j & ~qmask):
                F[i, j] = u[loc(i), loc(j)]
    return F


GATE_NAMES = ["I", "H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "SX", "RX", "RY", "RZ", "P", "U",
              "CX", "CY", "CZ", "SWAP", "CP", "CRX", "CRY", "CRZ", "CH", "CU"]


def static_state(ops: np.ndarray, n: int, params=None, pool=None) -> np.ndarray:
    """Dense-matrix simulation of a static (gate-only) op list."""
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    for op in ops:
        kind = int(op["kind"])
        if kind == 1:
            name = GATE_NAMES[int(op["gate"])]
            nq = 2 if name.startswith("C") or name == "SWAP" else 1
            ang = []
            for i in range(3):
                if op["pidx"][i] >= 0:
                    ang.append(float(op["angle"][i]) * float(params[op["pidx"][i]]))
                else:
                    ang.append(float(op["angle"][i]))
            psi = full_gate(n, name, [int(v) for v in op["q"][:nq]], ang) @ psi
        elif kind == 2:
            k = int(op["nq"])
            off = int(op["dense_off"])
            u = np.asarray(pool[off: off + (1 << 2 * k)]).reshape(1 << k, 1 << k)
            psi = full_dense(n, [int(v) for v in op["q"][:k]], u) @ psi
        else:
            raise ValueError("static_state: gates only")
    return psi


def pauli_matrix(n: int, x: int, z: int) -> np.ndarray:
    ops = {}
    for q in range(n):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        if xb and zb:
            ops[q] = PY
        elif xb:
            ops[q] = PX
        elif zb:
            ops[q] = PZ
    return embed(n, ops)


def hamiltonian(n: int, terms) -> np.ndarray:
    H = np.zeros((1 << n, 1 << n), dtype=complex)
    for t in terms:
        H += float(t["coeff"]) * pauli_matrix(n, int(t["x_mask"]), int(t["z_mask"]))
    return H


# ------------------------------------------------------------------ numpy Philox
def np_philox_block(ctr, key) -> np.ndarray:
    """Philox4x64-10 block for counter ``ctr`` via numpy (which pre-increments)."""
    c = [int(v) % (1 << 64) for v in ctr]
    # numpy generates from counter + 1: hand it ctr - 1 (256-bit borrow)
    val = sum(c[i] << (64 * i) for i in range(4))
    val = (val - 1) % (1 << 256)
    start = np.array([(val >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    return bg.random_raw(4).astype(np.uint64)


def np_uniform(seed, stream, shot, m) -> float:
    w = int(np_philox_block([shot, m, 0, 0], [seed, stream])[0])
    return (w >> 11) * 2.0 ** -53


# ------------------------------------------------------------------ CHP tableau
class Tableau:
    """Stabilizer rows only (enough to pin states of unitary Clifford circuits)."""

    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((n, n), dtype=np.uint8)
        self.z = np.eye(n, dtype=np.uint8)
        self.r = np.zeros(n, dtype=np.uint8)

    def h(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def cx(self, a, b):
        self.r ^= self.x[:, a] & self.z[:, b] & (self.x[:, b] ^ self.z[:, a] ^ 1)
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def pauli(self, a, p):
        if p == "X":
            self.r ^= self.z[:, a]
        elif p == "Z":
            self.r ^= self.x[:, a]
        else:
            self.r ^= self.x[:, a] ^ self.z[:, a]

    def apply(self, name, qs):
        if name == "H":
            self.h(qs[0])
        elif name == "S":
            self.s(qs[0])
        elif name == "SDG":
            for _ in range(3):
                self.s(qs[0])
        elif name in ("X", "Y", "Z"):
            self.pauli(qs[0], name)
        elif name == "CX":
            self.cx(*qs)
        elif name == "CZ":
            self.h(qs[1]); self.cx(*qs); self.h(qs[1])
        elif name == "SWAP":
            a, b = qs
            self.cx(a, b); self.cx(b, a); self.cx(a, b)
        else:
            raise ValueError(name)

    def generators(self):
        """[(sign, x_mask, z_mask)]"""
        out = []
        for i in range(self.n):
            xm = sum(int(self.x[i, q]) << q for q in range(self.n))
            zm = sum(int(self.z[i, q]) << q for q in range(self.n))
            out.append((-1 if self.r[i] else 1, xm, zm))
        return out

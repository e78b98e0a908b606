"""Seeded synthetic circuit generators.

Everything here draws *inputs* only (gate kinds, qubits, angles, predicates,
parameter sets, Hamiltonian terms, arrival times) with
``numpy.random.Generator(PCG64(seed))``.  No simulation arithmetic lives here;
the CUDA path and the oracle both consume what these functions return.

The paper's workloads are IBM-guide style feed-forward programs (Abstract:
conditional reset, if-else, multi-bit predicates, sequential feed-forward;
Fig. 2 and Sec. IV-C: conditional reset; Sec. IV-A.2: teleportation with
uncompute, random Clifford circuits with d in [10,100] and n in [2,20], QFT
and Bernstein-Vazirani) and a hardware-efficient VQE ansatz (Sec. IV-A.2,
Sec. IV-D).  The guide's own circuit files are not available, so the patterns
are regenerated from those descriptions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .ir import Circuit, Gate, Param, PAULI_DTYPE

TWO_PI = 2.0 * math.pi


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------------

_C1_GATES = ("H", "X", "RX", "RY", "RZ", "CX", "CZ")


def _random_gate(c: Circuit, r: np.random.Generator, n: int, kinds=_C1_GATES) -> None:
    k = kinds[int(r.integers(len(kinds)))]
    if k in ("CX", "CZ") and n >= 2:
        a, b = (int(v) for v in r.choice(n, size=2, replace=False))
        (c.cx if k == "CX" else c.cz)(a, b)
        return
    if k in ("CX", "CZ"):
        k = "H"
    q = int(r.integers(n))
    if k == "H":
        c.h(q)
    elif k == "X":
        c.x(q)
    else:
        getattr(c, k.lower())(q, float(r.uniform(0.0, TWO_PI)))


def _rotation_layer(c: Circuit, r: np.random.Generator, qubits) -> None:
    """A random single-qubit rotation (RX, RY or RZ, uniform kind) with theta~U[0,2pi) on each qubit."""
    for q in qubits:
        kind = int(r.integers(3))
        th = float(r.uniform(0.0, TWO_PI))
        (c.rx, c.ry, c.rz)[kind](q, th)


def _matching_layer(c: Circuit, r: np.random.Generator, qubits) -> None:
    """CX on a uniform random perfect matching of ``qubits`` (one left out if odd)."""
    perm = [qubits[i] for i in r.permutation(len(qubits))]
    for i in range(0, len(perm) - 1, 2):
        c.cx(perm[i], perm[i + 1])


def _deposit(bits: list[int], v: int) -> int:
    out = 0
    for i, b in enumerate(bits):
        if (v >> i) & 1:
            out |= 1 << b
    return out


# ----------------------------------------------------------------------------------
# the five benchmark workloads
# ----------------------------------------------------------------------------------

def plain_small(seed: int = 1, n: int = 5, n_gates: int = 40, every: int = 8) -> Circuit:
    """Plain-path feed-forward program: ``n_gates`` gates uniform over
    {H, X, RX, RY, RZ, CX, CZ} (angles U[0,2pi)); after every ``every`` gates a
    measure of a random qubit into the next classical bit j, followed by a
    conditional reset ``if (c[j]==1) x`` and an if-else on the 2-bit predicate
    {c[j], c[j-1]} (c[1] when j=0) whose branches are one random gate each."""
    r = rng(seed)
    c = Circuit(n)
    j = 0
    for g in range(1, n_gates + 1):
        _random_gate(c, r, n)
        if g % every == 0:
            q = int(r.integers(n))
            c.measure(q, j)
            c.cond(1 << j, 1 << j, lambda q=q: c.x(q))
            bits = [j, j - 1 if j > 0 else 1]
            mask = _deposit(bits, 3)
            value = _deposit(bits, int(r.integers(4)))
            c.cond(mask, value, lambda: _random_gate(c, r, n), lambda: _random_gate(c, r, n))
            j += 1
    return c


# generator seed of the layered program for each (n, state type) of the plain-path
# workload at full size: n=28/30 in complex128 and complex64
LAYERED_SEEDS = {(28, "c128"): 2, (28, "c64"): 3, (30, "c128"): 4, (30, "c64"): 5}


def layered(seed: int, n: int, layers: int = 20, block: int = 4) -> Circuit:
    """Layered dynamic circuit: each layer is a random rotation on every qubit
    then CX on a random perfect matching; after every ``block`` layers, measure
    two distinct random qubits into the next two classical bits, reset both,
    then ``cond(last three written bits == v)`` with X on the first and, in the
    else branch, Z on the second (v ~ U{0..7})."""
    r = rng(seed)
    c = Circuit(n)
    qs = list(range(n))
    cb = 0
    for layer in range(1, layers + 1):
        _rotation_layer(c, r, qs)
        _matching_layer(c, r, qs)
        if layer % block == 0:
            qa, qb = (int(v) for v in r.choice(n, size=2, replace=False))
            c.measure(qa, cb)
            c.measure(qb, cb + 1)
            c.reset(qa)
            c.reset(qb)
            bits = [cb + 1, cb, cb - 1 if cb > 0 else cb + 2]
            mask = _deposit(bits, 7)
            value = _deposit(bits, int(r.integers(8)))
            c.cond(mask, value, lambda qa=qa: c.x(qa), lambda qb=qb: c.z(qb))
            cb += 2
    return c


def sequential_feedforward(seed: int, n: int, layers: int = 10, rus_k: int = 4) -> Circuit:
    """Batching workload circuit on n data qubits plus one ancilla (index n):
    ``layers`` layers as in :func:`layered` (no mid-circuit measures), then for
    i = 0..n-2 measure q_i into c[i] and ``if (c[i]==1) ry(theta_i) q_{i+1}``;
    then repeat-until-success ``loop(rus_k) { if (c[63]==0) { reset a; ry(theta_r) a;
    measure a -> c[63] } }``."""
    r = rng(seed)
    c = Circuit(n + 1)
    qs = list(range(n))
    for _ in range(layers):
        _rotation_layer(c, r, qs)
        _matching_layer(c, r, qs)
    for i in range(n - 1):
        c.measure(i, i)
        th = float(r.uniform(0.0, TWO_PI))
        c.cond(1 << i, 1 << i, lambda i=i, th=th: c.ry(i + 1, th))
    a = n
    th_r = float(r.uniform(0.0, TWO_PI))

    def body():
        def attempt():
            c.reset(a)
            c.ry(a, th_r)
            c.measure(a, 63)
        c.cond(1 << 63, 0, attempt)

    c.loop(rus_k, body)
    c.rus_theta = th_r  # recorded for the success-probability pin
    return c


@dataclass
class BatchWorkload:
    circuits: dict  # n -> Circuit
    traj_n: np.ndarray  # per-trajectory data-qubit count
    seed: int = 6


def batching(seed: int = 6, n_traj: int = 65536, n_lo: int = 12, n_hi: int = 20,
             layers: int = 10) -> BatchWorkload:
    """Independent trajectories with n ~ U{n_lo..n_hi}; one seeded circuit per n,
    trajectory t keyed by Philox stream t."""
    r = rng(seed)
    traj_n = r.integers(n_lo, n_hi + 1, size=n_traj)
    circs = {n: sequential_feedforward(seed * 1000 + n, n, layers) for n in range(n_lo, n_hi + 1)}
    return BatchWorkload(circs, traj_n, seed)


def hea(n: int = 20, layers: int = 8) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta) then RZ(phi) on every qubit,
    then a CX ladder CX(0,1)..CX(n-2,n-1).  Layer L uses parameters
    2nL+q (RY) and 2nL+n+q (RZ); 2*n*layers parameters in all."""
    c = Circuit(n)
    for L in range(layers):
        for q in range(n):
            c.ry(q, Param(2 * n * L + q))
        for q in range(n):
            c.rz(q, Param(2 * n * L + n + q))
        for q in range(n - 1):
            c.cx(q, q + 1)
    return c


def hea_params(seed: int = 8, sets: int = 1024, n_params: int = 320) -> np.ndarray:
    return rng(seed).uniform(-math.pi, math.pi, size=(sets, n_params))


def heisenberg_fields(seed: int = 9, n: int = 20, n_terms: int = 200) -> np.ndarray:
    """Periodic 1D Heisenberg X_jX_{j+1}, Y_jY_{j+1}, Z_jZ_{j+1} over n bonds,
    plus random single-site X/Y/Z fields up to ``n_terms`` terms (duplicates
    kept); every coefficient ~N(0,1)."""
    r = rng(seed)
    terms = []
    for j in range(n):
        k = (j + 1) % n
        for p in "XYZ":
            terms.append((p, j, k))
    while len(terms) < n_terms:
        terms.append(("XYZ"[int(r.integers(3))], int(r.integers(n)), None))
    out = np.zeros(len(terms), dtype=PAULI_DTYPE)
    coeffs = r.normal(size=len(terms))
    for i, (p, a, b) in enumerate(terms):
        x = z = 0
        for q in (a,) if b is None else (a, b):
            if p in "XY":
                x |= 1 << q
            if p in "ZY":
                z |= 1 << q
        out[i] = (x, z, coeffs[i])
    return out


@dataclass
class Request:
    rid: int
    arrival: float
    n: int
    circuit: Circuit
    shots: int


def serving_stream(seed: int = 10, gen_seed: int = 11, rate: float = 200.0, duration: float = 60.0,
                   n_lo: int = 10, n_hi: int = 30, d_lo: int = 10, d_hi: int = 100,
                   max_shots: int = 4096, limit: int | None = None) -> list[Request]:
    """Poisson arrivals at ``rate``/s for ``duration`` s; per request n and depth
    log-uniform, 1-8 mid-circuit measures at random layer boundaries, each
    followed by a random feed-forward (a 1-3 bit predicate applying X or Z, or
    a loop(k<=4) repeat-until-success on the measured qubit), shots
    log-uniform in 1..max_shots."""
    ra = rng(seed)
    rg = rng(gen_seed)
    t = 0.0
    out: list[Request] = []
    rid = 0
    while True:
        t += float(ra.exponential(1.0 / rate))
        if t >= duration or (limit is not None and rid >= limit):
            break
        n = int(round(math.exp(rg.uniform(math.log(n_lo), math.log(n_hi)))))
        depth = int(round(math.exp(rg.uniform(math.log(d_lo), math.log(d_hi)))))
        n_meas = int(rg.integers(1, 9))
        shots = int(round(math.exp(rg.uniform(0.0, math.log(max_shots)))))
        out.append(Request(rid, t, n, _serving_circuit(rg, n, depth, n_meas), shots))
        rid += 1
    return out


def _serving_circuit(r: np.random.Generator, n: int, depth: int, n_meas: int) -> Circuit:
    c = Circuit(n)
    qs = list(range(n))
    where = sorted(int(v) for v in r.choice(np.arange(1, depth + 1), size=min(n_meas, depth), replace=False))
    cb = 0
    for layer in range(1, depth + 1):
        _rotation_layer(c, r, qs)
        _matching_layer(c, r, qs)
        while where and where[0] == layer:
            where.pop(0)
            q = int(r.integers(n))
            c.measure(q, cb)
            if r.random() < 0.5 or cb == 0:
                k = int(r.integers(1, 4))
                bits = [cb - i for i in range(k) if cb - i >= 0]
                mask = _deposit(bits, (1 << len(bits)) - 1)
                value = _deposit(bits, int(r.integers(1 << len(bits))))
                tq = int(r.integers(n))
                if r.random() < 0.5:
                    c.cond(mask, value, lambda tq=tq: c.x(tq))
                else:
                    c.cond(mask, value, lambda tq=tq: c.z(tq))
            else:
                k = int(r.integers(1, 5))
                th = float(r.uniform(0.0, TWO_PI))
                bit = cb

                def body(q=q, th=th, bit=bit):
                    def attempt():
                        c.reset(q)
                        c.ry(q, th)
                        c.measure(q, bit)
                    c.cond(1 << bit, 0, attempt)

                c.loop(k, body)
            cb = min(cb + 1, 62)
    return c


# ----------------------------------------------------------------------------------
# small programs used as pins and parity cases
# ----------------------------------------------------------------------------------

def conditional_reset(minus: bool = True) -> Circuit:
    """Fig. 2 / Sec. IV-C: prepare |+> (or |->), measure, if (c==1) X."""
    c = Circuit(1)
    if minus:
        c.x(0)
    c.h(0)
    c.measure(0, 0)
    c.cond(1, 1, lambda: c.x(0))
    return c


def teleport_uncompute(theta: float, phi: float, lam: float) -> Circuit:
    """Sec. IV-A.2: teleport U(theta,phi,lam)|0> from q0 to q2 with two
    mid-circuit measures and feed-forward, then apply the inverse of U on q2
    (U(-theta,-lam,-phi)); q2 returns to |0> deterministically."""
    c = Circuit(3)
    c.u(0, theta, phi, lam)
    c.h(1)
    c.cx(1, 2)
    c.cx(0, 1)
    c.h(0)
    c.measure(0, 0)
    c.measure(1, 1)
    c.cond(2, 2, lambda: c.x(2))
    c.cond(1, 1, lambda: c.z(2))
    c.u(2, -theta, -lam, -phi)
    return c


def ghz(n: int) -> Circuit:
    c = Circuit(n)
    c.h(0)
    for q in range(n - 1):
        c.cx(q, q + 1)
    return c


def qft_on_basis(n: int, x: int) -> Circuit:
    """Prepare |x> then the textbook QFT (Hadamards, controlled phases, final swaps),
    written for little-endian indices so that the output is sum_k e^{2 pi i x k/2^n}|k>/sqrt(2^n)."""
    c = Circuit(n)
    for q in range(n):
        if (x >> q) & 1:
            c.x(q)
    for j in reversed(range(n)):
        c.h(j)
        for k in reversed(range(j)):
            c.cp(k, j, math.pi / (1 << (j - k)))
    for q in range(n // 2):
        c.swap(q, n - 1 - q)
    return c


def bernstein_vazirani(n: int, secret: int) -> Circuit:
    """n input qubits and one target (index n): H on inputs, target in |->,
    CX from every input i with secret bit i set, H on inputs, measure inputs."""
    c = Circuit(n + 1)
    c.x(n)
    c.h(n)
    for q in range(n):
        c.h(q)
    for q in range(n):
        if (secret >> q) & 1:
            c.cx(q, n)
    for q in range(n):
        c.h(q)
    for q in range(n):
        c.measure(q, q)
    return c


def random_clifford(seed: int, n: int, depth: int) -> Circuit:
    """Random Clifford circuit over {H, S, SDG, X, Y, Z, CX, CZ, SWAP} (Sec. IV-A.2 static suite)."""
    r = rng(seed)
    c = Circuit(n)
    one = ("H", "S", "SDG", "X", "Y", "Z")
    two = ("CX", "CZ", "SWAP")
    for _ in range(depth):
        if n >= 2 and r.random() < 0.4:
            a, b = (int(v) for v in r.choice(n, size=2, replace=False))
            getattr(c, two[int(r.integers(3))].lower())(a, b)
        else:
            getattr(c, one[int(r.integers(6))].lower())(int(r.integers(n)))
    return c


def random_clifford_dynamic(seed: int, n: int, n_ops: int = 80, max_depth: int = 3) -> Circuit:
    """Random dynamic Clifford program: gates over {H, S, SDG, X, Y, Z, SX, CX,
    CY, CZ, SWAP}, measures into 6 classical bits, resets, nested if/else on
    1-3 bit predicates and bounded loops (the static suite's gate set, Sec.
    IV-A.2, with the feed-forward patterns of the Abstract)."""
    r = rng(seed)
    c = Circuit(n)
    one = ("h", "s", "sdg", "x", "y", "z", "sx")
    two = ("cx", "cy", "cz", "swap")
    state = {"left": n_ops}

    def gate():
        if n >= 2 and r.random() < 0.4:
            a, b = (int(v) for v in r.choice(n, size=2, replace=False))
            getattr(c, two[int(r.integers(len(two)))])(a, b)
        else:
            getattr(c, one[int(r.integers(len(one)))])(int(r.integers(n)))

    def block(depth: int, budget: int):
        for _ in range(budget):
            if state["left"] <= 0:
                return
            state["left"] -= 1
            u = r.random()
            if u < 0.6:
                gate()
            elif u < 0.75:
                c.measure(int(r.integers(n)), int(r.integers(6)))
            elif u < 0.82:
                c.reset(int(r.integers(n)))
            elif u < 0.94 and depth < max_depth:
                k = int(r.integers(1, 4))
                bits = [int(v) for v in r.choice(6, size=k, replace=False)]
                mask = _deposit(bits, (1 << k) - 1)
                value = _deposit(bits, int(r.integers(1 << k)))
                t = int(r.integers(1, 5))
                e = int(r.integers(0, 4))
                c.cond(mask, value, lambda: block(depth + 1, t),
                       (lambda: block(depth + 1, e)) if e else None)
            elif depth < max_depth:
                k = int(r.integers(1, 4))
                b = int(r.integers(1, 5))
                c.loop(k, lambda: block(depth + 1, b))

    while state["left"] > 0:
        block(0, state["left"])
    return c


def repetition_code(d: int, rounds: int, flip_every: int = 0, ghz: bool = False) -> Circuit:
    """Bit-flip repetition code of distance d (3 <= d <= 32): data qubits
    0..d-1, ancillas d..2d-2.  Each round measures the d-1 neighbour parities
    Z_j Z_{j+1} through an ancilla (CX, CX, measure into bit 32 + j, reset)
    and corrects a single flipped data qubit by feed-forward: qubit i (inner)
    when parities i-1 and i are set, qubit 0 when parity 0 alone is set among
    parities 0, 1, qubit d-1 when parity d-2 alone is set among d-3, d-2.
    flip_every > 0 applies X to data qubit (t mod d) before every
    flip_every-th round t.  ghz: the data starts in (|0...0> + |1...1>)/sqrt 2
    (H, CX chain), which every parity check leaves unchanged.  At the end the
    data qubits are read into bits 0..d-1: all zero (ghz=False) or all equal,
    each value with probability 1/2 (ghz=True), and a round's syndrome bits
    depend only on the flips."""
    if not 3 <= d <= 32:
        raise ValueError("distance out of range")
    c = Circuit(2 * d - 1)
    if ghz:
        c.h(0)
        for i in range(d - 1):
            c.cx(i, i + 1)
    for t in range(rounds):
        if flip_every and t % flip_every == 0:
            c.x(t % d)
        for j in range(d - 1):
            a = d + j
            c.cx(j, a).cx(j + 1, a)
            c.measure(a, 32 + j)
            c.reset(a)
        for i in range(d):
            if i == 0:
                mask, value = (1 << 32) | (1 << 33), 1 << 32
            elif i == d - 1:
                mask, value = (1 << (32 + d - 3)) | (1 << (32 + d - 2)), 1 << (32 + d - 2)
            else:
                mask = value = (1 << (32 + i - 1)) | (1 << (32 + i))
            c.cond(mask, value, lambda i=i: c.x(i))
    for i in range(d):
        c.measure(i, i)
    return c


_ALL_1Q = ("H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "SX")
_ALL_1Q_ANG = ("RX", "RY", "RZ", "P")
_ALL_2Q = ("CX", "CY", "CZ", "SWAP", "CH")
_ALL_2Q_ANG = ("CP", "CRX", "CRY", "CRZ")


def haar_unitary(r: np.random.Generator, k: int) -> np.ndarray:
    """A 2^k x 2^k unitary from the QR decomposition of a complex Gaussian
    matrix, phases of R's diagonal folded in (Haar-distributed)."""
    a = r.normal(size=(1 << k, 1 << k)) + 1j * r.normal(size=(1 << k, 1 << k))
    qm, rm = np.linalg.qr(a)
    return qm * (np.diag(rm) / np.abs(np.diag(rm)))


def dense_layers(seed: int, n: int, layers: int = 8, k: int = 4) -> Circuit:
    """Layers of dense k-qubit unitaries: each layer partitions the qubits at
    random into groups of k and applies a Haar-random unitary to each group;
    the n mod k qubits left over get a random RX/RY/RZ."""
    r = rng(seed)
    c = Circuit(n)
    for _ in range(layers):
        perm = [int(v) for v in r.permutation(n)]
        for g in range(n // k):
            c.dense(perm[g * k:(g + 1) * k], haar_unitary(r, k))
        for q in perm[(n // k) * k:]:
            kind = int(r.integers(3))
            (c.rx, c.ry, c.rz)[kind](q, float(r.uniform(0.0, TWO_PI)))
    return c


def random_static(seed: int, n: int, depth: int, dense_k: int = 0, params: int = 0) -> Circuit:
    """Random circuit over the whole gate vocabulary (optionally with dense
    k-qubit unitaries drawn from QR of a complex Gaussian, and parameter refs)."""
    r = rng(seed)
    c = Circuit(n)

    def ang():
        if params and r.random() < 0.5:
            return Param(int(r.integers(params)), float(r.choice([1.0, -1.0, 0.5, 2.0])))
        return float(r.uniform(0.0, TWO_PI))

    for _ in range(depth):
        u = r.random()
        if dense_k and n >= dense_k and u < 0.1:
            qs = [int(v) for v in r.choice(n, size=dense_k, replace=False)]
            c.dense(qs, haar_unitary(r, dense_k))
        elif n >= 2 and u < 0.35:
            a, b = (int(v) for v in r.choice(n, size=2, replace=False))
            if r.random() < 0.5:
                c.gate(Gate[_ALL_2Q[int(r.integers(len(_ALL_2Q)))]], [a, b])
            elif r.random() < 0.8:
                c.gate(Gate[_ALL_2Q_ANG[int(r.integers(len(_ALL_2Q_ANG)))]], [a, b], [ang()])
            else:
                c.gate(Gate.CU, [a, b], [ang(), ang(), ang()])
        elif u < 0.6:
            c.gate(Gate[_ALL_1Q[int(r.integers(len(_ALL_1Q)))]], [int(r.integers(n))])
        elif u < 0.9:
            c.gate(Gate[_ALL_1Q_ANG[int(r.integers(len(_ALL_1Q_ANG)))]], [int(r.integers(n))], [ang()])
        else:
            c.gate(Gate.U, [int(r.integers(n))], [ang(), ang(), ang()])
    return c


def random_dynamic(seed: int, n: int, n_ops: int = 60, max_depth: int = 3, dense_k: int = 0) -> Circuit:
    """Random dynamic program: gates, measures, resets, nested if/else on 1-3 bit
    predicates and bounded loops, to exercise every control-flow path."""
    r = rng(seed)
    c = Circuit(n)
    state = {"left": n_ops}

    def block(depth: int, budget: int):
        for _ in range(budget):
            if state["left"] <= 0:
                return
            state["left"] -= 1
            u = r.random()
            if u < 0.55:
                if dense_k and n >= dense_k and r.random() < 0.1:
                    qs = [int(v) for v in r.choice(n, size=dense_k, replace=False)]
                    a = r.normal(size=(1 << dense_k,) * 2) + 1j * r.normal(size=(1 << dense_k,) * 2)
                    qm, _ = np.linalg.qr(a)
                    c.dense(qs, qm)
                else:
                    _random_gate(c, r, n, ("H", "X", "RX", "RY", "RZ", "CX", "CZ"))
            elif u < 0.7:
                c.measure(int(r.integers(n)), int(r.integers(6)))
            elif u < 0.77:
                c.reset(int(r.integers(n)))
            elif u < 0.93 and depth < max_depth:
                k = int(r.integers(1, 4))
                bits = [int(v) for v in r.choice(6, size=k, replace=False)]
                mask = _deposit(bits, (1 << k) - 1)
                value = _deposit(bits, int(r.integers(1 << k)))
                t = int(r.integers(1, 5))
                e = int(r.integers(0, 4))
                c.cond(mask, value, lambda: block(depth + 1, t),
                       (lambda: block(depth + 1, e)) if e else None)
            elif depth < max_depth:
                k = int(r.integers(1, 4))
                b = int(r.integers(1, 5))
                c.loop(k, lambda: block(depth + 1, b))

    while state["left"] > 0:
        block(0, state["left"])
    return c

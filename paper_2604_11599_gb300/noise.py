"""Noise by trajectories: Pauli and readout channels lowered into the flat IR.

The paper mentions a noisy run of its conditional-reset circuit (Sec. IV-C)
and names noise among the things the state-vector path leaves for later
(Sec. VI).  Here a channel is sampled per trajectory with the same
counter-based draws as the measurements, so every engine that runs the IR
(plain path, batched launch, shot branching) runs noisy programs unchanged:

* a Bernoulli(p) decision is an ancilla qubit reset to |0>, rotated by
  RY(2 asin(sqrt p)) so that it reads 1 with probability p, and measured into
  a scratch classical bit;
* a Pauli channel (X, Y, Z with probabilities px, py, pz) first decides
  whether an error happens (px + py + pz), then which one (X with
  px / (px+py+pz), else Y with py / (py+pz), else Z), and applies it under
  COND records on the scratch bits;
* a readout error with probability p wraps the measurement in X ... X under
  the same decision: the record is flipped and the post-measurement state is
  the one of the true outcome.

Each decision costs one reset draw and one measurement draw of the ancilla
and one extra qubit for the whole program; the three scratch bits (61, 62,
63 by default) must not be used by the program.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .ir import OP_DTYPE, Circuit, Gate, Kind

TWO_QUBIT = {Gate.CX, Gate.CY, Gate.CZ, Gate.SWAP, Gate.CP, Gate.CRX, Gate.CRY, Gate.CRZ, Gate.CH, Gate.CU}


@dataclass
class NoiseModel:
    """Depolarising probability after every one-qubit gate (p1) and on each
    qubit of every two-qubit gate (p2), X/Y/Z equally likely; readout flip
    probability (p_meas); probability that a reset leaves |1> (p_reset)."""
    p1: float = 0.0
    p2: float = 0.0
    p_meas: float = 0.0
    p_reset: float = 0.0

    def __post_init__(self):
        for name in ("p1", "p2", "p_meas", "p_reset"):
            v = getattr(self, name)
            if not 0.0 <= v <= 1.0:
                raise ValueError(f"{name} = {v} is not a probability")


def bernoulli(c: Circuit, anc: int, bit: int, p: float) -> None:
    """Scratch bit `bit` := 1 with probability p (ancilla reset, RY, measure)."""
    c.reset(anc)
    c.ry(anc, 2.0 * math.asin(math.sqrt(min(max(p, 0.0), 1.0))))
    c.measure(anc, bit)


def pauli_channel(c: Circuit, q: int, px: float, py: float, pz: float, anc: int, bits=(61, 62, 63)) -> None:
    """X, Y or Z on qubit q with probabilities px, py, pz (nothing otherwise)."""
    tot = px + py + pz
    if tot <= 0.0:
        return
    if tot > 1.0 + 1e-12:
        raise ValueError("px + py + pz exceeds 1")
    b0, b1, b2 = bits

    def which():
        bernoulli(c, anc, b1, px / tot)

        def y_or_z():
            if py + pz <= 0.0:
                return
            bernoulli(c, anc, b2, py / (py + pz))
            c.cond(1 << b2, 1 << b2, lambda: c.y(q), lambda: c.z(q))

        c.cond(1 << b1, 1 << b1, lambda: c.x(q), y_or_z)

    bernoulli(c, anc, b0, min(tot, 1.0))
    c.cond(1 << b0, 1 << b0, which)


def depolarize(c: Circuit, q: int, p: float, anc: int, bits=(61, 62, 63)) -> None:
    pauli_channel(c, q, p / 3, p / 3, p / 3, anc, bits)


def noisy_measure(c: Circuit, q: int, cbit: int, p: float, anc: int, bits=(61, 62, 63)) -> None:
    """Measure q into cbit with the record flipped with probability p."""
    if p <= 0.0:
        c.measure(q, cbit)
        return
    b0 = bits[0]
    bernoulli(c, anc, b0, p)
    c.cond(1 << b0, 1 << b0, lambda: c.x(q))
    c.measure(q, cbit)
    c.cond(1 << b0, 1 << b0, lambda: c.x(q))


def noisy_reset(c: Circuit, q: int, p: float, anc: int, bits=(61, 62, 63)) -> None:
    """Reset q, leaving |1> with probability p."""
    c.reset(q)
    if p > 0.0:
        b0 = bits[0]
        bernoulli(c, anc, b0, p)
        c.cond(1 << b0, 1 << b0, lambda: c.x(q))


def with_noise(circ: Circuit, model: NoiseModel, anc: Optional[int] = None, bits=(61, 62, 63)) -> Circuit:
    """The same program with the model's channels after its gates, on its
    measurements and on its resets, on circ.n + 1 qubits (the last one is the
    ancilla unless `anc` names a qubit the program does not touch).  COND and
    LOOP structure is kept: a loop body's channels run on every iteration."""
    ops = circ.ops
    for b in bits:
        if not 0 <= b < 64:
            raise ValueError("scratch bits must lie in 0..63")
    used = set()
    for o in ops:
        k = int(o["kind"])
        if k == Kind.MEASURE:
            used.add(int(o["cbit"]))
        elif k == Kind.COND:
            m = int(o["mask"])
            used |= {i for i in range(64) if (m >> i) & 1}
    if used & set(bits):
        raise ValueError(f"the program uses scratch bits {sorted(used & set(bits))}")
    n = circ.n
    if anc is None:
        anc = n
        out = Circuit(n + 1)
    else:
        out = Circuit(max(n, anc + 1))
    out.dense_pool = list(circ.dense_pool)  # DENSE records keep their pool offsets
    out._dense_len = circ._dense_len
    out.n_params = circ.n_params

    def copy(o):
        r = np.zeros(1, dtype=OP_DTYPE)
        r[0] = o
        out._push(r)

    def emit(i0: int, i1: int):
        i = i0
        while i < i1:
            o = ops[i]
            k = int(o["kind"])
            if k in (Kind.GATE, Kind.DENSE):
                copy(o)
                if k == Kind.GATE:  # a dense gate takes the two-qubit rate on each of its qubits
                    g = int(o["gate"])
                    qs = [int(o["q"][0]), int(o["q"][1])] if g in TWO_QUBIT else [int(o["q"][0])]
                    p = model.p2 if g in TWO_QUBIT else model.p1
                else:
                    qs = [int(v) for v in o["q"][: int(o["nq"])]]
                    p = model.p2
                for q in qs:
                    depolarize(out, q, p, anc, bits)
                i += 1
            elif k == Kind.MEASURE:
                noisy_measure(out, int(o["q"][0]), int(o["cbit"]), model.p_meas, anc, bits)
                i += 1
            elif k == Kind.RESET:
                noisy_reset(out, int(o["q"][0]), model.p_reset, anc, bits)
                i += 1
            elif k == Kind.COND:
                tl, el = int(o["then_len"]), int(o["else_len"])
                t0, t1, e1 = i + 1, i + 1 + tl, i + 1 + tl + el
                out.cond(int(o["mask"]), int(o["value"]), lambda t0=t0, t1=t1: emit(t0, t1),
                         (lambda t1=t1, e1=e1: emit(t1, e1)) if el else None)
                i = e1
            elif k == Kind.LOOP:
                bl = int(o["body_len"])
                b0, b1 = i + 1, i + 1 + bl
                out.loop(int(o["loop_k"]), lambda b0=b0, b1=b1: emit(b0, b1))
                i = b1
            else:
                raise ValueError(f"unknown record kind {k}")

    emit(0, len(ops))
    return out


__all__ = ["NoiseModel", "bernoulli", "pauli_channel", "depolarize", "noisy_measure", "noisy_reset", "with_noise"]

"""Plain CPU model of the stabilizer-tableau algorithm the Clifford kernel runs
(test code: it pins the update rules against the state-vector oracle on the
CPU, so that the kernel's arithmetic has a checked statement in Python).

Aaronson and Gottesman, "Improved simulation of stabilizer circuits" (2004):
rows 0..n-1 are destabilisers, rows n..2n-1 stabilisers, each a Pauli string
with x bits, z bits (Y = both) and a sign bit r.  Gates conjugate every row;
a measurement of qubit q is random iff some stabiliser has x_q = 1.  Draws
follow the state-vector convention: the m-th draw of a shot uses u(seed,
stream, shot, m) and takes outcome 1 iff u >= p0 / (p0 + p1); a random
outcome of a stabiliser state has p0 = p1, so outcome 1 iff u >= 1/2.
"""
from __future__ import annotations

from paper_2604_11599_gb300.ir import Gate, Kind


def g_sum(ix: int, iz: int, hx: int, hz: int) -> int:
    """Sum over qubits of the exponent of i in (row i's Pauli) x (row h's Pauli)."""
    a, b, c, d = ix, iz, hx, hz
    plus = (a & b & ~c & d) | (a & ~b & c & d) | (~a & b & c & ~d)
    minus = (a & b & c & ~d) | (a & ~b & ~c & d) | (~a & b & c & d)
    return bin(plus).count("1") - bin(minus).count("1")


class Tableau:
    def __init__(self, n: int):
        self.n = n
        self.x = [1 << i for i in range(n)] + [0] * n
        self.z = [0] * n + [1 << i for i in range(n)]
        self.r = [0] * (2 * n)

    def rowsum(self, h: int, i: int) -> None:
        """Row h := row i * row h."""
        s = 2 * self.r[h] + 2 * self.r[i] + g_sum(self.x[i], self.z[i], self.x[h], self.z[h])
        self.r[h] = 1 if s % 4 == 2 else 0
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    # conjugation rules, one row at a time
    def h(self, q):
        for k in range(2 * self.n):
            xb, zb = (self.x[k] >> q) & 1, (self.z[k] >> q) & 1
            self.r[k] ^= xb & zb
            if xb != zb:
                self.x[k] ^= 1 << q
                self.z[k] ^= 1 << q

    def s(self, q):
        for k in range(2 * self.n):
            xb, zb = (self.x[k] >> q) & 1, (self.z[k] >> q) & 1
            self.r[k] ^= xb & zb
            self.z[k] ^= xb << q

    def sdg(self, q):
        for k in range(2 * self.n):
            xb, zb = (self.x[k] >> q) & 1, (self.z[k] >> q) & 1
            self.r[k] ^= xb & (zb ^ 1)
            self.z[k] ^= xb << q

    def sx(self, q):
        for k in range(2 * self.n):
            xb, zb = (self.x[k] >> q) & 1, (self.z[k] >> q) & 1
            self.r[k] ^= zb & (xb ^ 1)
            self.x[k] ^= zb << q

    def pauli(self, q, px: int, pz: int):
        """X (1,0), Z (0,1), Y (1,1): the sign flips where the row anticommutes."""
        for k in range(2 * self.n):
            xb, zb = (self.x[k] >> q) & 1, (self.z[k] >> q) & 1
            self.r[k] ^= (px & zb) ^ (pz & xb)

    def cx(self, c, t):
        for k in range(2 * self.n):
            xc, zc = (self.x[k] >> c) & 1, (self.z[k] >> c) & 1
            xt, zt = (self.x[k] >> t) & 1, (self.z[k] >> t) & 1
            self.r[k] ^= xc & zt & (xt ^ zc ^ 1)
            self.x[k] ^= xc << t
            self.z[k] ^= zt << c

    def cz(self, a, b):
        for k in range(2 * self.n):
            xa, za = (self.x[k] >> a) & 1, (self.z[k] >> a) & 1
            xb, zb = (self.x[k] >> b) & 1, (self.z[k] >> b) & 1
            self.r[k] ^= xa & xb & (za ^ zb)
            self.z[k] ^= (xb << a) | (xa << b)

    def swap(self, a, b):
        for k in range(2 * self.n):
            for arr in (self.x, self.z):
                ba, bb = (arr[k] >> a) & 1, (arr[k] >> b) & 1
                if ba != bb:
                    arr[k] ^= (1 << a) | (1 << b)

    def measure(self, q: int, u: float) -> int:
        n = self.n
        p = next((i for i in range(n, 2 * n) if (self.x[i] >> q) & 1), None)
        if p is not None:  # random outcome
            for i in range(2 * n):
                if i != p and (self.x[i] >> q) & 1:
                    self.rowsum(i, p)
            self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p], self.z[p], self.r[p]
            o = 1 if u >= 0.5 else 0
            self.x[p], self.z[p], self.r[p] = 0, 1 << q, o
            return o
        # deterministic: the sign of the product of the stabilisers whose destabiliser has x_q
        self.x.append(0)
        self.z.append(0)
        self.r.append(0)
        for i in range(n):
            if (self.x[i] >> q) & 1:
                self.rowsum(2 * n, i + n)
        o = self.r[2 * n]
        del self.x[2 * n], self.z[2 * n], self.r[2 * n]
        return o


def run(ops, n: int, uniform, seed: int = 0, stream: int = 0, shot: int = 0) -> int:
    """Classical register of one shot of a Clifford program (flat IR records).
    uniform(seed, stream, shot, m) supplies the m-th draw."""
    t = Tableau(n)
    st = {"creg": 0, "m": 0}

    def gate(g, q):
        if g == Gate.I:
            return
        if g == Gate.H:
            t.h(q[0])
        elif g == Gate.S:
            t.s(q[0])
        elif g == Gate.SDG:
            t.sdg(q[0])
        elif g == Gate.SX:
            t.sx(q[0])
        elif g == Gate.X:
            t.pauli(q[0], 1, 0)
        elif g == Gate.Y:
            t.pauli(q[0], 1, 1)
        elif g == Gate.Z:
            t.pauli(q[0], 0, 1)
        elif g == Gate.CX:
            t.cx(q[0], q[1])
        elif g == Gate.CY:  # S_t CX S_t^dagger: the rightmost factor acts first
            t.sdg(q[1])
            t.cx(q[0], q[1])
            t.s(q[1])
        elif g == Gate.CZ:
            t.cz(q[0], q[1])
        elif g == Gate.SWAP:
            t.swap(q[0], q[1])
        else:
            raise ValueError(f"gate {g} is not Clifford")

    def block(i0: int, i1: int):
        i = i0
        while i < i1:
            o = ops[i]
            k = int(o["kind"])
            if k == Kind.GATE:
                gate(int(o["gate"]), [int(v) for v in o["q"]])
                i += 1
            elif k in (Kind.MEASURE, Kind.RESET):
                q = int(o["q"][0])
                b = t.measure(q, uniform(seed, stream, shot, st["m"]))
                st["m"] += 1
                if k == Kind.MEASURE:
                    cb = int(o["cbit"])
                    st["creg"] = (st["creg"] & ~(1 << cb)) | (b << cb)
                elif b:
                    t.pauli(q, 1, 0)
                i += 1
            elif k == Kind.COND:
                tl, el = int(o["then_len"]), int(o["else_len"])
                if (st["creg"] & int(o["mask"])) == int(o["value"]):
                    block(i + 1, i + 1 + tl)
                else:
                    block(i + 1 + tl, i + 1 + tl + el)
                i += 1 + tl + el
            elif k == Kind.LOOP:
                bl = int(o["body_len"])
                for _ in range(int(o["loop_k"])):
                    block(i + 1, i + 1 + bl)
                i += 1 + bl
            else:
                raise ValueError("not a Clifford program")

    block(0, len(ops))
    return st["creg"]

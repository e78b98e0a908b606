"""OpenQASM 3 subset -> the flat IR of include/sv.h.

The paper's subject is OpenQASM 3 dynamic circuits (Sec. III): programs with
``input`` parameters (Sec. III-D), standard gates and the ``ctrl`` / ``inv``
modifiers (Sec. III-B), mid-circuit ``measure`` and ``reset``, ``if`` / ``else``
on classical bits and registers decided at run time (Sec. III-C), and bounded
loops (Abstract).  This module lowers that subset to ``ir.Circuit`` records,
which every engine of the library runs:

* declarations: ``qubit[n] q;`` / ``qubit q;`` / ``qreg q[n];``, ``bit[n] c;`` /
  ``bit c;`` / ``creg c[n];`` (all classical bits together <= 64), ``input
  float[64] theta;`` / ``input angle theta;`` (run-time parameters, in order of
  declaration), ``const float x = <expr>;``;
* gates: the standard library (h x y z s sdg t tdg sx id rx ry rz p phase u U u1
  u2 u3 cx CX cy cz ch swap cp cphase crx cry crz cu ccx cswap, and ``gphase``),
  the two-qubit rotations exporters emit (rxx ryy rzz rzx) and sxdg, a whole
  register as an operand broadcasts the gate over its qubits, ``gate``
  definitions are expanded inline, and the modifiers ``ctrl @`` / ``ctrl(k) @``,
  ``negctrl @`` / ``negctrl(k) @`` (control on |0>: X before and after on that
  qubit), ``inv @`` and ``pow(k) @`` (integer k >= 0), on standard and on user
  gates (a user gate's body is inverted record by record in reverse order, or
  controlled record by record);
* operands ``q``, ``q[i]`` and inclusive slices ``q[a:b]`` / ``q[a:s:b]``;
* ``def`` subroutines with qubit, bit (consecutive bits) and float / angle
  arguments, inlined at each call, returning nothing or one bit through
  ``return measure q;`` at the top of the body (``c[i] = f(...);``; a
  discarded result goes to bit 63); no classical declarations inside;
* ``c[i] = measure q[j];``, ``measure q[j] -> c[i];``, ``c = measure q;``,
  ``bit[n] c = measure q;``, ``measure q;`` (result into bit 63, which the
  program must leave undeclared), ``reset q;``, ``barrier ...;`` and
  ``delay[...] ...;`` (no effect on the state);
* ``if (c[i] == b)``, ``if (c == v)``, ``if (c[i])``, ``if (!c[i])``, ``!=``,
  ``true`` / ``false``, joined by ``&&`` (one COND predicate) and ``||`` (an
  if / else-if chain repeating the body), with ``!( ... )`` around the whole
  condition and an optional ``else``; predicates are read on the device;
* ``for uint i in [a:b]`` / ``[a:s:b]`` / ``{v, ...}``: a LOOP record when the
  body does not use the loop variable, unrolled otherwise; ``while`` is refused
  (unbounded).

Angles are constants or a constant times one ``input`` parameter (the IR's
``scale * params[idx]``); other expressions of parameters are refused.
Controlled forms without an IR gate are lowered to dense unitaries (constant
angles only).
"""
from __future__ import annotations

import math
import re
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple, Union

import numpy as np

from .ir import GATE_ARITY, Circuit, Gate, Kind, Param


class QasmError(ValueError):
    """A program outside the subset, or an error in it (with its line)."""


# ------------------------------------------------------------------ tokens
_TOKEN = re.compile(r"""
    (?P<ws>\s+|//[^\n]*|/\*.*?\*/)
  | (?P<num>(\d+\.\d*|\.\d+|\d+)([eE][+-]?\d+)?)
  | (?P<str>"[^"]*")
  | (?P<id>[A-Za-z_πτ][A-Za-z_0-9]*)
  | (?P<op>->|==|!=|<=|>=|\*\*|&&|\|\||[{}()\[\];,:=@+\-*/!<>])
""", re.S | re.X)


@dataclass
class Tok:
    kind: str
    text: str
    line: int


def _tokenize(src: str) -> List[Tok]:
    toks, pos, line = [], 0, 1
    while pos < len(src):
        m = _TOKEN.match(src, pos)
        if not m:
            raise QasmError(f"line {line}: unexpected character {src[pos]!r}")
        kind = m.lastgroup
        text = m.group(kind)
        if kind != "ws":
            toks.append(Tok(kind, text, line))
        line += text.count("\n")
        pos = m.end()
    toks.append(Tok("eof", "", line))
    return toks


# ------------------------------------------------------------------ linear angle values
@dataclass(frozen=True)
class Lin:
    """c0 + c1 * params[idx] (idx = -1: a constant)."""
    c0: float
    c1: float = 0.0
    idx: int = -1

    def const(self) -> bool:
        return self.idx < 0 or self.c1 == 0.0

    def __add__(self, o: "Lin") -> "Lin":
        if not self.const() and not o.const() and self.idx != o.idx:
            raise QasmError("an angle may depend on one input parameter only")
        idx = self.idx if not self.const() else o.idx
        return Lin(self.c0 + o.c0, self.c1 + o.c1, idx)

    def __neg__(self) -> "Lin":
        return Lin(-self.c0, -self.c1, self.idx)

    def scale(self, k: float) -> "Lin":
        return Lin(self.c0 * k, self.c1 * k, self.idx)

    def angle(self) -> Union[float, Param]:
        if self.const():
            return float(self.c0)
        if self.c0 != 0.0:
            raise QasmError("an angle must be a constant or a constant times an input parameter "
                            "(the IR has no offset)")
        return Param(self.idx, float(self.c1))


_FUNCS: Dict[str, Callable[[float], float]] = {
    "sin": math.sin, "cos": math.cos, "tan": math.tan, "exp": math.exp, "sqrt": math.sqrt,
    "arcsin": math.asin, "arccos": math.acos, "arctan": math.atan, "ln": math.log}
_CONSTS = {"pi": math.pi, "π": math.pi, "tau": 2 * math.pi, "τ": 2 * math.pi, "euler": math.e}


# ------------------------------------------------------------------ program state
@dataclass
class GateDef:
    params: List[str]
    qargs: List[str]
    body: List[Tok]


@dataclass
class SubDef:
    """A ``def`` subroutine: (kind, name, size) arguments -- kind 'qubit', 'bit'
    or 'float' (size 0: a single qubit or bit) -- and whether it returns a bit."""
    args: List[Tuple[str, str, int]]
    returns_bit: bool
    body: List[Tok]


@dataclass
class Program:
    """A lowered program: the IR circuit and the names it was written with."""
    circuit: Circuit
    n_qubits: int
    n_bits: int
    params: Dict[str, int] = field(default_factory=dict)
    qregs: Dict[str, Tuple[int, int]] = field(default_factory=dict)  # name -> (first qubit, size)
    cregs: Dict[str, Tuple[int, int]] = field(default_factory=dict)  # name -> (first bit, size)

    @property
    def ops(self) -> np.ndarray:
        return self.circuit.ops

    @property
    def pool(self) -> np.ndarray:
        return self.circuit.pool


# a measurement whose result is discarded (``measure q;``) writes this bit
HIDDEN_BIT = 63

# one-qubit standard gates: IR gate, number of angles
_G1 = {"h": (Gate.H, 0), "x": (Gate.X, 0), "y": (Gate.Y, 0), "z": (Gate.Z, 0), "s": (Gate.S, 0),
       "sdg": (Gate.SDG, 0), "t": (Gate.T, 0), "tdg": (Gate.TDG, 0), "sx": (Gate.SX, 0),
       "rx": (Gate.RX, 1), "ry": (Gate.RY, 1), "rz": (Gate.RZ, 1), "p": (Gate.P, 1), "phase": (Gate.P, 1),
       "u1": (Gate.P, 1), "u": (Gate.U, 3), "U": (Gate.U, 3), "u3": (Gate.U, 3)}
# two-qubit standard gates
_G2 = {"cx": (Gate.CX, 0), "CX": (Gate.CX, 0), "cy": (Gate.CY, 0), "cz": (Gate.CZ, 0), "ch": (Gate.CH, 0),
       "swap": (Gate.SWAP, 0), "cp": (Gate.CP, 1), "cphase": (Gate.CP, 1), "cu1": (Gate.CP, 1),
       "crx": (Gate.CRX, 1), "cry": (Gate.CRY, 1), "crz": (Gate.CRZ, 1), "cu3": (Gate.CU, 3)}
# controlled version of a one-qubit gate (one control)
_CTRL1 = {Gate.X: Gate.CX, Gate.Y: Gate.CY, Gate.Z: Gate.CZ, Gate.H: Gate.CH, Gate.P: Gate.CP,
          Gate.RX: Gate.CRX, Gate.RY: Gate.CRY, Gate.RZ: Gate.CRZ, Gate.U: Gate.CU}


def _u_matrix(th: float, ph: float, la: float) -> np.ndarray:
    c, s = math.cos(th / 2), math.sin(th / 2)
    return np.array([[c, -np.exp(1j * la) * s], [np.exp(1j * ph) * s, np.exp(1j * (ph + la)) * c]])


def _gate_matrix(g: Gate, a: Sequence[float]) -> np.ndarray:
    """2x2 matrix of a one-qubit IR gate (OpenQASM 3 standard-library meanings)."""
    h = 1 / math.sqrt(2)
    m = {Gate.H: [[h, h], [h, -h]], Gate.X: [[0, 1], [1, 0]], Gate.Y: [[0, -1j], [1j, 0]],
         Gate.Z: [[1, 0], [0, -1]], Gate.S: [[1, 0], [0, 1j]], Gate.SDG: [[1, 0], [0, -1j]],
         Gate.T: [[1, 0], [0, np.exp(1j * math.pi / 4)]], Gate.TDG: [[1, 0], [0, np.exp(-1j * math.pi / 4)]],
         Gate.SX: [[(1 + 1j) / 2, (1 - 1j) / 2], [(1 - 1j) / 2, (1 + 1j) / 2]]}.get(g)
    if m is not None:
        return np.array(m, dtype=np.complex128)
    if g == Gate.RX:
        c, s = math.cos(a[0] / 2), math.sin(a[0] / 2)
        return np.array([[c, -1j * s], [-1j * s, c]])
    if g == Gate.RY:
        c, s = math.cos(a[0] / 2), math.sin(a[0] / 2)
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if g == Gate.RZ:
        return np.diag([np.exp(-0.5j * a[0]), np.exp(0.5j * a[0])])
    if g == Gate.P:
        return np.diag([1, np.exp(1j * a[0])])
    if g == Gate.U:
        return _u_matrix(*a)
    raise QasmError(f"no matrix for {g.name}")


def _controlled_k(m: np.ndarray, nc: int) -> np.ndarray:
    """A 2^k x 2^k unitary with nc controls in front: local bits 0..nc-1 are the
    controls, nc.. the unitary's qubits; it acts when every control bit is 1."""
    d = m.shape[0]
    out = np.eye(d << nc, dtype=np.complex128)
    cm = (1 << nc) - 1
    for a in range(d):
        for b in range(d):
            out[cm | (a << nc), cm | (b << nc)] = m[a, b]
    return out


def _neg(a):
    return Param(a.idx, -a.scale) if isinstance(a, Param) else -a


def _inverse1(g: Gate, angles: List) -> Tuple[Gate, List]:
    """Inverse of a one-qubit IR gate with its angles (literals or parameter references)."""
    if g in (Gate.H, Gate.X, Gate.Y, Gate.Z):
        return g, []
    pairs = {Gate.S: Gate.SDG, Gate.SDG: Gate.S, Gate.T: Gate.TDG, Gate.TDG: Gate.T}
    if g in pairs:
        return pairs[g], []
    if g in (Gate.RX, Gate.RY, Gate.RZ, Gate.P):
        return g, [_neg(angles[0])]
    if g == Gate.U:  # U(t, p, l)^dagger = U(-t, -l, -p)
        return g, [_neg(angles[0]), _neg(angles[2]), _neg(angles[1])]
    if g == Gate.SX:
        return Gate.SX, ["inverse"]
    raise QasmError(f"no inverse for {g.name}")


def _controlled(m: np.ndarray, k: int) -> np.ndarray:
    """Matrix over (controls q[0..k-1], target q[k]) with local bit r <-> q[r]:
    the target acts when every control bit is 1."""
    dim = 1 << (k + 1)
    out = np.eye(dim, dtype=np.complex128)
    cm = (1 << k) - 1
    for a in range(2):
        for b in range(2):
            out[cm | (a << k), cm | (b << k)] = m[a, b]
    return out


class _Lowerer:
    def __init__(self, toks: List[Tok]):
        self.t = toks
        self.i = 0
        self.qregs: Dict[str, Tuple[int, int]] = {}
        self.cregs: Dict[str, Tuple[int, int]] = {}
        self.params: Dict[str, int] = {}
        self.consts: Dict[str, float] = {}
        self.gates: Dict[str, GateDef] = {}
        self.subs: Dict[str, SubDef] = {}
        self.ret_bit: Optional[int] = None  # inside a subroutine returning a bit: where `return measure` writes
        self.in_sub = False
        self.depth = 0  # block nesting (return is allowed at the top of a subroutine body only)
        self.nq = 0
        self.nb = 0
        self.ops: List[Callable[[Circuit], None]] = []  # emitted after the qubit count is known

    # -- token helpers ----------------------------------------------------------------
    def peek(self, k: int = 0) -> Tok:
        return self.t[min(self.i + k, len(self.t) - 1)]

    def next(self) -> Tok:
        tok = self.t[self.i]
        self.i += 1
        return tok

    def err(self, msg: str, tok: Optional[Tok] = None) -> QasmError:
        tok = tok or self.peek()
        return QasmError(f"line {tok.line}: {msg}")

    def expect(self, text: str) -> Tok:
        tok = self.next()
        if tok.text != text:
            raise self.err(f"expected {text!r}, found {tok.text or 'end of input'!r}", tok)
        return tok

    def ident(self) -> str:
        tok = self.next()
        if tok.kind != "id":
            raise self.err(f"expected a name, found {tok.text!r}", tok)
        return tok.text

    def accept(self, text: str) -> bool:
        if self.peek().text == text:
            self.i += 1
            return True
        return False

    # -- expressions --------------------------------------------------------------------
    def expr(self, env: Dict[str, Lin]) -> Lin:
        v = self.term(env)
        while self.peek().text in ("+", "-"):
            op = self.next().text
            r = self.term(env)
            v = v + (r if op == "+" else -r)
        return v

    def term(self, env: Dict[str, Lin]) -> Lin:
        v = self.power(env)
        while self.peek().text in ("*", "/"):
            op = self.next().text
            r = self.power(env)
            if op == "*":
                if v.const():
                    v = r.scale(v.c0)
                elif r.const():
                    v = v.scale(r.c0)
                else:
                    raise self.err("a product of two input parameters is not an angle of the IR")
            else:
                if not r.const() or r.c0 == 0:
                    raise self.err("division by a parameter or by zero")
                v = v.scale(1.0 / r.c0)
        return v

    def power(self, env: Dict[str, Lin]) -> Lin:
        v = self.unary(env)
        if self.accept("**"):
            e = self.power(env)
            if not (v.const() and e.const()):
                raise self.err("powers of input parameters are not angles of the IR")
            v = Lin(v.c0 ** e.c0)
        return v

    def unary(self, env: Dict[str, Lin]) -> Lin:
        if self.accept("-"):
            return -self.unary(env)
        if self.accept("+"):
            return self.unary(env)
        return self.atom(env)

    def atom(self, env: Dict[str, Lin]) -> Lin:
        tok = self.next()
        if tok.kind == "num":
            return Lin(float(tok.text))
        if tok.text == "(":
            v = self.expr(env)
            self.expect(")")
            return v
        if tok.kind == "id":
            name = tok.text
            if name in env:
                return env[name]
            if name in _FUNCS and self.peek().text == "(":
                self.expect("(")
                a = self.expr(env)
                self.expect(")")
                if not a.const():
                    raise self.err(f"{name}() of an input parameter is not an angle of the IR", tok)
                return Lin(_FUNCS[name](a.c0))
            if name in self.consts:
                return Lin(self.consts[name])
            if name in _CONSTS:
                return Lin(_CONSTS[name])
            if name in self.params:
                return Lin(0.0, 1.0, self.params[name])
            raise self.err(f"unknown name {name!r}", tok)
        raise self.err(f"unexpected {tok.text!r} in an expression", tok)

    def int_expr(self, env: Dict[str, Lin]) -> int:
        v = self.expr(env)
        if not v.const() or v.c0 != int(v.c0):
            raise self.err("expected an integer")
        return int(v.c0)

    # -- operands -----------------------------------------------------------------------
    def qoperand(self, env: Dict[str, Lin], qmap: Optional[Dict[str, List[int]]]) -> List[int]:
        """Qubits of an operand: one, or a whole register (broadcast)."""
        name = self.ident()
        if qmap is not None and name in qmap:
            regs = qmap[name]
        elif name in self.qregs:
            first, size = self.qregs[name]
            regs = list(range(first, first + size))
        else:
            raise self.err(f"unknown qubit {name!r}")
        if self.accept("["):
            return [regs[k] for k in self.index_or_slice(env, name, len(regs))]
        return list(regs)

    def index_or_slice(self, env, name: str, size: int) -> List[int]:
        """After '[': one index, or an inclusive slice a:b / a:s:b (OpenQASM 3 ranges)."""
        k = self.int_expr(env)
        ks = [k]
        if self.accept(":"):
            e = self.int_expr(env)
            step = 1
            if self.accept(":"):
                step, e = e, self.int_expr(env)
            if step == 0:
                raise self.err("a slice with step 0")
            ks = list(range(k, e + (1 if step > 0 else -1), step))
        self.expect("]")
        for i in ks:
            if not 0 <= i < size:
                raise self.err(f"index {i} outside {name}[{size}]")
        return ks

    def coperand(self, env: Dict[str, Lin]) -> List[int]:
        name = self.ident()
        if name not in self.cregs:
            raise self.err(f"unknown bit {name!r}")
        first, size = self.cregs[name]
        if self.accept("["):
            return [first + k for k in self.index_or_slice(env, name, size)]
        return list(range(first, first + size))

    # -- program ------------------------------------------------------------------------
    def program(self) -> None:
        if self.peek().text == "OPENQASM":
            self.next()
            self.next()
            self.expect(";")
        while self.peek().kind != "eof":
            self.statement({}, None, self.ops)

    def block(self, env, qmap, out) -> None:
        self.depth += 1
        if self.accept("{"):
            while not self.accept("}"):
                if self.peek().kind == "eof":
                    raise self.err("unterminated block")
                self.statement(env, qmap, out)
        else:
            self.statement(env, qmap, out)
        self.depth -= 1

    def statement(self, env, qmap, out) -> None:
        tok = self.peek()
        t = tok.text
        if t == "include":
            self.next()
            name = self.next()
            if name.kind != "str" or name.text.strip('"') not in ("stdgates.inc", "qelib1.inc"):
                raise self.err("only stdgates.inc can be included", name)
            self.expect(";")
        elif t in ("qubit", "qreg"):
            self.declare_qubits()
        elif t in ("bit", "creg"):
            self.declare_bits(env, qmap, out)
        elif t == "input":
            self.declare_input()
        elif t == "const":
            self.declare_const()
        elif t == "gate":
            self.define_gate()
        elif t == "def":
            self.define_sub()
        elif t == "return":
            return self.return_stmt(env, qmap, out, tok)
        elif t in ("barrier", "delay"):  # no effect on the state (timing only)
            while self.next().text != ";":
                pass
        elif t == "reset":
            self.next()
            qs = self.qoperand(env, qmap)
            self.expect(";")
            out.extend((lambda q: lambda c: c.reset(q))(q) for q in qs)
        elif t == "measure":
            self.next()
            qs = self.qoperand(env, qmap)
            if self.accept(";"):  # result discarded: the draw still happens, into the hidden bit
                if self.nb >= 64:
                    raise self.err("a measurement without a destination needs bit 63 free", tok)
                out.extend((lambda q: lambda c: c.measure(q, HIDDEN_BIT))(q) for q in qs)
                return
            self.expect("->")
            bs = self.coperand(env)
            self.expect(";")
            self.emit_measure(qs, bs, out, tok)
        elif t == "if":
            self.if_stmt(env, qmap, out)
        elif t == "for":
            self.for_stmt(env, qmap, out)
        elif t == "while":
            raise self.err("while loops are unbounded: only bounded for loops are supported")
        elif tok.kind == "id" and t in self.cregs and self.peek(1).text in ("=", "["):
            bs = self.coperand(env)
            self.expect("=")
            if self.peek().kind == "id" and self.peek().text in self.subs:
                if len(bs) != 1:
                    raise self.err("a subroutine returns one bit", tok)
                self.call_sub(env, qmap, out, bs[0])
                return
            self.expect("measure")
            qs = self.qoperand(env, qmap)
            self.expect(";")
            self.emit_measure(qs, bs, out, tok)
        elif tok.kind == "id" and t in self.subs:
            self.call_sub(env, qmap, out, None)
        elif tok.kind == "id":
            self.gate_call(env, qmap, out)
        else:
            raise self.err(f"unexpected {t!r}")

    def declare_qubits(self) -> None:
        kw = self.next().text
        if kw == "qubit":
            size = 1
            if self.accept("["):
                size = self.int_expr({})
                self.expect("]")
            name = self.ident()
        else:
            name = self.ident()
            self.expect("[")
            size = self.int_expr({})
            self.expect("]")
        self.expect(";")
        if name in self.qregs or size < 1:
            raise self.err(f"bad qubit register {name!r}")
        self.qregs[name] = (self.nq, size)
        self.nq += size

    def declare_bits(self, env=None, qmap=None, out=None) -> None:
        if self.in_sub:
            raise self.err("classical declarations inside a subroutine are not supported")
        kw = self.next().text
        tok = self.peek()
        if kw == "bit":
            size = 1
            if self.accept("["):
                size = self.int_expr({})
                self.expect("]")
            name = self.ident()
        else:
            name = self.ident()
            self.expect("[")
            size = self.int_expr({})
            self.expect("]")
        init = kw == "bit" and self.accept("=")  # bit[n] c = measure q;
        if init:
            self.expect("measure")
            qs = self.qoperand(env or {}, qmap)
        self.expect(";")
        if name in self.cregs or size < 1:
            raise self.err(f"bad bit register {name!r}")
        if self.nb + size > 64:
            raise self.err("more than 64 classical bits")
        self.cregs[name] = (self.nb, size)
        self.nb += size
        if init:
            self.emit_measure(qs, list(range(self.nb - size, self.nb)), out, tok)

    def declare_input(self) -> None:
        self.next()
        ty = self.ident()
        if ty not in ("float", "angle"):
            raise self.err("inputs are float or angle parameters")
        if self.accept("["):
            self.int_expr({})
            self.expect("]")
        name = self.ident()
        self.expect(";")
        self.params[name] = len(self.params)

    def declare_const(self) -> None:
        self.next()
        self.ident()  # type
        if self.accept("["):
            self.int_expr({})
            self.expect("]")
        name = self.ident()
        self.expect("=")
        v = self.expr({})
        self.expect(";")
        if not v.const():
            raise self.err("a const needs a constant value")
        self.consts[name] = v.c0

    def define_gate(self) -> None:
        self.next()
        name = self.ident()
        params: List[str] = []
        if self.accept("("):
            if not self.accept(")"):
                params.append(self.ident())
                while self.accept(","):
                    params.append(self.ident())
                self.expect(")")
        qargs = [self.ident()]
        while self.accept(","):
            qargs.append(self.ident())
        self.expect("{")
        depth, body = 1, []
        while True:
            tok = self.next()
            if tok.kind == "eof":
                raise self.err("unterminated gate body")
            depth += tok.text == "{"
            depth -= tok.text == "}"
            if depth == 0:
                break
            body.append(tok)
        self.gates[name] = GateDef(params, qargs, body)

    def define_sub(self) -> None:
        tok = self.next()
        name = self.ident()
        if name in self.subs or name in self.gates:
            raise self.err(f"{name!r} is defined twice", tok)
        args: List[Tuple[str, str, int]] = []
        self.expect("(")
        if not self.accept(")"):
            while True:
                kind = self.ident()
                size = 0
                if self.accept("["):
                    size = self.int_expr({})
                    self.expect("]")
                if kind in ("float", "angle"):
                    kind, size = "float", 0
                elif kind not in ("qubit", "bit"):
                    raise self.err(f"subroutine arguments are qubit, bit, float or angle, not {kind!r}")
                args.append((kind, self.ident(), size))
                if self.accept(")"):
                    break
                self.expect(",")
        returns_bit = False
        if self.accept("->"):
            if self.ident() != "bit":
                raise self.err("a subroutine returns a bit or nothing")
            returns_bit = True
        self.expect("{")
        depth, body = 1, []
        while True:
            t = self.next()
            if t.kind == "eof":
                raise self.err("unterminated subroutine body")
            depth += t.text == "{"
            depth -= t.text == "}"
            if depth == 0:
                break
            body.append(t)
        self.subs[name] = SubDef(args, returns_bit, body)

    def call_sub(self, env, qmap, out, dest: Optional[int]) -> None:
        """Inlines a subroutine call: its body lowered with the arguments bound."""
        tok = self.peek()
        name = self.ident()
        sd = self.subs[name]
        if dest is not None and not sd.returns_bit:
            raise self.err(f"{name!r} returns nothing", tok)
        sub_env: Dict[str, Lin] = {}
        sub_q: Dict[str, List[int]] = {}
        sub_c: Dict[str, Tuple[int, int]] = {}
        self.expect("(")
        for k, (kind, arg, size) in enumerate(sd.args):
            if k:
                self.expect(",")
            if kind == "float":
                sub_env[arg] = self.expr(env)
            elif kind == "qubit":
                qs = self.qoperand(env, qmap)
                if len(qs) != max(size, 1):
                    raise self.err(f"argument {arg!r} of {name!r} takes {max(size, 1)} qubits", tok)
                sub_q[arg] = qs
            else:
                bs = self.coperand(env)
                if len(bs) != max(size, 1) or bs != list(range(bs[0], bs[0] + len(bs))):
                    raise self.err(f"argument {arg!r} of {name!r} takes {max(size, 1)} consecutive bits", tok)
                sub_c[arg] = (bs[0], len(bs))
        self.expect(")")
        self.expect(";")
        if self.depth > 64:
            raise self.err("subroutine calls nested too deeply (recursion?)", tok)
        sub = _Lowerer(sd.body + [Tok("eof", "", tok.line)])
        sub.qregs, sub.cregs = {}, sub_c
        sub.params, sub.consts, sub.gates, sub.subs = self.params, self.consts, self.gates, self.subs
        sub.nq, sub.nb = self.nq, self.nb
        sub.in_sub = True
        sub.depth = self.depth + 1
        sub.ret_bit = (dest if dest is not None else HIDDEN_BIT) if sd.returns_bit else None
        if sub.ret_bit == HIDDEN_BIT and self.nb >= 64:
            raise self.err("a discarded return value needs bit 63 free", tok)
        sub.depth0 = sub.depth
        while sub.peek().kind != "eof":
            if sub.statement(dict(env, **sub_env), sub_q, out) == "return":
                break

    def return_stmt(self, env, qmap, out, tok):
        self.next()
        if self.ret_bit is None:
            raise self.err("return outside a subroutine that returns a bit", tok)
        if self.depth != getattr(self, "depth0", -1):
            raise self.err("return is allowed only at the top of a subroutine body", tok)
        self.expect("measure")
        qs = self.qoperand(env, qmap)
        self.expect(";")
        if len(qs) != 1:
            raise self.err("return measure takes one qubit", tok)
        self.emit_measure(qs, [self.ret_bit], out, tok)
        return "return"

    def emit_measure(self, qs, bs, out, tok) -> None:
        if len(qs) != len(bs):
            raise self.err(f"measuring {len(qs)} qubits into {len(bs)} bits", tok)
        out.extend((lambda q, b: lambda c: c.measure(q, b))(q, b) for q, b in zip(qs, bs))

    # -- control flow -------------------------------------------------------------------
    # Conditions: a disjunction (||) of conjunctions (&&) of bit tests and register
    # equalities.  A conjunction is one COND predicate (mask, value); a disjunction
    # becomes an if / else-if chain whose branches repeat the body, so exactly one
    # runs; a leading !( ... ) or a register != swaps the branches.
    def cond_value(self, env) -> int:
        if self.peek().text in ("true", "false"):
            return 1 if self.next().text == "true" else 0
        return self.int_expr(env)

    def cond_literal(self, env) -> Tuple[int, int, bool]:
        """(mask, value, negated): one test; negated marks `register != v` on several bits."""
        if self.accept("!"):
            bits = self.coperand(env)
            if len(bits) != 1:
                raise self.err("'!' applies to a single bit")
            return 1 << bits[0], 0, False
        if self.accept("("):
            terms, neg = self.cond_disj(env)
            self.expect(")")
            if len(terms) != 1 or neg:
                raise self.err("'||' or a register '!=' inside a conjunction is not supported")
            return terms[0][0], terms[0][1], False
        bits = self.coperand(env)
        op = None
        if self.peek().text in ("==", "!="):
            op = self.next().text
            v = self.cond_value(env)
        elif len(bits) == 1:
            v = 1
        else:
            raise self.err("a register condition needs '== value'")
        if v < 0 or v >= (1 << len(bits)):
            raise self.err(f"value {v} does not fit {len(bits)} bits")
        mask = sum(1 << b for b in bits)
        value = sum(((v >> k) & 1) << b for k, b in enumerate(bits))
        if op == "!=":
            if len(bits) == 1:
                return mask, mask ^ value, False
            return mask, value, True
        return mask, value, False

    def cond_conj(self, env) -> Tuple[Tuple[int, int, bool], bool]:
        """((mask, value, possible), negated) of literals joined by &&."""
        mask = value = 0
        possible, negated, n = True, False, 0
        while True:
            m, v, ng = self.cond_literal(env)
            n += 1
            negated = negated or ng
            if (value ^ v) & mask & m:  # the same bit required 0 and 1
                possible = False
            mask, value = mask | m, value | v
            if not self.accept("&&"):
                break
        if negated and n > 1:
            raise self.err("a register '!=' inside a conjunction is not supported")
        return (mask, value, possible), negated

    def cond_disj(self, env) -> Tuple[List[Tuple[int, int, bool]], bool]:
        terms, negs = [], []
        while True:
            t, ng = self.cond_conj(env)
            terms.append(t)
            negs.append(ng)
            if not self.accept("||"):
                break
        if any(negs) and len(terms) > 1:
            raise self.err("a register '!=' inside a disjunction is not supported")
        return terms, negs[0]

    def if_stmt(self, env, qmap, out) -> None:
        self.next()
        self.expect("(")
        if self.peek().text == "!" and self.peek(1).text == "(":
            self.next()
            self.next()
            terms, neg = self.cond_disj(env)
            self.expect(")")
            neg = not neg
        else:
            terms, neg = self.cond_disj(env)
        self.expect(")")
        then_ops: List[Callable] = []
        else_ops: List[Callable] = []
        self.block(env, qmap, then_ops)
        if self.accept("else"):
            self.block(env, qmap, else_ops)
        if neg:
            then_ops, else_ops = else_ops, then_ops
        terms = [(m, v) for m, v, ok in terms if ok] or [(0, 1)]  # (0, 1): never true

        def emit(c, then_ops=then_ops, else_ops=else_ops, terms=terms):
            def level(i):
                mask, value = terms[i]
                rest = (lambda: level(i + 1)) if i + 1 < len(terms) else (
                    (lambda: [f(c) for f in else_ops]) if else_ops else None)
                c.cond(mask, value, lambda: [f(c) for f in then_ops], rest)
            level(0)
        out.append(emit)

    def for_stmt(self, env, qmap, out) -> None:
        self.next()
        if self.peek().text in ("int", "uint", "float", "angle", "bit"):  # the loop variable's type
            self.next()
            if self.accept("["):
                self.int_expr({})
                self.expect("]")
        var = self.ident()
        self.expect("in")
        if self.accept("["):
            a = self.int_expr(env)
            self.expect(":")
            b = self.int_expr(env)
            step = 1
            if self.accept(":"):
                step, b = b, self.int_expr(env)
            self.expect("]")
            if step == 0:
                raise self.err("a loop step of 0")
            values = list(range(a, b + (1 if step > 0 else -1), step))  # ranges include their end
        else:
            self.expect("{")
            values = [self.int_expr(env)]
            while self.accept(","):
                values.append(self.int_expr(env))
            self.expect("}")
        start = self.i
        uses = self._block_uses(var)
        if not uses:  # one LOOP record
            body: List[Callable] = []
            self.block(env, qmap, body)
            k = len(values)
            if k > (1 << 16):
                raise self.err("a loop of more than 65536 iterations")
            out.append(lambda c, body=body, k=k: c.loop(k, lambda: [f(c) for f in body]))
            return
        for v in values:  # the body uses the loop variable: unrolled
            self.i = start
            self.block({**env, var: Lin(float(v))}, qmap, out)

    def _block_uses(self, var: str) -> bool:
        j, depth = self.i, 0
        while True:
            tok = self.t[j]
            if tok.kind == "eof":
                return False
            if tok.kind == "id" and tok.text == var:
                return True
            if tok.text == "{":
                depth += 1
            elif tok.text == "}":
                depth -= 1
                if depth == 0:
                    return False
            elif tok.text == ";" and depth == 0:
                return False
            j += 1

    # -- gate calls -----------------------------------------------------------------------
    def gate_call(self, env, qmap, out) -> None:
        mods: List[Tuple[str, int]] = []
        while self.peek().text in ("ctrl", "inv", "pow", "negctrl"):
            m = self.next().text
            k = 1
            if m in ("ctrl", "negctrl", "pow") and self.accept("("):
                k = self.int_expr(env)
                self.expect(")")
            self.expect("@")
            mods.append((m, k))
        tok = self.peek()
        name = self.ident()
        args: List[Lin] = []
        if self.accept("("):
            if not self.accept(")"):
                args.append(self.expr(env))
                while self.accept(","):
                    args.append(self.expr(env))
                self.expect(")")
        if name == "gphase" and self.peek().text == ";":  # a global phase takes no qubits
            self.expect(";")
            self.apply(name, args, [], mods, out, tok)
            return
        operands = [self.qoperand(env, qmap)]
        while self.accept(","):
            operands.append(self.qoperand(env, qmap))
        self.expect(";")
        width = max(len(o) for o in operands)
        for o in operands:
            if len(o) not in (1, width):
                raise self.err("registers of different sizes in one gate call", tok)
        for k in range(width):  # broadcast over registers
            qs = [o[k] if len(o) > 1 else o[0] for o in operands]
            if len(set(qs)) != len(qs):
                raise self.err("a gate with a repeated qubit", tok)
            self.apply(name, args, qs, mods, out, tok)

    def apply(self, name: str, args: List[Lin], qs: List[int], mods, out, tok) -> None:
        # modifiers apply right to left: pow, then inv, then ctrl on the outside
        n_ctrl = 0
        inv = False
        reps = 1
        for m, k in reversed(mods):
            if m == "pow":
                if k < 0:
                    raise self.err("pow(k) with k < 0", tok)
                reps *= k
            elif m == "inv":
                inv = not inv
            else:
                n_ctrl += k
        # control qubits come first, in the order of their modifiers; negctrl ones act on |0>
        neg, at = [], 0
        for m, k in mods:
            if m in ("ctrl", "negctrl"):
                if m == "negctrl":
                    neg += qs[at: at + k]
                at += k
        if name == "gphase":
            if n_ctrl != len(qs):
                raise self.err("gphase takes control qubits only", tok)
        elif n_ctrl >= len(qs):
            raise self.err("more controls than qubits", tok)
        ctrls, targets = qs[:n_ctrl], qs[n_ctrl:]
        for q in neg:
            out.append((lambda q: lambda c: c.x(q))(q))
        for _ in range(reps):
            self.apply_one(name, args, ctrls, targets, inv, out, tok)
        for q in neg:
            out.append((lambda q: lambda c: c.x(q))(q))

    def apply_one(self, name, args, ctrls, targets, inv, out, tok) -> None:
        if name in self.gates:
            self.expand(name, args, targets, inv, ctrls, out, tok)
            return
        if name in ("id", "I"):
            return
        if name == "gphase":  # e^{i theta}: a phase on the controls, exact even without them
            if len(args) != 1:
                raise self.err("gphase takes one angle", tok)
            th = -args[0] if inv else args[0]
            if ctrls:
                self.emit1(Gate.P, [th.angle()], ctrls[:-1], ctrls[-1], out, tok)
            elif self.nq:
                for g in (Gate.P, Gate.X, Gate.P, Gate.X):  # P(t) X P(t) X = e^{it} I on qubit 0
                    self.emit1(g, [th.angle()] if g == Gate.P else [], [], 0, out, tok)
            return
        if name == "sxdg":
            if args or len(targets) != 1:
                raise self.err("sxdg takes one qubit", tok)
            self.apply_one("sx", args, ctrls, targets, not inv, out, tok)
            return
        if name in ("rzz", "rxx", "ryy", "rzx"):  # exp(-i t/2 P_a P_b) = basis change, CX, RZ(t), CX, back
            if len(args) != 1 or len(targets) != 2:
                raise self.err(f"{name} takes one angle and two qubits", tok)
            a, b = targets
            th = -args[0] if inv else args[0]
            pre = {"rzz": [], "rxx": [(Gate.H, [], a), (Gate.H, [], b)],
                   "ryy": [(Gate.RX, [math.pi / 2], a), (Gate.RX, [math.pi / 2], b)],
                   "rzx": [(Gate.H, [], b)]}[name]
            post = [(g, [-v for v in ang], q) for g, ang, q in pre]
            for g, ang, q in pre:
                self.emit1(g, ang, [], q, out, tok)
            self.emit1(Gate.X, [], [a], b, out, tok)
            self.emit1(Gate.RZ, [th.angle()], ctrls, b, out, tok)
            self.emit1(Gate.X, [], [a], b, out, tok)
            for g, ang, q in post:
                self.emit1(g, ang, [], q, out, tok)
            return
        if name == "u2":
            name, args = "u", [Lin(math.pi / 2)] + list(args)
        if name in _G1:
            g, na = _G1[name]
            if len(args) != na or len(targets) != 1:
                raise self.err(f"{name} takes {na} angles and one qubit", tok)
            g, angles = self.invert1(g, args) if inv else (g, [a.angle() for a in args])
            self.emit1(g, angles, ctrls, targets[0], out, tok)
            return
        if name in ("cu",):  # cu(theta, phi, lambda, gamma): controlled U with a control phase
            if len(args) not in (3, 4) or len(targets) != 2:
                raise self.err("cu takes 3 or 4 angles and two qubits", tok)
            gamma = args[3] if len(args) == 4 else Lin(0.0)
            if inv:
                gamma = -gamma
            g, angles = self.invert1(Gate.U, args[:3]) if inv else (Gate.U, [a.angle() for a in args[:3]])
            self.emit1(g, angles, ctrls + [targets[0]], targets[1], out, tok)
            if gamma.c0 != 0 or not gamma.const():
                self.emit1(Gate.P, [gamma.angle()], ctrls, targets[0], out, tok)
            return
        if name in _G2:
            g, na = _G2[name]
            if len(args) != na or len(targets) != 2:
                raise self.err(f"{name} takes {na} angles and two qubits", tok)
            if g in (Gate.SWAP, Gate.CX, Gate.CZ):
                if ctrls:
                    base = {Gate.CX: Gate.X, Gate.CZ: Gate.Z}.get(g)
                    if base is None:
                        raise self.err("ctrl @ swap is not supported", tok)
                    self.emit1(base, [], ctrls + [targets[0]], targets[1], out, tok)
                else:
                    out.append((lambda g, q: lambda c: c.gate(g, q))(g, list(targets)))
                return
            base = {Gate.CY: Gate.Y, Gate.CH: Gate.H, Gate.CP: Gate.P, Gate.CRX: Gate.RX, Gate.CRY: Gate.RY,
                    Gate.CRZ: Gate.RZ, Gate.CU: Gate.U}[g]
            b, angles = self.invert1(base, args) if inv else (base, [a.angle() for a in args])
            self.emit1(b, angles, ctrls + [targets[0]], targets[1], out, tok)
            return
        if name == "ccx":
            if len(targets) != 3 or args:
                raise self.err("ccx takes three qubits", tok)
            self.emit1(Gate.X, [], ctrls + targets[:2], targets[2], out, tok)
            return
        if name == "cswap":
            if len(targets) != 3 or args:
                raise self.err("cswap takes three qubits", tok)
            c, a, b = targets
            for g_ctrl, tgt in ((b, a), (a, b), (b, a)):  # swap = three CX; the middle one controlled
                cs = ctrls + [c, g_ctrl] if (g_ctrl, tgt) == (a, b) else [g_ctrl]
                self.emit1(Gate.X, [], cs, tgt, out, tok)
            return
        raise self.err(f"unknown gate {name!r}", tok)

    def invert1(self, g: Gate, args: List[Lin]) -> Tuple[Gate, List]:
        self_inv = {Gate.H, Gate.X, Gate.Y, Gate.Z}
        pairs = {Gate.S: Gate.SDG, Gate.SDG: Gate.S, Gate.T: Gate.TDG, Gate.TDG: Gate.T}
        if g in self_inv:
            return g, []
        if g in pairs:
            return pairs[g], []
        if g in (Gate.RX, Gate.RY, Gate.RZ, Gate.P):
            return g, [(-args[0]).angle()]
        if g == Gate.U:  # U(t, p, l)^dagger = U(-t, -l, -p)
            return g, [(-args[0]).angle(), (-args[2]).angle(), (-args[1]).angle()]
        if g == Gate.SX:
            return Gate.SX, ["inverse"]
        raise self.err(f"no inverse for {g.name}")

    def emit1(self, g: Gate, angles: List, ctrls: List[int], target: int, out, tok) -> None:
        """A one-qubit gate with any number of controls."""
        if angles == ["inverse"]:  # SX^dagger as a dense matrix
            m = _gate_matrix(Gate.SX, []).conj().T
            if ctrls:
                m = _controlled(m, len(ctrls))
            qs = list(ctrls) + [target]
            out.append((lambda q, m: lambda c: c.dense(q, m))(qs, m))
            return
        if not ctrls:
            out.append((lambda g, q, a: lambda c: c.gate(g, q, a))(g, [target], angles))
            return
        if len(ctrls) == 1 and g in _CTRL1:
            out.append((lambda g, q, a: lambda c: c.gate(g, q, a))(_CTRL1[g], [ctrls[0], target], angles))
            return
        if any(isinstance(a, Param) for a in angles):
            raise self.err("controls on a parametrised gate beyond the IR's controlled gates", tok)
        if len(ctrls) + 1 > 4:
            raise self.err("a dense unitary on more than four qubits", tok)
        m = _controlled(_gate_matrix(g, angles), len(ctrls))
        qs = list(ctrls) + [target]
        out.append((lambda q, m: lambda c: c.dense(q, m))(qs, m))

    def expand(self, name, args, targets, inv, ctrls, out, tok) -> None:
        gd = self.gates[name]
        if len(args) != len(gd.params) or len(targets) != len(gd.qargs):
            raise self.err(f"{name} takes {len(gd.params)} angles and {len(gd.qargs)} qubits", tok)
        env = dict(zip(gd.params, args))
        qmap = {q: [t] for q, t in zip(gd.qargs, targets)}
        body: List[Callable] = []
        sub = _Lowerer(gd.body + [Tok("eof", "", tok.line)])
        sub.qregs, sub.cregs, sub.params, sub.consts, sub.gates = {}, {}, self.params, self.consts, self.gates
        sub.nq = self.nq
        while sub.peek().kind != "eof":
            sub.gate_call(env, qmap, body)
        if not inv and not ctrls:
            out.extend(body)
            return
        # inv / ctrl on a user gate: its body as IR records, inverted (reversed, each
        # record by its inverse) and/or controlled record by record
        tmp = Circuit(max(self.nq, 1))
        for f in body:
            f(tmp)
        recs, pool = tmp.ops, tmp.pool
        if inv:
            recs = recs[::-1]
        for r in recs:
            self.emit_record(r, pool, inv, list(ctrls), out, tok)

    def emit_record(self, r, pool, inv: bool, ctrls: List[int], out, tok) -> None:
        """One GATE or DENSE record of a user gate's body, inverted if `inv`, with
        the extra controls `ctrls`."""
        if int(r["kind"]) == int(Kind.DENSE):
            k = int(r["nq"])
            qs = [int(q) for q in r["q"][:k]]
            off = int(r["dense_off"])
            m = np.asarray(pool[off: off + (1 << (2 * k))]).reshape(1 << k, 1 << k)
            if inv:
                m = m.conj().T
            if ctrls:
                if len(ctrls) + k > 4:
                    raise self.err("a dense unitary on more than four qubits", tok)
                m = _controlled_k(m, len(ctrls))
                qs = list(ctrls) + qs
            out.append((lambda q, m: lambda c: c.dense(q, m))(qs, m))
            return
        g = Gate(int(r["gate"]))
        na = GATE_ARITY[g][1]
        angles = [Param(int(r["pidx"][i]), float(r["angle"][i])) if int(r["pidx"][i]) >= 0 else float(r["angle"][i])
                  for i in range(na)]
        qs = [int(q) for q in r["q"][: GATE_ARITY[g][0]]]
        if g == Gate.SWAP:  # three CX, the middle one reversed: self-inverse in either order
            a, b = qs
            for c_, t_ in ((a, b), (b, a), (a, b)):
                self.emit1(Gate.X, [], ctrls + [c_], t_, out, tok)
            return
        base = {Gate.CX: Gate.X, Gate.CY: Gate.Y, Gate.CZ: Gate.Z, Gate.CH: Gate.H, Gate.CP: Gate.P,
                Gate.CRX: Gate.RX, Gate.CRY: Gate.RY, Gate.CRZ: Gate.RZ, Gate.CU: Gate.U}.get(g)
        inner = [qs[0]] if base is not None else []
        target = qs[-1]
        b = base if base is not None else g
        if inv:
            b, angles = _inverse1(b, angles)
        self.emit1(b, angles, ctrls + inner, target, out, tok)


def lower(src: str) -> Program:
    """Lowers an OpenQASM 3 program of the subset above to the flat IR."""
    low = _Lowerer(_tokenize(src))
    low.program()
    if low.nq == 0:
        raise QasmError("the program declares no qubits")
    c = Circuit(low.nq)
    for f in low.ops:
        f(c)
    c.n_params = max(c.n_params, len(low.params))
    return Program(c, low.nq, low.nb, dict(low.params), dict(low.qregs), dict(low.cregs))


def _main(argv: Optional[Sequence[str]] = None) -> int:
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Run an OpenQASM 3 program (subset) on the GPU.")
    ap.add_argument("file")
    ap.add_argument("--shots", type=int, default=1024)
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--param", type=float, action="append", default=[], help="input values, in declaration order")
    ap.add_argument("--engine", default="auto", choices=["auto", "branched", "per-shot", "clifford"],
                    help="auto: tableaux for Clifford programs, else shot branching (batched launch for small "
                         "programs); branched: one trajectory per distinct outcome path (the same records as "
                         "per-shot); clifford: stabilizer tableaux (Clifford gates only, up to 64 qubits)")
    a = ap.parse_args(argv)
    with open(a.file) as f:
        prog = lower(f.read())
    from . import sv

    if a.engine == "auto":
        from . import engines

        cregs, _ = engines.sample(prog.ops, prog.n_qubits, a.shots, dtype=a.dtype, params=a.param or None,
                                  pool=prog.pool if len(prog.pool) else None, seed=a.seed)
    elif a.engine == "clifford":
        with sv.Clifford(prog.n_qubits, prog.ops) as cl:
            cregs = cl.sample(a.shots, seed=a.seed)
    else:
        with sv.State(prog.n_qubits, a.dtype) as st:
            if len(prog.pool):
                st.set_dense_pool(prog.pool)
            run = st.sample_branched if a.engine == "branched" else st.sample
            cregs, _ = run(prog.ops, a.shots, params=a.param or None, seed=a.seed)
    counts: Dict[str, int] = {}
    for v in cregs:
        key = format(int(v), f"0{max(1, prog.n_bits)}b")
        counts[key] = counts.get(key, 0) + 1
    print(json.dumps({"qubits": prog.n_qubits, "bits": prog.n_bits, "shots": a.shots,
                      "counts": dict(sorted(counts.items()))}))
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())

"""FP64 CPU oracle for dynamic-circuit state-vector simulation.

TEST INFRASTRUCTURE ONLY: this package is loaded by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py``.  The CUDA product path never imports it, and it imports nothing
from the product package: it reads op lists as raw 120-byte records (the
``sv_op`` input format) and Pauli terms as 24-byte records (``sv_pauli``).

The C source (``sv_oracle.c``) is the plain amplitude-loop definition; this
wrapper adds the gradient checks built from it (parameter shift and central
finite differences; Sec. IV-D checks that energies agree across backends).

Pinned by tests/test_oracle_*.py against closed forms, numpy's independent
Philox, scipy matrix exponentials and dense Kronecker products.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

OP_ITEMSIZE = 120
PAULI_ITEMSIZE = 24
TERMINAL_DRAW = 1 << 32  # draw index of the terminal sample of a shot

DRAW_DTYPE = np.dtype(
    [("qubit", "<i4"), ("is_reset", "<i4"), ("outcome", "<i4"), ("forced", "<i4"),
     ("p0", "<f8"), ("p1", "<f8"), ("u", "<f8"), ("margin", "<f8")]
)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-D_GNU_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    u64, i32, vp, sz, dp = C.c_uint64, C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(C.c_double)
    lib.orc_philox4x64_10.argtypes = [vp, vp, vp]
    lib.orc_uniform.argtypes = [u64, u64, u64, u64]
    lib.orc_uniform.restype = C.c_double
    lib.orc_gate_matrix.argtypes = [C.c_int, vp, vp]
    lib.orc_gate_matrix.restype = C.c_int
    lib.orc_run.argtypes = [C.c_int, vp, sz, vp, sz, vp, sz, u64, u64, u64, vp, sz, vp, vp,
                            vp, sz, vp, vp, sz, vp]
    lib.orc_run.restype = C.c_int
    lib.orc_sample.argtypes = [C.c_int, vp, u64, u64, u64, u64, u64, vp, vp]
    lib.orc_sample.restype = C.c_int
    lib.orc_expval.argtypes = [C.c_int, vp, vp, sz, vp, vp]
    lib.orc_expval.restype = C.c_int
    lib.orc_norm2.argtypes = [vp, C.c_int]
    lib.orc_norm2.restype = C.c_double
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_get_threads.restype = C.c_int
    _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def set_threads(k: int) -> None:
    _load().orc_set_threads(int(k))


def get_threads() -> int:
    return int(_load().orc_get_threads())


# ------------------------------------------------------------------------- Philox
def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def uniform(seed: int, stream: int, shot: int, m: int) -> float:
    return float(_load().orc_uniform(seed, stream, shot, m))


def gate_matrix(gate: int, angles: Sequence[float] = (0.0, 0.0, 0.0)):
    """Returns (shape, 2x2 matrix): shape 1 = one-qubit, 2 = controlled, 3 = swap."""
    a = np.zeros(3, dtype=np.float64)
    a[: len(angles)] = angles
    m = np.zeros(4, dtype=np.complex128)
    shape = _load().orc_gate_matrix(int(gate), a.ctypes.data, m.ctypes.data)
    return shape, m.reshape(2, 2)


# ------------------------------------------------------------------------- runs
@dataclass
class Trajectory:
    psi: np.ndarray
    creg: int
    draws: np.ndarray
    norms: Optional[np.ndarray]
    status: int


def _ops_bytes(ops: np.ndarray) -> np.ndarray:
    ops = np.ascontiguousarray(ops)
    if ops.dtype.itemsize != OP_ITEMSIZE:
        raise ValueError("op records must be 120 bytes")
    return ops


def run(ops: np.ndarray, n: int, params=None, seed: int = 0, stream: int = 0, shot: int = 0,
        pool=None, forced=None, trace_norms: bool = False, max_draws: int = 4096,
        out: Optional[np.ndarray] = None) -> Trajectory:
    """One trajectory from |0..0> (every draw keyed by (seed, stream, shot, m))."""
    lib = _load()
    ops = _ops_bytes(ops)
    N = 1 << n
    psi = out if out is not None else np.empty(N, dtype=np.complex128)
    prm = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    pl = None if pool is None or len(pool) == 0 else np.ascontiguousarray(pool, dtype=np.complex128)
    fo = None if forced is None else np.ascontiguousarray(forced, dtype=np.int32)
    draws = np.zeros(max_draws, dtype=DRAW_DTYPE)
    creg = C.c_uint64(0)
    nd = C.c_size_t(0)
    nn = C.c_size_t(0)
    max_norms = 1 << 16 if trace_norms else 0
    norms = np.zeros(max_norms, dtype=np.float64) if trace_norms else None
    st = lib.orc_run(n, ops.ctypes.data, len(ops), _ptr(prm), 0 if prm is None else prm.size,
                     _ptr(pl), 0 if pl is None else pl.size, seed, stream, shot,
                     _ptr(fo), 0 if fo is None else fo.size, psi.ctypes.data, C.byref(creg),
                     draws.ctypes.data, max_draws, C.byref(nd), _ptr(norms), max_norms, C.byref(nn))
    k = min(nd.value, max_draws)
    return Trajectory(psi, int(creg.value), draws[:k].copy(),
                      None if norms is None else norms[: min(nn.value, max_norms)].copy(), int(st))


def sample(psi: np.ndarray, shots: int, seed: int = 0, stream: int = 0, shot0: int = 0,
           m_index: int = TERMINAL_DRAW):
    """Terminal samples (basis indices) and their relative CDF margins."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(round(math.log2(psi.size)))
    out = np.zeros(shots, dtype=np.uint64)
    mg = np.zeros(shots, dtype=np.float64)
    st = _load().orc_sample(n, psi.ctypes.data, shots, seed, stream, shot0, m_index, out.ctypes.data,
                            mg.ctypes.data)
    if st:
        raise RuntimeError(f"orc_sample failed: {st}")
    return out, mg


def expval(psi: np.ndarray, terms: np.ndarray):
    """(per-term <P_t>, sum_t c_t <P_t>)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    terms = np.ascontiguousarray(terms)
    if terms.dtype.itemsize != PAULI_ITEMSIZE:
        raise ValueError("Pauli records must be 24 bytes")
    n = int(round(math.log2(psi.size)))
    per = np.zeros(len(terms), dtype=np.float64)
    tot = C.c_double(0)
    st = _load().orc_expval(n, psi.ctypes.data, terms.ctypes.data, len(terms), per.ctypes.data,
                            C.byref(tot))
    if st:
        raise RuntimeError(f"orc_expval failed: {st}")
    return per, float(tot.value)


def norm2(psi: np.ndarray) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(_load().orc_norm2(psi.ctypes.data, int(round(math.log2(psi.size)))))


def run_shots(ops: np.ndarray, n: int, shots: int, params=None, seed: int = 0, stream: int = 0,
              pool=None, terminal: bool = False):
    """Records (and optionally terminal samples) of shots 0..shots-1."""
    cregs = np.zeros(shots, dtype=np.uint64)
    bits = np.zeros(shots, dtype=np.uint64) if terminal else None
    margins = []
    psi = np.empty(1 << n, dtype=np.complex128)
    for s in range(shots):
        tr = run(ops, n, params, seed, stream, s, pool, out=psi)
        if tr.status:
            raise RuntimeError(f"oracle run failed: {tr.status}")
        cregs[s] = tr.creg
        margins.append(tr.draws["margin"].min() if len(tr.draws) else np.inf)
        if terminal:
            b, _ = sample(psi, 1, seed, stream, s)
            bits[s] = b[0]
    return cregs, bits, np.asarray(margins)


# ------------------------------------------------------------------------- energies and gradients
def energy(ops, n, params, terms, pool=None, seed: int = 0, stream: int = 0, shot: int = 0) -> float:
    tr = run(ops, n, params, seed, stream, shot, pool)
    if tr.status:
        raise RuntimeError(f"oracle run failed: {tr.status}")
    return expval(tr.psi, terms)[1]


def param_shift_grad(ops, n, params, terms, pool=None) -> np.ndarray:
    """Parameter-shift gradient: for a parameter that enters one rotation
    exp(-i theta P / 2) with multiplier 1, dE/dtheta = (E(theta+pi/2) - E(theta-pi/2))/2."""
    p = np.array(params, dtype=np.float64)
    g = np.zeros_like(p)
    for k in range(p.size):
        pp = p.copy(); pp[k] += math.pi / 2
        pm = p.copy(); pm[k] -= math.pi / 2
        g[k] = 0.5 * (energy(ops, n, pp, terms, pool) - energy(ops, n, pm, terms, pool))
    return g


def finite_diff_grad(ops, n, params, terms, pool=None, h: float = 1e-5) -> np.ndarray:
    """Central finite differences (E(theta+h) - E(theta-h)) / 2h."""
    p = np.array(params, dtype=np.float64)
    g = np.zeros_like(p)
    for k in range(p.size):
        pp = p.copy(); pp[k] += h
        pm = p.copy(); pm[k] -= h
        g[k] = (energy(ops, n, pp, terms, pool) - energy(ops, n, pm, terms, pool)) / (2 * h)
    return g

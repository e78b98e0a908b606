"""Python binding of libsv (argument marshalling only).

Every function maps onto one C-ABI entry point of ``include/sv.h`` with the
same name; all simulation work runs in the CUDA library.  PyTorch, when it is
importable, supplies the device memory of the state (a tensor the handle
views, zero-copy) and the CUDA stream the library enqueues on.

Importing this module loads ``libsv.so``; it raises if the library was not
built (``python -m paper_2604_11599_gb300.build``) -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .ir import OP_DTYPE, PAULI_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsv.so")

SV_C64, SV_C128 = 0, 1
STATUS = {0: "SV_OK", -1: "SV_ERR_ARG", -2: "SV_ERR_OOM", -3: "SV_ERR_CUDA", -4: "SV_ERR_TIMEOUT",
          -5: "SV_ERR_UNSUPPORTED", -6: "SV_ERR_NUMERIC"}

DRAW_DTYPE = np.dtype([("qubit", "<i4"), ("is_reset", "<i4"), ("outcome", "<i4"), ("pad", "<i4"),
                       ("p0", "<f8"), ("p1", "<f8"), ("u", "<f8")])


class SVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ProgramStats(C.Structure):
    _fields_ = [("records", C.c_uint64), ("unrolled_ops", C.c_uint64), ("gates", C.c_uint64),
                ("draws", C.c_uint64), ("passes", C.c_uint64), ("stages", C.c_uint64),
                ("flags", C.c_uint64), ("tile_bits", C.c_int32), ("low_bits", C.c_int32),
                ("plan_bytes", C.c_uint64), ("specialised", C.c_int32), ("compile_seconds", C.c_double),
                ("block_barriers", C.c_uint64), ("warp_barriers", C.c_uint64), ("kernels_per_run", C.c_uint64)]


class WorkCounts(C.Structure):
    _fields_ = [("bytes_read", C.c_uint64), ("bytes_written", C.c_uint64), ("gates", C.c_uint64),
                ("draws", C.c_uint64), ("passes", C.c_uint64), ("updates", C.c_uint64)]


class GradStats(C.Structure):
    _fields_ = [("forward_passes", C.c_uint64), ("backward_passes", C.c_uint64), ("gates", C.c_uint64),
                ("term_groups", C.c_uint32), ("terms", C.c_uint32), ("state_qubits", C.c_uint32),
                ("resident_sets", C.c_uint32), ("specialised", C.c_uint32), ("pad", C.c_uint32),
                ("compile_seconds", C.c_double)]


class BranchStats(C.Structure):
    _fields_ = [("shots", C.c_uint64), ("paths", C.c_uint64), ("levels", C.c_uint64), ("max_draws", C.c_uint64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded libsv (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsv.so is not built ({LIB_PATH}); run python -m paper_2604_11599_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, sz, u64, i32, st = C.c_void_p, C.c_size_t, C.c_uint64, C.c_int, C.c_int
    sig = {
        "sv_create": ([i32, i32, vp, sz, C.POINTER(vp)], st),
        "sv_destroy": ([vp], st),
        "sv_bind_stream": ([vp, vp], st),
        "sv_set_dense_pool": ([vp, vp, sz], st),
        "sv_prepare": ([vp, vp, sz, C.POINTER(vp)], st),
        "sv_program_free": ([vp], st),
        "sv_program_info": ([vp, C.POINTER(ProgramStats)], st),
        "sv_launch": ([vp, vp, vp, sz, u64, u64, u64], st),
        "sv_run": ([vp, vp, sz, vp, sz, u64, u64, u64, vp], st),
        "sv_get_creg": ([vp, vp], st),
        "sv_get_trace": ([vp, vp, sz, C.POINTER(sz)], st),
        "sv_sample": ([vp, vp, sz, vp, sz, u64, u64, u64, vp, vp], st),
        "sv_sample_state": ([vp, u64, u64, u64, u64, vp], st),
        "sv_sample_state_device": ([vp, u64, u64, u64, u64, vp], st),
        "sv_sample_branched": ([vp, vp, sz, vp, sz, u64, u64, u64, vp, C.POINTER(BranchStats)], st),
        "sv_batch_sample_branched": ([vp, vp, vp, vp, sz, u64, vp, C.POINTER(BranchStats)], st),
        "sv_clifford_create": ([i32, vp, sz, vp, C.POINTER(vp)], st),
        "sv_clifford_sample": ([vp, u64, u64, u64, u64, vp], st),
        "sv_clifford_destroy": ([vp], st),
        "sv_expval": ([vp, vp, sz, vp, vp], st),
        "sv_expval_static": ([vp, i32, i32, vp, sz, vp, vp], st),
        "sv_get_amplitudes": ([vp, vp, sz, sz], st),
        "sv_set_amplitudes": ([vp, vp, sz, sz], st),
        "sv_state_buffer": ([vp, C.POINTER(vp), C.POINTER(sz)], st),
        "sv_set_tuning": ([vp, i32, i32, i32], st),
        "sv_sync": ([vp], st),
        "sv_profile": ([vp, i32], st),
        "sv_set_cache": ([vp, i32], st),
        "sv_set_jit": ([vp, i32], st),
        "sv_set_dense_tc": ([vp, i32], st),
        "sv_jit_check": ([i32, i32, vp, sz, vp, sz, C.c_char_p, sz], st),
        "sv_jit_check_adjoint": ([i32, i32, vp, sz, vp, sz, C.c_char_p, sz], st),
        "sv_jit_check_batch": ([i32, sz, vp, vp, vp, C.c_char_p, sz], st),
        "sv_plan_info": ([i32, i32, vp, sz, vp, sz, i32, i32, i32, C.POINTER(ProgramStats)], st),
        "sv_profile_read": ([vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.POINTER(C.c_double)], st),
        "sv_profile_work": ([vp, C.POINTER(WorkCounts)], st),
        "sv_selftest_wait": ([vp, C.c_uint32], st),
        "sv_set_tile_select": ([vp, i32], st),
        "sv_set_stage_pairs": ([vp, i32], st),
        "sv_set_jit_blocks": ([vp, i32], st),
        "sv_grad_info": ([vp, C.POINTER(GradStats)], st),
        "sv_batch_profile": ([vp, i32], st),
        "sv_batch_work": ([vp, C.POINTER(WorkCounts)], st),
        "sv_batch_create": ([i32, vp, C.POINTER(vp)], st),
        "sv_batch_add_program": ([vp, i32, vp, sz, vp, sz, vp, sz, C.POINTER(C.c_uint32)], st),
        "sv_batch_set_items": ([vp, vp, vp, vp, sz], st),
        "sv_batch_launch": ([vp, u64], st),
        "sv_batch_results": ([vp, vp], st),
        "sv_batch_run": ([vp, vp, vp, vp, sz, u64, vp], st),
        "sv_batch_destroy": ([vp], st),
        "sv_batch_set_tuning": ([vp, i32, i32], st),
        "sv_grad_create": ([i32, i32, vp, sz, vp, sz, vp, sz, vp, C.POINTER(vp)], st),
        "sv_grad_run": ([vp, vp, sz, sz, vp, vp], st),
        "sv_grad_destroy": ([vp], st),
        "sv_grad_set_jit": ([vp, i32], st),
        "sv_batch_set_jit": ([vp, i32], st),
        "sv_batch_jit_info": ([vp, C.POINTER(i32), C.POINTER(C.c_double)], st),
        "sv_expval_grad_batch": ([i32, i32, vp, sz, vp, sz, sz, vp, sz, vp, vp, vp], st),
        "sv_last_error": ([], C.c_char_p),
        "sv_version": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int) -> None:
    if status != 0:
        raise SVError(status, lib().sv_last_error().decode())


def _ops(ops: np.ndarray) -> np.ndarray:
    ops = np.ascontiguousarray(ops)
    if ops.dtype != OP_DTYPE:
        raise TypeError("ops must be an array of ir.OP_DTYPE records")
    return ops


def _f64(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None or a.size == 0 else a.ctypes.data


def _torch():
    try:
        import torch  # noqa: F401
        return torch
    except Exception:  # pragma: no cover - torch is part of the image
        return None


class Program:
    """A lowered program (``sv_prepare``); launch it with :meth:`State.launch`."""

    def __init__(self, handle: int, owner: "State"):
        self._h = handle
        self.owner = owner

    @property
    def stats(self) -> dict:
        s = ProgramStats()
        _check(lib().sv_program_info(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ProgramStats._fields_}

    def free(self):
        if self._h:
            _check(lib().sv_program_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class State:
    """A state vector of ``n`` qubits (``sv_create``) in |0...0>."""

    def __init__(self, n: int, dtype: str = "c64", buffer=None, stream=None):
        self.n = int(n)
        self.dtype = dtype
        self.dt = SV_C64 if dtype == "c64" else SV_C128
        self.amp = np.complex64 if dtype == "c64" else np.complex128
        torch = _torch()
        n_int = max(self.n, 10)  # the library pads small states to 10 qubits
        self._buf = buffer
        if self._buf is None and torch is not None and torch.cuda.is_available() and 1 <= self.n <= 34:
            real = torch.float32 if dtype == "c64" else torch.float64
            self._buf = torch.empty(2 << n_int, dtype=real, device="cuda")
        ptr, nbytes = None, 0
        if self._buf is not None:
            ptr = self._buf.data_ptr()
            nbytes = self._buf.numel() * self._buf.element_size()
        h = C.c_void_p()
        _check(lib().sv_create(self.n, self.dt, ptr, nbytes, C.byref(h)))
        self._h = h.value
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        if stream is not None:
            _check(lib().sv_bind_stream(self._h, stream))
        self._pool = None

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().sv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- configuration
    def bind_stream(self, stream) -> None:
        _check(lib().sv_bind_stream(self._h, stream))

    def set_dense_pool(self, pool) -> None:
        p = np.ascontiguousarray(pool, dtype=np.complex128)
        self._pool = p
        _check(lib().sv_set_dense_pool(self._h, _ptr(p), p.size))

    def set_jit(self, enable: bool) -> None:
        """Per-program specialised sweep kernels (compiled on a program's first launch)."""
        _check(lib().sv_set_jit(self._h, 1 if enable else 0))

    def set_dense_tc(self, enable: bool) -> None:
        """Dense four-qubit gates on the tensor cores (complex64, 2^12-amplitude tiles; on by default)."""
        _check(lib().sv_set_dense_tc(self._h, 1 if enable else 0))

    def set_cache(self, enable: bool) -> None:
        _check(lib().sv_set_cache(self._h, 1 if enable else 0))

    def set_jit_blocks(self, blocks_per_sm: int = 0) -> None:
        """CTAs per SM of the specialised kernels (0: the default for the dtype)."""
        _check(lib().sv_set_jit_blocks(self._h, int(blocks_per_sm)))

    def set_tile_select(self, closure: bool = True) -> None:
        """Tile qubits chosen for the gates they unlock (True) or by first fit."""
        _check(lib().sv_set_tile_select(self._h, 1 if closure else 0))

    def set_stage_pairs(self, mode: int = 0) -> None:
        """Complex64 stage packing: 0 fewest stages, 1/2 weigh 16-byte pair accesses."""
        _check(lib().sv_set_stage_pairs(self._h, int(mode)))

    def set_tuning(self, tile_bits: int = 0, low_bits: int = 0, max_pass_gates: int = 0) -> None:
        _check(lib().sv_set_tuning(self._h, tile_bits, low_bits, max_pass_gates))

    # -------------------------------------------------------------- running
    def prepare(self, ops: np.ndarray) -> Program:
        ops = _ops(ops)
        h = C.c_void_p()
        _check(lib().sv_prepare(self._h, _ptr(ops), len(ops), C.byref(h)))
        return Program(h.value, self)

    def launch(self, prog: Program, dev_params=None, seed: int = 0, stream_id: int = 0, shot: int = 0) -> None:
        """Asynchronous run with device-resident parameters (a CUDA tensor of float64 or None)."""
        ptr, n = None, 0
        if dev_params is not None:
            ptr, n = dev_params.data_ptr(), dev_params.numel()
        _check(lib().sv_launch(self._h, prog._h, ptr, n, seed, stream_id, shot))

    def run(self, ops: np.ndarray, params=None, seed: int = 0, stream_id: int = 0, shot: int = 0,
            wait: bool = True) -> Optional[int]:
        ops = _ops(ops)
        p = _f64(params)
        creg = C.c_uint64(0)
        _check(lib().sv_run(self._h, _ptr(ops), len(ops), _ptr(p), 0 if p is None else p.size,
                            seed, stream_id, shot, C.byref(creg) if wait else None))
        return int(creg.value) if wait else None

    def creg(self) -> int:
        v = C.c_uint64(0)
        _check(lib().sv_get_creg(self._h, C.byref(v)))
        return int(v.value)

    def trace(self, max_draws: int = 4096) -> np.ndarray:
        out = np.zeros(max_draws, dtype=DRAW_DTYPE)
        n = C.c_size_t(0)
        _check(lib().sv_get_trace(self._h, out.ctypes.data, max_draws, C.byref(n)))
        return out[: min(n.value, max_draws)].copy()

    def sample(self, ops: np.ndarray, shots: int, params=None, seed: int = 0, stream_id: int = 0,
               terminal: bool = False):
        ops = _ops(ops)
        p = _f64(params)
        cregs = np.zeros(shots, dtype=np.uint64)
        bits = np.zeros(shots, dtype=np.uint64) if terminal else None
        _check(lib().sv_sample(self._h, _ptr(ops), len(ops), _ptr(p), 0 if p is None else p.size, shots, seed,
                               stream_id, _ptr(cregs), _ptr(bits)))
        return cregs, bits

    def sample_branched(self, ops: np.ndarray, shots: int, params=None, seed: int = 0, stream_id: int = 0):
        """The registers sample() gives, one trajectory per distinct outcome path
        (``sv_sample_branched``); returns (cregs, stats)."""
        ops = _ops(ops)
        p = _f64(params)
        cregs = np.zeros(shots, dtype=np.uint64)
        st = BranchStats()
        _check(lib().sv_sample_branched(self._h, _ptr(ops), len(ops), _ptr(p), 0 if p is None else p.size, shots,
                                        seed, stream_id, _ptr(cregs), C.byref(st)))
        return cregs, st.as_dict()

    def sample_state(self, shots: int, seed: int = 0, stream_id: int = 0, shot0: int = 0) -> np.ndarray:
        out = np.zeros(shots, dtype=np.uint64)
        _check(lib().sv_sample_state(self._h, shots, seed, stream_id, shot0, _ptr(out)))
        return out

    def sample_state_device(self, out, seed: int = 0, stream_id: int = 0, shot0: int = 0) -> None:
        """Terminal samples into a device tensor (uint64 / int64, one per shot);
        asynchronous on the bound stream."""
        _check(lib().sv_sample_state_device(self._h, int(out.numel()), seed, stream_id, shot0, out.data_ptr()))

    def expval(self, terms: np.ndarray):
        terms = np.ascontiguousarray(terms)
        if terms.dtype != PAULI_DTYPE:
            raise TypeError("terms must be an array of ir.PAULI_DTYPE records")
        tot = C.c_double(0)
        per = np.zeros(len(terms), dtype=np.float64)
        _check(lib().sv_expval(self._h, _ptr(terms), len(terms), C.byref(tot), _ptr(per)))
        return float(tot.value), per

    def amplitudes(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        count = (1 << self.n) - first if count is None else count
        out = np.empty(count, dtype=self.amp)
        _check(lib().sv_get_amplitudes(self._h, out.ctypes.data, first, count))
        return out

    def set_amplitudes(self, values, first: int = 0) -> None:
        v = np.ascontiguousarray(values, dtype=self.amp)
        _check(lib().sv_set_amplitudes(self._h, v.ctypes.data, first, v.size))

    def sync(self) -> None:
        _check(lib().sv_sync(self._h))

    def profile(self, enable: bool = True) -> None:
        _check(lib().sv_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """Pass-kernel time, launches and the device work counters since
        profiling was enabled or last read (then reset)."""
        w = WorkCounts()
        _check(lib().sv_profile_work(self._h, C.byref(w)))
        ms, n, b = C.c_double(0), C.c_uint64(0), C.c_double(0)
        _check(lib().sv_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(b)))
        out = {"ms": ms.value, "launches": int(n.value), "bytes": b.value}
        out.update({k: int(getattr(w, k)) for k, _ in WorkCounts._fields_})
        return out

    def selftest_wait(self, polls: int = 1000) -> None:
        """Runs a bounded device wait that always runs out; raises SVError
        (SV_ERR_TIMEOUT) exactly as a timed-out pass does."""
        _check(lib().sv_selftest_wait(self._h, int(polls)))

    def tensor(self):
        """Zero-copy torch view (complex) of the state, or None without torch."""
        if self._buf is None:
            return None
        torch = _torch()
        return torch.view_as_complex(self._buf.view(-1, 2))[: 1 << self.n]


def plan_info(ops: np.ndarray, n: int, dtype: str = "c64", pool=None, tile_bits: int = 0, low_bits: int = 0,
              max_pass_gates: int = 0) -> dict:
    """Host-only lowering statistics (``sv_plan_info``); needs no GPU."""
    ops = _ops(ops)
    p = None if pool is None else np.ascontiguousarray(pool, dtype=np.complex128)
    s = ProgramStats()
    _check(lib().sv_plan_info(n, SV_C64 if dtype == "c64" else SV_C128, _ptr(ops), len(ops), _ptr(p),
                              0 if p is None else p.size, tile_bits, low_bits, max_pass_gates, C.byref(s)))
    return {k: getattr(s, k) for k, _ in ProgramStats._fields_}


class Batch:
    """Many trajectories in one persistent launch (``sv_batch_*``)."""

    def __init__(self, dtype: str = "c64", stream=None):
        self.dtype = dtype
        torch = _torch()
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        _check(lib().sv_batch_create(SV_C64 if dtype == "c64" else SV_C128, stream, C.byref(h)))
        self._h = h.value
        self.n_items = 0

    def add_program(self, ops: np.ndarray, n: int, params=None, pool=None) -> int:
        ops = _ops(ops)
        p = _f64(params)
        pl = None if pool is None or len(pool) == 0 else np.ascontiguousarray(pool, dtype=np.complex128)
        pid = C.c_uint32(0)
        _check(lib().sv_batch_add_program(self._h, n, _ptr(ops), len(ops), _ptr(p), 0 if p is None else p.size,
                                          _ptr(pl), 0 if pl is None else pl.size, C.byref(pid)))
        return int(pid.value)

    def set_tuning(self, low_bits: int = 0, max_pass_gates: int = 0) -> None:
        """Planner tuning of programs added from now on (``sv_batch_set_tuning``)."""
        _check(lib().sv_batch_set_tuning(self._h, low_bits, max_pass_gates))

    def set_items(self, prog_ids, stream_ids, shots) -> None:
        pr = np.ascontiguousarray(prog_ids, dtype=np.uint32)
        sid = np.ascontiguousarray(stream_ids, dtype=np.uint64)
        sh = np.ascontiguousarray(shots, dtype=np.uint64)
        if not (pr.size == sid.size == sh.size):
            raise ValueError("item arrays differ in length")
        _check(lib().sv_batch_set_items(self._h, _ptr(pr), _ptr(sid), _ptr(sh), pr.size))
        self.n_items = pr.size

    def launch(self, seed: int = 0) -> None:
        _check(lib().sv_batch_launch(self._h, seed))

    def results(self) -> np.ndarray:
        out = np.zeros(self.n_items, dtype=np.uint64)
        _check(lib().sv_batch_results(self._h, _ptr(out)))
        return out

    def run(self, prog_ids, stream_ids, shots, seed: int = 0) -> np.ndarray:
        self.set_items(prog_ids, stream_ids, shots)
        self.launch(seed)
        return self.results()

    def sample_branched(self, prog_ids, stream_ids, n_shots, seed: int = 0):
        """Request r: n_shots[r] shots (counters 0..) of program prog_ids[r] on
        stream stream_ids[r], one trajectory per distinct outcome path
        (``sv_batch_sample_branched``); returns (cregs request after request, stats)."""
        pr = np.ascontiguousarray(prog_ids, dtype=np.uint32)
        sid = np.ascontiguousarray(stream_ids, dtype=np.uint64)
        ns = np.ascontiguousarray(n_shots, dtype=np.uint64)
        if not (pr.size == sid.size == ns.size):
            raise ValueError("request arrays differ in length")
        cregs = np.zeros(int(ns.sum()), dtype=np.uint64)
        st = BranchStats()
        _check(lib().sv_batch_sample_branched(self._h, _ptr(pr), _ptr(sid), _ptr(ns), pr.size, seed, _ptr(cregs),
                                              C.byref(st)))
        self.n_items = 0
        return cregs, st.as_dict()

    def profile(self, enable: bool = True) -> None:
        """Device work counters of the following launches (zeroed on enable)."""
        _check(lib().sv_batch_profile(self._h, 1 if enable else 0))

    def work(self) -> dict:
        w = WorkCounts()
        _check(lib().sv_batch_work(self._h, C.byref(w)))
        return {k: int(getattr(w, k)) for k, _ in WorkCounts._fields_}

    def set_jit(self, on: bool = True) -> None:
        """Launches run a kernel specialised to the programs added so far (compiled
        at the next launch) instead of the generic one."""
        _check(lib().sv_batch_set_jit(self._h, 1 if on else 0))

    def jit_info(self) -> dict:
        spec, secs = C.c_int(0), C.c_double(0)
        _check(lib().sv_batch_jit_info(self._h, C.byref(spec), C.byref(secs)))
        return {"specialised": bool(spec.value), "compile_seconds": float(secs.value)}

    def close(self):
        if getattr(self, "_h", None):
            lib().sv_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Clifford:
    """Clifford programs on up to 64 qubits by stabilizer tableaux, one warp per
    shot (``sv_clifford_*``)."""

    def __init__(self, n: int, ops: np.ndarray, stream=None):
        ops = _ops(ops)
        torch = _torch()
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        _check(lib().sv_clifford_create(n, _ptr(ops), len(ops), stream, C.byref(h)))
        self._h = h.value
        self.n = n

    def sample(self, shots: int, seed: int = 0, stream_id: int = 0, shot0: int = 0) -> np.ndarray:
        out = np.zeros(shots, dtype=np.uint64)
        _check(lib().sv_clifford_sample(self._h, shots, seed, stream_id, shot0, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().sv_clifford_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Grad:
    """Energies and adjoint gradients of <H> for batches of parameter sets
    (``sv_grad_*``); parameters and results live on the GPU as torch tensors."""

    def __init__(self, ops: np.ndarray, n: int, terms: np.ndarray, dtype: str = "c64", pool=None, stream=None):
        ops = _ops(ops)
        terms = np.ascontiguousarray(terms)
        if terms.dtype != PAULI_DTYPE:
            raise TypeError("terms must be an array of ir.PAULI_DTYPE records")
        torch = _torch()
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        pl = None if pool is None or len(pool) == 0 else np.ascontiguousarray(pool, dtype=np.complex128)
        h = C.c_void_p()
        _check(lib().sv_grad_create(n, SV_C64 if dtype == "c64" else SV_C128, _ptr(ops), len(ops), _ptr(pl),
                                    0 if pl is None else pl.size, _ptr(terms), len(terms), stream, C.byref(h)))
        self._h = h.value
        self.n, self.dtype = n, dtype

    def run(self, params):
        """params: [P, n_params] float64 CUDA tensor -> (energies [P], gradients [P, n_params])."""
        import torch

        params = params.detach().contiguous()
        if params.dtype != torch.float64 or not params.is_cuda or params.dim() != 2:
            raise TypeError("params must be a 2-D float64 CUDA tensor")
        P, n_params = params.shape
        val = torch.empty(P, dtype=torch.float64, device=params.device)
        grad = torch.empty(P, n_params, dtype=torch.float64, device=params.device)
        _check(lib().sv_grad_run(self._h, params.data_ptr(), P, n_params, val.data_ptr(), grad.data_ptr()))
        return val, grad

    def set_jit(self, on: bool = True) -> None:
        """Specialised kernel for this program (default) or the generic one."""
        _check(lib().sv_grad_set_jit(self._h, 1 if on else 0))

    def info(self) -> dict:
        """Passes, gates, term groups and resident sets of one parameter set's
        work; whether the specialised kernel runs, and its compile seconds."""
        g = GradStats()
        _check(lib().sv_grad_info(self._h, C.byref(g)))
        out = {k: int(getattr(g, k)) for k, _ in GradStats._fields_ if k not in ("pad", "compile_seconds")}
        out["compile_seconds"] = float(g.compile_seconds)
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().sv_grad_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expval_grad_batch(ops: np.ndarray, n: int, params: np.ndarray, terms: np.ndarray, dtype: str = "c64"):
    """``sv_expval_grad_batch`` with host arrays: (energies [P], gradients [P, n_params])."""
    ops = _ops(ops)
    p = np.ascontiguousarray(params, dtype=np.float64)
    if p.ndim != 2:
        raise ValueError("params must be [P, n_params]")
    terms = np.ascontiguousarray(terms)
    val = np.zeros(p.shape[0])
    grad = np.zeros_like(p)
    torch = _torch()
    stream = torch.cuda.current_stream().cuda_stream if torch is not None and torch.cuda.is_available() else None
    _check(lib().sv_expval_grad_batch(n, SV_C64 if dtype == "c64" else SV_C128, _ptr(ops), len(ops), _ptr(p),
                                      p.shape[0], p.shape[1], _ptr(terms), len(terms), _ptr(val), _ptr(grad), stream))
    return val, grad


def sv_expval_static(dev_state_ptr: int, n: int, dtype: str, terms: np.ndarray, dev_out_ptr: int,
                     stream: Optional[int] = None) -> None:
    """``sv_expval_static``: per-term <P_t> of a device-resident state into a
    caller-owned device array, with no device allocation by the library (for
    callers whose device memory is owned by their own allocator or pool)."""
    terms = np.ascontiguousarray(terms)
    if terms.dtype != PAULI_DTYPE:
        raise TypeError("terms must be an array of ir.PAULI_DTYPE records")
    _check(lib().sv_expval_static(dev_state_ptr, n, SV_C64 if dtype == "c64" else SV_C128, _ptr(terms), len(terms),
                                  dev_out_ptr, stream))


def jit_check(ops: np.ndarray, n: int, dtype: str = "c64", pool=None) -> str:
    """Compiles a program's specialised module on the host (no GPU); returns the log, raises on failure."""
    ops = _ops(ops)
    pl = None if pool is None or len(pool) == 0 else np.ascontiguousarray(pool, dtype=np.complex128)
    buf = C.create_string_buffer(8192)
    st = lib().sv_jit_check(n, SV_C64 if dtype == "c64" else SV_C128, _ptr(ops), len(ops), _ptr(pl),
                            0 if pl is None else pl.size, buf, 8192)
    if st != 0:
        raise SVError(st, buf.value.decode(errors="replace"))
    return buf.value.decode(errors="replace")


def jit_check_adjoint(ops: np.ndarray, n: int, dtype: str = "c64", pool=None) -> str:
    """Compiles a program's specialised adjoint kernel on the host (no GPU); returns the log, raises on failure."""
    ops = _ops(ops)
    pl = None if pool is None or len(pool) == 0 else np.ascontiguousarray(pool, dtype=np.complex128)
    buf = C.create_string_buffer(8192)
    st = lib().sv_jit_check_adjoint(n, SV_C64 if dtype == "c64" else SV_C128, _ptr(ops), len(ops), _ptr(pl),
                                    0 if pl is None else pl.size, buf, 8192)
    if st != 0:
        raise SVError(st, buf.value.decode(errors="replace"))
    return buf.value.decode(errors="replace")


def jit_check_batch(programs, dtype: str = "c64") -> str:
    """Compiles the batched kernel specialised to [(ops, n), ...] on the host
    (no GPU); returns the log, raises on failure."""
    arrs = [_ops(o) for o, _ in programs]
    k = len(arrs)
    ns = (C.c_int * k)(*[int(n) for _, n in programs])
    ptrs = (C.c_void_p * k)(*[a.ctypes.data for a in arrs])
    lens = (C.c_size_t * k)(*[len(a) for a in arrs])
    buf = C.create_string_buffer(8192)
    st = lib().sv_jit_check_batch(SV_C64 if dtype == "c64" else SV_C128, k, ns, ptrs, lens, buf, 8192)
    if st != 0:
        raise SVError(st, buf.value.decode(errors="replace"))
    return buf.value.decode(errors="replace")


def version() -> str:
    return lib().sv_version().decode()

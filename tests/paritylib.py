"""Helpers that compare the CUDA path with the oracle (test code).

Tolerances (from the benchmark spec of the method's targets):
  amplitudes max-abs 1e-12 (complex128) / 2e-5 (complex64);
  expectation values 1e-10 / 1e-5;
  measurement records bit-exact, except draws whose oracle margin
  |u - p0/(p0+p1)| is below the near-threshold band (1e-9 for complex128;
  1e-5 for complex64, whose FP32 state moves p by ~1e-6).  A trajectory that
  diverges at such a draw is re-run in the oracle with the GPU's outcomes
  forced, and its amplitudes must then agree.

Every comparison tallies its draws under a label: how many there were, how
many lie within 1e-9 of the threshold, how many within the band, and how many
trajectories needed the forced re-run.  conftest.py prints the tallies at the
end of the session.
"""
import numpy as np

AMP_TOL = {"c64": 2e-5, "c128": 1e-12}
EXP_TOL = {"c64": 1e-5, "c128": 1e-10}
BAND = {"c64": 1e-5, "c128": 1e-9}

# label -> {"draws", "near_1e-9", "near_band", "forced", "mismatch_in_band"}
NEAR: dict = {}


def tally(label, margins, dtype, forced=0, mismatch_in_band=0):
    """Adds one trajectory's oracle draw margins to the counts of `label`."""
    d = NEAR.setdefault(label, {"draws": 0, "near_1e-9": 0, "near_band": 0, "forced": 0,
                                "mismatch_in_band": 0, "band": BAND[dtype]})
    m = np.asarray(margins, dtype=np.float64)
    d["draws"] += int(m.size)
    d["near_1e-9"] += int((m < 1e-9).sum())
    d["near_band"] += int((m < BAND[dtype]).sum())
    d["forced"] += int(forced)
    d["mismatch_in_band"] += int(mismatch_in_band)
    return d


def _records_agree(g_out, ref, orc_rerun, dtype):
    """Bit-exact records, or a divergence inside the band followed by a forced
    oracle re-run; returns (reference trajectory to compare with, forced?)."""
    r_out = list(ref.draws["outcome"])
    if g_out == r_out:
        return ref, False
    near = ref.draws["margin"] < BAND[dtype]
    k = next(i for i in range(min(len(g_out), len(r_out)) + 1)
             if i >= len(g_out) or i >= len(r_out) or g_out[i] != r_out[i])
    assert k < len(r_out) and near[k], (
        f"records diverge at draw {k} away from the threshold (margin {ref.draws['margin'][k]:.3g})")
    ref = orc_rerun(np.array(g_out, dtype=np.int32))
    assert list(ref.draws["outcome"]) == g_out
    return ref, True


def compare_run(st, orc, ops, n, dtype, params=None, seed=0, stream=0, shot=0, pool=None,
                check_amps=True, stats=None, label=None):
    """Runs one trajectory on both sides and asserts parity. Returns the GPU creg."""
    creg = st.run(ops, params, seed, stream, shot)
    gtr = st.trace()
    ref = orc.run(ops, n, params, seed, stream, shot, pool)
    assert ref.status == 0
    margins = ref.draws["margin"]
    near = margins < BAND[dtype]
    if stats is not None:
        stats["draws"] = stats.get("draws", 0) + len(ref.draws)
        stats["near_1e-9"] = stats.get("near_1e-9", 0) + int((margins < 1e-9).sum())
        stats["near_band"] = stats.get("near_band", 0) + int(near.sum())
    ref, forced = _records_agree(
        list(gtr["outcome"]), ref,
        lambda f: orc.run(ops, n, params, seed, stream, shot, pool, forced=f), dtype)
    if forced and stats is not None:
        stats["forced"] = stats.get("forced", 0) + 1
    tally(label or "other parity tests", margins, dtype, forced=int(forced))
    assert creg == ref.creg
    if check_amps:
        psi = st.amplitudes()
        err = float(np.max(np.abs(psi.astype(np.complex128) - ref.psi)))
        assert err <= AMP_TOL[dtype], f"max-abs amplitude error {err:.3g} > {AMP_TOL[dtype]}"
        return creg, err
    return creg, 0.0


def compare_large(st, orc, ops, n, dtype, seed=0, stream=0, shot=0, label=None, chunk=1 << 24):
    """compare_run for states too large to copy whole: the oracle writes into
    one preallocated FP64 vector and the GPU amplitudes are read back and
    compared chunk by chunk.  Returns (creg, max-abs amplitude error)."""
    creg = st.run(ops, seed=seed, stream_id=stream, shot=shot)
    gtr = st.trace()
    psi = np.empty(1 << n, dtype=np.complex128)
    ref = orc.run(ops, n, seed=seed, stream=stream, shot=shot, out=psi)
    assert ref.status == 0
    margins = ref.draws["margin"]
    ref, forced = _records_agree(
        list(gtr["outcome"]), ref,
        lambda f: orc.run(ops, n, seed=seed, stream=stream, shot=shot, forced=f, out=psi), dtype)
    tally(label or f"n={n} {dtype}", margins, dtype, forced=int(forced))
    assert creg == ref.creg
    err = 0.0
    for first in range(0, 1 << n, chunk):
        cnt = min(chunk, (1 << n) - first)
        g = st.amplitudes(first, cnt)
        err = max(err, float(np.max(np.abs(g.astype(np.complex128) - psi[first:first + cnt]))))
    assert err <= AMP_TOL[dtype], f"max-abs amplitude error {err:.3g} > {AMP_TOL[dtype]}"
    return creg, err


# ------------------------------------------------------------- oracle worker processes
# Trajectories of small states run one per process, each oracle single-threaded.
# The pool uses the spawn start method, so it never inherits a CUDA context.
def _orc_init():
    import oracle

    oracle.build()
    oracle.set_threads(1)


def _orc_traj(job):
    import oracle

    ops, n, seed, stream, shot = job
    tr = oracle.run(ops, n, seed=seed, stream=stream, shot=shot)
    return tr.status, tr.creg, tr.draws["margin"].copy(), tr.draws["outcome"].copy()


def oracle_pool(workers=None):
    import multiprocessing as mp
    import os

    k = workers or max(1, min(16, os.cpu_count() or 1))
    return mp.get_context("spawn").Pool(k, initializer=_orc_init)

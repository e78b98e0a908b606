#!/usr/bin/env python
"""Benchmark of the plain dynamic-circuit path: amplitude-gate updates/s.

Workload (one step = one trajectory of the whole program): the layered
dynamic circuit on n=30 qubits in complex64 -- 20 layers of a random rotation
on every qubit then CX on a random perfect matching, a measure + reset of two
random qubits every 4 layers and a 3-bit feed-forward cond (X / Z), generator
seed 5, Philox seed 0, shot = step index.  The 8 GiB state is larger than L2,
so no flush is needed between steps.

value     updates/s = (gates + measures + resets) * 2^n per step / device time,
          inputs resident (the lowered program is on the device), CUDA events
          on the launching stream, K steps after W warm-up steps.
e2e       the same metric through sv_run with host buffers: every step lowers
          the op list and copies the plan to the device (program cache off;
          compiled kernels are reused), runs, and reads the classical register
          back.
roofline  the state-sweep pass kernel (k_pass): algorithmic bytes (state read
          + written once per storing pass) / its event-timed duration,
          against the measured HBM copy bandwidth.
cpu_baseline / --impl reference
          the FP64 oracle on the machine's host cores over a bounded prefix of the
          same n=30 program (gates only), in the same metric.

Multi-GPU: the path shards by independent trajectories; each rank runs its own
replica (no collective on the data path), time is the max over ranks and
value the sum of all ranks' updates over that time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude-gate updates/s"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batching / VQE / serving measurements")
    ap.add_argument("--no-jit", action="store_true", help="use the generic pass kernels")
    ap.add_argument("--circuit", default="layered", choices=["layered", "dense4"],
                    help="layered: the plain dynamic-circuit workload; dense4: layers of dense 4-qubit unitaries")
    ap.add_argument("--no-dense-tc", action="store_true", help="dense 4-qubit gates on the FP32 pipes")
    ap.add_argument("--first-fit", action="store_true", help="plan tiles by first fit instead of by the gates they unlock")
    ap.add_argument("--stage-pairs", type=int, default=None, choices=(0, 1, 2),
                    help="complex64 stage packing: 0 fewest stages, 1/2 weigh 16-byte pair accesses")
    ap.add_argument("--jit-blocks", type=int, default=0, help="CTAs per SM of the specialised kernels (0: default)")
    ap.add_argument("--form", default=None, choices=["batching", "adjoint", "sample_expval"],
                    help="run only this auxiliary measurement (for profiling) and print its JSON")
    ap.add_argument("--items", type=int, default=65536, help="--form batching: trajectories")
    ap.add_argument("--jit", action="store_true", help="--form batching: the kernel specialised to the programs")
    ap.add_argument("--sets", type=int, default=1024, help="--form adjoint: parameter sets")
    ap.add_argument("--tile-bits", type=int, default=0, help="qubits per shared-memory tile (0: default 12)")
    ap.add_argument("--low-bits", type=int, default=0, help="contiguous low qubits per tile (0: default 4)")
    return ap.parse_args()


def workload_name(n, dtype, kind="layered"):
    cx = "complex64" if dtype == "c64" else "complex128"
    if kind == "dense4":
        return (f"dense-unitary circuit, n={n}, {cx}: 6 layers of Haar-random 4-qubit unitaries on a random "
                f"partition of the qubits, RX/RY/RZ on the n mod 4 left over; 1 trajectory per step")
    return (f"plain layered dynamic circuit, n={n}, {cx}: "
            f"20 layers (rotation on every qubit + CX perfect matching), measure+reset 2 qubits every 4 layers, "
            f"3-bit cond X/Z; 1 trajectory per step")


def circuit(n, dtype, kind="layered"):
    from paper_2604_11599_gb300 import workloads

    if kind == "dense4":
        return workloads.dense_layers(12, n, layers=6)
    return workloads.layered(workloads.LAYERED_SEEDS.get((n, dtype), 5), n, layers=20)


# FP64 operations the sweep kernels execute per amplitude for each IR gate (complex128):
# factored RX / RY one FMA per component (4), one-qubit diagonals a complex multiply on
# half the amplitudes (3), CX / X / SWAP register renames (0), other one-qubit gates a
# 2x2 complex product (14), controlled ones the same on half (7), plus 6 per storing
# pass for the pass factor.  Nominal GB300 FP64 rate: 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25

# DRAM bytes (read + write) over the state bytes the pass kernels counted, for
# all 32 specialised pass launches of one step of the n=26 complex64 layered
# program (ncu dram__bytes_read.sum + dram__bytes_write.sum: 16.111 GB read,
# 14.948 GB written, against 16.106 + 16.643 GB counted; writes fall short of
# the count because the last tiles stored are still in L2 when a launch ends).
# Summarised in profiles/sv_jit_passes_layered_n30_c64.md.  A pass's traffic
# is proportional to the state, so a launch at any n moves this fraction of the
# bytes it counts.
PASS_DRAM_OVER_COUNTED = 31.059e9 / 32.749e9


def fp64_ops_per_step(ops, n_passes, n):
    from paper_2604_11599_gb300.ir import Gate, Kind

    per = {Gate.RX: 4, Gate.RY: 4, Gate.RZ: 3, Gate.P: 3, Gate.S: 3, Gate.SDG: 3, Gate.T: 3, Gate.TDG: 3,
           Gate.Z: 3, Gate.CX: 0, Gate.X: 0, Gate.SWAP: 0, Gate.CZ: 0, Gate.I: 0}
    total = 0
    for r in ops:
        if int(r["kind"]) != int(Kind.GATE):
            continue
        g = Gate(int(r["gate"]))
        total += per.get(g, 7 if g >= Gate.CX else 14)
    return float(total + 6 * n_passes) * float(1 << n)


def near_threshold(st, prog, steps, stream_id, dtype):
    """The timed steps' draws again (untimed): how many fell within 1e-9 of the
    outcome threshold, and within the dtype's parity band, by the margins the
    GPU itself computed, |u - p0/(p0+p1)|."""
    import numpy as np

    band = 1e-5 if dtype == "c64" else 1e-9
    tot = n9 = nb = 0
    mn = float("inf")
    for i in range(steps):
        st.launch(prog, seed=0, stream_id=stream_id, shot=i)
        tr = st.trace()
        if len(tr):
            m = np.abs(tr["u"] - tr["p0"] / (tr["p0"] + tr["p1"]))
            tot += len(m)
            n9 += int((m < 1e-9).sum())
            nb += int((m < band).sum())
            mn = min(mn, float(m.min()))
    return {"draws": tot, "within_1e-9": n9, f"within_{band:g}": nb, "min_margin": mn,
            "margins": "GPU-side |u - p0/(p0+p1)| of the timed steps' draws"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(n, dtype, seconds, gates_cap=None, kind="layered"):
    """The oracle over the longest gate-only prefix of the program that fits in
    `seconds`; returns (updates/s, sample description, threads)."""
    import numpy as np

    import oracle

    oracle.build()
    c = circuit(n, dtype, kind)
    ops = c.ops
    pool = c.pool if len(c.pool) else None
    gate_only = 0
    while gate_only < len(ops) and ops[gate_only]["kind"] in (1, 2):
        gate_only += 1
    psi = np.empty(1 << n, dtype=np.complex128)
    # calibrate on 4 gates, then size the prefix to the time budget
    t0 = time.perf_counter()
    oracle.run(ops[:4], n, pool=pool, out=psi)
    t_small = time.perf_counter() - t0
    per_gate = max(t_small / 4, 1e-6)
    k = int(max(4, min(gate_only, seconds / per_gate)))
    if gates_cap:
        k = min(k, gates_cap)
    t0 = time.perf_counter()
    tr = oracle.run(ops[:k], n, pool=pool, out=psi)
    dt = time.perf_counter() - t0
    assert tr.status == 0
    ups = k * float(1 << n) / dt
    return ups, f"first {k} gates (gate-only prefix) of the n={n} program, FP64, one trajectory", \
        oracle.get_threads(), dt


def clifford_form(sv, W, np):
    """Clifford programs on the stabilizer tableaux against the state-vector engines."""
    cl = {}
    rep = W.repetition_code(32, 10, flip_every=1, ghz=True)
    rnd = W.random_clifford_dynamic(21, 64, n_ops=150)
    for name, circ, nq in (("repetition_d32_10_rounds_63q", rep, 63), ("random_dynamic_64q_150_ops", rnd, 64)):
        with sv.Clifford(nq, circ.ops) as h:
            h.sample(1000)
            t0 = time.perf_counter()
            h.sample(1_000_000, seed=1)
            cl[name] = {"tableau_shots_per_s": 1e6 / (time.perf_counter() - t0), "shots": 1_000_000}
    rep10 = W.repetition_code(10, 10, flip_every=1, ghz=True)
    with sv.Clifford(19, rep10.ops) as h:
        h.sample(1000)
        t0 = time.perf_counter()
        h.sample(100_000, seed=1)
        t_tab = time.perf_counter() - t0
    with sv.Batch("c64") as b:
        p = b.add_program(rep10.ops, 19)
        b.run([p] * 8, np.zeros(8), np.arange(8))
        t0 = time.perf_counter()
        b.run([p] * 1000, np.zeros(1000), np.arange(1000))
        t_sv = time.perf_counter() - t0
        b.sample_branched([p], [0], [1000])
        t0 = time.perf_counter()
        _, bst = b.sample_branched([p], [0], [100_000])
        t_br = time.perf_counter() - t0
    cl["repetition_d10_10_rounds_19q"] = {"tableau_shots_per_s": 1e5 / t_tab,
                                          "sv_batched_per_shot_shots_per_s": 1000 / t_sv,
                                          "sv_batched_branched_shots_per_s": 1e5 / t_br,
                                          "branched_paths": bst["paths"]}
    return cl


def measure_forms(sv, torch):
    """The three serving-style forms against the plain path on the same GPU
    (bounded runs; the circuits are the seeded workloads of the tests)."""
    import numpy as np

    from paper_2604_11599_gb300 import serve, workloads as W

    out = {}
    # batching: 65,536 trajectories of the sequential feed-forward + RUS circuit, n = 12..20 (+1 ancilla)
    wl = W.batching(seed=6, n_traj=65536)
    with sv.Batch("c64") as b:
        pid = {n: b.add_program(c.ops, n + 1) for n, c in wl.circuits.items()}
        ids = np.array([pid[int(n)] for n in wl.traj_n])
        b.set_items(ids, np.arange(len(ids)), np.zeros(len(ids)))
        b.launch(0)
        b.results()
        t0 = time.perf_counter()
        b.launch(0)
        b.results()
        tb = time.perf_counter() - t0
        b.profile(True)  # the same launch once more with the device work counters on
        b.launch(0)
        b.results()
        bw = b.work()
        b.profile(False)
        # the kernel specialised to these programs (compiled once, then launched like the generic one)
        b.set_jit(True)
        b.launch(0)
        b.results()
        t0 = time.perf_counter()
        b.launch(0)
        b.results()
        tj = time.perf_counter() - t0
        bj = b.jit_info()
    sample = wl.traj_n[:256]
    states = {}
    for n in sorted(set(int(v) for v in sample)):
        states[n] = sv.State(n + 1, "c64")
        states[n].run(wl.circuits[n].ops)
    t0 = time.perf_counter()
    for i, n in enumerate(sample):
        states[int(n)].run(wl.circuits[int(n)].ops, seed=0, stream_id=i)
    tp = time.perf_counter() - t0
    for st in states.values():
        st.close()
    out["batching"] = {"workload": "65,536 trajectories, n~U{12..20}+ancilla, 10 layers, sequential feed-forward "
                                   "+ loop(4) RUS, complex64, one persistent launch",
                       "trajectories_per_s": len(ids) / tb, "plain_path_trajectories_per_s": 256 / tp,
                       "plain_path_sample": "first 256 trajectories, one sv_run each", "seconds": tb,
                       "updates_per_s": bw["updates"] / tb,
                       "updates_counted": "executed gates and draws x 2^n (n = 13..21 with the ancilla), counted "
                                          "on the device in a second, identical launch",
                       "state_bytes_per_s": (bw["bytes_read"] + bw["bytes_written"]) / tb,
                       "state_bytes_frac_of_hbm": (bw["bytes_read"] + bw["bytes_written"]) / tb / 1e9
                       / measured_peaks()[0]["hbm_gbs"],
                       "state_bytes_note": "tile reads and writes of the per-CTA state slots (2^13..2^21 "
                                           "amplitudes, largely L2-resident), against the HBM copy peak",
                       "specialised": {"trajectories_per_s": len(ids) / tj, "seconds": tj,
                                       "updates_per_s": bw["updates"] / tj, "kernel": "sv_jit_batch",
                                       "specialised": bj["specialised"], "compile_seconds": bj["compile_seconds"],
                                       "note": "sv_batch_set_jit(1): stage programs compiled for the 9 programs"}}
    # plain small program, 1,000 shots, complex128
    c = W.plain_small()
    with sv.State(5, "c128") as st:
        st.sample(c.ops, 50)
        t0 = time.perf_counter()
        st.sample(c.ops, 1000)
        tps = time.perf_counter() - t0
        lat = []  # per-shot latency of the plain path: one sv_run (creg read back) per shot
        for shot in range(300):
            t1 = time.perf_counter()
            st.run(c.ops, seed=0, shot=shot)
            lat.append(time.perf_counter() - t1)
        lat.sort()
        m_all = []  # near-threshold draws of the 1,000 shots (GPU-side margins, untimed)
        for shot in range(1000):
            st.run(c.ops, seed=0, shot=shot)
            tr = st.trace()
            m_all.extend(np.abs(tr["u"] - tr["p0"] / (tr["p0"] + tr["p1"])).tolist())
        m_all = np.asarray(m_all)
        st.sample_branched(c.ops, 50)
        t0 = time.perf_counter()
        _, pst = st.sample_branched(c.ops, 1000)
        tpb = time.perf_counter() - t0
    with sv.Batch("c128") as b:
        p = b.add_program(c.ops, 5)
        b.run([p] * 1000, np.zeros(1000), np.arange(1000))
        t0 = time.perf_counter()
        b.run([p] * 1000, np.zeros(1000), np.arange(1000))
        tbs = time.perf_counter() - t0
        b.sample_branched([p], [0], [1000])
        t0 = time.perf_counter()
        _, bst = b.sample_branched([p], [0], [1000])
        tbb = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, bst5 = b.sample_branched([p], [0], [100_000])
        tbb5 = time.perf_counter() - t0
    out["plain_small_1000_shots"] = {"plain_path_shots_per_s": 1000 / tps, "batched_shots_per_s": 1000 / tbs,
                                     "plain_shot_latency_p50_ms": 1000 * lat[len(lat) // 2],
                                     "plain_shot_latency_p99_ms": 1000 * lat[int(0.99 * len(lat))],
                                     "branched_plain_path_shots_per_s": 1000 / tpb,
                                     "branched_batched_shots_per_s": 1000 / tbb,
                                     "branched_paths": pst["paths"], "branched_levels": bst["levels"],
                                     "branched_batched_100k_shots_per_s": 100_000 / tbb5,
                                     "branched_100k_paths": bst5["paths"],
                                     "near_threshold_draws": {"draws": int(m_all.size),
                                                              "within_1e-9": int((m_all < 1e-9).sum()),
                                                              "min_margin": float(m_all.min())}}
    # autotuned batched launch: gates per pass timed on 2,048 trajectories of the same mix, then the
    # 65,536-trajectory launch again with the chosen setting (cache in a scratch file)
    try:
        from paper_2604_11599_gb300 import tune

        progs = [(c.ops, n + 1) for n, c in wl.circuits.items()]
        with tempfile.TemporaryDirectory() as td:
            t0 = time.perf_counter()
            best = tune.tune_batch(progs, "c64", cache=tune.Cache(os.path.join(td, "tune.json")), reps=1,
                                   n_items=2048, candidates=tune.batch_candidates(lows=(0,), gates=(0, 8, 16, 32)))
            t_tune = time.perf_counter() - t0
        with sv.Batch("c64") as b:
            b.set_tuning(best.low_bits, best.max_pass_gates)
            pid = {n: b.add_program(c.ops, n + 1) for n, c in wl.circuits.items()}
            ids = np.array([pid[int(n)] for n in wl.traj_n])
            b.set_items(ids, np.arange(len(ids)), np.zeros(len(ids)))
            b.launch(0)
            b.results()
            t0 = time.perf_counter()
            b.launch(0)
            b.results()
            tt = time.perf_counter() - t0
        out["batching"].update({"autotuned_trajectories_per_s": len(ids) / tt, "autotuned_setting": best.label(),
                                "autotune_seconds": t_tune})
    except Exception as e:  # an auxiliary measurement must not cost the bench line
        out["batching"]["autotune_error"] = repr(e)
    # Clifford programs: stabilizer tableaux (one warp per shot) against the state-vector engines
    try:
        out["clifford"] = clifford_form(sv, W, np)
    except Exception as e:
        out["clifford"] = {"error": repr(e)}
    # noise by trajectories: the n=5 program with depolarising, readout and reset channels (ancilla lowering)
    try:
        from paper_2604_11599_gb300 import noise

        nz = noise.with_noise(W.plain_small(), noise.NoiseModel(p1=1e-3, p2=1e-2, p_meas=1e-2, p_reset=1e-2))
        with sv.Batch("c128") as b:
            p = b.add_program(nz.ops, nz.n)
            b.run([p] * 64, np.zeros(64), np.arange(64))
            t0 = time.perf_counter()
            b.run([p] * 1000, np.zeros(1000), np.arange(1000))
            t_ps = time.perf_counter() - t0
            b.sample_branched([p], [0], [1000])
            t0 = time.perf_counter()
            _, nst = b.sample_branched([p], [0], [10_000])
            t_br = time.perf_counter() - t0
        out["noise"] = {"workload": "the n=5 plain-path program with depolarising (1e-3 / 1e-2), readout (1e-2) and "
                                    "reset (1e-2) channels lowered through one ancilla, complex128",
                        "records": int(len(nz.ops)), "batched_per_shot_shots_per_s": 1000 / t_ps,
                        "batched_branched_shots_per_s": 1e4 / t_br, "branched_paths": nst["paths"]}
    except Exception as e:
        out["noise"] = {"error": repr(e)}
    # VQE: n=20 hardware-efficient ansatz, 320 parameters, 200 Pauli terms
    c = W.hea(20, 8)
    terms = W.heisenberg_fields(9, 20, 200)
    vqe = {}
    for dt in ("c64", "c128"):
        sets = 1024
        h = sv.Grad(c.ops, 20, terms, dt)
        gi = h.info()
        prm = torch.tensor(W.hea_params(8, sets, 320), device="cuda")
        h.run(prm[:4])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.run(prm)
        torch.cuda.synchronize()
        dts = time.perf_counter() - t0
        amp = 8 if dt == "c64" else 16
        S = float(1 << gi["state_qubits"]) * amp
        # per set: |0> written, forward passes read + write psi, lambda = H psi gathers psi once per
        # term group and writes lambda, backward passes read + write psi and lambda
        per_set = S * (1 + 2 * gi["forward_passes"] + gi["term_groups"] + 2 + 4 * gi["backward_passes"])
        upd = float(gi["gates"]) * 3 * float(1 << gi["state_qubits"])  # forward, then U^dagger on psi and lambda
        vqe[dt] = {"parameter_sets": sets, "gradient_sets_per_s": sets / dts, "seconds": dts,
                   "updates_per_s": sets * upd / dts,
                   "updates_counted": "(forward gates + backward gates on psi and on lambda) x 2^20 per set",
                   "state_bytes_per_s": sets * per_set / dts,
                   "state_bytes_frac_of_hbm": sets * per_set / dts / 1e9 / measured_peaks()[0]["hbm_gbs"],
                   "work_per_set": gi}
        h.close()
    out["vqe_adjoint"] = vqe
    # the plain path's other sizes and state types (the headline line is n=30 complex64)
    p2 = {}
    for n2, dt2 in ((28, "c64"), (28, "c128"), (30, "c128")):
        p2[f"n{n2}_{dt2}"] = plain_line(sv, torch, n2, dt2)
    out["plain_layered_other_sizes"] = p2
    # terminal sampling and Pauli-sum expectation on an n=28 complex64 state (one read of the
    # state per sampling call; one per group of terms that share an X mask)
    peaks, kind = measured_peaks()
    n_s = 28
    c = W.layered(3, n_s, layers=2)
    terms = W.heisenberg_fields(9, n_s, 10 * n_s)
    xs = [int(x) for x in terms["x_mask"]]
    groups = len(set(xs))
    reads = sum((xs.count(x) + 15) // 16 for x in set(xs))  # one read of the state per launch of <= 16 terms
    sbytes = float(1 << n_s) * 8
    shots = 1 << 20
    with sv.State(n_s, "c64") as st:
        st.set_jit(True)
        st.run(c.ops)
        dev_out = torch.empty(shots, dtype=torch.int64, device="cuda")
        st.sample_state_device(dev_out, seed=1)
        st.sample_state(1 << 16)
        st.expval(terms)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st.sample_state_device(dev_out, seed=2)
        e1.record()
        e1.synchronize()
        ts = e0.elapsed_time(e1) / 1000.0
        t0 = time.perf_counter()
        st.sample_state(shots, seed=2)
        ts_host = time.perf_counter() - t0
        t0 = time.perf_counter()
        st.expval(terms)
        te = time.perf_counter() - t0
    out["sample_expval"] = {
        "state": f"n={n_s} complex64 after 2 layered layers",
        "sampling": {"shots": shots, "seconds": ts, "shots_per_s": shots / ts,
                     "timing": "CUDA events around sv_sample_state_device (CDF build from one read of the state, "
                               "block scan, one search per shot); samples left on the device",
                     "state_reads_gbs": sbytes / ts / 1e9, "hbm_frac": sbytes / ts / 1e9 / peaks["hbm_gbs"],
                     "host_output_seconds": ts_host,
                     "host_output_note": "sv_sample_state, wall clock, samples copied to a host array"},
        "expval": {"terms": int(len(terms)), "x_groups": groups, "state_reads": reads, "seconds": te,
                   "timing": "wall clock of sv_expval (grouping, launches, result copy)",
                   "state_reads_gbs": reads * sbytes / te / 1e9,
                   "hbm_frac": reads * sbytes / te / 1e9 / peaks["hbm_gbs"], "hbm_peak_kind": f"of {kind}"}}
    # dense four-qubit unitaries, n=30 complex64: tensor cores against the FP32 pipes
    from paper_2604_11599_gb300.ir import Kind

    c = W.dense_layers(12, 30, layers=6)
    n_dense = int((c.ops["kind"] == int(Kind.DENSE)).sum())
    dense = {"workload": "n=30 complex64, 6 layers of Haar-random dense 4-qubit unitaries on a random partition "
                         "(7 per layer) + RX/RY/RZ on the 2 qubits left over; 1 trajectory per step",
             "dense_gates_per_step": n_dense}
    with sv.State(30, "c64") as st:
        st.set_jit(True)
        st.set_dense_pool(c.pool)
        prog = st.prepare(c.ops)
        upd = float(prog.stats["gates"]) * float(1 << 30)
        for tc in (True, False):
            st.set_dense_tc(tc)
            for _ in range(2):
                st.launch(prog)
            torch.cuda.synchronize()
            st.profile(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                st.launch(prog)
            e1.record()
            e1.synchronize()
            prof = st.profile_read()
            st.profile(False)
            ms = e0.elapsed_time(e1) / 3
            gbs = prof["bytes"] / (prof["ms"] / 1000.0) / 1e9
            useful = n_dense * float(1 << 30) * 128.0 * 3  # 128 flops / amplitude / dense gate, 3 steps
            dense["tensor_cores" if tc else "fp32_pipes"] = {
                "updates_per_s": upd / (ms / 1000.0), "ms_per_step": ms, "pass_kernels_gbs": gbs,
                "hbm_frac": gbs / peaks["hbm_gbs"], "hbm_peak_kind": f"of {kind}",
                "dense_tflops_useful": useful / (prof["ms"] / 1000.0) / 1e12}
    out["dense4"] = dense
    # serving, the stated request mix (n log-uniform 10-30, depth 10-100, 1-8 measures with
    # cond/loop feed-forward, shots log-uniform 1-4,096, Poisson 200 req/s) on a shortened stream
    out["serving"] = serving_form(sv, torch, W, serve, np)
    return out


def plain_line(sv, torch, n, dtype, steps=3, warmup=2):
    """One configuration of the plain layered workload: device time of whole
    trajectories, updates and bytes counted by the pass kernels."""
    c = circuit(n, dtype)
    peaks, kind = measured_peaks()
    with sv.State(n, dtype) as st:
        st.set_jit(True)
        prog = st.prepare(c.ops)
        st.launch(prog, shot=999)
        for i in range(warmup):
            st.launch(prog, shot=1000 + i)
        torch.cuda.synchronize()
        st.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            st.launch(prog, shot=i)
        e1.record()
        e1.synchronize()
        prof = st.profile_read()
        st.profile(False)
        stats = prog.stats
    ms = e0.elapsed_time(e1) / steps
    gbs = prof["bytes"] / (prof["ms"] / 1000.0) / 1e9
    line = {"workload": workload_name(n, dtype), "ms_per_step": ms,
            "updates_per_s": prof["updates"] / steps / (ms / 1000.0), "passes": stats["passes"],
            "pass_kernels_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"], "hbm_peak_kind": f"of {kind}"}
    if dtype == "c128":
        tf = fp64_ops_per_step(c.ops, stats["passes"], n) / (prof["ms"] / steps / 1000.0) / 1e12
        line.update({"bound": "alu", "fp64_tflops": tf, "fp64_frac_of_nominal": tf / FP64_PEAK_TFLOPS})
    return line


def serving_form(sv, torch, W, serve, np, duration=0.5):
    """The serving configuration's request mix, Poisson 200 req/s, cut to
    `duration` seconds of arrivals (draining a 60 s stream takes far longer
    than a bench run), served to completion by the continuous-batching server.
    The sequential plain path (one request at a time, one trajectory per shot)
    would need shots x (one trajectory) per request -- hours for the n=28..30
    requests -- so it is modelled: one trajectory of every request is timed on
    the plain path, its service time is shots x that time, and a FIFO queue
    over the same arrivals gives its wall time and latencies."""
    stream = W.serving_stream(seed=10, gen_seed=11, rate=200.0, duration=duration, n_lo=10, n_hi=30,
                              d_lo=10, d_hi=100, max_shots=4096)
    reqs = serve.requests_from_stream(stream)
    shots = int(sum(r.shots for r in reqs))
    be = serve.GpuBackend("c64", seed=0)
    srv = serve.Server(be)
    warm = W.serving_stream(seed=12, gen_seed=13, rate=200.0, duration=0.05, n_lo=10, n_hi=20, d_lo=10,
                            d_hi=20, max_shots=64)
    srv.serve(serve.requests_from_stream(warm))
    res, st_srv = srv.serve(reqs)
    srv.close()
    # the sequential plain path, modelled from one timed trajectory of each request
    t1 = {}
    for r in reqs:
        with sv.State(r.n, "c64") as st:
            st.run(r.ops, seed=0, stream_id=r.rid, shot=0)
            t0 = time.perf_counter()
            st.run(r.ops, seed=0, stream_id=r.rid, shot=1)
            t1[r.rid] = time.perf_counter() - t0
    clock, lat = 0.0, []
    for r in sorted(reqs, key=lambda q: (q.arrival, q.rid)):
        clock = max(clock, r.arrival) + r.shots * t1[r.rid]
        lat.append(clock - r.arrival)
    ns = np.array([r.n for r in reqs])
    offered_span = max(r.arrival for r in reqs)
    return {
        "workload": (f"{len(reqs)} requests: Poisson 200 req/s for {duration:g} s (the configuration's 60 s "
                     "shortened so that the stream drains within the bench run), n log-uniform 10-30, depth "
                     "log-uniform 10-100 layers, 1-8 mid-circuit measures each with cond or loop(k<=4) "
                     "feed-forward, shots log-uniform 1-4,096, complex64, admission by HBM footprint"),
        "requests": len(reqs), "shots": shots, "requests_n_ge_28": int((ns >= 28).sum()),
        "offered": {"requests_per_s": len(reqs) / duration, "shots_per_s": shots / duration,
                    "arrival_span_s": offered_span},
        "server": dict(st_srv, drain_after_last_arrival_s=st_srv["wall_s"] - offered_span,
                       achieved_requests_per_s=len(reqs) / st_srv["wall_s"]),
        "sequential_plain_path_model": {
            "shots_per_s": shots / clock, "wall_s": clock,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "how": "one trajectory per request timed on the plain path (sv_run, record read back); service "
                   "time = shots x that time; FIFO over the same arrivals"},
        "server_vs_sequential_shots_per_s": (shots / st_srv["wall_s"]) / (shots / clock),
    }


def single_form(args):
    """One auxiliary measurement on its own (the commands the kernel profiles use)."""
    import numpy as np
    import torch

    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv, workloads as W

    out = {"form": args.form}
    if args.form == "batching":
        wl = W.batching(seed=6, n_traj=args.items)
        with sv.Batch("c64") as b:
            b.set_jit(args.jit)
            pid = {n: b.add_program(c.ops, n + 1) for n, c in wl.circuits.items()}
            ids = np.array([pid[int(n)] for n in wl.traj_n])
            b.set_items(ids, np.arange(len(ids)), np.zeros(len(ids)))
            for _ in range(2):
                t0 = time.perf_counter()
                b.launch(0)
                b.results()
                dt = time.perf_counter() - t0
            ji = b.jit_info()
        out.update({"trajectories": args.items, "seconds": dt, "trajectories_per_s": args.items / dt,
                    "specialised": ji["specialised"], "compile_seconds": ji["compile_seconds"]})
    elif args.form == "adjoint":
        c = W.hea(20, 8)
        terms = W.heisenberg_fields(9, 20, 200)
        h = sv.Grad(c.ops, 20, terms, args.dtype)
        prm = torch.tensor(W.hea_params(8, args.sets, 320), device="cuda")
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.run(prm)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        out.update({"sets": args.sets, "seconds": dt, "gradient_sets_per_s": args.sets / dt, "work_per_set": h.info()})
        h.close()
    else:
        n = 28
        c = W.layered(3, n, layers=2)
        terms = W.heisenberg_fields(9, n, 10 * n)
        with sv.State(n, "c64") as st:
            st.run(c.ops)
            dev = torch.empty(1 << 20, dtype=torch.int64, device="cuda")
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st.sample_state_device(dev, seed=5)
                torch.cuda.synchronize()
                ts = time.perf_counter() - t0
                t0 = time.perf_counter()
                st.expval(terms)
                te = time.perf_counter() - t0
        out.update({"state": "n=28 complex64", "sample_1M_seconds": ts, "expval_280_terms_seconds": te})
    print(json.dumps(out), flush=True)


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores, same metric and config."""
    if rank != 0:
        return
    per_step = max(1.0, min(12.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    desc = threads = None
    for i in range(args.warmup + args.steps):
        ups, desc, threads, dt = oracle_sample(args.n, args.dtype, per_step, kind=args.circuit)
        if i >= args.warmup:
            vals.append((ups, dt))
    ups = statistics.median(v for v, _ in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.median(d for _, d in vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(args.n, args.dtype, args.circuit), "n": args.n},
        "cpu_baseline": {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": ups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    faulthandler.enable()  # a crash in native code prints the Python stack that led to it
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.form:
        return single_form(args)

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import replicas, sv

    n, dtype = args.n, args.dtype
    stream_id = replicas.stream_of(rank)  # ranks simulate independent trajectories
    c = circuit(n, dtype, args.circuit)
    st = sv.State(n, dtype)
    st.set_jit(not args.no_jit)
    st.set_dense_tc(not args.no_dense_tc)
    st.set_tile_select(not args.first_fit)
    if args.stage_pairs is not None:
        st.set_stage_pairs(args.stage_pairs)
    st.set_jit_blocks(args.jit_blocks)
    if args.tile_bits or args.low_bits:
        st.set_tuning(args.tile_bits, args.low_bits, 0)
    if len(c.pool):
        st.set_dense_pool(c.pool)
    prog = st.prepare(c.ops)
    st.launch(prog, seed=0, shot=999)  # first launch compiles the specialised kernels (once per program)
    torch.cuda.synchronize()
    stats = prog.stats
    stream = torch.cuda.current_stream()

    for i in range(args.warmup):
        st.launch(prog, seed=0, stream_id=stream_id, shot=1000 + i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    st.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        st.launch(prog, seed=0, stream_id=stream_id, shot=i)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    prof = st.profile_read()
    st.profile(False)
    clk = clocks.stop()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    # updates of the work that ran: gate records executed (not-taken if/else arms
    # excluded) and draws executed, counted by the pass kernels on the device
    upd = float(prof["gates"] + prof["draws"]) * float(1 << n) / args.steps
    value = replicas.whole_job_rate(upd, ms / 1000.0, world)
    near = near_threshold(st, prog, args.steps, stream_id, dtype) if rank == 0 else None

    # end to end through the public API with host buffers, plan lowered + copied each step
    e2e = None
    if not args.no_e2e:
        st.set_cache(False)
        st.run(c.ops, seed=0, shot=0)  # warm
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            st.run(c.ops, seed=0, stream_id=stream_id, shot=i)  # waits for the classical register
        dt = replicas.max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
        st.set_cache(True)
        e2e = {"value": replicas.whole_job_rate(upd, dt, world), "unit": UNIT,
               "h2d_bytes_per_step": int(stats["plan_bytes"]), "d2h_bytes_per_step": 8,
               "ms_per_step": dt * 1000.0}

    peaks, kind = measured_peaks()
    achieved = prof["bytes"] / (prof["ms"] / 1000.0) / 1e9 if prof["ms"] > 0 else 0.0
    full_pass = float(1 << n) * (8 if dtype == "c64" else 16) * 2  # algorithmic bytes of a loading, storing pass
    per_launch = prof["bytes"] / max(1, prof["launches"])
    traffic = (PASS_DRAM_OVER_COUNTED * per_launch
               if (dtype == "c64" and args.circuit == "layered" and not args.first_fit and not args.low_bits
                   and args.stage_pairs is None
                   and not args.tile_bits) else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "traffic_note": ("DRAM read + write bytes per pass launch: the ncu capture of all pass launches of "
                                 "one n=26 step (DRAM bytes / counted bytes = "
                                 f"{PASS_DRAM_OVER_COUNTED:.4f}) x this step's counted bytes per launch; a pass "
                                 f"that loads and stores every tile counts {full_pass:.4g}") if traffic else None,
                "kernel": "sv_jit_passes (k_pass specialised)" if stats["specialised"] else "k_pass",
                "peak_kind": f"of {kind}", "bytes_per_launch": prof["bytes"] / max(1, prof["launches"]),
                "avg_launch_ms": prof["ms"] / max(1, prof["launches"]),
                "bytes_counted": "state bytes the pass kernels read and wrote, counted on the device "
                                 "(tiles copied in, tiles stored); passes that moved nothing add nothing",
                "bytes_read_per_step": prof["bytes_read"] / args.steps,
                "bytes_written_per_step": prof["bytes_written"] / args.steps,
                "passes_moving_data_per_step": prof["passes"] / args.steps}
    if dtype == "c128":  # FP64-bound: the arithmetic the kernels execute against the FP64 rate
        flops = fp64_ops_per_step(c.ops, stats["passes"], n)
        tf = flops / (prof["ms"] / 1000.0) / 1e12 if prof["ms"] > 0 else 0.0
        roofline = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP64_PEAK_TFLOPS, "traffic": None, "kernel": roofline["kernel"],
                    "peak_kind": "of nominal (GB300 FP64 1.25 TFLOP/s; 0.60 TFMA/s measured by a probe)",
                    "fp64_ops_per_step": flops, "hbm_achieved_gbs": achieved,
                    "hbm_frac_of_measured": achieved / peaks["hbm_gbs"]}

    forms = None
    if rank == 0 and not args.no_forms:
        forms = measure_forms(sv, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ups, desc, threads, dt = oracle_sample(n, dtype, args.cpu_seconds, kind=args.circuit)
        cpu = {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "seconds": dt}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if dtype == "c64" else "f64", "data": "synthetic",
            "config": {"workload": workload_name(n, dtype, args.circuit), "n": n, "state": dtype,
                       "gates_per_step": prof["gates"] / args.steps, "draws_per_step": prof["draws"] / args.steps,
                       "gate_records_in_program": stats["gates"],
                       "passes_per_step": stats["passes"], "tile_bits": stats["tile_bits"],
                       "low_bits": stats["low_bits"], "l2": "inputs larger than L2 (state 2^n amplitudes)",
                       "specialised_kernels": bool(stats["specialised"]),
                       "compile_seconds": round(stats["compile_seconds"], 2),
                       "parallelism": f"replicas x{world}"},
            "near_threshold_draws": near,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * stats["kernels_per_run"], "clocks": clk, "forms": forms,
        }
        print(json.dumps(line), flush=True)
    st.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

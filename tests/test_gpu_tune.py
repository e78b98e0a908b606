"""Autotuner on the GPU: it returns one of the candidates, caches it by
device, size, dtype and program structure, and the chosen setting keeps
parity with the oracle (plain path and batched launch)."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import tune, workloads as W

from paritylib import BAND, compare_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


def test_tune_plain_caches_and_keeps_parity(svmod, orc, tmp_path):
    n = 14
    c = W.layered(2, n, layers=4)
    path = str(tmp_path / "tune.json")
    cands = [tune.Setting(10, 3, 0, False), tune.Setting(12, 4, 0, False), tune.Setting(12, 4, 0, True)]
    best = tune.tune_plain(c.ops, n, "c64", cache=tune.Cache(path), candidates=cands, reps=2)
    assert best in cands
    disk = tune.Cache(path)
    assert len(disk.data) == 1
    (key, entry), = disk.data.items()
    assert f"|n{n}|c64|" in key and set(entry["ms"]) == {s.label() for s in cands}
    # a program of the same structure with other angles hits the cache (no candidates to time)
    ops2 = c.ops.copy()
    ops2["angle"] += 0.25
    assert tune.tune_plain(ops2, n, "c64", cache=disk, candidates=[]) == best
    with svmod.State(n, "c64") as st:
        tune.apply(st, best)
        compare_run(st, orc, c.ops, n, "c64", seed=1)


def test_tune_batch_keeps_parity(svmod, orc, tmp_path):
    circ = W.sequential_feedforward(5, 6, layers=2)
    progs = [(circ.ops, 7)]
    cands = [tune.Setting(12, 0, 0), tune.Setting(12, 0, 8)]
    best = tune.tune_batch(progs, "c128", cache=tune.Cache(str(tmp_path / "b.json")), candidates=cands, reps=1,
                           n_items=256)
    assert best in cands
    with svmod.Batch("c128") as b:
        b.set_tuning(best.low_bits, best.max_pass_gates)
        p = b.add_program(circ.ops, 7)
        got = b.run(np.full(64, p), np.zeros(64), np.arange(64), seed=0)
    want, _, margins = orc.run_shots(circ.ops, 7, 64, seed=0)
    ok = margins > BAND["c128"]
    assert np.array_equal(got[ok], want[ok])

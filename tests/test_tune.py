"""Autotuner logic without a GPU: the search picks the fastest measurable
candidate, candidate settings are ones the planner accepts, the cache round
trips, and the program key ignores literal angles only."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import tune, workloads as W
from paper_2604_11599_gb300.ir import Circuit


def test_autotune_picks_fastest_and_skips_failures():
    cands = [tune.Setting(10, 3, 0, False), tune.Setting(12, 4, 0, True), tune.Setting(14, 6, 16, False)]
    cost = {cands[0]: 5.0, cands[1]: 2.0, cands[2]: 1.0}
    calls = []

    def measure(s):
        calls.append(s)
        if s == cands[2]:
            raise KeyError("this one cannot run")
        return cost[s]

    best, table = tune.autotune(measure, cands, reps=3, errors=(KeyError,))
    assert best == cands[1] and set(table) == {cands[0], cands[1]}
    assert calls.count(cands[0]) == 3
    with pytest.raises(RuntimeError):
        tune.autotune(lambda s: (_ for _ in ()).throw(KeyError()), cands, errors=(KeyError,))


def test_autotune_uses_the_median():
    a, b = tune.Setting(10, 3), tune.Setting(12, 4)
    seq = {a: iter([1.0, 9.0, 9.0]), b: iter([5.0, 5.0, 5.0])}
    best, table = tune.autotune(lambda s: next(seq[s]), [a, b], reps=3)
    assert best == b and table[a] == 9.0


@pytest.mark.parametrize("n,dtype", [(8, "c64"), (16, "c128"), (24, "c64")])
def test_plain_candidates_plan_on_the_host(n, dtype):
    c = W.layered(1, n, layers=3)
    cands = tune.plain_candidates(n, dtype, c.ops)
    assert cands and all(s.tile_bits <= max(n, 10) and s.tile_bits - s.low_bits <= 9 for s in cands)
    from paper_2604_11599_gb300 import sv

    for s in cands:  # each one plans (the check inside plain_candidates kept only these)
        st = sv.plan_info(c.ops, n, dtype, None, s.tile_bits, s.low_bits, s.max_pass_gates)
        assert st["tile_bits"] == s.tile_bits and st["low_bits"] == s.low_bits
    assert any(s.jit for s in cands) and any(not s.jit for s in cands)


def test_batch_candidates_ranges():
    for s in tune.batch_candidates():
        assert s.tile_bits == 12 and (s.low_bits == 0 or 3 <= s.low_bits <= 12)
        assert 0 <= s.max_pass_gates <= 128


def test_structure_hash_ignores_literal_angles_only():
    def prog(theta, q=0, param=False):
        c = Circuit(3)
        c.h(0)
        if param:
            from paper_2604_11599_gb300.ir import Param

            c.rx(q, Param(0, theta))
        else:
            c.rx(q, theta)
        c.measure(q, 0)
        return c.ops

    assert tune.structure_hash(prog(0.1)) == tune.structure_hash(prog(2.3))
    assert tune.structure_hash(prog(0.1)) != tune.structure_hash(prog(0.1, q=1))
    # a parameter reference is structure (its scale is kept)
    assert tune.structure_hash(prog(1.0, param=True)) != tune.structure_hash(prog(2.0, param=True))
    assert tune.structure_hash(prog(0.1)) != tune.structure_hash(prog(0.1, param=True))


def test_cache_round_trip(tmp_path, monkeypatch):
    p = tmp_path / "t.json"
    c = tune.Cache(str(p))
    s = tune.Setting(13, 5, 16, True)
    c.put("plain|dev|n20|c64|abc", s, {s: 1.5})
    c.save()
    d = tune.Cache(str(p))
    assert d.get("plain|dev|n20|c64|abc") == s and d.get("missing") is None
    assert d.data["plain|dev|n20|c64|abc"]["ms"] == {s.label(): 1.5}
    monkeypatch.setenv("SV_TUNE_CACHE", str(tmp_path / "env.json"))
    assert tune.Cache().path == str(tmp_path / "env.json")
    (tmp_path / "bad.json").write_text("{not json")
    assert tune.Cache(str(tmp_path / "bad.json")).data == {}

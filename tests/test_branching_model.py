"""Shot branching, stated as a CPU model over the oracle: one representative
trajectory per outcome path (its recorded masses p0, p1 and outcomes), every
shot walked down the tree with its own Philox numbers and the rule
u >= p0/(p0+p1), new paths started by the smallest shot that leaves the tree
at a draw.  Because equal outcome prefixes mean equal states, the records
must equal the oracle's per-shot records exactly, with one trajectory per
distinct outcome sequence."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W


def branched_records(orc, ops, n, shots, seed=0, stream=0):
    paths = []  # [draws (p0, p1, outcome, child), creg]

    def add(shot):
        tr = orc.run(ops, n, seed=seed, stream=stream, shot=shot)
        assert tr.status == 0
        paths.append([[[float(d["p0"]), float(d["p1"]), int(d["outcome"]), -1] for d in tr.draws], tr.creg])
        return len(paths) - 1

    add(0)
    where = [(0, 0)] * shots  # (path, next draw); None once at the end of a path
    runs = 1
    while True:
        claims = {}
        for s in range(shots):
            if where[s] is None:
                continue
            j, i = where[s]
            while True:
                draws, _ = paths[j]
                if i == len(draws):
                    where[s] = None
                    break
                p0, p1, o, child = draws[i]
                u = orc.uniform(seed, stream, s, i)
                mine = (1 if u >= p0 / (p0 + p1) else 0) if p0 + p1 > 0 else 0
                if mine == o:
                    i += 1
                elif child >= 0:
                    j, i = child, i + 1
                else:
                    claims.setdefault((j, i), s)
                    where[s] = (j, i)
                    break
        if not claims:
            break
        for (j, i), s in sorted(claims.items()):
            k = add(s)
            runs += 1
            # the new path replays its parent's masses up to the draw it leaves at
            assert len(paths[k][0]) > i and all(
                a[:2] == b[:2] for a, b in zip(paths[j][0][: i + 1], paths[k][0][: i + 1]))
            paths[j][0][i][3] = k
    # final assignment: walk again (every shot now ends at a path's end)
    regs = np.zeros(shots, dtype=np.uint64)
    for s in range(shots):
        j, i = 0, 0
        while True:
            draws, creg = paths[j]
            if i == len(draws):
                regs[s] = creg
                break
            p0, p1, o, child = draws[i]
            u = orc.uniform(seed, stream, s, i)
            mine = (1 if u >= p0 / (p0 + p1) else 0) if p0 + p1 > 0 else 0
            if mine == o:
                i += 1
            else:
                assert child >= 0
                j, i = child, i + 1
    return regs, runs


@pytest.mark.parametrize("make,n", [(lambda: W.plain_small(), 5), (lambda: W.sequential_feedforward(3, 4, layers=2), 5),
                                    (lambda: W.random_dynamic(9, 6, n_ops=50), 6)])
def test_branching_reproduces_per_shot_records(orc, make, n):
    c = make()
    shots = 300
    got, runs = branched_records(orc, c.ops, n, shots, seed=2)
    want, _, _ = orc.run_shots(c.ops, n, shots, seed=2)
    assert np.array_equal(got, want)
    # one trajectory per distinct outcome sequence among the shots
    seqs = {tuple(orc.run(c.ops, n, seed=2, shot=s).draws["outcome"].tolist()) for s in range(shots)}
    assert runs == len(seqs)

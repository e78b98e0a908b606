"""Adjoint gradients of <H> (batched over parameter sets) against the oracle:
energies, parameter-shift gradients, finite-difference gradients, autograd."""
import math

import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import Circuit, Gate, Param

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-10}


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


def stencil_grad(orc, ops, n, p, terms, pool=None, h=1e-3):
    """4-point central stencil on the oracle's FP64 energy (error O(h^4))."""
    g = np.zeros_like(p)
    for k in range(p.size):
        f = []
        for d in (2, 1, -1, -2):
            q = p.copy()
            q[k] += d * h
            f.append(orc.energy(ops, n, q, terms, pool))
        g[k] = (-f[0] + 8 * f[1] - 8 * f[2] + f[3]) / (12 * h)
    return g


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_hea_energy_and_param_shift(svmod, orc, dtype):
    n, layers = 5, 2
    c = W.hea(n=n, layers=layers)
    terms = W.heisenberg_fields(seed=9, n=n, n_terms=25)
    scale = float(np.abs(terms["coeff"]).sum())
    params = np.random.default_rng(1).uniform(-math.pi, math.pi, size=(6, c.n_params))
    val, grad = svmod.expval_grad_batch(c.ops, n, params, terms, dtype)
    for s in range(len(params)):
        e = orc.energy(c.ops, n, params[s], terms)
        assert abs(val[s] - e) <= TOL[dtype] * scale
        g = orc.param_shift_grad(c.ops, n, params[s], terms)
        assert np.max(np.abs(grad[s] - g)) <= TOL[dtype] * scale


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_general_gates_shared_and_scaled_params(svmod, orc, dtype):
    """Every parametrised gate kind (RX RY RZ P U CRX CRY CRZ CP CU), parameters
    shared across gates and scaled, fixed gates and dense 2/3-qubit unitaries."""
    n = 5
    r = np.random.default_rng(4)
    c = Circuit(n)
    for q in range(n):
        c.h(q)
    kinds = [Gate.RX, Gate.RY, Gate.RZ, Gate.P, Gate.U, Gate.CRX, Gate.CRY, Gate.CRZ, Gate.CP, Gate.CU]
    for rep in range(3):
        for g in kinds:
            nq = 2 if g.name.startswith("C") else 1
            qs = [int(v) for v in r.choice(n, size=nq, replace=False)]
            na = 3 if g in (Gate.U, Gate.CU) else 1
            angs = [Param(int(r.integers(6)), float(r.choice([1.0, -0.5, 2.0]))) for _ in range(na)]
            c.gate(g, qs, angs)
            c.gate(Gate.CX, [int(v) for v in r.choice(n, size=2, replace=False)])
        for k in (2, 3):
            qs = [int(v) for v in r.choice(n, size=k, replace=False)]
            a = r.normal(size=(1 << k, 1 << k)) + 1j * r.normal(size=(1 << k, 1 << k))
            u, _ = np.linalg.qr(a)
            c.dense(qs, u)
    terms = W.heisenberg_fields(seed=2, n=n, n_terms=20)
    scale = float(np.abs(terms["coeff"]).sum())
    params = r.uniform(-2, 2, size=(3, 6))
    h = svmod.Grad(c.ops, n, terms, dtype, pool=c.pool)
    import torch

    val, grad = h.run(torch.tensor(params, device="cuda"))
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    assert h.info()["specialised"] == 1  # the kernel specialised to this program ran
    # the generic kernel (gate records read at run time) on the same sets
    h.set_jit(False)
    val_g, grad_g = h.run(torch.tensor(params, device="cuda"))
    assert h.info()["specialised"] == 0
    val_g, grad_g = val_g.cpu().numpy(), grad_g.cpu().numpy()
    for s in range(len(params)):
        e = orc.energy(c.ops, n, params[s], terms, c.pool)
        g = stencil_grad(orc, c.ops, n, params[s], terms, c.pool)
        tol = max(TOL[dtype], 1e-9) * scale
        for v, gr in ((val, grad), (val_g, grad_g)):
            assert abs(v[s] - e) <= TOL[dtype] * scale
            assert np.max(np.abs(gr[s] - g)) <= tol, np.max(np.abs(gr[s] - g))


def test_autograd_backward(svmod):
    import torch

    from paper_2604_11599_gb300.autograd import energy

    n = 4
    c = W.hea(n=n, layers=2)
    terms = W.heisenberg_fields(seed=1, n=n, n_terms=12)
    h = svmod.Grad(c.ops, n, terms, "c128")
    p = torch.tensor(np.random.default_rng(0).uniform(-1, 1, size=(4, c.n_params)), device="cuda",
                     requires_grad=True)
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], device="cuda", dtype=torch.float64)
    (energy(p, h) * w).sum().backward()
    _, g = h.run(p.detach())
    assert torch.allclose(p.grad, w[:, None] * g, atol=1e-14, rtol=0)
    # a few optimisation steps lower the energy
    q = p.detach()[0].clone().requires_grad_(True)
    opt = torch.optim.SGD([q], lr=0.05)
    e0 = float(energy(q, h).detach())
    for _ in range(20):
        opt.zero_grad()
        energy(q, h).backward()
        opt.step()
    assert float(energy(q, h).detach()) < e0


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_vqe_config_full_size_spot_check(svmod, orc, dtype):
    """n=20 hardware-efficient ansatz, 8 layers, 320 parameters, 200 Pauli terms:
    energy against the oracle and three gradient entries against parameter shift."""
    n = 20
    c = W.hea(n=n, layers=8)
    terms = W.heisenberg_fields(seed=9, n=n, n_terms=200)
    scale = float(np.abs(terms["coeff"]).sum())
    params = W.hea_params(seed=8, sets=4, n_params=320)
    val, grad = svmod.expval_grad_batch(c.ops, n, params, terms, dtype)
    s = 1
    assert abs(val[s] - orc.energy(c.ops, n, params[s], terms)) <= TOL[dtype] * scale
    for k in (0, 157, 319):
        pp, pm = params[s].copy(), params[s].copy()
        pp[k] += math.pi / 2
        pm[k] -= math.pi / 2
        g = 0.5 * (orc.energy(c.ops, n, pp, terms) - orc.energy(c.ops, n, pm, terms))
        assert abs(grad[s, k] - g) <= TOL[dtype] * scale


def test_adjoint_rejects_dynamic_programs(svmod):
    c = Circuit(3)
    c.rx(0, Param(0))
    c.measure(0, 0)
    terms = W.heisenberg_fields(seed=1, n=3, n_terms=4)
    with pytest.raises(svmod.SVError, match="UNSUPPORTED"):
        svmod.expval_grad_batch(c.ops, 3, np.zeros((1, 1)), terms, "c64")

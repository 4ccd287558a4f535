"""Batched instances: gradients and the on-device Adam loop against the
oracle (adjoint gradients driving a float64 host Adam)."""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2104_03293_gb300 import build, qs as _qs
    build.build()
    return _qs


def _batch(qs, insts):
    bt = qs.Batch([inst.n for inst in insts])
    for i, inst in enumerate(insts):
        bt.set_ising(i, inst.h, inst.edges, inst.J)
    return bt


@pytest.mark.parametrize("objective", [0, 1])
def test_batched_grad_matches_oracle(qs, objective):
    items = I.config2(count=8, n_lo=11, n_hi=17, p_lo=1, p_hi=4)
    insts = [inst for inst, _, _ in items]
    bt = _batch(qs, insts)
    bt.evolve([g for _, g, _ in items], [b for _, _, b in items])
    v, dg, db = bt.grad(objective)
    bt.close()
    for i, (inst, g, b) in enumerate(items):
        vr, dgr, dbr = oracle.adjoint(inst, g, b, objective)
        scale = max(1.0, np.max(np.abs(np.concatenate([dgr, dbr]))))
        assert abs(v[i] - vr) <= 1e-5 * max(1.0, abs(vr)), (i, v[i], vr)
        assert np.max(np.abs(dg[i] - dgr)) <= 1e-4 * scale, (i, dg[i], dgr)
        assert np.max(np.abs(db[i] - dbr)) <= 1e-4 * scale, (i, db[i], dbr)


def _aqa_init(items):
    gs, bs = [], []
    for inst, p, tau in items:
        g, b = oracle.aqa_angles(tau, np.arange(1, p + 1) / (p + 1))
        gs.append(g)
        bs.append(b)
    return gs, bs


def test_batched_adam_graph_matches_host_adam(qs):
    """Five Adam steps (lr 0.01, bias-corrected) from the AQA initialisation:
    graph replay and plain launches agree bit for bit; both follow a float64
    host Adam driven by oracle gradients; E and P_ground reported at the
    final angles equal the oracle's at those angles."""
    items = I.config4(count=5, n_lo=12, n_hi=15, p_lo=3, p_hi=6)
    insts = [inst for inst, _, _ in items]
    g0, b0 = _aqa_init(items)
    steps = 5
    out = {}
    for graph in (True, False):
        bt = _batch(qs, insts)
        bt.evolve(g0, b0)
        gf, bf = bt.adam(g0, b0, steps, use_graph=graph)
        E, P = bt.results()
        bt.close()
        out[graph] = (gf, bf, E, P)
    gf, bf, E, P = out[True]
    for a, c in zip(gf + bf, out[False][0] + out[False][1]):
        assert np.array_equal(a, c)
    assert np.array_equal(E, out[False][2]) and np.array_equal(P, out[False][3])
    for i, inst in enumerate(insts):
        p = len(g0[i])
        theta = np.concatenate([g0[i], b0[i]])
        m, v = np.zeros(2 * p), np.zeros(2 * p)
        small = np.zeros(2 * p, dtype=bool)
        for t in range(1, steps + 1):
            _, dg, db = oracle.adjoint(inst, theta[:p], theta[p:], 0)
            grad = np.concatenate([dg, db])
            small |= np.abs(grad) < 1e-3 * max(1.0, np.max(np.abs(grad)))
            theta, m, v = oracle.adam_step(theta, grad, m, v, t)
        got = np.concatenate([gf[i], bf[i]])
        # components whose gradient came near zero may take either sign of
        # the normalised Adam step; bound them by the step size instead
        tol = np.where(small, 2 * steps * 0.01, 1e-4 * np.maximum(1.0, np.abs(theta)))
        assert np.all(np.abs(got - theta) <= tol), (i, got, theta)
        Er, Pr = oracle.expect(inst, gf[i], bf[i])
        bound = float(np.abs(inst.h).sum() + np.abs(inst.J).sum())
        assert abs(E[i] - Er) <= 1e-5 * max(abs(Er), bound, 1.0) and abs(P[i] - Pr) <= 1e-5


def test_autograd_functions_match_the_adjoint(qs):
    """energy() (free angles) and aqa_energy() (tau and the schedule knots)
    through torch.autograd against the oracle adjoint and chain rule."""
    import torch
    inst = I.erdos_renyi_ising(14, seed=21, h_values=(-1, 0, 1), j_values=(-1, 0, 1))
    st = qs.State(inst.n)
    st.set_instance(inst)
    g0, b0 = I.uniform_angles(4, 22)
    gamma = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
    beta = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
    F = qs.energy(gamma, beta, st, qs.QS_OBJ_ENERGY)
    F.backward()
    vr, dgr, dbr = oracle.adjoint(inst, g0, b0, 0)
    scale = max(1.0, np.max(np.abs(np.concatenate([dgr, dbr]))))
    assert abs(F.item() - vr) <= 1e-5 * max(1.0, abs(vr))
    assert np.max(np.abs(gamma.grad.numpy() - dgr)) <= 1e-4 * scale
    assert np.max(np.abs(beta.grad.numpy() - dbr)) <= 1e-4 * scale
    sk = np.arange(1, 6) / 6.0
    tau = torch.tensor(0.75, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(sk, dtype=torch.float64, requires_grad=True)
    P = qs.aqa_energy(tau, s, st, qs.QS_OBJ_GROUND)
    P.backward()
    g, b = oracle.aqa_angles(0.75, sk)
    vr, dgr, dbr = oracle.adjoint(inst, g, b, 1)
    dt_r, ds_r = oracle.aqa_chain(0.75, sk, dgr, dbr)
    assert abs(P.item() - vr) <= 1e-5
    assert abs(tau.grad.item() - dt_r) <= 1e-4 * max(1.0, abs(dt_r))
    assert np.max(np.abs(s.grad.numpy() - ds_r)) <= 1e-4 * max(1.0, np.max(np.abs(ds_r)))
    st.close()

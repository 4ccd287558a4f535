"""Batched instances: gradients and the on-device Adam loop against the
oracle (adjoint gradients driving a float64 host Adam)."""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import instances as I
from tolerances import assert_grad, assert_readout, p_tol, value_tol

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
        assert abs(v[i] - vr) <= value_tol(objective, inst, vr), (i, v[i], vr)
        assert_grad(np.concatenate([dg[i], db[i]]), np.concatenate([dgr, dbr]), what=i)


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
        assert_readout(inst, E[i], P[i], Er, Pr, i)


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
    assert abs(F.item() - vr) <= value_tol(0, inst, vr)
    assert_grad(np.concatenate([gamma.grad.numpy(), beta.grad.numpy()]), np.concatenate([dgr, dbr]))
    sk = np.arange(1, 6) / 6.0
    tau = torch.tensor(0.75, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(sk, dtype=torch.float64, requires_grad=True)
    P = qs.aqa_energy(tau, s, st, qs.QS_OBJ_GROUND)
    P.backward()
    g, b = oracle.aqa_angles(0.75, sk)
    vr, dgr, dbr = oracle.adjoint(inst, g, b, 1)
    dt_r, ds_r = oracle.aqa_chain(0.75, sk, dgr, dbr)
    assert abs(P.item() - vr) <= p_tol(vr) and vr > 0.05
    assert_grad(np.concatenate([[tau.grad.item()], s.grad.numpy()]), np.concatenate([[dt_r], ds_r]))
    # the paper's second-order map (Appendix A) with its chain rule
    sk2 = np.arange(5) / 4.0
    tau2 = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    s2 = torch.tensor(sk2, dtype=torch.float64, requires_grad=True)
    P2 = qs.aqa_energy(tau2, s2, st, qs.QS_OBJ_GROUND, order=2)
    P2.backward()
    g2, b2 = oracle.aqa_angles_second_order(0.8, sk2)
    vr2, dgr2, dbr2 = oracle.adjoint(inst, g2, b2, 1)
    dt2, ds2 = oracle.aqa_chain_second_order(0.8, sk2, dgr2, dbr2)
    assert abs(P2.item() - vr2) <= p_tol(vr2)
    assert_grad(np.concatenate([[tau2.grad.item()], s2.grad.numpy()]), np.concatenate([[dt2], ds2]))
    st.close()


def _sample(items, k, seed):
    """k indices spanning the qubit range: the smallest and largest n, the
    deepest p, then a seeded draw of the rest."""
    ns = np.array([it[0].n for it in items])
    ps = np.array([len(it[1]) if hasattr(it[1], "__len__") else it[1] for it in items])
    pick = [int(np.argmin(ns)), int(np.argmax(ns)), int(np.argmax(ps))]
    rng = np.random.default_rng(seed)
    rest = [i for i in rng.permutation(len(items)) if i not in pick]
    return sorted(set(pick + [int(i) for i in rest[:k - len(set(pick))]]))


@pytest.mark.slow
def test_config2_full_batch_against_oracle(qs):
    """All 512 instances of the batched workload (n ~ U{16..24}, p ~
    U{1..10}) in one batch; E and P of 16 instances spanning n = 16..24
    against the oracle, every instance against its own one-at-a-time run."""
    items = I.config2()
    insts = [it[0] for it in items]
    bt = _batch(qs, insts)
    bt.evolve([it[1] for it in items], [it[2] for it in items])
    E, P = bt.results()
    bt.close()
    idx = _sample(items, 16, 2)
    assert min(insts[i].n for i in idx) == 16 and max(insts[i].n for i in idx) == 24
    for i in idx:
        inst, g, b = items[i]
        Er, Pr = oracle.expect(inst, g, b)
        assert_readout(inst, E[i], P[i], Er, Pr, i)
    # one at a time (single states use the packed-pair sweeps from 24 qubits,
    # the batch the scalar ones: equal up to float32 rounding order)
    for i in range(0, 512, 37):
        inst, g, b = items[i]
        with qs.State(inst.n) as st:
            st.set_instance(inst)
            st.evolve(g, b)
            Es, Ps, _ = st.readout()
        assert_readout(inst, E[i], P[i], Es, Ps, i)


@pytest.mark.slow
def test_config4_full_batch_adam_against_oracle(qs):
    """All 64 instances of the optimiser workload (n ~ U{18..22}, p ~
    U{5..20}, AQA initialisation): the batched gradient at the initial angles
    against the oracle adjoint, then 200 Adam steps replayed from a CUDA
    graph, and E, P reported at the final angles against the oracle's
    readout at those angles, on 16 instances spanning n and p."""
    items = I.config4()
    insts = [it[0] for it in items]
    g0, b0 = _aqa_init(items)
    bt = _batch(qs, insts)
    bt.evolve(g0, b0)
    v, dg, db = bt.grad(0)
    idx = _sample([(it[0], it[1]) for it in items], 16, 4)
    assert max(items[i][1] for i in idx) == max(it[1] for it in items)
    for i in idx[:6]:
        vr, dgr, dbr = oracle.adjoint(insts[i], g0[i], b0[i], 0)
        assert abs(v[i] - vr) <= value_tol(0, insts[i], vr), (i, v[i], vr)
        assert_grad(np.concatenate([dg[i], db[i]]), np.concatenate([dgr, dbr]), what=i)
    gf, bf = bt.adam(g0, b0, 200, use_graph=True)
    E, P = bt.results()
    bt.close()
    E0 = np.array([oracle.expect(insts[i], g0[i], b0[i])[0] for i in idx])
    for j, i in enumerate(idx):
        Er, Pr = oracle.expect(insts[i], gf[i], bf[i])
        assert_readout(insts[i], E[i], P[i], Er, Pr, i)
    # 200 steps of minimisation lower the energy of every sampled instance
    assert np.all(E[idx] < E0), (E[idx], E0)


def test_queue_withheld_dependency_times_out(qs):
    """Failure detection without a GPU fault: a work queue whose instance 1
    waits for one tile that no sweep provides gives up after its 50 ms limit;
    the error reaches the host as QS_ETIMEOUT, no copy is left in flight, and
    the next evolve of the same batch is correct again."""
    insts = [I.erdos_renyi_ising(n, I.workload_seed(2, 900 + n)) for n in (16, 18, 20)]
    gs, bs = zip(*[I.uniform_angles(3, I.workload_seed(2, 950 + k)) for k in range(3)])
    bt = _batch(qs, insts)
    try:
        bt.test_withhold(1, 0.05)
        bt.evolve(list(gs), list(bs))
        with pytest.raises(qs.QSError) as exc:
            bt.results()
        assert exc.value.code == qs.QS_ETIMEOUT
        bt.evolve(list(gs), list(bs))
        E, P = bt.results()
    finally:
        bt.close()
    for i, inst in enumerate(insts):
        Er, Pr, _ = oracle.readout(inst, oracle.evolve(inst, gs[i], bs[i]))
        assert_readout(inst, E[i], P[i], Er, Pr, i)


def test_batch_launch_rules_and_autotune(qs):
    """Every work-queue launch rule (CTAs per SM, instance windows that
    order the queue window by window) gives the oracle's readouts and
    gradients; the batch autotuner keeps one of them."""
    items = I.config2(count=10, n_lo=13, n_hi=19, p_lo=1, p_hi=5)
    insts = [inst for inst, _, _ in items]
    gs, bs = [g for _, g, _ in items], [b for _, _, b in items]
    bt = _batch(qs, insts)
    ref = [oracle.readout(x, oracle.evolve(x, g, b))[:2] for x, g, b in items]
    adj = [oracle.adjoint(x, g, b, 0) for x, g, b in items]
    try:
        for rule in [(0, 0), (1, 0), (0, 1 << 20), (1, 4 << 20), (0, 1)]:
            bt.set_launch_rule(*rule)
            bt.evolve(gs, bs)
            E, P = bt.results()
            for i, inst in enumerate(insts):
                assert_readout(inst, E[i], P[i], ref[i][0], ref[i][1], (rule, i))
            v, dg, db = bt.grad(0)
            for i, inst in enumerate(insts):
                assert_grad(np.concatenate([dg[i], db[i]]), np.concatenate([adj[i][1], adj[i][2]]), what=(rule, i))
        bt.evolve(gs, bs)
        c, w, ms = bt.autotune()
        assert c in (0, 1) and w in (0, 256 << 20, 64 << 20) and ms > 0
        bt.evolve(gs, bs)
        E, P = bt.results()
        for i, inst in enumerate(insts):
            assert_readout(inst, E[i], P[i], ref[i][0], ref[i][1], ("tuned", i))
    finally:
        bt.close()

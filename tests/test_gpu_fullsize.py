"""CUDA path at the full sizes of the benchmark, checked through properties
the oracle can compute exactly.

A cost whose couplings split into components on disjoint qubit sets gives a
product state (phase and mixer both factorise), so an n = 34 state built
from two 17-qubit components must equal psi_A (x) psi_B, with
E = E_A + E_B and P_ground = P_A P_B.  These runs use the same tile shapes,
sweep plan and launch configuration as the n = 34 forward and the n = 33
adjoint of the benchmark (shapes depend only on n).  Sampled amplitudes are
compared one by one; the sampled squared error, scaled to the full state,
estimates the state-norm error.
"""
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


def _component(n, k):
    return I.erdos_renyi_ising(n, I.workload_seed(5, 100 + k), h_values=(-1, 0, 1), j_values=(-1, 0, 1))


def _angles(p, tau=0.75):
    s = np.arange(1, p + 1) / (p + 1)
    return oracle.aqa_angles(tau, s)


def _sampled_norm_error(buf, psiA, psiB, nA, n, count=1 << 16, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, size=count), [0, (1 << n) - 1]]))
    got = buf[torch.from_numpy(idx).to(buf.device)].cpu().numpy().astype(np.complex128)
    want = psiA[idx & ((1 << nA) - 1)] * psiB[idx >> nA]
    return np.sqrt(np.sum(np.abs(got - want) ** 2) * (2.0 ** n) / idx.size)


@pytest.mark.parametrize("n,nA,dtype", [(34, 17, "c64"), (30, 15, "c128")])
def test_factorised_state_at_full_size(qs, n, nA, dtype):
    import torch
    A, B = _component(nA, 0), _component(n - nA, 1)
    U = I.union([A, B])
    g, b = _angles(4)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    buf = torch.empty(1 << n, dtype=tdt, device="cuda")
    st = qs.State(n, dtype, buffer=buf)
    try:
        st.set_instance(U)
        cmin, cmax, arg, cnt, _ = st.cost_info()
        gA, gB = oracle.ground(A), oracle.ground(B)
        assert (cmin, cmax) == (gA[0] + gB[0], gA[1] + gB[1])
        assert (arg, cnt) == (gA[2] + (gB[2] << nA), gA[3] * gB[3])
        st.evolve(g, b)
        E, P, N = st.readout()
        psiA, psiB = oracle.evolve(A, g, b), oracle.evolve(B, g, b)
        EA, PA, _ = oracle.readout(A, psiA)
        EB, PB, _ = oracle.readout(B, psiB)
        bound = float(np.abs(U.h).sum() + np.abs(U.J).sum())
        assert abs(E - (EA + EB)) <= 1e-5 * max(abs(EA + EB), bound, 1.0), (E, EA + EB)
        assert abs(P - PA * PB) <= 1e-5, (P, PA * PB)
        assert abs(N - 1.0) <= 1e-5
        st.canonicalize()
        err = _sampled_norm_error(buf, psiA, psiB, nA, n)
        assert err <= (1e-4 if dtype == "c64" else 1e-10), err
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()


@pytest.mark.parametrize("objective", [1, 0])
def test_factorised_adjoint_n33(qs, objective):
    """Gradient at n = 33 with psi and lambda in the two halves of one
    buffer (the benchmark's layout): the derivative of E_A + E_B, or of
    P_A P_B, by the product rule from the two components' oracle adjoints."""
    import torch
    n, nA = 33, 16
    A, B = _component(nA, 2), _component(n - nA, 3)
    U = I.union([A, B])
    g, b = _angles(3)
    buf = torch.empty(1 << (n + 1), dtype=torch.complex64, device="cuda")
    halves = buf.view(2, -1)
    st = qs.State(n, "c64", buffer=halves[0])
    try:
        st.set_adjoint_buffer(halves[1])
        st.set_instance(U)
        v, dg, db = st.grad(g, b, objective)
        FA, dgA, dbA = oracle.adjoint(A, g, b, objective)
        FB, dgB, dbB = oracle.adjoint(B, g, b, objective)
        if objective == 0:
            vr, dgr, dbr = FA + FB, dgA + dgB, dbA + dbB
        else:
            vr, dgr, dbr = FA * FB, dgA * FB + FA * dgB, dbA * FB + FA * dbB
        scale = max(1.0, np.max(np.abs(np.concatenate([dgr, dbr]))))
        assert abs(v - vr) <= 1e-5 * max(1.0, abs(vr)), (v, vr)
        assert np.max(np.abs(dg - dgr)) <= 1e-4 * scale, (dg, dgr)
        assert np.max(np.abs(db - dbr)) <= 1e-4 * scale, (db, dbr)
    finally:
        st.close()
        del halves, buf
        torch.cuda.empty_cache()


def test_config3_gradient_against_finite_differences(qs):
    """n = 26, p = 10 MaxCut: complex64 adjoint against central differences
    of <H_C> taken on the complex128 path (step 1e-4)."""
    inst, g, b = I.config3()
    st = qs.State(inst.n, "c64")
    st.set_instance(inst)
    v, dg, db = st.grad(g, b, 0)
    st.close()
    ref = qs.State(inst.n, "c128")
    ref.set_instance(inst)

    def E(gg, bb):
        ref.evolve(gg, bb)
        return ref.expect()

    h = 1e-4
    fd = []
    for k in range(2 * len(g)):
        d = np.zeros(2 * len(g))
        d[k] = h
        fd.append((E(g + d[:len(g)], b + d[len(g):]) - E(g - d[:len(g)], b - d[len(g):])) / (2 * h))
    ref.close()
    fd = np.array(fd)
    got = np.concatenate([dg, db])
    scale = max(1.0, np.max(np.abs(fd)))
    assert np.max(np.abs(got - fd)) <= 1e-3 * scale, np.max(np.abs(got - fd))


def test_flat_cost_and_fields_only(qs):
    """No couplings: zero weights make every state a ground state (E = 0,
    P = 1); fields only give a product of single-qubit states."""
    n = 14
    st = qs.State(n)
    st.set_ising(np.zeros(n), np.zeros((0, 2)), np.zeros(0))
    assert st.cost_info()[:4] == (0, 0, 0, 1 << n)
    st.evolve([0.3, 0.9], [0.2, 1.3])
    E, P, N = st.readout()
    assert abs(E) <= 1e-6 and abs(P - 1.0) <= 1e-5 and abs(N - 1.0) <= 1e-5
    inst = I._canon(n, np.arange(n) % 3 - 1.0, [], [], "fields")
    st.set_instance(inst)
    g, b = I.uniform_angles(3, 9)
    st.evolve(g, b)
    ref = oracle.evolve(inst, g, b)
    assert np.linalg.norm(st.copy_state() - ref) <= 1e-4
    st.close()


def test_shape_rules_and_autotuner(qs):
    """Every candidate shape plan gives the oracle's state (n = 24: strided,
    packed-pair and run-structured shapes), and the autotuner keeps one of
    them and still matches."""
    inst = I.erdos_renyi_ising(24, I.workload_seed(5, 200), h_values=(-1, 0, 1), j_values=(-1, 0, 1))
    g, b = _angles(3)
    ref = oracle.evolve(inst, g, b)
    Er, Pr, _ = oracle.readout(inst, ref)
    st = qs.State(inst.n)
    st.set_instance(inst)
    for rule in [(0, 18), (1, 20), (1, 22), (1, 24), (-1, -1)]:
        st.set_shape_rule(*rule)
        st.evolve(g, b)
        E, P, _ = st.readout()
        assert np.linalg.norm(st.copy_state() - ref) <= 1e-4, rule
        assert abs(E - Er) <= 1e-5 * max(abs(Er), 1.0) and abs(P - Pr) <= 1e-5
    ra, sp, ms = st.autotune(2)
    assert (ra, sp) in [(0, 18), (1, 20), (1, 22), (1, 24)] and ms > 0
    st.evolve(g, b)
    assert np.linalg.norm(st.copy_state() - ref) <= 1e-4
    v, dg, db = st.grad(g, b, 1)
    vr, dgr, dbr = oracle.adjoint(inst, g, b, 1)
    scale = max(1.0, float(np.abs(np.concatenate([dgr, dbr])).max()))
    assert abs(v - vr) <= 1e-5 and np.abs(dg - dgr).max() <= 1e-4 * scale
    st.close()

"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test checks the oracle against something it does not share code with:
dense matrix exponentials built from Pauli Kronecker products (scipy), a
published closed form, exact special cases, symmetries of the definitions,
brute force on tiny inputs, central finite differences, the adiabatic limit
and torch's own Adam.  A plausible slip in the oracle (a swapped bit order, a
dropped field term, the mixer before the phase, a wrong sign in the rotation,
a wrong adjoint term) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2104_03293_gb300 import instances as I

I2 = np.eye(2)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def pauli(n, ops):
    """Kronecker product with qubit n-1 leftmost, so qubit j acts on bit j."""
    M = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        M = np.kron(M, ops.get(q, I2))
    return M


def dense_hc(inst):
    H = np.zeros((1 << inst.n, 1 << inst.n), dtype=np.complex128)
    for i in range(inst.n):
        H += inst.h[i] * pauli(inst.n, {i: PZ})
    for (a, b), w in zip(inst.edges, inst.J):
        H += w * pauli(inst.n, {int(a): PZ, int(b): PZ})
    return H


def dense_hd(n):
    return sum(pauli(n, {i: PX}) for i in range(n))


def dense_state(inst, gamma, beta):
    n = inst.n
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    HC, HD = dense_hc(inst), dense_hd(n)
    for g, b in zip(gamma, beta):
        psi = scipy.linalg.expm(-1j * g * HC) @ psi
        psi = scipy.linalg.expm(-1j * b * HD) @ psi
    return psi


def small_instances():
    out = [
        I.erdos_renyi_ising(1, 11, h_values=(1.5,)),
        I.erdos_renyi_ising(2, 12, mean_degree=1.0),
        I.erdos_renyi_ising(3, 13, mean_degree=2.0),
        I.erdos_renyi_ising(5, 14),
        I.maxcut_regular3(6, 15),
        I.erdos_renyi_ising(8, 16, mean_degree=3.0),
        I.maxcut_regular3(10, 17),
    ]
    return out


# ---------------------------------------------------------------- P1: dense expm
@pytest.mark.parametrize("idx", range(7))
def test_evolve_matches_dense_expm(idx):
    inst = small_instances()[idx]
    for p in (1, 3):
        g, b = I.uniform_angles(p, 100 + idx * 7 + p)
        ref = dense_state(inst, g, b)
        got = oracle.evolve(inst, g, b)
        assert np.linalg.norm(got - ref) <= 1e-12


@pytest.mark.parametrize("idx", range(7))
def test_cost_matches_pauli_diagonal(idx):
    inst = small_instances()[idx]
    diag = np.real(np.diag(dense_hc(inst)))
    assert np.array_equal(oracle.cost_all(inst), diag)


# ---------------------------------------------------------------- P7: brute force
@pytest.mark.parametrize("idx", range(7))
def test_ground_matches_brute_force(idx):
    inst = small_instances()[idx]
    diag = np.real(np.diag(dense_hc(inst)))
    cmin, cmax, arg, cnt = oracle.ground(inst)
    assert cmin == diag.min() and cmax == diag.max()
    mins = np.flatnonzero(diag == diag.min())
    assert arg == mins[0] and cnt == mins.size


def test_ground_ties_take_lowest_index():
    # h = 0 MaxCut: Z2 symmetric, the ground set has >= 2 states.
    inst = I.maxcut_regular3(8, 3)
    cmin, _, arg, cnt = oracle.ground(inst)
    costs = []
    for z in range(1 << inst.n):
        s = [1 - 2 * ((z >> i) & 1) for i in range(inst.n)]
        costs.append(sum(w * s[a] * s[b] for (a, b), w in zip(inst.edges, inst.J)))
    assert cnt >= 2 and cnt % 2 == 0
    assert arg == min(z for z, c in enumerate(costs) if c == cmin)


# ---------------------------------------------------------------- P2: closed form
def wang_edge_cut(du, dv, lam, Gam, beta):
    """p = 1 MaxCut edge cut expectation of Wang, Hadfield, Jiang, Rieffel,
    Phys. Rev. A 97, 022304 (2018), for C = sum (1 - Z_u Z_v)/2 with phase
    e^{-i Gam C}; du, dv are the full degrees, lam the triangles on (u, v)."""
    c = math.cos(Gam)
    return (0.5 + 0.25 * math.sin(4 * beta) * math.sin(Gam) * (c ** (du - 1) + c ** (dv - 1))
            - 0.25 * math.sin(2 * beta) ** 2 * c ** (du + dv - 2 - 2 * lam) * (1 - math.cos(2 * Gam) ** lam))


@pytest.mark.parametrize("n,seed", [(8, 1), (10, 2), (12, 3), (12, 4), (14, 5)])
def test_p1_maxcut_closed_form(n, seed):
    inst = I.maxcut_regular3(n, seed)
    adj = {i: set() for i in range(n)}
    for a, b in inst.edges:
        adj[int(a)].add(int(b)); adj[int(b)].add(int(a))
    rng = np.random.default_rng(seed)
    for _ in range(3):
        g, b = rng.uniform(0, np.pi, size=2)
        # H_C = sum Z Z:  e^{-i g sum ZZ} = e^{-i Gam C} up to a global phase, Gam = -2 g
        Gam = -2.0 * g
        E = 0.0
        for u, v in inst.edges:
            u, v = int(u), int(v)
            lam = len(adj[u] & adj[v])
            E += 1.0 - 2.0 * wang_edge_cut(len(adj[u]), len(adj[v]), lam, Gam, b)
        got, _ = oracle.expect(inst, [g], [b])
        assert abs(got - E) <= 1e-11


# ---------------------------------------------------------------- P3: special angles
@pytest.mark.parametrize("inst", [I.maxcut_regular3(10, 9), I.erdos_renyi_ising(11, 10)])
def test_zero_and_special_angles(inst):
    cmin, _, _, cnt = oracle.ground(inst)
    N = 1 << inst.n
    E, P = oracle.expect(inst, [0.0], [0.0])
    assert abs(E) <= 1e-13 and abs(P - cnt / N) <= 1e-15
    # beta = 0: the diagonal phase leaves |psi|^2 uniform
    E, P = oracle.expect(inst, [0.7, 1.3], [0.0, 0.0])
    assert abs(E) <= 1e-12 and abs(P - cnt / N) <= 1e-14
    # gamma = 0: |+> is an eigenvector of H_D
    E, P = oracle.expect(inst, [0.0, 0.0], [0.4, 2.1])
    assert abs(E) <= 1e-12
    # beta = pi/2: e^{-i pi/2 X} = -i X flips every bit after the phase
    g = 0.37
    psi = oracle.evolve(inst, [g], [np.pi / 2])
    diag = oracle.cost_all(inst)
    z = np.arange(N)
    expect = (-1j) ** inst.n * np.exp(-1j * g * diag[z ^ (N - 1)]) * 2.0 ** (-inst.n / 2)
    assert np.max(np.abs(psi - expect)) <= 1e-13


def test_plus_state():
    psi = oracle.plus_state(7)
    assert np.allclose(psi, 2.0 ** -3.5, atol=0, rtol=1e-15)


# ---------------------------------------------------------------- P4 / P5
def test_norm_and_round_trip():
    inst = I.erdos_renyi_ising(12, 21)
    g, b = I.uniform_angles(6, 22)
    psi = oracle.evolve(inst, g, b)
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-13
    # undo the layers in reverse order with negated angles, gate by gate
    for k in range(len(g) - 1, -1, -1):
        for i in range(inst.n):
            oracle.gate_x(psi, inst.n, i, -b[k])
        for (a, c), w in zip(inst.edges, inst.J):
            oracle.gate_zz(psi, inst.n, int(a), int(c), -g[k] * w)
        for i in range(inst.n):
            oracle.gate_z(psi, inst.n, i, -g[k] * inst.h[i])
    assert np.max(np.abs(psi - 2.0 ** (-inst.n / 2))) <= 1e-13


# ---------------------------------------------------------------- P6: symmetries
def test_symmetries():
    inst = I.erdos_renyi_ising(11, 31)
    g, b = I.uniform_angles(4, 32)
    psi = oracle.evolve(inst, g, b)
    # sign flip of all angles conjugates the state (H_C real, |+> real)
    assert np.max(np.abs(oracle.evolve(inst, -g, -b) - psi.conj())) <= 1e-13
    # beta -> beta + pi multiplies each layer by (-1)^n  (beta periodic in [0, pi))
    b2 = b.copy(); b2[1] += np.pi
    assert np.max(np.abs(oracle.evolve(inst, g, b2) - (-1) ** inst.n * psi)) <= 1e-12
    # gamma -> gamma + 2 pi leaves the state unchanged for integer costs
    g2 = g.copy(); g2[2] += 2 * np.pi
    assert np.max(np.abs(oracle.evolve(inst, g2, b) - psi)) <= 1e-12
    # h = 0: psi_z = psi_{complement of z}
    mc = I.maxcut_regular3(10, 33)
    phi = oracle.evolve(mc, g, b)
    N = 1 << mc.n
    assert np.max(np.abs(phi - phi[np.arange(N) ^ (N - 1)])) <= 1e-14


# ---------------------------------------------------------------- P8: adjoint
@pytest.mark.parametrize("objective", [0, 1])
@pytest.mark.parametrize("n,p,seed", [(4, 1, 41), (6, 4, 42), (9, 3, 43)])
def test_adjoint_matches_central_differences(objective, n, p, seed):
    inst = I.erdos_renyi_ising(n, seed)
    g, b = I.uniform_angles(p, seed + 1)
    val, dg, db = oracle.adjoint(inst, g, b, objective)
    E, P = oracle.expect(inst, g, b)
    assert abs(val - (E if objective == 0 else P)) <= 1e-13
    eps = 1e-5

    def F(gg, bb):
        return oracle.expect(inst, gg, bb)[objective]

    scale = max(1.0, float(np.max(np.abs(np.concatenate([dg, db])))))
    for k in range(p):
        e = np.zeros(p); e[k] = eps
        fd_g = (F(g + e, b) - F(g - e, b)) / (2 * eps)
        fd_b = (F(g, b + e) - F(g, b - e)) / (2 * eps)
        assert abs(dg[k] - fd_g) <= 1e-7 * scale
        assert abs(db[k] - fd_b) <= 1e-7 * scale


# ---------------------------------------------------------------- P9: AQA sign
def test_aqa_adiabatic_limit_fixes_the_sign():
    # 6 qubits, integer weights, unique ground state (checked below)
    inst = I.erdos_renyi_ising(6, 4, mean_degree=3.0)
    cmin, _, _, cnt = oracle.ground(inst)
    assert cnt == 1
    p, tau = 400, 0.1
    s = np.arange(1, p + 1) / (p + 1)
    g, b = oracle.aqa_angles(tau, s)
    assert np.all(b < 0) and np.all(g > 0)
    _, P = oracle.expect(inst, g, b)
    assert P > 0.99
    # the literal +tau(1 - s) sign anneals towards the top of the spectrum
    _, P_wrong = oracle.expect(inst, g, -b)
    assert P_wrong < 1e-6


def test_aqa_chain_rule_matches_differences():
    inst = I.erdos_renyi_ising(7, 51)
    p, tau = 5, 0.75
    s = np.arange(1, p + 1) / (p + 1)

    def F(t, ss):
        g, b = oracle.aqa_angles(t, ss)
        return oracle.expect(inst, g, b)[1]

    g, b = oracle.aqa_angles(tau, s)
    _, dg, db = oracle.adjoint(inst, g, b, 1)
    dtau, ds = oracle.aqa_chain(tau, s, dg, db)
    eps = 1e-6
    assert abs(dtau - (F(tau + eps, s) - F(tau - eps, s)) / (2 * eps)) <= 1e-7
    for k in range(p):
        e = np.zeros(p); e[k] = eps
        assert abs(ds[k] - (F(tau, s + e) - F(tau, s - e)) / (2 * eps)) <= 1e-7


def test_second_order_map_is_a_product_of_symmetric_steps():
    """Appendix A: with the second-order angles the QAOA state equals
    U(s_p)...U(s_1)|+> up to a global phase, U(s) = e^{i tau A H_D/2}
    e^{-i tau B H_C} e^{i tau A H_D/2}, with s_k = (k-1)/(p-1)."""
    inst = I.erdos_renyi_ising(6, 61)
    p, tau = 5, 0.6
    s = np.arange(p) / (p - 1)
    g, b = oracle.aqa_angles_second_order(tau, s)
    psi = oracle.evolve(inst, g, b)
    HC, HD = dense_hc(inst), dense_hd(inst.n)
    ref = np.full(1 << inst.n, 2.0 ** (-inst.n / 2), dtype=np.complex128)
    for sk in s:
        half = scipy.linalg.expm(1j * tau * (1 - sk) * HD / 2)
        ref = half @ scipy.linalg.expm(-1j * tau * sk * HC) @ half @ ref
    phase = np.vdot(psi, ref)
    assert abs(abs(phase) - 1.0) <= 1e-12
    assert np.linalg.norm(ref - phase * psi) <= 1e-12


def test_second_order_chain_rule_matches_differences():
    """dP/dtau and dP/ds_k under the second-order map (Eqs. beta_k-gamma_k,
    Appendix A): the oracle's chain rule applied to its adjoint against
    central differences of P_ground taken through the map itself."""
    inst = I.erdos_renyi_ising(7, 52)
    p, tau = 6, 0.8
    s = np.arange(p) / (p - 1)

    def F(t, ss):
        g, b = oracle.aqa_angles_second_order(t, ss)
        return oracle.expect(inst, g, b)[1]

    g, b = oracle.aqa_angles_second_order(tau, s)
    _, dg, db = oracle.adjoint(inst, g, b, 1)
    dtau, ds = oracle.aqa_chain_second_order(tau, s, dg, db)
    eps = 1e-6
    assert abs(dtau - (F(tau + eps, s) - F(tau - eps, s)) / (2 * eps)) <= 1e-7
    for k in range(p):
        e = np.zeros(p); e[k] = eps
        assert abs(ds[k] - (F(tau, s + e) - F(tau, s - e)) / (2 * eps)) <= 1e-7
    # the first-order chain rule applied to the second-order angles is wrong
    # (it misses the knot s_{k+1} inside beta_k): the pin can tell them apart
    _, ds1 = oracle.aqa_chain(tau, s, dg, db)
    assert np.max(np.abs(ds1 - ds)) > 1e-3


# ---------------------------------------------------------------- spin expectations
@pytest.mark.parametrize("idx", [1, 3, 4, 5])
def test_zexp_matches_dense_pauli_expectations(idx):
    """<Z_i> after every layer (Sec. III.B.2, Fig. 6) against
    <psi_k| Z_i |psi_k> with Z_i the Kronecker product and psi_k from dense
    matrix exponentials."""
    inst = small_instances()[idx]
    p = 3
    g, b = I.uniform_angles(p, 300 + idx)
    got = oracle.evolve_zexp(inst, g, b)
    assert got.shape == (p, inst.n)
    for k in range(p):
        psi = dense_state(inst, g[:k + 1], b[:k + 1])
        for i in range(inst.n):
            ref = np.vdot(psi, pauli(inst.n, {i: PZ}) @ psi).real
            assert abs(got[k, i] - ref) <= 1e-12


def test_zexp_special_cases_and_closed_form():
    inst = I.erdos_renyi_ising(9, 71)
    # gamma = 0: the state stays |+> (an eigenvector of H_D); beta = 0: the
    # phase leaves |psi|^2 uniform.  Either way every <Z_i> vanishes.
    assert np.max(np.abs(oracle.evolve_zexp(inst, [0.0, 0.0], [0.3, 1.1]))) <= 1e-14
    assert np.max(np.abs(oracle.evolve_zexp(inst, [0.4, 0.9], [0.0, 0.0]))) <= 1e-14
    # fields only, one layer: each qubit evolves alone, e^{-i b X} e^{-i g h Z}|+>
    # has <Z> = sin(2 b) sin(2 g h) (a 2 x 2 computation)
    h = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    fields = I._canon(5, h, [], [], "fields")
    g, b = 0.37, 0.81
    got = oracle.evolve_zexp(fields, [g], [b])[0]
    assert np.max(np.abs(got - np.sin(2 * b) * np.sin(2 * g * h))) <= 1e-14
    # and then E = sum_i h_i <Z_i> at every layer
    g3, b3 = I.uniform_angles(3, 72)
    z = oracle.evolve_zexp(fields, g3, b3)
    for k in range(3):
        E, _ = oracle.expect(fields, g3[:k + 1], b3[:k + 1])
        assert abs(E - float(h @ z[k])) <= 1e-13


# ---------------------------------------------------------------- Adam
def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    theta = rng.normal(size=6)
    t_param = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t_param], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(6); v = np.zeros(6)
    for step in range(1, 8):
        grad = rng.normal(size=6)
        theta, m, v = oracle.adam_step(theta, grad, m, v, step)
        opt.zero_grad()
        t_param.grad = torch.tensor(grad, dtype=torch.float64)
        opt.step()
        assert np.max(np.abs(theta - t_param.detach().numpy())) <= 1e-14


# ------------------------------------------------ QSDS product formula, Eq. (AQA4)
def _dense_qsds(inst, tau, A, B):
    n = inst.n
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    HX = dense_hd(n)
    HZ = sum(inst.h[i] * pauli(n, {i: PZ}) for i in range(n))
    HZZ = dense_hc(inst) - HZ
    for a, b in zip(A, B):
        S = scipy.linalg.expm(0.5j * tau * (a * HX - b * HZ))  # h~x = A, h~z = -B h
        Zc = scipy.linalg.expm(-1j * tau * b * HZZ)            # J~z = -B J
        psi = S @ (Zc @ (S @ psi))
    return psi


@pytest.mark.parametrize("idx", range(4))
def test_qsds_matches_dense_product_formula(idx):
    """Eq. (AQA4) with the fields of Eq. (AQA3): the oracle's single-spin
    2 x 2 exponentials and ZZ gates against dense matrix exponentials of the
    full single-spin and coupling Hamiltonians, step by step."""
    inst = small_instances()[idx]
    nsteps = 5
    s = np.arange(nsteps) / nsteps
    A, B = 1.0 - s, s
    got = oracle.qsds_evolve(inst, 0.6, A, B)
    want = _dense_qsds(inst, 0.6, A, B)
    assert np.max(np.abs(got - want)) <= 1e-12
    assert abs(np.linalg.norm(got) - 1.0) <= 1e-13


def test_qsds_without_fields_is_the_second_order_qaoa_map():
    """With h = 0 the single-spin steps are pure x rotations that commute, so
    merging consecutive half steps gives the QAOA state with gamma_k =
    tau B_k and beta_k = -tau (A_k + A_{k+1}) / 2 (the last one -tau A / 2),
    up to the global phase exp(i tau A_0 n / 2) of the first half step on
    |+>^n (the structure of Appendix A)."""
    inst = I.maxcut_regular3(8, 91)
    nsteps, tau = 6, 0.45
    s = (np.arange(nsteps) + 0.5) / nsteps
    A, B = 1.0 - s, s
    got = oracle.qsds_evolve(inst, tau, A, B)
    g = tau * B
    b = -0.5 * tau * (A + np.append(A[1:], 0.0))
    want = oracle.evolve(inst, g, b) * np.exp(0.5j * tau * A[0] * inst.n)
    assert np.max(np.abs(got - want)) <= 1e-12


def test_gate_u_general_matrix():
    """A general 2 x 2 matrix on qubit j against the dense Kronecker product."""
    rng = np.random.default_rng(5)
    n = 5
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    u = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    for j in range(n):
        want = pauli(n, {j: u}) @ psi
        got = oracle.gate_u(n, psi.copy(), j, u)
        assert np.max(np.abs(got - want)) <= 1e-12

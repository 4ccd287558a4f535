"""Layers with general single-spin unitaries (qs_evolve_su2) and the product
formula of Eq. (AQA4) (qs_qsds_layers) through the C ABI, against the
oracle: the step-by-step Eq. (AQA4) state of oracle.qsds_evolve, and random
per-qubit unitaries applied with the oracle's general gate.

Tolerances as for the other state parity tests: ||psi - psi_ref||_2 <= 1e-4
(complex64) or 1e-10 (complex128); E and P_ground as in tests/tolerances.py.
Sizes cover the padded small state and contiguous and strided tiles (one
and two strided shapes); the run-structured tiles of 33 and 34 qubits are
not reached at these sizes.
"""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import instances as I
from tolerances import assert_readout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2104_03293_gb300 import build, qs as _qs
    build.build()
    return _qs


def _linear(nsteps):
    s = (np.arange(nsteps) + 0.5) / nsteps
    return 1.0 - s, s


@pytest.mark.parametrize("n,dtype,nsteps", [(12, "c64", 8), (12, "c128", 5), (17, "c64", 10), (21, "c128", 4),
                                            (24, "c64", 8), (25, "c64", 3)])
def test_qsds_product_formula_against_oracle(qs, n, dtype, nsteps):
    inst = I.erdos_renyi_ising(n, I.workload_seed(6, 400 + n))
    tau = 0.7
    A, B = _linear(nsteps)
    g, u = qs.qsds_layers(n, tau, A, B, inst.h)
    st = qs.State(n, dtype)
    try:
        st.set_instance(inst)
        st.evolve_su2(g, u)
        E, P, N = st.readout()
        psi = st.copy_state().astype(np.complex128)
    finally:
        st.close()
    ref = oracle.qsds_evolve(inst, tau, A, B)
    err = np.linalg.norm(psi - ref)
    assert err <= (1e-4 if dtype == "c64" else 1e-10), (n, dtype, err)
    Er, Pr, _ = oracle.readout(inst, ref)
    assert_readout(inst, E, P, Er, Pr, (n, dtype))
    assert abs(N - 1.0) <= 1e-5
    assert Pr > 2.0 ** -n  # the annealing moves weight onto the ground state


@pytest.mark.parametrize("n", [13, 20])
def test_random_single_spin_unitaries(qs, n):
    """Random unitaries per layer and qubit (Haar-like from QR), random
    phases: the GPU state against the oracle's general 2 x 2 gates."""
    inst = I.erdos_renyi_ising(n, I.workload_seed(6, 500 + n))
    rng = np.random.default_rng(n)
    p = 3
    g = rng.uniform(0, np.pi, size=p)
    u = np.empty((p, n, 2, 2), dtype=np.complex128)
    for k in range(p):
        for q in range(n):
            z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
            qm, r = np.linalg.qr(z)
            u[k, q] = qm * (np.diag(r) / np.abs(np.diag(r)))
    st = qs.State(n, "c64")
    try:
        st.set_instance(inst)
        st.evolve_su2(g, u)
        psi = st.copy_state().astype(np.complex128)
    finally:
        st.close()
    ref = oracle.evolve(inst, [0.0], [0.0])
    for k in range(p):
        ref = oracle.evolve(inst, [g[k]], [0.0], psi=ref)
        for q in range(n):
            oracle.gate_u(n, ref, q, u[k, q])
    assert np.linalg.norm(psi - ref) <= 1e-4


def test_x_rotations_reproduce_qaoa(qs):
    """U = exp(-i beta X) on every qubit is the QAOA mixer: evolve_su2 and
    evolve give the same state (the tangent-form sweeps against the general
    butterfly)."""
    inst = I.erdos_renyi_ising(22, I.workload_seed(6, 600))
    g, b = I.uniform_angles(4, I.workload_seed(6, 601))
    u = np.empty((4, inst.n, 2, 2), dtype=np.complex128)
    for k in range(4):
        c, s = np.cos(b[k]), np.sin(b[k])
        u[k, :] = np.array([[c, -1j * s], [-1j * s, c]])
    st = qs.State(inst.n, "c64")
    try:
        st.set_instance(inst)
        st.evolve_su2(g, u)
        a = st.copy_state()
        E1, P1, _ = st.readout()
        st.evolve(g, b)
        bb = st.copy_state()
        E2, P2, _ = st.readout()
    finally:
        st.close()
    assert np.linalg.norm(a.astype(np.complex128) - bb.astype(np.complex128)) <= 1e-5
    assert abs(E1 - E2) <= 1e-5 * max(1.0, abs(E2)) and abs(P1 - P2) <= 1e-4 * P2 + 1e-9

"""Per-layer spin expectations <Z_i> (Sec. III.B.2, Fig. 6) through the C ABI
(qs_evolve_zexp) against the oracle's plain per-qubit sums after every layer.

Tolerance: per layer k, max_i |z_ki - zref_ki| <= rel * max_i |zref_ki| + abs,
rel = 1e-5 (complex64) or 1e-10 (complex128), relative to the layer's largest
magnetisation.  Instances carry fields (ER(4), h, J ~ U{-2..2}), so the
magnetisations are of order 0.1-1 under AQA angles; random angles put the
stored array in the flipped frame on some layers (cotangent form).  Sizes
cover the padded small state (one tile shape, several layers per sweep),
contiguous, strided and packed-pair phase sweeps, and, through a factorised
instance, the n = 34 shapes of the benchmark.
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


def _aqa(p, tau=0.75):
    s = np.arange(1, p + 1) / (p + 1)
    return oracle.aqa_angles(tau, s)


def _check(z, zr, rel, what):
    assert z.shape == zr.shape, (what, z.shape, zr.shape)
    for k in range(zr.shape[0]):
        scale = float(np.max(np.abs(zr[k])))
        err = float(np.max(np.abs(z[k] - zr[k])))
        assert err <= rel * scale + 1e-9, (what, k, err, scale)


@pytest.mark.parametrize("n,dtype,p,kind", [
    (12, "c64", 10, "aqa"), (12, "c128", 5, "rand"), (17, "c64", 10, "aqa"), (17, "c64", 6, "rand"),
    (21, "c64", 12, "aqa"), (21, "c128", 4, "rand"), (24, "c64", 10, "aqa"), (24, "c64", 5, "rand"),
])
def test_zexp_against_oracle(qs, n, dtype, p, kind):
    inst = I.erdos_renyi_ising(n, I.workload_seed(6, n))
    g, b = _aqa(p) if kind == "aqa" else I.uniform_angles(p, I.workload_seed(6, 100 + n))
    st = qs.State(n, dtype)
    try:
        st.set_instance(inst)
        z = st.evolve_zexp(g, b)
        E, P, _ = st.readout()
        # the evolve leaves the same state and readout as a plain evolve (same
        # arithmetic; only the fused accumulations differ)
        st2 = qs.State(n, dtype)
        st2.set_instance(inst)
        st2.evolve(g, b)
        E2, P2, _ = st2.readout()
        st2.close()
    finally:
        st.close()
    assert abs(E - E2) <= 1e-9 * max(1.0, abs(E2)) and abs(P - P2) <= 1e-9 * P2 + 1e-15
    zr = oracle.evolve_zexp(inst, g, b)
    _check(z, zr, 1e-5 if dtype == "c64" else 1e-10, (n, dtype, p, kind))
    if kind == "aqa":
        assert float(np.max(np.abs(zr[-1]))) > 0.05  # the comparison has something to catch


def test_zexp_zero_field_symmetry(qs):
    # MaxCut (h = 0): psi_z = psi_{not z}, so every <Z_i> vanishes
    inst = I.maxcut_regular3(18, I.workload_seed(6, 7))
    g, b = I.uniform_angles(4, I.workload_seed(6, 8))
    st = qs.State(inst.n, "c64")
    try:
        st.set_instance(inst)
        z = st.evolve_zexp(g, b)
    finally:
        st.close()
    assert float(np.max(np.abs(z))) <= 1e-6


def test_zexp_repeatable_and_p0(qs):
    inst = I.erdos_renyi_ising(20, I.workload_seed(6, 9))
    g, b = _aqa(9)
    st = qs.State(inst.n, "c64")
    try:
        st.set_instance(inst)
        z1 = st.evolve_zexp(g, b)
        z2 = st.evolve_zexp(g, b)
        assert np.array_equal(z1, z2)  # fixed reduction order: bit-identical
        assert st.evolve_zexp([], []).shape == (0, inst.n)
    finally:
        st.close()


def test_zexp_factorised_full_size(qs):
    # n = 34 from two 17-qubit components: <Z_i> of the product state is the
    # component's own <Z_i> (the other factor has unit norm)
    import torch
    comp = [I.erdos_renyi_ising(17, I.workload_seed(5, 100 + k), h_values=(-1, 0, 1), j_values=(-1, 0, 1))
            for k in range(2)]
    U = I.union(comp)
    g, b = _aqa(20)
    buf = torch.empty(1 << 34, dtype=torch.complex64, device="cuda")
    st = qs.State(34, "c64", buffer=buf)
    try:
        st.set_instance(U)
        z = st.evolve_zexp(g, b)
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()
    zr = np.concatenate([oracle.evolve_zexp(c, g, b) for c in comp], axis=1)
    _check(z, zr, 1e-5, "n34 factorised")

"""Tile loads of the strided packed-pair forward sweeps on the GPU (plan rule
fields pair_tma and pair_l2): tensor-map copies, and cp.async copies with
128- or 256-byte L2 fetches, give states bit-identical to the default
cp.async loads (the same arithmetic on the same values), and the oracle's
state where the oracle runs: the whole state at n = 24 and 27 (lean
strided sweeps) and n = 26 with the strided shapes in reverse order (the
packed-pair shape's sweeps merged around the phases), a product instance of two oracle-sized components at
n = 32 (two strided shapes of 2^3-amplitude rows, the merged sweeps
included) and n = 34 (the bench's shapes and the default ones).
"""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import instances as I
from tolerances import e_tol, p_tol

pytestmark = pytest.mark.gpu

LOADS = [(0, 1), (0, 2), (1, 0), (1, 2)]


@pytest.fixture(scope="module")
def qs():
    from paper_2104_03293_gb300 import build, qs as _qs
    build.build()
    return _qs


def _set_load(st, rule, tma, l2):
    r = list(rule) + [0] * (8 - len(rule))
    r[5], r[6] = tma, l2
    st.set_plan_rule(r)


@pytest.mark.parametrize("n,order", [(24, 0), (27, 0), (26, 1)])
def test_loads_against_oracle(qs, n, order):
    inst = I.erdos_renyi_ising(n, I.workload_seed(7, n))
    s = np.arange(1, 6) / 6.0
    g, b = oracle.aqa_angles(0.8, s)
    ref = oracle.evolve(inst, g, b)
    st = qs.State(n)
    try:
        st.set_instance(inst)
        rule = list(st.plan_rule())
        rule[7] = order  # 1: the packed-pair shape last, its sweeps merged
        st.set_plan_rule(rule)
        st.evolve(g, b)
        base = st.copy_state()
        assert np.linalg.norm(base.astype(np.complex128) - ref) <= 1e-4
        Eb = st.readout()
        for tma, l2 in LOADS:
            _set_load(st, rule, tma, l2)
            st.evolve(g, b)
            got = st.copy_state()
            assert np.array_equal(got.view(np.uint32), base.view(np.uint32)), (tma, l2)
            assert st.readout() == Eb
    finally:
        st.close()


def _checksum(buf):
    import torch
    v = torch.view_as_real(buf).view(-1).view(torch.int32)
    tot, step = 0, 1 << 28
    for i in range(0, v.numel(), step):
        tot += int(v[i:i + step].to(torch.int64).sum())
    return tot


@pytest.mark.parametrize("n,rule", [(32, [0, 18, 3, 0, 4]), (34, [1, 20, -1, 0, 4]), (34, [-1, -1, -1, 0, 4])])
def test_loads_full_size(qs, n, rule):
    import torch
    nA = n // 2
    A = I.erdos_renyi_ising(nA, I.workload_seed(7, 200 + n))
    B = I.erdos_renyi_ising(n - nA, I.workload_seed(7, 300 + n))
    U = I.union([A, B])
    s = np.arange(1, 7) / 7.0
    g, b = oracle.aqa_angles(0.75, s)
    buf = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    st = qs.State(n, buffer=buf)
    rng = np.random.default_rng(n)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, size=1 << 16), [0, (1 << n) - 1]]))
    tidx = torch.from_numpy(idx).to(buf.device)
    try:
        st.set_instance(U)
        _set_load(st, rule, 0, 0)
        st.evolve(g, b)
        E0 = st.readout()
        sum0 = _checksum(buf)
        samp0 = buf[tidx].cpu().numpy()
        psiA, psiB = oracle.evolve(A, g, b), oracle.evolve(B, g, b)
        EA, PA, _ = oracle.readout(A, psiA)
        EB, PB, _ = oracle.readout(B, psiB)
        assert abs(E0[0] - (EA + EB)) <= e_tol(U, EA + EB) and abs(E0[1] - PA * PB) <= p_tol(PA * PB)
        want = psiA[idx & ((1 << nA) - 1)] * psiB[idx >> nA]
        # global phase: the tiled path's state equals the oracle's up to the
        # canonical phase, compared after qs_canonicalize below
        for tma, l2 in LOADS:
            _set_load(st, rule, tma, l2)
            st.evolve(g, b)
            assert st.readout() == E0, (tma, l2)
            assert _checksum(buf) == sum0, (tma, l2)
            assert np.array_equal(buf[tidx].cpu().numpy().view(np.uint32), samp0.view(np.uint32)), (tma, l2)
        st.canonicalize()
        got = buf[tidx].cpu().numpy().astype(np.complex128)
        err = np.sqrt(np.sum(np.abs(got - want) ** 2) * (2.0 ** n) / idx.size)
        assert err <= 1e-4, err
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()

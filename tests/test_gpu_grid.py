"""p = 1 landscape scan (Sec. III.B.1, Fig. 4) through the batched path,
against the oracle at every grid point."""
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


def test_grid_scan_matches_oracle(qs):
    inst = I.erdos_renyi_ising(12, I.workload_seed(6, 0), h_values=(-1, 0, 1), j_values=(-1, 0, 1))
    gammas = np.arange(8) * (2 * np.pi / 8)
    betas = np.arange(6) * (np.pi / 6)
    E, P = qs.grid_scan(inst.h, inst.edges, inst.J, gammas, betas)
    assert E.shape == (8, 6) and P.shape == (8, 6)
    bound = float(np.abs(inst.h).sum() + np.abs(inst.J).sum())
    for a, g in enumerate(gammas):
        for c, b in enumerate(betas):
            Er, Pr = oracle.expect(inst, [g], [b])
            assert abs(E[a, c] - Er) <= 1e-5 * max(abs(Er), bound, 1.0), (a, c, E[a, c], Er)
            assert abs(P[a, c] - Pr) <= 1e-4 * Pr + 1e-9, (a, c, P[a, c], Pr)
    # gamma = 0 or beta = 0 leaves |+>^n's statistics: E = sum h_i <Z_i> + ... = 0, P = count / 2^n
    cmin, cmax, arg, cnt = oracle.ground(inst)
    assert np.all(np.abs(E[0, :]) <= 1e-5 * max(bound, 1.0)) and np.all(np.abs(E[:, 0]) <= 1e-5 * max(bound, 1.0))
    P0 = cnt / 2.0 ** inst.n
    assert np.allclose(P[0, :], P0, rtol=1e-4, atol=1e-9) and np.allclose(P[:, 0], P0, rtol=1e-4, atol=1e-9)


def test_grid_scan_rejects_an_empty_grid(qs):
    inst = I.erdos_renyi_ising(12, I.workload_seed(6, 1))
    with pytest.raises(qs.QSError):
        qs.grid_scan(inst.h, inst.edges, inst.J, [], [0.1])

"""An exact-cover instance (Sec. III.A.3, half-integer weights) on the CUDA
path: the enumeration finds the planted cover, and an AQA run with the
angles divided by the rescaling factor r of Eq. (rescale) matches the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import exact_cover as X
from paper_2104_03293_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2104_03293_gb300 import build, qs as _qs
    build.build()
    return _qs


@pytest.mark.parametrize("n,f", [(14, 40), (20, 50)])
def test_exact_cover_on_the_cuda_path(qs, n, f):
    a, x = I.exact_cover(n, f, I.workload_seed(7, 100 + n))
    h, e, J, C = X.ising_from_exact_cover(a)
    inst = I._canon(n, h, e, J, "exact_cover")
    r = X.rescale_factor(h, J)
    st = qs.State(n)
    st.set_ising(h, e, J)
    cmin, cmax, arg, cnt, shift = st.cost_info()  # costs in units of 2^-shift
    rmin, rmax, rarg, rcnt = oracle.ground(inst)
    assert (cmin, cmax) == (rmin * 2 ** shift, rmax * 2 ** shift) and (arg, cnt) == (rarg, rcnt)
    assert rmin + C == 0 and oracle.cost(inst, arg) + C == 0
    g, b = qs.aqa_angles(0.75, np.arange(1, 6) / 6.0)
    st.evolve(np.asarray(g) / r, b)
    E, P, N = st.readout()
    Er, Pr = oracle.expect(inst, np.asarray(g) / r, b)
    bound = float(np.abs(h).sum() + np.abs(J).sum())
    assert abs(E - Er) <= 1e-5 * max(abs(Er), bound, 1.0) and abs(P - Pr) <= 1e-4 * Pr + 1e-9 and abs(N - 1) <= 1e-5
    if n <= 14:
        assert np.linalg.norm(st.copy_state() - oracle.evolve(inst, np.asarray(g) / r, b)) <= 1e-4
    st.close()

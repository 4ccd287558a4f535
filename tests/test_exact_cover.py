"""Exact cover to Ising (Sec. III.A.3): the mapping of the package against
the objective of Eq. (exactcover) written out in the oracle, for every
assignment of small seeded instances; the rescaling of Eq. (rescale)."""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import exact_cover as X
from paper_2104_03293_gb300 import instances as I

CASES = [(4, 6, 1, None), (6, 10, 2, None), (8, 20, 3, None), (10, 30, 4, 0.3), (12, 40, 5, None), (12, 24, 6, 0.05)]


def _mapped(a):
    h, e, J, C = X.ising_from_exact_cover(a)
    return I._canon(a.shape[0], h, e, J, "exact_cover"), C


@pytest.mark.parametrize("n,f,seed,q", CASES)
def test_mapping_equals_the_objective_for_every_assignment(n, f, seed, q):
    a, x = I.exact_cover(n, f, I.workload_seed(7, seed), extra_density=q)
    inst, C = _mapped(a)
    direct = oracle.exact_cover_cost_all(a)
    assert np.array_equal(oracle.cost_all(inst) + C, direct.astype(np.float64))
    # half-integer weights (the engine's integer path takes them exactly)
    assert np.all(2 * inst.h == np.round(2 * inst.h)) and np.all(2 * inst.J == np.round(2 * inst.J))


@pytest.mark.parametrize("n,f,seed,q", CASES)
def test_planted_solution_is_a_ground_state(n, f, seed, q):
    a, x = I.exact_cover(n, f, I.workload_seed(7, seed), extra_density=q)
    assert np.all(a[x == 1].sum(axis=0) == 1)  # the planted rows cover every column once
    inst, C = _mapped(a)
    cmin, _, arg, cnt = oracle.ground(inst)
    z = int(sum(int(b) << i for i, b in enumerate(x)))
    assert cmin + C == 0 and oracle.cost(inst, z) + C == 0
    assert oracle.cost(inst, arg) + C == 0 and cnt >= 1


def test_rescale_factor_follows_its_definition():
    # h in [-3, 1], J in [0.5, 2]: max(1/2, -3/-2, 2/1, 0.5/-1, 0) = 2
    assert X.rescale_factor([-3.0, 1.0], [0.5, 2.0]) == 2.0
    # h = [1], J in [-1.5, 0.5]: max(1/2, 1/-2, 0.5/1, -1.5/-1, 0) = 1.5
    assert X.rescale_factor([1.0], [-1.5, 0.5]) == 1.5
    assert X.rescale_factor([0.0], []) == 0.0
    for n, f, seed, q in CASES:
        a, _ = I.exact_cover(n, f, I.workload_seed(7, seed), extra_density=q)
        h, _, J, _ = X.ising_from_exact_cover(a)
        r = X.rescale_factor(h, J)
        assert r > 0 and np.all(np.abs(h) / r <= X.H_MAX + 1e-12) and np.all(np.abs(J) / r <= X.J_MAX + 1e-12)
        # the sign of the fields (spin convention) does not change r
        assert X.rescale_factor(-h, J) == r


def test_rescaled_cost_equals_scaled_angles():
    """Evolving H_C / r with gamma is evolving H_C with gamma / r."""
    a, _ = I.exact_cover(8, 16, I.workload_seed(7, 9))
    inst, _ = _mapped(a)
    r = X.rescale_factor(inst.h, inst.J)
    scaled = inst.copy()
    scaled.h, scaled.J = inst.h / r, inst.J / r
    g, b = oracle.aqa_angles(0.75, np.arange(1, 4) / 4.0)
    psi_a = oracle.evolve(scaled, g, b)
    psi_b = oracle.evolve(inst, np.asarray(g) / r, b)
    assert np.linalg.norm(psi_a - psi_b) <= 1e-12


def test_bad_matrices_are_rejected():
    with pytest.raises(ValueError):
        X.ising_from_exact_cover(np.array([[0, 2], [1, 0]]))
    with pytest.raises(ValueError):
        X.ising_from_exact_cover(np.zeros((0, 3)))

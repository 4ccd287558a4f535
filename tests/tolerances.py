"""Tolerances of the parity tests (CUDA path against the oracle).

* state: ||psi - psi_ref||_2 <= 1e-4 for complex64, 1e-10 for complex128;
* <H_C>: |E - E_ref| <= 1e-5 max(|E_ref|, sum|h| + sum|J|, 1) (relative to the
  cost scale when E_ref happens to lie near zero);
* ground-state probability: |P - P_ref| <= 1e-4 P_ref + 1e-9, relative, so a
  small P is compared at its own scale (a zero readout fails);
* gradients: max|g - g_ref| <= 1e-4 max|g_ref| + 1e-12, relative to the
  largest component of the reference gradient, with no floor of one.
"""
import numpy as np


def e_tol(inst, E_ref):
    return 1e-5 * max(abs(E_ref), float(np.abs(inst.h).sum() + np.abs(inst.J).sum()), 1.0)


def p_tol(P_ref):
    return 1e-4 * abs(P_ref) + 1e-9


def value_tol(objective, inst, ref):
    return e_tol(inst, ref) if objective == 0 else p_tol(ref)


def assert_grad(got, ref, rel=1e-4, what=""):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    assert err <= rel * scale + 1e-12, (what, err, scale, got, ref)


def assert_readout(inst, E, P, Er, Pr, what=""):
    assert abs(E - Er) <= e_tol(inst, Er), (what, E, Er)
    assert abs(P - Pr) <= p_tol(Pr), (what, P, Pr)

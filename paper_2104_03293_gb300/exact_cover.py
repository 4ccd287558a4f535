"""Exact cover as an Ising cost (Sec. III.A.3).

The problem of Eq. (exactcover) -- minimise over x in {0,1}^N the sum over
the F columns of (sum_i a_if x_i - 1)^2 -- becomes a diagonal H_C of the
form of Eq. (HC) by x_i -> (1 + sigma_i)/2 (Eq. xtosigma).  Multiplying out
the square gives the fields, couplings and constant of Eqs. (HChi)-(HCC):

    h_i  = sum_j (a a^T)_ij / 2 - (a b)_i,     J_ij = (a a^T)_ij / 2  (i < j),
    C    = b^T b + sum_{i<j} (a a^T)_ij / 2 + sum_i ((a a^T)_ii - 2 (a b)_i) / 2,

with b the all-ones F-vector; all of them are half-integers, which the
engine's integer cost path takes as they are.  The paper's spin is
sigma_i = 2 x_i - 1 (|0> is the -1 eigenstate); the engine's is
s_i = 1 - 2 bit_i with bit_i = x_i, so s_i = -sigma_i: the fields change
sign and the couplings do not.  Then, for every basis state z,

    sum_f (sum_i a_if bit_i(z) - 1)^2 = C_engine(z) + C.

Eq. (rescale) divides h, J and C by r to bring instances to a common range
(|h| <= 2, |J| <= 1).  Evolving H_C / r with angle gamma is evolving H_C
with gamma / r, so the engine keeps the half-integer weights and the
caller divides the phase angles (and the energies) by r.
"""
from __future__ import annotations

import numpy as np

H_MAX, J_MAX = 2.0, 1.0  # h_max = -h_min, J_max = -J_min of Eq. (rescale)


def ising_from_exact_cover(a):
    """Map the 0/1 problem matrix a [N, F] to the engine's Ising cost.

    Returns (h [N], edges [m, 2] with i < j, J [m], C): fields and couplings
    in the engine's spin convention (s = 1 - 2 bit) and the additive
    constant of Eq. (HCC)."""
    a = np.asarray(a, dtype=np.int64)
    if a.ndim != 2 or a.shape[0] < 1 or np.any((a != 0) & (a != 1)):
        raise ValueError("a must be a non-empty 0/1 matrix [N, F]")
    aat = a @ a.T
    ab = a.sum(axis=1)
    h_sigma = aat.sum(axis=1) / 2.0 - ab                       # Eq. (HChi)
    iu, ju = np.triu_indices(a.shape[0], k=1)
    keep = aat[iu, ju] != 0
    edges = np.stack([iu[keep], ju[keep]], axis=1).astype(np.int32)
    J = aat[iu, ju][keep] / 2.0                                # Eq. (HCJij)
    C = (a.shape[1] + aat[iu, ju].sum() / 2.0
         + (np.diag(aat) - 2 * ab).sum() / 2.0)                # Eq. (HCC)
    return -h_sigma, edges, J, float(C)


def rescale_factor(h, J) -> float:
    """r of Eq. (rescale) for fields h and couplings J (the same in either
    spin convention: the h terms use the largest field over h_max and the
    smallest over h_min = -h_max)."""
    h = np.asarray(h, dtype=np.float64)
    J = np.asarray(J, dtype=np.float64)
    terms = [0.0]
    if h.size:
        terms += [h.max() / H_MAX, h.min() / -H_MAX]
    if J.size:
        terms += [J.max() / J_MAX, J.min() / -J_MAX]
    return float(max(terms))

"""CPU oracle for the QAOA / AQA hot path (arXiv 2104.03293).

TEST INFRASTRUCTURE ONLY.  The functions here are the plain, slow reference
that the CUDA path is checked against.  Only the test-suite, the smoke check
and the CPU-baseline leg of ``bench.py`` may import this package; the product
library never calls it and shares no code with it.

The numerical work is in ``oracle.c`` (complex128, gate by gate, see its
header for the equations it follows).  This module compiles it with the host
C compiler on first use, wraps it with ctypes, and adds the few host-side
formulas that are plain algebra:

* the first-order AQA angle map, the linear schedule A(s) = 1 - s, B(s) = s
  with gamma_k = tau * B(s_k) and beta_k = -tau * A(s_k).  The sign follows
  Eqs. (beta_k)-(gamma_k): the annealing driver is H_I = -H_D (Eq. HI), so a
  step of the annealing Hamiltonian contributes e^{+i tau A H_D}, i.e. a
  negative beta;
* the paper's second-order map, Eqs. (beta_k)-(gamma_k) verbatim;
* the chain rule from (dgamma, dbeta) to (dtau, ds_k) for both maps;
* the per-layer spin expectations <Z_i> recorded during AQA (in ``oracle.c``);
* quantum spin dynamics by the product formula of Eq. (AQA4), step by step,
  with exact single-spin x + z exponentials (in ``oracle.c``);
* a float64 Adam step (bias-corrected) used to drive oracle gradients;
* the exact-cover objective of Eq. (exactcover) from its definition, over
  all assignments (the pin of the exact-cover to Ising mapping).

Every function works on the instance fields ``n, h, edges, J`` as produced by
``paper_2104_03293_gb300.instances`` (the shared seeded input generator).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (OpenMP if available)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    cc = os.environ.get("CC", "gcc")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.c_double
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.orc_cost.restype = D
        lib.orc_cost.argtypes = [I, P, I, P, P, ctypes.c_uint64]
        lib.orc_cost_all.argtypes = [I, P, I, P, P, P]
        lib.orc_ground.argtypes = [I, P, I, P, P, P, P, P, P]
        lib.orc_init_plus.argtypes = [I, P]
        lib.orc_gate_z.argtypes = [I, P, I, D]
        lib.orc_gate_zz.argtypes = [I, P, I, I, D]
        lib.orc_gate_x.argtypes = [I, P, I, D]
        lib.orc_layer.argtypes = [I, P, P, I, P, P, D, D]
        lib.orc_evolve.argtypes = [I, P, P, I, P, P, I, P, P, I]
        lib.orc_readout.argtypes = [I, P, P, I, P, P, D, P, P, P]
        lib.orc_adjoint.argtypes = [I, P, I, P, P, I, P, P, I, D, P, P, P, P, P]
        lib.orc_zexp.argtypes = [I, P, P]
        lib.orc_evolve_zexp.argtypes = [I, P, P, I, P, P, I, P, P, P]
        lib.orc_gate_u.argtypes = [I, P, I, P]
        lib.orc_qsds_evolve.argtypes = [I, P, P, I, P, P, I, D, P, P]
        lib.orc_set_threads.argtypes = [I]
        lib.orc_num_threads.restype = I
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fields(inst):
    h = np.ascontiguousarray(inst.h, dtype=np.float64)
    e = np.ascontiguousarray(inst.edges, dtype=np.int32).reshape(-1, 2)
    J = np.ascontiguousarray(inst.J, dtype=np.float64)
    assert h.shape == (inst.n,) and J.shape == (e.shape[0],)
    return h, e, J


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(t: int) -> None:
    """Number of host threads of the oracle's OpenMP loops (t >= 1)."""
    _load().orc_set_threads(int(t))


def cost(inst, z: int) -> float:
    """C(z) of Eq. (HC) for one basis state."""
    h, e, J = _fields(inst)
    return float(_load().orc_cost(inst.n, _ptr(h), e.shape[0], _ptr(e), _ptr(J), int(z)))


def cost_all(inst) -> np.ndarray:
    """C(z) for all 2^n basis states (float64)."""
    h, e, J = _fields(inst)
    out = np.empty(1 << inst.n, dtype=np.float64)
    _load().orc_cost_all(inst.n, _ptr(h), e.shape[0], _ptr(e), _ptr(J), _ptr(out))
    return out


def ground(inst):
    """(cmin, cmax, argmin, count) by enumeration of all 2^n basis states."""
    h, e, J = _fields(inst)
    cmin = np.zeros(1); cmax = np.zeros(1)
    arg = np.zeros(1, dtype=np.int64); cnt = np.zeros(1, dtype=np.int64)
    _load().orc_ground(inst.n, _ptr(h), e.shape[0], _ptr(e), _ptr(J),
                       _ptr(cmin), _ptr(cmax), _ptr(arg), _ptr(cnt))
    return float(cmin[0]), float(cmax[0]), int(arg[0]), int(cnt[0])


def exact_cover_cost_all(a) -> np.ndarray:
    """The exact-cover objective of Eq. (exactcover), sum over the F columns
    of (sum_i a_if x_i - 1)^2, for every x in {0,1}^N (x_i = bit i of the
    basis index), written out from its definition (int64)."""
    a = np.asarray(a, dtype=np.int64)
    N, F = a.shape
    z = np.arange(1 << N, dtype=np.int64)
    x = (z[:, None] >> np.arange(N, dtype=np.int64)[None, :]) & 1     # [2^N, N]
    covered = x @ a                                                   # [2^N, F]
    return ((covered - 1) ** 2).sum(axis=1)


def plus_state(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().orc_init_plus(n, _ptr(psi))
    return psi


def gate_z(psi, n, i, theta):
    _load().orc_gate_z(n, _ptr(psi), i, float(theta))


def gate_zz(psi, n, i, j, theta):
    _load().orc_gate_zz(n, _ptr(psi), i, j, float(theta))


def gate_x(psi, n, j, beta):
    _load().orc_gate_x(n, _ptr(psi), j, float(beta))


def evolve(inst, gamma, beta, psi=None) -> np.ndarray:
    """|beta, gamma> of Eq. (QAOA_state), starting from |+>^n (or from psi)."""
    h, e, J = _fields(inst)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    assert g.shape == b.shape
    from_plus = psi is None
    if psi is None:
        psi = np.empty(1 << inst.n, dtype=np.complex128)
    else:
        assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << inst.n
    _load().orc_evolve(inst.n, _ptr(psi), _ptr(h), e.shape[0], _ptr(e), _ptr(J),
                       g.size, _ptr(g), _ptr(b), int(from_plus))
    return psi


def readout(inst, psi, cmin=None):
    """(E, P_ground, norm) of a state; the ground set is all minimal-cost z."""
    h, e, J = _fields(inst)
    if cmin is None:
        cmin = ground(inst)[0]
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    E = np.zeros(1); P = np.zeros(1); nrm = np.zeros(1)
    _load().orc_readout(inst.n, _ptr(psi), _ptr(h), e.shape[0], _ptr(e), _ptr(J), float(cmin),
                        _ptr(E), _ptr(P), _ptr(nrm))
    return float(E[0]), float(P[0]), float(nrm[0])


def gate_u(n, psi, j, u) -> np.ndarray:
    """Apply the 2 x 2 matrix u (complex, [[u00, u01], [u10, u11]]) to qubit j
    of psi in place (Eq. twocomponentupdates with a general matrix)."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(4).view(np.float64))
    _load().orc_gate_u(n, _ptr(psi), int(j), _ptr(uu))
    return psi


def qsds_evolve(inst, tau, A, B) -> np.ndarray:
    """The second-order product formula of Eq. (AQA4), step by step from
    |+>^n, with the fields of Eq. (AQA3): per step S(tau/2) Z(tau) S(tau/2),
    S = exp[i tau/2 sum_i (A_l X_i - B_l h_i Z_i)], Z = exp[-i tau B_l sum J Z Z]."""
    h, e, J = _fields(inst)
    a = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(B, dtype=np.float64)
    assert a.shape == b.shape
    psi = np.empty(1 << inst.n, dtype=np.complex128)
    _load().orc_qsds_evolve(inst.n, _ptr(psi), _ptr(h), e.shape[0], _ptr(e), _ptr(J), a.size, float(tau),
                            _ptr(a), _ptr(b))
    return psi


def zexp(inst, psi) -> np.ndarray:
    """<Z_i> = sum_z |psi_z|^2 s_i(z) for every qubit i of one state."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(inst.n)
    _load().orc_zexp(inst.n, _ptr(psi), _ptr(out))
    return out


def evolve_zexp(inst, gamma, beta) -> np.ndarray:
    """<Z_i> after every layer of Eq. (QAOA_state) from |+>^n: array [p, n]
    (the spin expectation values recorded during AQA, Sec. III.B.2, Fig. 6)."""
    h, e, J = _fields(inst)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    assert g.shape == b.shape
    psi = np.empty(1 << inst.n, dtype=np.complex128)
    out = np.zeros((g.size, inst.n))
    _load().orc_evolve_zexp(inst.n, _ptr(psi), _ptr(h), e.shape[0], _ptr(e), _ptr(J),
                            g.size, _ptr(g), _ptr(b), _ptr(out))
    return out


def expect(inst, gamma, beta):
    """(E, P_ground) of |beta, gamma>."""
    E, P, _ = readout(inst, evolve(inst, gamma, beta))
    return E, P


def adjoint(inst, gamma, beta, objective: int = 0, cmin=None):
    """(F, dF/dgamma, dF/dbeta) with F = <H_C> (objective 0) or P_ground (1)."""
    h, e, J = _fields(inst)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    if cmin is None:
        cmin = ground(inst)[0]
    N = 1 << inst.n
    psi = np.empty(N, dtype=np.complex128)
    lam = np.empty(N, dtype=np.complex128)
    val = np.zeros(1)
    dg = np.zeros(g.size); db = np.zeros(g.size)
    _load().orc_adjoint(inst.n, _ptr(h), e.shape[0], _ptr(e), _ptr(J), g.size, _ptr(g), _ptr(b),
                        int(objective), float(cmin), _ptr(psi), _ptr(lam), _ptr(val), _ptr(dg), _ptr(db))
    return float(val[0]), dg, db


# ---------------------------------------------------------------------------
# Host-side algebra: AQA angle maps, chain rule, Adam
# ---------------------------------------------------------------------------

def aqa_angles(tau: float, s) -> tuple:
    """First-order AQA on the linear schedule A(s) = 1 - s, B(s) = s.

    gamma_k = tau * B(s_k) and beta_k = -tau * A(s_k): one first-order
    Trotter step of H(s) = A(s) H_I + B(s) H_C (Eqs. HI, Hofs) with
    H_I = -H_D, so the driver factor is e^{+i tau A(s_k) H_D}."""
    s = np.asarray(s, dtype=np.float64)
    return tau * s, -tau * (1.0 - s)


def aqa_chain(tau: float, s, dgamma, dbeta):
    """(dF/dtau, dF/ds_k) for the map of ``aqa_angles``."""
    s = np.asarray(s, dtype=np.float64)
    dg = np.asarray(dgamma, dtype=np.float64)
    db = np.asarray(dbeta, dtype=np.float64)
    dtau = float(np.sum(dg * s - db * (1.0 - s)))
    ds = tau * (dg + db)
    return dtau, ds


def aqa_angles_second_order(tau: float, s) -> tuple:
    """Eqs. (beta_k)-(gamma_k) with A(s) = 1 - s, B(s) = s:
    beta_k = -tau (A(s_{k+1}) + A(s_k)) / 2 for k < p, beta_p = -tau A(s_p) / 2,
    gamma_k = tau B(s_k)."""
    s = np.asarray(s, dtype=np.float64)
    A = 1.0 - s
    beta = np.empty_like(s)
    beta[:-1] = -tau * (A[1:] + A[:-1]) / 2.0
    beta[-1] = -tau * A[-1] / 2.0
    return tau * s, beta


def aqa_chain_second_order(tau: float, s, dgamma, dbeta):
    """(dF/dtau, dF/ds_k) for the map of ``aqa_angles_second_order``.

    Written from that map term by term: gamma_k = tau s_k gives s_k dF/dgamma_k
    to dtau and tau dF/dgamma_k to ds_k; beta_k = -tau (A(s_{k+1}) + A(s_k)) / 2
    (k < p) and beta_p = -tau A(s_p) / 2 give beta_k / tau dF/dbeta_k to dtau
    and, with dA/ds = -1, tau / 2 dF/dbeta_k to ds_k and to ds_{k+1}."""
    s = np.asarray(s, dtype=np.float64)
    dg = np.asarray(dgamma, dtype=np.float64)
    db = np.asarray(dbeta, dtype=np.float64)
    p = s.size
    A = 1.0 - s
    dtau = 0.0
    ds = np.zeros(p)
    for k in range(p):
        dtau += s[k] * dg[k]
        ds[k] += tau * dg[k]
        if k + 1 < p:
            dtau += -(A[k + 1] + A[k]) / 2.0 * db[k]
            ds[k] += tau / 2.0 * db[k]
            ds[k + 1] += tau / 2.0 * db[k]
        else:
            dtau += -A[k] / 2.0 * db[k]
            ds[k] += tau / 2.0 * db[k]
    return float(dtau), ds


def adam_step(theta, grad, m, v, t, lr=0.01, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (minimisation); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v

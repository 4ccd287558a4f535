"""Python binding of the C ABI in include/qs.h (ctypes, marshalling only).

Every numerical step runs in libqs.so.  PyTorch only supplies device memory
(optional caller-owned state buffers) and the current CUDA stream.  If the
library has not been built, or no CUDA device is present, the calls raise:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional, Sequence

import numpy as np

from .build import INCLUDE, LIB

QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_ENOTINT, QS_ESTATE = range(7)
QS_C64, QS_C128 = 0, 1
QS_OBJ_ENERGY, QS_OBJ_GROUND = 0, 1
QS_PATH_TILED, QS_PATH_PLAIN = 0, 1
PLAN_RULE_INTS = 8  # QS_PLAN_RULE_INTS
MIN_PHYS_QUBITS = 13

_STATUS = {0: "QS_OK", 1: "QS_EINVAL", 2: "QS_ENOMEM", 3: "QS_ECUDA", 4: "QS_ETIMEOUT", 5: "QS_ENOTINT",
           6: "QS_ESTATE"}


class QSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI = ctypes.POINTER(ctypes.c_int)
_PI32 = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "qs_create": [ctypes.POINTER(_P), _I, _I, _P, _P, ctypes.c_size_t],
    "qs_destroy": [_P],
    "qs_set_path": [_P, _I],
    "qs_set_ising": [_P, _PD, _I, _PI32, _PD],
    "qs_evolve": [_P, _I, _PD, _PD, _I],
    "qs_expect": [_P, _PD],
    "qs_ground_prob": [_P, _PD, _PI64, _PI64, _PI64],
    "qs_readout": [_P, _PD, _PD, _PD],
    "qs_cost_info": [_P, _PI64, _PI64, _PI64, _PI64, _PI],
    "qs_enumerate_noalloc": [_I, _PD, _I, _PI32, _PD, _P, _PI64, _PI64, _PI64, _PI64, _PI],
    "qs_set_shape_rule": [_P, _I, _I],
    "qs_autotune": [_P, _I, _PI, _PI, _PD],
    "qs_set_plan_rule": [_P, _PI],
    "qs_get_plan_rule": [_P, _PI],
    "qs_autotune_ex": [_P, _I, _I, _PI, _PI, _PD, _PI, _PD],
    "qs_batch_set_launch_rule": [_P, _I, ctypes.c_int64],
    "qs_batch_autotune": [_P, _PI, _PI64, _PD],
    "qs_grad": [_P, _I, _PD, _PD, _I, _PD, _PD, _PD],
    "qs_evolve_zexp": [_P, _I, _PD, _PD, _PD],
    "qs_evolve_su2": [_P, _I, _PD, _PD],
    "qs_qsds_layers": [_I, _I, _D, _PD, _PD, _PD, _PD, _PD],
    "qs_set_adjoint_buffer": [_P, _P, ctypes.c_size_t],
    "qs_copy_state": [_P, _P, ctypes.c_size_t],
    "qs_state_ptr": [_P, ctypes.POINTER(_P), _PI],
    "qs_canonicalize": [_P],
    "qs_plan_info": [_P, _I, _PI, _PI],
    "qs_plan_sweeps": [_I, _I, _I, _PI, _PI],
    "qs_aqa_angles": [_I, _D, _PD, _PD, _PD],
    "qs_aqa_angles_2nd": [_I, _D, _PD, _PD, _PD],
    "qs_aqa_chain": [_I, _D, _PD, _PD, _PD, _PD, _PD],
    "qs_aqa_chain_2nd": [_I, _D, _PD, _PD, _PD, _PD, _PD],
    "qs_launch_count": [_PI64],
    "qs_plan_shape": [_I, _I, _I, _PI, _PI, _PI, _PI, _PI, _PI],
    "qs_pair_tile_map": [_I, _I, _I, _I, _I, _I, _PI, _PI, _PI, _PI, _PI, _PI],
    "qs_last_error": [],
    "qs_version": [],
    "qs_batch_create": [ctypes.POINTER(_P), _I, _PI, _I, _P],
    "qs_batch_set_ising": [_P, _I, _PD, _I, _PI32, _PD],
    "qs_batch_evolve": [_P, _PI, _PI64, _PD, _PD],
    "qs_batch_results": [_P, _PD, _PD],
    "qs_batch_grad": [_P, _I, _PD, _PD, _PD],
    "qs_batch_adam": [_P, _I, _D, _D, _D, _D, _PD, _PD, _I],
    "qs_batch_destroy": [_P],
    "qs_batch_test_withhold": [_P, _I, _D],
    "qs_batch_partition": [_I, _PI, _PI, _I, _PI, _PD],
}


def _tune_key(n: int, dtype: int) -> str:
    """Autotuner cache key: GPU model, SM count, n and dtype."""
    name, sms = "gpu", 0
    try:
        import torch
        if torch.cuda.is_available():
            pr = torch.cuda.get_device_properties(torch.cuda.current_device())
            name, sms = pr.name, pr.multi_processor_count
    except Exception:
        pass
    return f"{name}|sm{sms}|n{n}|{'c64' if dtype == QS_C64 else 'c128'}"


def header_functions() -> list[str]:
    """Names of every function declared in include/qs.h."""
    txt = open(os.path.join(INCLUDE, "qs.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(qs_\w+)\s*\(", txt, flags=re.M)))


def lib():
    """Load libqs.so (raises if it is missing: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_2104_03293_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("qs_last_error", "qs_version") else _I
        _lib = L
        return L


def _check(rc: int):
    if rc != QS_OK:
        raise QSError(rc, lib().qs_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream or None
        except Exception:
            return None
        return None
    if isinstance(stream, int):
        return stream or None
    return getattr(stream, "cuda_stream", None) or None


def _ising_arrays(n: int, h, edges, J):
    """Contiguous (h, edges, J) for the C calls, with the lengths the C side
    reads checked here: h has n entries and J one per edge."""
    h = _f64(h)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    J = _f64(J)
    if h.ndim != 1 or h.size != n:
        raise ValueError(f"h has {h.size} entries, expected {n}")
    if J.ndim != 1 or J.size != e.shape[0]:
        raise ValueError(f"J has {J.size} entries for {e.shape[0]} edges")
    return h, e, J


def _angles(gamma, beta):
    g, b = _f64(np.atleast_1d(gamma)), _f64(np.atleast_1d(beta))  # a scalar is one layer
    if g.ndim != 1 or g.shape != b.shape:
        raise ValueError("gamma and beta must be 1-D and of the same length")
    return g, b


def phys_qubits(n: int) -> int:
    return max(n, MIN_PHYS_QUBITS)


class State:
    """An n-qubit state on the GPU (qs_create / qs_destroy)."""

    def __init__(self, n: int, dtype: str = "c64", stream=None, buffer=None):
        self.n = int(n)
        if dtype in ("c64", "complex64", QS_C64):
            self.dtype = QS_C64
        elif dtype in ("c128", "complex128", QS_C128):
            self.dtype = QS_C128
        else:
            raise ValueError(f"dtype {dtype!r}: expected 'c64' or 'c128'")
        self.elem = 8 if self.dtype == QS_C64 else 16
        self._buffer = buffer  # keep a caller tensor alive
        self._adj = None
        ptr, nbytes = None, 0
        if buffer is not None:
            ptr = buffer.data_ptr()
            nbytes = buffer.numel() * buffer.element_size()
        h = _P()
        _check(lib().qs_create(ctypes.byref(h), self.n, self.dtype, _stream_ptr(stream), ptr, nbytes))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_path(self, path: int):
        _check(lib().qs_set_path(self._h, int(path)))

    def set_ising(self, h, edges, J):
        h, e, J = _ising_arrays(self.n, h, edges, J)
        _check(lib().qs_set_ising(self._h, _dptr(h), int(e.shape[0]), e.ctypes.data_as(_PI32), _dptr(J)))

    def set_instance(self, inst):
        self.set_ising(inst.h, inst.edges, inst.J)

    def evolve(self, gamma, beta, from_plus: bool = True):
        g, b = _angles(gamma, beta)
        _check(lib().qs_evolve(self._h, int(g.size), _dptr(g), _dptr(b), int(bool(from_plus))))

    def evolve_zexp(self, gamma, beta) -> np.ndarray:
        """Evolve from |+>^n and return <Z_i> after every layer, array [p, n]."""
        g, b = _angles(gamma, beta)
        out = np.zeros((g.size, self.n))
        _check(lib().qs_evolve_zexp(self._h, int(g.size), _dptr(g), _dptr(b), _dptr(out)))
        return out

    def evolve_su2(self, gamma, u):
        """Layers exp(-i gamma_k H_C) then per-qubit 2 x 2 matrices u[k, i]
        (complex array [p, n, 2, 2]) from |+>^n."""
        g = _f64(np.atleast_1d(gamma))
        uu = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(g.size, self.n, 2, 2))
        flat = np.ascontiguousarray(uu.reshape(-1).view(np.float64))
        _check(lib().qs_evolve_su2(self._h, int(g.size), _dptr(g), _dptr(flat)))

    def readout(self):
        E, P, N = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().qs_readout(self._h, ctypes.byref(E), ctypes.byref(P), ctypes.byref(N)))
        return E.value, P.value, N.value

    def expect(self) -> float:
        E = ctypes.c_double()
        _check(lib().qs_expect(self._h, ctypes.byref(E)))
        return E.value

    def ground_prob(self):
        P = ctypes.c_double()
        a, c, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().qs_ground_prob(self._h, ctypes.byref(P), ctypes.byref(a), ctypes.byref(c), ctypes.byref(k)))
        return P.value, a.value, c.value, k.value

    def cost_info(self):
        vals = [ctypes.c_int64() for _ in range(4)]
        s = ctypes.c_int()
        _check(lib().qs_cost_info(self._h, *[ctypes.byref(v) for v in vals], ctypes.byref(s)))
        return tuple(v.value for v in vals) + (s.value,)

    def set_shape_rule(self, runs_a: int = -1, split: int = -1):
        _check(lib().qs_set_shape_rule(self._h, int(runs_a), int(split)))

    def autotune(self, p_trial: int = 2):
        """Time the candidate tile-shape plans, keep the fastest: (runs_a, split, ms)."""
        r, sp, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().qs_autotune(self._h, int(p_trial), ctypes.byref(r), ctypes.byref(sp), ctypes.byref(ms)))
        return r.value, sp.value, ms.value

    def plan_rule(self) -> tuple:
        """(runs_a, split, cmin, ctas_per_sm, pair_cluster, pair_tma, pair_l2,
        order) of the handle."""
        v = (ctypes.c_int * PLAN_RULE_INTS)()
        _check(lib().qs_get_plan_rule(self._h, v))
        return tuple(v)

    def set_plan_rule(self, rule):
        """Set a plan rule; a shorter rule keeps the remaining fields at their
        defaults (cp.async tile loads, default L2 fetch size, planned order
        of the strided shapes)."""
        r = [int(x) for x in rule]
        if len(r) > PLAN_RULE_INTS or len(r) < 5:
            raise ValueError(f"a plan rule has 5 to {PLAN_RULE_INTS} ints")
        r += [0] * (PLAN_RULE_INTS - len(r))
        v = (ctypes.c_int * PLAN_RULE_INTS)(*r)
        _check(lib().qs_set_plan_rule(self._h, v))

    def autotune_plan(self, p_trial: int = 2, cache: Optional[str] = None):
        """Search the plan rules (qs_autotune_ex) and keep the fastest.  Returns
        (rule, ms, candidates) with candidates a list of (rule, ms).  With a
        JSON cache file (argument or QS_TUNE_CACHE), a rule stored for this
        GPU model, SM count, n and dtype is applied without timing, and a new
        search is stored there."""
        cache = cache or os.environ.get("QS_TUNE_CACHE")
        key = _tune_key(self.n, self.dtype)
        if cache and os.path.exists(cache):
            import json
            with open(cache) as f:
                entry = json.load(f).get(key)
            if entry and len(entry["rule"]) == PLAN_RULE_INTS:
                self.set_plan_rule(entry["rule"])
                return tuple(entry["rule"]), float(entry["ms"]), [(tuple(r), m) for r, m in entry["candidates"]]
        cap, k = 64, PLAN_RULE_INTS
        rules, ms_c = (ctypes.c_int * (k * cap))(), (ctypes.c_double * cap)()
        best, nc, ms = (ctypes.c_int * k)(), ctypes.c_int(), ctypes.c_double()
        _check(lib().qs_autotune_ex(self._h, int(p_trial), cap, ctypes.byref(nc), rules, ms_c, best, ctypes.byref(ms)))
        cands = [(tuple(rules[k * i:k * i + k]), ms_c[i]) for i in range(min(nc.value, cap))]
        if cache:
            import json
            data = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    data = json.load(f)
            data[key] = {"rule": list(best), "ms": ms.value, "p_trial": int(p_trial),
                         "candidates": [[list(r), m] for r, m in cands]}
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1)
            os.replace(tmp, cache)
        return tuple(best), ms.value, cands

    def set_adjoint_buffer(self, buffer):
        self._adj = buffer
        ptr = None if buffer is None else buffer.data_ptr()
        nbytes = 0 if buffer is None else buffer.numel() * buffer.element_size()
        _check(lib().qs_set_adjoint_buffer(self._h, ptr, nbytes))

    def grad(self, gamma, beta, objective: int = QS_OBJ_ENERGY):
        g, b = _angles(gamma, beta)
        dg, db = np.zeros_like(g), np.zeros_like(b)
        v = ctypes.c_double()
        _check(lib().qs_grad(self._h, int(g.size), _dptr(g), _dptr(b), int(objective), ctypes.byref(v), _dptr(dg),
                             _dptr(db)))
        return v.value, dg, db

    def copy_state(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == QS_C64 else np.complex128)
        _check(lib().qs_copy_state(self._h, out.ctypes.data_as(_P), out.nbytes))
        return out

    def state_ptr(self):
        p, f = _P(), ctypes.c_int()
        _check(lib().qs_state_ptr(self._h, ctypes.byref(p), ctypes.byref(f)))
        return p.value, f.value

    def canonicalize(self):
        _check(lib().qs_canonicalize(self._h))

    def plan_info(self, p: int):
        s, w = ctypes.c_int(), ctypes.c_int()
        _check(lib().qs_plan_info(self._h, int(p), ctypes.byref(s), ctypes.byref(w)))
        return s.value, w.value


def enumerate_noalloc(h, edges, J, cuda_stream=None):
    """qs_enumerate_noalloc: (cmin, cmax, argmin, ground_count, shift) of the
    Ising cost, computed with the library's static device scratch."""
    h, e, J = _ising_arrays(np.asarray(h).size, h, edges, J)
    vals = [ctypes.c_int64() for _ in range(4)]
    s = ctypes.c_int()
    _check(lib().qs_enumerate_noalloc(int(h.size), _dptr(h), int(e.shape[0]), e.ctypes.data_as(_PI32), _dptr(J),
                                      _stream_ptr(cuda_stream),
                                      *[ctypes.byref(v) for v in vals], ctypes.byref(s)))
    return tuple(v.value for v in vals) + (s.value,)


def plan_sweeps(n: int, p: int, dtype: int = QS_C64):
    """(tile shapes, HBM sweeps for p layers) of the tiled path (host only)."""
    s, w = ctypes.c_int(), ctypes.c_int()
    _check(lib().qs_plan_sweeps(int(n), int(dtype), int(p), ctypes.byref(s), ctypes.byref(w)))
    return s.value, w.value


def plan_shapes(n: int, dtype: int = QS_C64):
    """Tile shapes of the tiled path: list of dicts (kind, K, c, g0, n1, g1)."""
    out = []
    for k in range(8):
        vals = [ctypes.c_int() for _ in range(6)]
        rc = lib().qs_plan_shape(int(n), int(dtype), k, *[ctypes.byref(v) for v in vals])
        if rc != QS_OK:
            break
        out.append(dict(zip(("kind", "K", "c", "g0", "n1", "g1"), (v.value for v in vals))))
    return out


def pair_tile_map(n: int, c: int, g0: int, n1: int, g1: int, g: int):
    """Tensor-map view of a strided complex64 tile shape for a first read into
    layout g (host only): dict(rank, kbit, start, width, box, landing), or
    None when the shape does not fit a five-dimensional box."""
    rank, kbit = ctypes.c_int(), ctypes.c_int()
    arr = [(ctypes.c_int * 5)() for _ in range(3)]
    land = (ctypes.c_int * 13)()
    rc = lib().qs_pair_tile_map(int(n), int(c), int(g0), int(n1), int(g1), int(g), ctypes.byref(rank),
                                ctypes.byref(kbit), arr[0], arr[1], arr[2], land)
    if rc != QS_OK:
        return None
    r = rank.value
    return {"rank": r, "kbit": kbit.value, "start": list(arr[0])[:r], "width": list(arr[1])[:r],
            "box": list(arr[2])[:r], "landing": list(land)}


def aqa_angles(tau: float, s) -> tuple:
    s = _f64(s)
    g, b = np.zeros_like(s), np.zeros_like(s)
    _check(lib().qs_aqa_angles(int(s.size), float(tau), _dptr(s), _dptr(g), _dptr(b)))
    return g, b


def qsds_layers(n: int, tau: float, A, B, hfield):
    """(gamma [nsteps + 1], u [nsteps + 1, n, 2, 2]) reproducing the product
    formula of Eq. (AQA4) with evolve_su2 (host)."""
    a, b, h = _f64(A), _f64(B), _f64(hfield)
    assert a.shape == b.shape and h.shape == (n,)
    g = np.zeros(a.size + 1)
    flat = np.zeros((a.size + 1) * n * 8)
    _check(lib().qs_qsds_layers(int(n), int(a.size), float(tau), _dptr(a), _dptr(b), _dptr(h), _dptr(g), _dptr(flat)))
    return g, flat.view(np.complex128).reshape(a.size + 1, n, 2, 2)


def aqa_angles_2nd(tau: float, s) -> tuple:
    s = _f64(s)
    g, b = np.zeros_like(s), np.zeros_like(s)
    _check(lib().qs_aqa_angles_2nd(int(s.size), float(tau), _dptr(s), _dptr(g), _dptr(b)))
    return g, b


def aqa_chain(tau: float, s, dgamma, dbeta):
    s, dg, db = _f64(s), _f64(dgamma), _f64(dbeta)
    ds = np.zeros_like(s)
    dt = ctypes.c_double()
    _check(lib().qs_aqa_chain(int(s.size), float(tau), _dptr(s), _dptr(dg), _dptr(db), ctypes.byref(dt), _dptr(ds)))
    return dt.value, ds


def aqa_chain_2nd(tau: float, s, dgamma, dbeta):
    """(dF/dtau, dF/ds_k) under the second-order map of aqa_angles_2nd."""
    s, dg, db = _f64(s), _f64(dgamma), _f64(dbeta)
    ds = np.zeros_like(s)
    dt = ctypes.c_double()
    _check(lib().qs_aqa_chain_2nd(int(s.size), float(tau), _dptr(s), _dptr(dg), _dptr(db), ctypes.byref(dt),
                                  _dptr(ds)))
    return dt.value, ds


def version() -> str:
    return lib().qs_version().decode()


def launch_count() -> int:
    """Kernels launched by libqs.so in this process so far."""
    c = ctypes.c_int64()
    _check(lib().qs_launch_count(ctypes.byref(c)))
    return c.value


class Batch:
    """Independent instances evolved together (qs_batch_*)."""

    def __init__(self, ns: Sequence[int], stream=None):
        n = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
        self.count = int(n.size)
        self.ns = n
        h = _P()
        _check(lib().qs_batch_create(ctypes.byref(h), self.count, n.ctypes.data_as(_PI), QS_C64, _stream_ptr(stream)))
        self._h = h
        self.p = None
        self.off = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_ising(self, idx: int, h, edges, J):
        if not 0 <= int(idx) < self.count:
            raise ValueError(f"instance index {idx} out of range [0, {self.count})")
        h, e, J = _ising_arrays(int(self.ns[int(idx)]), h, edges, J)
        _check(lib().qs_batch_set_ising(self._h, int(idx), _dptr(h), int(e.shape[0]), e.ctypes.data_as(_PI32),
                                        _dptr(J)))

    def _layout(self, gammas, betas=None):
        if len(gammas) != self.count or (betas is not None and len(betas) != self.count):
            raise ValueError(f"expected one angle list per instance ({self.count})")
        if betas is not None and any(len(g) != len(b) for g, b in zip(gammas, betas)):
            raise ValueError("gamma and beta lists differ in length for some instance")
        p = np.ascontiguousarray(np.asarray([len(g) for g in gammas], dtype=np.int32))
        off = np.zeros(self.count, dtype=np.int64)
        off[1:] = np.cumsum(p[:-1])
        return p, off

    def evolve(self, gammas, betas):
        p, off = self._layout(gammas, betas)
        g = _f64(np.concatenate([np.asarray(x, dtype=np.float64) for x in gammas]) if p.sum() else np.zeros(1))
        b = _f64(np.concatenate([np.asarray(x, dtype=np.float64) for x in betas]) if p.sum() else np.zeros(1))
        self.p, self.off = p, off
        _check(lib().qs_batch_evolve(self._h, p.ctypes.data_as(_PI), off.ctypes.data_as(_PI64), _dptr(g), _dptr(b)))

    def results(self):
        E, P = np.zeros(self.count), np.zeros(self.count)
        _check(lib().qs_batch_results(self._h, _dptr(E), _dptr(P)))
        return E, P

    def _split(self, flat):
        return [flat[o:o + k].copy() for o, k in zip(self.off, self.p)]

    def grad(self, objective: int = QS_OBJ_ENERGY):
        if self.p is None:
            raise QSError(QS_ESTATE, "Batch.grad: evolve the batch first (it fixes each instance's angles)")
        tot = int(self.p.sum())
        v = np.zeros(self.count)
        dg, db = np.zeros(max(tot, 1)), np.zeros(max(tot, 1))
        _check(lib().qs_batch_grad(self._h, int(objective), _dptr(v), _dptr(dg), _dptr(db)))
        return v, self._split(dg), self._split(db)

    def set_launch_rule(self, ctas_per_sm: int = 0, window_bytes: int = 0):
        _check(lib().qs_batch_set_launch_rule(self._h, int(ctas_per_sm), int(window_bytes)))

    def autotune(self):
        """Time the queue's launch rules on the last evolve's angles, keep the
        fastest: (ctas_per_sm, window_bytes, ms).  A new evolve is needed
        before results()."""
        c, w, ms = ctypes.c_int(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().qs_batch_autotune(self._h, ctypes.byref(c), ctypes.byref(w), ctypes.byref(ms)))
        return c.value, w.value, ms.value

    def test_withhold(self, idx: int, wait_limit_s: float):
        """Failure-detection test: the next evolve withholds one dependency of
        instance idx and gives up after wait_limit_s (results then raise
        QS_ETIMEOUT; the batch stays usable)."""
        _check(lib().qs_batch_test_withhold(self._h, int(idx), float(wait_limit_s)))

    def adam(self, gammas, betas, steps: int, lr=0.01, b1=0.9, b2=0.999, eps=1e-8, use_graph: bool = True):
        if self.p is None:
            raise QSError(QS_ESTATE, "Batch.adam: evolve the batch first (it fixes each instance's p)")
        p, _ = self._layout(gammas, betas)
        if not np.array_equal(p, self.p):
            raise ValueError("Batch.adam: the angle lists must have the lengths of the last evolve")
        g = _f64(np.concatenate([np.asarray(x, dtype=np.float64) for x in gammas]))
        b = _f64(np.concatenate([np.asarray(x, dtype=np.float64) for x in betas]))
        _check(lib().qs_batch_adam(self._h, int(steps), lr, b1, b2, eps, _dptr(g), _dptr(b), int(bool(use_graph))))
        return self._split(g), self._split(b)


def batch_partition(ns, ps, world: int):
    """qs_batch_partition: (rank of each instance, work per rank), the
    greedy longest-first bin-packing of max(p, 1) 2^n over `world` ranks."""
    n = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
    p = np.ascontiguousarray(np.asarray(ps, dtype=np.int32))
    if n.shape != p.shape or n.ndim != 1:
        raise ValueError("ns and ps must be 1-D and of the same length")
    rank_of = np.zeros(n.size, dtype=np.int32)
    load = np.zeros(max(int(world), 1))
    _check(lib().qs_batch_partition(int(n.size), n.ctypes.data_as(_PI), p.ctypes.data_as(_PI), int(world),
                                    rank_of.ctypes.data_as(_PI), _dptr(load)))
    return rank_of, load


def grid_scan(h, edges, J, gammas, betas, stream=None, return_batch: bool = False):
    """p = 1 landscapes of one instance over a (gamma, beta) grid (the
    energy and success-probability maps of Sec. III.B.1, Fig. 4, scanned there
    on 64 x 64 points, beta in [0, pi), gamma in [0, 2 pi)): E and
    P_ground at every point of gammas x betas, from one batched evolve of
    len(gammas) * len(betas) copies of the instance (qs_batch_*), each copy
    with its own p = 1 angles.  Returns two arrays of shape (len(gammas),
    len(betas)); with return_batch, also the evolved Batch (caller closes it).
    Every copy holds its own cost program (built by qs_batch_set_ising)."""
    h = _f64(h)
    gammas = np.asarray(gammas, dtype=np.float64).ravel()
    betas = np.asarray(betas, dtype=np.float64).ravel()
    G, B = gammas.size, betas.size
    if G == 0 or B == 0:
        raise QSError(QS_EINVAL, "grid_scan: empty angle grid")
    bt = Batch([h.size] * (G * B), stream=stream)
    try:
        for i in range(G * B):
            bt.set_ising(i, h, edges, J)
        bt.evolve(np.repeat(gammas, B).reshape(-1, 1), np.tile(betas, G).reshape(-1, 1))
        E, P = bt.results()
    except BaseException:
        bt.close()
        raise
    if return_batch:
        return E.reshape(G, B), P.reshape(G, B), bt
    bt.close()
    return E.reshape(G, B), P.reshape(G, B)


def _torch_energy_function():
    import torch

    class QSEnergy(torch.autograd.Function):
        """F(gamma, beta) = <H_C> or P_ground of a State; backward uses qs_grad."""

        @staticmethod
        def forward(ctx, gamma, beta, state, objective=QS_OBJ_ENERGY):
            g = gamma.detach().cpu().double().numpy()
            b = beta.detach().cpu().double().numpy()
            val, dg, db = state.grad(g, b, objective)
            ctx.save_for_backward(torch.from_numpy(dg).to(gamma.dtype), torch.from_numpy(db).to(beta.dtype))
            return torch.tensor(val, dtype=gamma.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            dg, db = ctx.saved_tensors
            return grad_out * dg, grad_out * db, None, None

    return QSEnergy


def energy(gamma, beta, state: State, objective: int = QS_OBJ_ENERGY):
    """Differentiable objective through torch.autograd (gradients from qs_grad)."""
    return _torch_energy_function().apply(gamma, beta, state, objective)


def _torch_aqa_function():
    import torch

    class QSAqa(torch.autograd.Function):
        """F(tau, s) of the AQA angles (order 1: qs_aqa_angles, order 2:
        qs_aqa_angles_2nd); backward uses qs_grad and the matching chain rule
        (qs_aqa_chain or qs_aqa_chain_2nd)."""

        @staticmethod
        def forward(ctx, tau, s, state, objective=QS_OBJ_ENERGY, order=1):
            t = float(tau.detach().cpu().double())
            sk = s.detach().cpu().double().numpy()
            g, b = aqa_angles(t, sk) if order == 1 else aqa_angles_2nd(t, sk)
            val, dg, db = state.grad(g, b, objective)
            dt, ds = aqa_chain(t, sk, dg, db) if order == 1 else aqa_chain_2nd(t, sk, dg, db)
            ctx.save_for_backward(torch.tensor(dt, dtype=tau.dtype), torch.from_numpy(ds).to(s.dtype))
            return torch.tensor(val, dtype=tau.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            dt, ds = ctx.saved_tensors
            return grad_out * dt, grad_out * ds, None, None, None

    return QSAqa


def aqa_energy(tau, s, state: State, objective: int = QS_OBJ_ENERGY, order: int = 1):
    """Differentiable AQA objective in (tau, schedule knots s_k) through
    torch.autograd, for the first-order map (order 1) or the paper's
    second-order map of Appendix A (order 2)."""
    if order not in (1, 2):
        raise ValueError("order must be 1 or 2")
    return _torch_aqa_function().apply(tau, s, state, objective, order)

"""Plain FP64 CPU oracle of the MR-LBM adaptive step (arXiv 2102.12163).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path never
does.  The C source (``mrlbm_oracle.c``) follows the paper's definitions with
dense per-level arrays; this module only compiles it and marshals numpy arrays.

Parity status: every operator is pinned by a test against a fact the paper or
the mathematics fixes (see ``tests/test_oracle_*.py``).  The vectorial D1Q2^2
shallow-water equilibrium is not printed in the paper (it is built by analogy
with the vectorial Euler scheme of Section 5.3 and the flux of the shallow
water system of Section 5.2); it is pinned by the closed-form flux and by the
convergence of its uniform scheme to the exact entropy solution of the dam
break, not by a value the paper gives.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrlbm_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

BC_PERIODIC, BC_COPY = 0, 1
COLLIDE_LEAVES, COLLIDE_RECONSTRUCTED = 0, 1
EQ_ADVECTION, EQ_BURGERS, EQ_SW, EQ_EULER = 0, 1, 2, 3
EQ_SW_D1Q3, EQ_SW_D1Q5 = 4, 5  # shallow water, one velocity set for h and hu (Section 5.2)
NFIELDS = {EQ_ADVECTION: 1, EQ_BURGERS: 1, EQ_SW: 2, EQ_EULER: 3, EQ_SW_D1Q3: 2, EQ_SW_D1Q5: 2}
NPOP = {EQ_ADVECTION: 2, EQ_BURGERS: 2, EQ_SW: 4, EQ_EULER: 6, EQ_SW_D1Q3: 3, EQ_SW_D1Q5: 5}


def build(force: bool = False) -> str:
    """Compile the oracle with -ffp-contract=off (no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mrlbm_oracle.h"))
    ):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("Jmin", ctypes.c_int), ("Jmax", ctypes.c_int), ("gamma", ctypes.c_int),
        ("mu_bar", ctypes.c_int), ("bc", ctypes.c_int), ("eps", ctypes.c_double),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("eq", ctypes.c_int),
        ("lambda_", ctypes.c_double), ("s", ctypes.c_double * 3), ("eqp", ctypes.c_double),
        ("collision", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp, ucp, ip, lp = P(ctypes.c_double), P(ctypes.c_ubyte), P(ctypes.c_int), P(ctypes.c_long)
        sp = P(_Params)
        sig = {
            "orc_nfields": (ctypes.c_int, [ctypes.c_int]),
            "orc_collide": (None, [ctypes.c_void_p]),
            "orc_npop": (ctypes.c_int, [ctypes.c_int]),
            "orc_create": (ctypes.c_void_p, [sp]),
            "orc_free": (None, [ctypes.c_void_p]),
            "orc_total_cells": (ctypes.c_long, [ctypes.c_void_p]),
            "orc_set_initial": (None, [ctypes.c_void_p, dp]),
            "orc_set_state": (ctypes.c_int, [ctypes.c_void_p, ucp, dp]),
            "orc_get_state": (None, [ctypes.c_void_p, ucp, dp]),
            "orc_adapt": (None, [ctypes.c_void_p]),
            "orc_lbm_step": (None, [ctypes.c_void_p]),
            "orc_step": (None, [ctypes.c_void_p]),
            "orc_lbm_step_uncompacted": (None, [ctypes.c_void_p, dp]),
            "orc_get_trace": (None, [ctypes.c_void_p, dp, ucp, ucp, ucp]),
            "orc_leaves": (ctypes.c_long, [ctypes.c_void_p, ip, lp, dp, ctypes.c_long]),
            "orc_reconstruct_finest": (None, [ctypes.c_void_p, dp]),
            "orc_reconstruct_moments": (None, [ctypes.c_void_p, dp]),
            "orc_mass": (None, [ctypes.c_void_p, dp]),
            "orc_uniform_step": (None, [sp, dp]),
            "orc_equilibrium_populations": (None, [sp, dp, dp, ctypes.c_long]),
            "orc_moments": (None, [sp, dp, dp, ctypes.c_long]),
            "orc_prediction_coefficients": (None, [ctypes.c_int, dp]),
            "orc_predict_level": (None, [ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, dp]),
            "orc_project_level": (None, [dp, ctypes.c_long, dp]),
            "orc_mr_encode": (None, [ctypes.c_int] * 4 + [dp, dp]),
            "orc_mr_decode": (None, [ctypes.c_int] * 4 + [dp, dp]),
            "orc_grade": (None, [ctypes.c_int] * 4 + [ucp]),
            "orc_check_graded": (ctypes.c_int, [ctypes.c_int] * 4 + [ucp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


@dataclass
class Params:
    """Problem parameters in the paper's notation (Sections 2-5)."""

    Jmin: int
    Jmax: int
    eq: int
    lam: float
    eps: float = 1e-4
    gamma: int = 1
    mu_bar: int = 0
    bc: int = BC_PERIODIC
    a: float = -1.0
    b: float = 1.0
    s: tuple = (1.0, 1.0, 1.0)
    eqp: float = 0.0
    collision: int = 0  # 0 leaves collision, 1 reconstructed collision (Section 4.5)
    _c: _Params = field(default=None, repr=False, compare=False)

    def c(self) -> _Params:
        s = list(self.s) + [1.0] * (3 - len(self.s))
        return _Params(self.Jmin, self.Jmax, self.gamma, self.mu_bar, self.bc, self.eps,
                       self.a, self.b, self.eq, self.lam, (ctypes.c_double * 3)(*s[:3]), self.eqp,
                       self.collision)

    @property
    def nf(self) -> int:
        return NFIELDS[self.eq]

    @property
    def q(self) -> int:
        return NPOP[self.eq]


def level_offsets(Jmin: int, Jmax: int) -> list[int]:
    off, o = {}, 0
    for l in range(Jmin, Jmax + 1):
        off[l] = o
        o += 1 << l
    off[Jmax + 1] = o
    return off


class Oracle:
    """One instance of the adaptive scheme on the CPU."""

    def __init__(self, p: Params):
        self.p = p
        self._pc = p.c()
        self._h = lib().orc_create(ctypes.byref(self._pc))
        if not self._h:
            raise ValueError(f"invalid oracle parameters {p}")
        self.S = lib().orc_total_cells(self._h)
        self.off = level_offsets(p.Jmin, p.Jmax)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    # state -----------------------------------------------------------
    def set_initial(self, m_cons: np.ndarray) -> None:
        m = np.ascontiguousarray(m_cons, dtype=np.float64).reshape(self.p.nf, 1 << self.p.Jmax)
        lib().orc_set_initial(self._h, _d(m))

    def set_state(self, R: np.ndarray, values: np.ndarray) -> None:
        R = np.ascontiguousarray(R, dtype=np.uint8)
        v = np.ascontiguousarray(values, dtype=np.float64).reshape(self.p.q, self.S)
        rc = lib().orc_set_state(self._h, _u8(R), _d(v))
        if rc:
            raise ValueError(f"not a graded tree (code {rc})")

    def get_state(self):
        R = np.zeros(self.S, np.uint8)
        v = np.zeros((self.p.q, self.S), np.float64)
        lib().orc_get_state(self._h, _u8(R), _d(v))
        return R, v

    # scheme ----------------------------------------------------------
    def adapt(self) -> None:
        lib().orc_adapt(self._h)

    def collide(self) -> None:
        """The collision phase alone (leaves or reconstructed, per the parameters)."""
        lib().orc_collide(self._h)

    def lbm_step(self) -> None:
        lib().orc_lbm_step(self._h)

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            lib().orc_step(self._h)

    def lbm_step_uncompacted(self) -> np.ndarray:
        out = np.zeros((self.p.q, self.S), np.float64)
        lib().orc_lbm_step_uncompacted(self._h, _d(out))
        return out

    def trace(self):
        D = np.zeros(self.S, np.float64)
        T = np.zeros(self.S, np.uint8)
        H = np.zeros(self.S, np.uint8)
        G = np.zeros(self.S, np.uint8)
        lib().orc_get_trace(self._h, _d(D), _u8(T), _u8(H), _u8(G))
        return D, T, H, G

    def leaves(self):
        n = lib().orc_leaves(self._h, None, None, None, 0)
        lv = np.zeros(n, np.int32)
        ix = np.zeros(n, np.int64)
        f = np.zeros((self.p.q, max(n, 1)), np.float64)
        lib().orc_leaves(self._h, lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         ix.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _d(f), n)
        return lv, ix, f[:, :n]

    def finest(self) -> np.ndarray:
        out = np.zeros((self.p.q, 1 << self.p.Jmax), np.float64)
        lib().orc_reconstruct_finest(self._h, _d(out))
        return out

    def finest_moments(self) -> np.ndarray:
        out = np.zeros((self.p.nf, 1 << self.p.Jmax), np.float64)
        lib().orc_reconstruct_moments(self._h, _d(out))
        return out

    def mass(self) -> np.ndarray:
        out = np.zeros(self.p.nf, np.float64)
        lib().orc_mass(self._h, _d(out))
        return out

    def tree_levels(self, R: np.ndarray | None = None) -> dict:
        if R is None:
            R, _ = self.get_state()
        return {l: R[self.off[l]: self.off[l + 1]].astype(bool) for l in range(self.p.Jmin, self.p.Jmax + 1)}


# free functions --------------------------------------------------------------

def uniform_step(p: Params, f: np.ndarray, n: int = 1) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    pc = p.c()
    for _ in range(n):
        lib().orc_uniform_step(ctypes.byref(pc), _d(f))
    return f


def equilibrium(p: Params, m_cons: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(m_cons, dtype=np.float64)
    n = m.shape[-1]
    f = np.zeros((p.q, n), np.float64)
    pc = p.c()
    lib().orc_equilibrium_populations(ctypes.byref(pc), _d(m.reshape(p.nf, n)), _d(f), n)
    return f


def moments(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.shape[-1]
    m = np.zeros((p.nf, n), np.float64)
    pc = p.c()
    lib().orc_moments(ctypes.byref(pc), _d(f), _d(m), n)
    return m


def prediction_coefficients(gamma: int) -> np.ndarray:
    c = np.zeros(3, np.float64)
    lib().orc_prediction_coefficients(gamma, _d(c))
    return c[:gamma].copy()


def predict_level(gamma: int, bc: int, coarse: np.ndarray) -> np.ndarray:
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    fine = np.zeros(2 * coarse.size, np.float64)
    lib().orc_predict_level(gamma, bc, _d(coarse), coarse.size, _d(fine))
    return fine


def project_level(fine: np.ndarray) -> np.ndarray:
    fine = np.ascontiguousarray(fine, dtype=np.float64)
    coarse = np.zeros(fine.size // 2, np.float64)
    lib().orc_project_level(_d(fine), coarse.size, _d(coarse))
    return coarse


def mr_encode(Jmin, Jmax, gamma, bc, finest):
    finest = np.ascontiguousarray(finest, dtype=np.float64)
    packed = np.zeros(level_offsets(Jmin, Jmax)[Jmax + 1], np.float64)
    lib().orc_mr_encode(Jmin, Jmax, gamma, bc, _d(finest), _d(packed))
    return packed


def mr_decode(Jmin, Jmax, gamma, bc, packed):
    packed = np.ascontiguousarray(packed, dtype=np.float64)
    finest = np.zeros(1 << Jmax, np.float64)
    lib().orc_mr_decode(Jmin, Jmax, gamma, bc, _d(packed), _d(finest))
    return finest


def grade(Jmin, Jmax, gamma, bc, R):
    R = np.ascontiguousarray(R, dtype=np.uint8).copy()
    lib().orc_grade(Jmin, Jmax, gamma, bc, _u8(R))
    return R


def check_graded(Jmin, Jmax, gamma, bc, R) -> int:
    R = np.ascontiguousarray(R, dtype=np.uint8)
    return lib().orc_check_graded(Jmin, Jmax, gamma, bc, _u8(R))

"""Helpers shared by the oracle and parity tests (no method arithmetic here)."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2102_12163_gb300 import workloads as W


def params_of(inst: W.Instance) -> O.Params:
    return O.Params(Jmin=inst.Jmin, Jmax=inst.Jmax, eq=inst.eq, lam=inst.lam, eps=inst.eps, gamma=inst.gamma,
                    mu_bar=inst.mu_bar, bc=inst.bc, a=inst.a, b=inst.b, s=inst.s, eqp=inst.eqp,
                    collision=inst.collision)


def oracle_of(inst: W.Instance) -> O.Oracle:
    o = O.Oracle(params_of(inst))
    o.set_initial(inst.m0)
    return o


def poly_averages(coef, edges):
    """Exact cell averages of the polynomial sum_i coef[i] x^i over cells [e_k, e_k+1]."""
    prim = np.zeros_like(edges)
    for i, c in enumerate(coef):
        prim = prim + c * edges ** (i + 1) / (i + 1)
    return np.diff(prim) / np.diff(edges)


def levels(Jmin, Jmax, arr):
    off = O.level_offsets(Jmin, Jmax)
    return {l: arr[off[l]:off[l + 1]] for l in range(Jmin, Jmax + 1)}


def is_graded(Jmin, Jmax, gamma, bc, R) -> bool:
    """Definition of a graded tree (Section 3.3) checked literally on a cell set."""
    L = levels(Jmin, Jmax, np.asarray(R).astype(bool))
    if not L[Jmin].all():
        return False
    for l in range(Jmin + 1, Jmax + 1):
        n, npar = 1 << l, 1 << (l - 1)
        for k in np.nonzero(L[l])[0]:
            if not L[l][k ^ 1]:
                return False
            for d in range(-gamma, gamma + 1):
                kk = (k >> 1) + d
                if bc == O.BC_PERIODIC:
                    kk %= npar
                elif kk < 0 or kk >= npar:
                    continue
                if not L[l - 1][kk]:
                    return False
    return True


def leaves_of(Jmin, Jmax, R):
    L = levels(Jmin, Jmax, np.asarray(R).astype(bool))
    out = []
    for l in range(Jmin, Jmax + 1):
        for k in np.nonzero(L[l])[0]:
            if l == Jmax or not (L[l + 1][2 * k] or L[l + 1][2 * k + 1]):
                out.append((l, int(k)))
    return out


def random_graded_tree(Jmin, Jmax, rng, density=0.1, bc=O.BC_PERIODIC, gamma=1):
    """A graded tree from a random seed set of cells closed by the oracle's grading."""
    S = O.level_offsets(Jmin, Jmax)[Jmax + 1]
    off = O.level_offsets(Jmin, Jmax)
    R = np.zeros(S, np.uint8)
    R[off[Jmin]:off[Jmin + 1]] = 1
    for l in range(Jmin + 1, Jmax + 1):
        pick = rng.random(1 << l) < density * (0.6 ** (Jmax - l))
        pick = pick | np.roll(pick, 1) if rng.random() < 0.5 else pick
        R[off[l]:off[l + 1]] |= pick.astype(np.uint8)
    # sibling closure of the seed set before grading
    for l in range(Jmin + 1, Jmax + 1):
        seg = R[off[l]:off[l + 1]].reshape(-1, 2)
        seg[:] = seg.max(axis=1, keepdims=True)
    return O.grade(Jmin, Jmax, gamma, bc, R)


def relerr(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    scale = max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    return float(np.max(np.abs(a - b))) / scale if a.size else 0.0


def prescribed_detail_state(Jmin, Jmax, bc, q, details, base=0.5, other=0.25):
    """Full tree whose population 0 has exactly the given details
    {(level, pair p): d} on a constant coarse average (dyadic values, so the
    multiresolution round trip is exact); the other populations are constant."""
    off = O.level_offsets(Jmin, Jmax)
    S = off[Jmax + 1]
    packed = np.zeros(S)
    packed[off[Jmin]:off[Jmin + 1]] = base
    for (l, p), d in details.items():
        packed[off[l] + 2 * p] = d
    vals = np.full((q, S), other)
    vals[0, off[Jmax]:] = O.mr_decode(Jmin, Jmax, 1, bc, packed)
    return np.ones(S, np.uint8), vals

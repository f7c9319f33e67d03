"""Pins of the oracle's enlargement operator H (Section 4.2: the dilation by
sigma = max |w^h| of every cell of R(T(Lambda^n)) and the refinement rule of
eq. HartenLossOfRegularity) against traces computed by hand.

Every case starts from the full tree with population 0 built from prescribed
details (one or two nonzero pairs, dyadic values, so the multiresolution round
trip is exact and the oracle's max |detail| equals the prescribed modulus).
The expected sets R(H(T(Lambda^n))) below are written out cell by cell; they
were worked out on paper from the two rules, not computed by code.

Levels Jmin = 2 .. Jmax = 6, eps = 1/8, so eps_l = 2^(l - 6) / 8 is 1/64,
2/64, 4/64, 8/64 on levels 3, 4, 5, 6 (Prop. ErrorControl), and the Harten
level 2^(mu_bar + 1) eps_l is 2 eps_l for mu_bar = 0 and 16 eps_l for mu_bar = 3.

The last test plants mistakes in a copy of the oracle (compiled on the CPU)
and checks that these pins catch each one.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O

JMIN, JMAX, EPS = 2, 6, 1.0 / 8.0
U = 1.0 / 64.0  # detail unit: eps_l = 1, 2, 4, 8 units on levels 3..6
ALL = "all"

# (bc, mu_bar, {(level, pair): detail}, {level: cells of R(H(T)) on that level})
# every level not listed holds no cell of R(H(T)); level Jmin is always whole
CASES = {
    # a kept pair well inside level 4: rule (a) adds the neighbouring pairs 2 and 4;
    # 3 units < 2 eps_4 = 4 units, so rule (b) adds nothing
    "interior": (O.BC_PERIODIC, 0, {(4, 3): 3 * U}, {4: [4, 5, 6, 7, 8, 9]}),
    # the detail equals 2 eps_4 exactly: kept and refined (">=" as printed), the
    # four children 2k .. 2k + 3 of the even cell k = 6 join level 5
    "harten_tie": (O.BC_PERIODIC, 0, {(4, 3): 4 * U}, {4: [4, 5, 6, 7, 8, 9], 5: [12, 13, 14, 15]}),
    # just below 2 eps_4: kept, not refined
    "harten_below": (O.BC_PERIODIC, 0, {(4, 3): 4 * U - 2.0 ** -20}, {4: [4, 5, 6, 7, 8, 9]}),
    # mu_bar = 3: the Harten level is 16 eps_4 = 32 units; 31 units do not refine, 32 do
    "mu3_below": (O.BC_PERIODIC, 3, {(4, 3): 31 * U}, {4: [4, 5, 6, 7, 8, 9]}),
    "mu3_at": (O.BC_PERIODIC, 3, {(4, 3): 32 * U}, {4: [4, 5, 6, 7, 8, 9], 5: [12, 13, 14, 15]}),
    # on level Jmax - 1 the refinement reaches the finest level: k = 20 -> cells 40..43
    "harten_at_jmax_minus_1": (O.BC_PERIODIC, 0, {(5, 10): 8 * U},
                               {5: [18, 19, 20, 21, 22, 23], 6: [40, 41, 42, 43]}),
    # on level Jmax rule (b) does not apply, however large the detail
    "no_harten_at_jmax": (O.BC_PERIODIC, 0, {(6, 20): 100 * U}, {6: [38, 39, 40, 41, 42, 43]}),
    # a detail below eps_5 (3 < 4 units): nothing kept on level 5, nothing added
    "below_threshold": (O.BC_PERIODIC, 0, {(5, 10): 3 * U}, {}),
    # the first pair of level 4: periodic wraps to the last pair, copy clips it
    "left_periodic": (O.BC_PERIODIC, 0, {(4, 0): 3 * U}, {4: [0, 1, 2, 3, 14, 15]}),
    "left_copy": (O.BC_COPY, 0, {(4, 0): 3 * U}, {4: [0, 1, 2, 3]}),
    # the last pair of level 4
    "right_periodic": (O.BC_PERIODIC, 0, {(4, 7): 3 * U}, {4: [0, 1, 12, 13, 14, 15]}),
    "right_copy": (O.BC_COPY, 0, {(4, 7): 3 * U}, {4: [12, 13, 14, 15]}),
    # level Jmin + 1 (8 cells), detail equal to eps_3 (kept on ">="), below 2 eps_3
    "first_refined_level_periodic": (O.BC_PERIODIC, 0, {(3, 0): 1 * U}, {3: [0, 1, 2, 3, 6, 7]}),
    "first_refined_level_copy": (O.BC_COPY, 0, {(3, 0): 1 * U}, {3: [0, 1, 2, 3]}),
    # two kept pairs two pairs apart: their dilations meet in pair 5 (no gap left)
    "two_pairs": (O.BC_PERIODIC, 0, {(4, 3): 3 * U, (4, 6): 3 * U},
                  {4: [4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15]}),
    # refinement on level 4 at the right edge under the copy boundary: the four
    # children of k = 14 are cells 28..31 of level 5, all inside the domain
    "harten_right_copy": (O.BC_COPY, 0, {(4, 7): 5 * U}, {4: [12, 13, 14, 15], 5: [28, 29, 30, 31]}),
}


def _params(eq, bc, mu_bar):
    q = O.NPOP[eq]
    return O.Params(Jmin=JMIN, Jmax=JMAX, eq=eq, lam=2.0, eps=EPS, mu_bar=mu_bar, bc=bc, eqp=1.0,
                    s=(1.5, 1.0, 1.0)), q


def _state(bc, q, details):
    """Full tree; population 0 from the given details on a constant coarse
    average, the other populations constant (no detail)."""
    off = O.level_offsets(JMIN, JMAX)
    S = off[JMAX + 1]
    packed = np.zeros(S)
    packed[off[JMIN]:off[JMIN + 1]] = 0.5
    for (l, p), d in details.items():
        packed[off[l] + 2 * p] = d
    vals = np.full((q, S), 0.25)
    vals[0, off[JMAX]:] = O.mr_decode(JMIN, JMAX, 1, bc, packed)
    return np.ones(S, np.uint8), vals


def _trace(L, p, q, R, vals):
    """orc_set_state + orc_adapt + orc_get_trace through the library handle L."""
    pc = p.c()
    h = L.orc_create(ctypes.byref(pc))
    assert h
    try:
        S = L.orc_total_cells(h)
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_ubyte)
        R = np.ascontiguousarray(R)
        vals = np.ascontiguousarray(vals)
        assert L.orc_set_state(h, R.ctypes.data_as(up), vals.ctypes.data_as(dp)) == 0
        L.orc_adapt(h)
        D = np.zeros(S)
        T, H, G = (np.zeros(S, np.uint8) for _ in range(3))
        L.orc_get_trace(h, D.ctypes.data_as(dp), T.ctypes.data_as(up), H.ctypes.data_as(up), G.ctypes.data_as(up))
        return D, T, H
    finally:
        L.orc_free(h)


def _expected_H(expect):
    off = O.level_offsets(JMIN, JMAX)
    H = np.zeros(off[JMAX + 1], np.uint8)
    H[off[JMIN]:off[JMIN + 1]] = 1
    for l, cells in expect.items():
        H[off[l] + np.asarray(cells, int)] = 1
    return H


def _check(L, name, eq):
    bc, mu_bar, details, expect = CASES[name]
    p, q = _params(eq, bc, mu_bar)
    R, vals = _state(bc, q, details)
    D, T, H = _trace(L, p, q, R, vals)
    off = O.level_offsets(JMIN, JMAX)
    # the prescribed details are what the oracle measures
    for (l, pp), d in details.items():
        assert D[off[l] + 2 * pp] == d and D[off[l] + 2 * pp + 1] == d
    assert np.count_nonzero(D) == 2 * len(details)
    exp = _expected_H(expect)
    bad = np.nonzero(H != exp)[0]
    return [(l, int(c - off[l])) for c in bad for l in range(JMIN, JMAX + 1) if off[l] <= c < off[l + 1]]


@pytest.mark.parametrize("name", sorted(CASES))
def test_enlargement_trace_d1q2(name):
    """D1Q2 schemes: sigma = 1."""
    assert _check(O.lib(), name, O.EQ_BURGERS) == []


@pytest.mark.parametrize("name", ["interior", "harten_tie", "left_periodic", "left_copy", "right_periodic",
                                  "right_copy", "first_refined_level_periodic", "two_pairs"])
def test_enlargement_trace_d1q5(name):
    """D1Q5 (Section 5.2 runs it with sigma = 2): the same cells as sigma = 1.
    Rule (a) adds (l, k + delta), |delta| <= sigma, for both cells 2p, 2p + 1
    of a kept pair, i.e. cells 2p - sigma .. 2p + 1 + sigma, and R(H) holds
    siblings together: for sigma = 1 and sigma = 2 alike that is the pairs
    p - 1, p, p + 1 (see the next test)."""
    assert _check(O.lib(), name, O.EQ_SW_D1Q5) == []


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_COPY])
def test_dilation_by_one_and_two_agree_on_sibling_closed_sets(bc):
    """Brute force over every sibling-closed subset of a level of 16 cells:
    dilating by sigma = 1 or sigma = 2 cells and closing under siblings gives
    the same set, while sigma = 3 does not.  (So a D1Q5 run with sigma = 1
    would build the same trees; the pin of sigma is the trace above.)"""
    n = 16

    def dil(cells, s):
        out = set()
        for k in cells:
            for d in range(-s, s + 1):
                kk = k + d
                if bc == O.BC_PERIODIC:
                    kk %= n
                elif not 0 <= kk < n:
                    continue
                out |= {kk, kk ^ 1}
        return out

    differ3 = 0
    for mask in range(1 << (n // 2)):
        cells = {c for p in range(n // 2) if (mask >> p) & 1 for c in (2 * p, 2 * p + 1)}
        assert dil(cells, 1) == dil(cells, 2)
        differ3 += dil(cells, 3) != dil(cells, 1)
    assert differ3 > 0


# mistakes planted in a copy of the oracle: (description, original text, planted text)
MUTATIONS = [
    ("Harten factor 2^(mu_bar + 2)", "ldexp(eps_l, p->mu_bar + 1)", "ldexp(eps_l, p->mu_bar + 2)"),
    ("Harten rule on > instead of >=", "st->D[CELL(st, l, k)] >= big", "st->D[CELL(st, l, k)] > big"),
    ("two children instead of four", "for (int d = 0; d < 4; ++d) st->H", "for (int d = 0; d < 2; ++d) st->H"),
    ("children from k instead of 2k", "st->H[CELL(st, l + 1, 2 * k + d)]", "st->H[CELL(st, l + 1, k + d)]"),
    ("no dilation (sigma = 0)", "for (int d = -sigma; d <= sigma; ++d) add_pair(st->H",
     "for (int d = 0; d <= 0; ++d) add_pair(st->H"),
    ("one-sided dilation", "for (int d = -sigma; d <= sigma; ++d) add_pair(st->H",
     "for (int d = 0; d <= sigma; ++d) add_pair(st->H"),
    ("Harten rule on the threshold", "&& st->D[CELL(st, l, k)] >= big", "&& st->D[CELL(st, l, k)] >= eps_l"),
]


def _build_mutant(tmp_path, old, new, tag):
    src_dir = os.path.dirname(O._SRC)
    text = open(O._SRC).read()
    assert text.count(old) == 1, old
    d = tmp_path / tag
    d.mkdir()
    (d / "mrlbm_oracle.c").write_text(text.replace(old, new))
    (d / "mrlbm_oracle.h").write_text(open(os.path.join(src_dir, "mrlbm_oracle.h")).read())
    so = d / "liborc_mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(d / "mrlbm_oracle.c"), "-lm"])
    L = ctypes.CDLL(str(so))
    vp = ctypes.c_void_p
    L.orc_create.restype = vp
    L.orc_create.argtypes = [ctypes.POINTER(O._Params)]
    L.orc_free.argtypes = [vp]
    L.orc_total_cells.restype = ctypes.c_long
    L.orc_total_cells.argtypes = [vp]
    L.orc_set_state.restype = ctypes.c_int
    L.orc_set_state.argtypes = [vp, ctypes.POINTER(ctypes.c_ubyte), ctypes.POINTER(ctypes.c_double)]
    L.orc_adapt.argtypes = [vp]
    L.orc_get_trace.argtypes = [vp] + [ctypes.POINTER(ctypes.c_double)] + [ctypes.POINTER(ctypes.c_ubyte)] * 3
    return L


def test_planted_mistakes_are_caught(tmp_path):
    for i, (what, old, new) in enumerate(MUTATIONS):
        L = _build_mutant(tmp_path, old, new, f"m{i}")
        failing = [n for n in sorted(CASES) for eq in (O.EQ_BURGERS, O.EQ_SW_D1Q5) if _check(L, n, eq)]
        assert failing, f"planted mistake not caught: {what}"
    # the unmutated source compiled the same way passes every case
    L = _build_mutant(tmp_path, "ldexp(eps_l, p->mu_bar + 1)", "ldexp(eps_l, p->mu_bar + 1)", "clean")
    assert not [n for n in sorted(CASES) for eq in (O.EQ_BURGERS, O.EQ_SW_D1Q5) if _check(L, n, eq)]

"""C ABI checks that need no GPU: the library loads, exports every entry point
of include/mrlbm.h, validates its arguments, and its reconstruction tables
agree with the oracle's reconstruction."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2102_12163_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mrlbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"mr_status\s+(\w+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    L = capi.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(capi.exported_symbols())


def test_argument_validation():
    L = capi.load()
    h = ctypes.c_void_p()
    assert L.mr_mesh_init(ctypes.byref(h), 1, 8, 1, 1e-4, -1.0, 1.0, 0, 0, 0) == capi.MR_ERR_ARG
    assert L.mr_mesh_init(ctypes.byref(h), 2, 30, 1, 1e-4, -1.0, 1.0, 0, 0, 0) == capi.MR_ERR_ARG
    assert L.mr_mesh_init(ctypes.byref(h), 2, 8, 4, 1e-4, -1.0, 1.0, 0, 0, 0) == capi.MR_ERR_ARG
    assert L.mr_mesh_init(ctypes.byref(h), 2, 8, 1, -1.0, -1.0, 1.0, 0, 0, 0) == capi.MR_ERR_ARG
    assert L.mr_mesh_init(ctypes.byref(h), 2, 8, 1, 1e-4, 1.0, -1.0, 0, 0, 0) == capi.MR_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    L.mr_last_error(None, buf, 256)
    assert b"b > a" in buf.value
    assert L.mr_mesh_init(ctypes.byref(h), 2, 8, 1, 1e-4, -1.0, 1.0, 0, 0, 0) == capi.MR_OK
    sz = ctypes.c_size_t()
    # scheme not set yet
    assert L.mr_workspace_size(h, ctypes.byref(sz)) == capi.MR_ERR_STATE
    s = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    c = ctypes.c_double(0.5)
    assert L.lbm_scheme(h, 1, 3, 1.0, s, capi.MR_EQ_ADVECTION, ctypes.byref(c)) == capi.MR_ERR_ARG
    assert L.lbm_scheme(h, 2, 2, 1.0, s, capi.MR_EQ_ADVECTION, ctypes.byref(c)) == capi.MR_ERR_ARG
    assert L.lbm_scheme(h, 1, 2, 1.0, s, capi.MR_EQ_ADVECTION, ctypes.byref(c)) == capi.MR_OK
    assert L.mr_workspace_size(h, ctypes.byref(sz)) == capi.MR_OK
    small = sz.value
    assert small > 0
    # stepping before a workspace is bound is refused, not run
    assert L.mr_advance(h, 1) == capi.MR_ERR_STATE
    assert L.mr_set_launch(h, 100, 0) == capi.MR_ERR_ARG
    assert L.mr_destroy(h) == capi.MR_OK
    # workspace grows with the finest level
    assert L.mr_mesh_init(ctypes.byref(h), 2, 12, 1, 1e-4, -1.0, 1.0, 0, 0, 0) == capi.MR_OK
    assert L.lbm_scheme(h, 1, 2, 1.0, s, capi.MR_EQ_ADVECTION, ctypes.byref(c)) == capi.MR_OK
    assert L.mr_workspace_size(h, ctypes.byref(sz)) == capi.MR_OK
    assert sz.value > 8 * small
    L.mr_destroy(h)


def test_batch_creation_checks_every_descriptor():
    L = capi.load()
    descs = (capi.mr_instance_desc * 3)()
    for d in descs:
        d.Jmin, d.Jmax, d.gamma, d.bc, d.eq = 2, 8, 1, 0, capi.MR_EQ_BURGERS
        d.eps, d.a, d.b, d.lambda_ = 1e-3, -1.0, 1.0, 1.0
        d.s[0] = d.s[1] = d.s[2] = 1.0
    h = ctypes.c_void_p()
    assert L.mr_batch_create(ctypes.byref(h), descs, 3, capi.MR_FP32_MIXED) == capi.MR_OK
    L.mr_destroy(h)
    # prediction stencils gamma = 1, 2, 3 are built; 0 and 4 are refused
    descs[1].gamma, descs[2].gamma = 2, 3
    assert L.mr_batch_create(ctypes.byref(h), descs, 3, capi.MR_FP64) == capi.MR_OK
    L.mr_destroy(h)
    for bad in (0, 4):
        descs[1].gamma = bad
        assert L.mr_batch_create(ctypes.byref(h), descs, 3, capi.MR_FP64) == capi.MR_ERR_ARG
    descs[1].gamma = 2
    descs[2].s[0] = 2.5
    assert L.mr_batch_create(ctypes.byref(h), descs, 3, capi.MR_FP64) == capi.MR_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    L.mr_last_error(None, buf, 256)
    assert b"instance 2" in buf.value
    # the lattice velocity lambda is taken in [2^-16, 2^16], where the FP64
    # collision's division by a lambda that is no power of two (Markstein's
    # correction) stays away from overflow and underflow
    descs[2].s[0] = 1.0
    for lam, ok in ((2.0 ** 16, True), (3.0 * 2.0 ** -16, True), (2.0 ** -16, True),
                    (2.0 ** 16 * 1.5, False), (2.0 ** -17, False), (0.0, False), (float("nan"), False)):
        descs[0].lambda_ = lam
        rc = L.mr_batch_create(ctypes.byref(h), descs, 3, capi.MR_FP64)
        assert rc == (capi.MR_OK if ok else capi.MR_ERR_ARG), lam
        if ok:
            L.mr_destroy(h)


def _table(dj, kind):
    out = (ctypes.c_double * 4)()
    assert capi.load().mr_reconstruction_coefficients(dj, kind, out) == capi.MR_OK
    return np.array(out[: 2 if kind in (2, 5) else 4])


def _full_tree_to(Jmin, Jmax, lmax):
    off = O.level_offsets(Jmin, Jmax)
    R = np.zeros(off[Jmax + 1], np.uint8)
    for l in range(Jmin, lmax + 1):
        R[off[l]:off[l + 1]] = 1
    return R, off


@pytest.mark.parametrize("dj", [1, 2, 3, 5, 8])
def test_reconstruction_tables_match_the_oracle(dj):
    """The per-level-gap tables of the CUDA path give the first / last finest
    cell of a leaf exactly as the oracle's level-by-level prediction does."""
    Jmin, l = 2, 5
    Jmax = l + dj
    rng = np.random.default_rng(dj)
    p = O.Params(Jmin=Jmin, Jmax=Jmax, eq=O.EQ_BURGERS, lam=1.0, bc=O.BC_PERIODIC)
    cf, t1 = _table(dj, 0), _table(dj, 1)
    # (a) all leaves on level l: first cell from (k-2..k+1), last from mirrored weights
    R, off = _full_tree_to(Jmin, Jmax, l)
    o = O.Oracle(p)
    vals = rng.normal(size=(2, o.S))
    o.set_state(R, vals)
    fin = o.finest()[0]
    V = vals[0, off[l]:off[l + 1]]
    n = 1 << l
    for k in range(n):
        win = V[[(k - 2) % n, (k - 1) % n, k, (k + 1) % n]]
        assert abs(fin[k << dj] - cf @ win) < 1e-13
        winr = V[[(k - 1) % n, k, (k + 1) % n, (k + 2) % n]]
        assert abs(fin[((k + 1) << dj) - 1] - cf[::-1] @ winr) < 1e-13
    # (b) finer left neighbour: refine cell k-1 of level l
    k = 9
    R2 = R.copy()
    R2[off[l + 1] + 2 * (k - 1)] = R2[off[l + 1] + 2 * (k - 1) + 1] = 1
    assert O.check_graded(Jmin, Jmax, 1, O.BC_PERIODIC, R2) == 0
    o.set_state(R2, vals)
    fin = o.finest()[0]
    V1 = vals[0, off[l + 1]:off[l + 2]]
    # children of the leaf k predicted from its level-l window (V[k-1] is the projection)
    vkm1 = 0.5 * (V1[2 * k - 2] + V1[2 * k - 1])
    tt = -0.125 * (V[k + 1] - vkm1)
    w1 = np.array([V1[2 * k - 2], V1[2 * k - 1], V[k] + tt, V[k] - tt])
    assert abs(fin[k << dj] - t1 @ w1) < 1e-13


@pytest.mark.parametrize("dj", [1, 2, 4, 7])
def test_copy_boundary_tables_match_the_oracle(dj):
    Jmin, l = 2, 4
    Jmax = l + dj
    rng = np.random.default_rng(100 + dj)
    p = O.Params(Jmin=Jmin, Jmax=Jmax, eq=O.EQ_BURGERS, lam=1.0, bc=O.BC_COPY)
    R, off = _full_tree_to(Jmin, Jmax, l)
    o = O.Oracle(p)
    vals = rng.normal(size=(2, o.S))
    o.set_state(R, vals)
    fin = o.finest()[0]
    V = vals[0, off[l]:off[l + 1]]
    bf = _table(dj, 2)
    n = 1 << l
    assert abs(fin[0] - bf @ V[[0, 1]]) < 1e-13
    assert abs(fin[-1] - bf @ V[[n - 1, n - 2]]) < 1e-13
    # the cells next to the boundary use the interior weights on a clamped window
    cf = _table(dj, 0)
    assert abs(fin[1 << dj] - cf @ V[[0, 0, 1, 2]]) < 1e-13
    assert abs(fin[(1 << dj) - 1] - cf[::-1] @ V[[0, 0, 1, 2]]) < 1e-13


def test_tables_are_exact_dyadic_rationals():
    from fractions import Fraction

    for dj in range(0, 17):
        for kind in (0, 1, 2, 3, 4, 5):
            if kind in (1, 4) and dj == 0:
                continue
            t = _table(dj, kind)
            assert sum(Fraction(x) for x in t) == 1  # weights reproduce constants
            for x in t:
                assert (Fraction(x) * 8 ** dj).denominator == 1


@pytest.mark.parametrize("dj", [1, 2, 3, 6])
def test_second_cell_tables_match_the_oracle(dj):
    """Second finest cell from a leaf edge (streamed by the |v| = 2 lambda
    populations of D1Q5): interior, finer-neighbour and copy-boundary weights
    against the oracle's level-by-level prediction."""
    Jmin, l = 2, 5
    Jmax = l + dj
    rng = np.random.default_rng(200 + dj)
    cf2, t12, bf2 = _table(dj, 3), _table(dj, 4), _table(dj, 5)
    R, off = _full_tree_to(Jmin, Jmax, l)
    n = 1 << l
    for bc in (O.BC_PERIODIC, O.BC_COPY):
        p = O.Params(Jmin=Jmin, Jmax=Jmax, eq=O.EQ_BURGERS, lam=1.0, bc=bc)
        o = O.Oracle(p)
        vals = rng.normal(size=(2, o.S))
        o.set_state(R, vals)
        fin = o.finest()[0]
        V = vals[0, off[l]:off[l + 1]]
        for k in range(2, n - 2):
            assert abs(fin[(k << dj) + 1] - cf2 @ V[[k - 2, k - 1, k, k + 1]]) < 1e-13
            assert abs(fin[((k + 1) << dj) - 2] - cf2[::-1] @ V[[k - 1, k, k + 1, k + 2]]) < 1e-13
        if bc == O.BC_COPY:
            assert abs(fin[1] - bf2 @ V[[0, 1]]) < 1e-13
            assert abs(fin[-2] - bf2 @ V[[n - 1, n - 2]]) < 1e-13
    # finer left neighbour
    p = O.Params(Jmin=Jmin, Jmax=Jmax, eq=O.EQ_BURGERS, lam=1.0, bc=O.BC_PERIODIC)
    o = O.Oracle(p)
    vals = rng.normal(size=(2, o.S))
    k = 9
    R2 = R.copy()
    R2[off[l + 1] + 2 * (k - 1)] = R2[off[l + 1] + 2 * (k - 1) + 1] = 1
    o.set_state(R2, vals)
    fin = o.finest()[0]
    V = vals[0, off[l]:off[l + 1]]
    V1 = vals[0, off[l + 1]:off[l + 2]]
    vkm1 = 0.5 * (V1[2 * k - 2] + V1[2 * k - 1])
    tt = -0.125 * (V[k + 1] - vkm1)
    w1 = np.array([V1[2 * k - 2], V1[2 * k - 1], V[k] + tt, V[k] - tt])
    assert abs(fin[(k << dj) + 1] - t12 @ w1) < 1e-13

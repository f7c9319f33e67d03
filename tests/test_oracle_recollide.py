"""Pins of the oracle's reconstructed collision (Section 4.5, eq.
reconstructedCollision) against facts the paper and the mathematics fix."""
import numpy as np
import pytest

import oracle as O
from oracle_helpers import oracle_of, params_of, random_graded_tree
from paper_2102_12163_gb300 import workloads as W

ALL = [W.EQ_ADVECTION, W.EQ_BURGERS, W.EQ_SW, W.EQ_EULER, W.EQ_SW_D1Q3, W.EQ_SW_D1Q5]


def _pair(inst, seed, bc):
    """Two oracles, leaves and reconstructed collision, on one random graded tree."""
    rng = np.random.default_rng(seed)
    p = params_of(inst)
    R = random_graded_tree(inst.Jmin, inst.Jmax, rng, density=0.25, bc=bc)
    m = np.array([[1.0], [0.1], [2.0]])[: p.nf]
    if inst.eq in (W.EQ_ADVECTION, W.EQ_BURGERS):
        m = np.array([[0.4]])
    base = O.equilibrium(p, m)[:, :1]
    S = O.level_offsets(inst.Jmin, inst.Jmax)[inst.Jmax + 1]
    vals = base + 0.05 * rng.normal(size=(p.q, S))
    a = O.Oracle(p)
    b = O.Oracle(params_of(inst.with_(collision=W.COLLIDE_RECONSTRUCTED)))
    a.set_state(R, vals)
    b.set_state(R, vals)
    return a, b


@pytest.mark.parametrize("eq", ALL)
def test_full_tree_is_the_leaves_collision(eq):
    """Every leaf on the finest level: the average over one reconstructed cell
    is the leaf itself, so the two collisions coincide (eps = 0 runs)."""
    inst = W.random_smooth(7, eq, seed=40 + eq, eps=0.0)
    a = oracle_of(inst)
    b = oracle_of(inst.with_(collision=W.COLLIDE_RECONSTRUCTED))
    for _ in range(6):
        a.step()
        b.step()
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    assert np.max(np.abs(a.get_state()[1] - b.get_state()[1])) < 1e-14


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_COPY])
def test_linear_equilibrium_is_the_leaves_collision(bc):
    """Advection: m^{1,eq} = c m^0 is linear, and the projection of the
    reconstruction of a leaf is the leaf (consistency of prediction and
    projection, Section 3.1), so averaging the equilibria over the finest
    cells changes nothing on any tree."""
    inst = W.random_smooth(9, W.EQ_ADVECTION, seed=50 + bc, bc=bc)
    a, b = _pair(inst, 51 + bc, bc)
    a.lbm_step()
    b.lbm_step()
    assert np.max(np.abs(a.get_state()[1] - b.get_state()[1])) < 1e-13


def _collided(inst, seed, bc):
    a, b = _pair(inst, seed, bc)
    a.collide()
    b.collide()
    lv, ix, fa = a.leaves()
    _, _, fb = b.leaves()
    return lv, fa, fb


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_COPY])
def test_convex_equilibrium_averages_above_the_leaf_value(bc):
    """Burgers, s = 1: the relaxed moment after the collision is the mean over
    the leaf's reconstructed finest cells of (m^0)^2 / 2, which by Jensen is at
    least (mean m^0)^2 / 2 = the leaves collision's value, and strictly larger
    where the reconstruction varies; the conserved moment is untouched; leaves
    on the finest level are collided identically."""
    inst = W.random_smooth(9, W.EQ_BURGERS, seed=60 + bc, bc=bc).with_(s=(1.0,))
    lv, fa, fb = _collided(inst, 61 + bc, bc)
    assert np.allclose(fa[0] + fa[1], fb[0] + fb[1], rtol=0, atol=1e-15)
    ra, rb = fa[0] - fa[1], fb[0] - fb[1]
    assert np.all(rb >= ra - 1e-15)
    coarse = lv < inst.Jmax
    assert np.max(rb[coarse] - ra[coarse]) > 1e-9
    fine = lv == inst.Jmax
    assert np.max(np.abs(fa[:, fine] - fb[:, fine])) == 0.0


@pytest.mark.parametrize("eq", [W.EQ_SW, W.EQ_EULER, W.EQ_SW_D1Q3, W.EQ_SW_D1Q5])
def test_nonlinear_systems_differ_only_on_coarse_leaves(eq):
    """The conserved moments stay; the two collisions agree on leaves of the
    finest level (one reconstructed cell) and differ on coarser ones."""
    inst = W.random_smooth(9, eq, seed=70 + eq, bc=O.BC_PERIODIC)
    lv, fa, fb = _collided(inst, 71 + eq, O.BC_PERIODIC)
    p = params_of(inst)
    assert np.allclose(O.moments(p, fa), O.moments(p, fb), rtol=0, atol=1e-14)
    fine = lv == inst.Jmax
    assert np.max(np.abs(fa[:, fine] - fb[:, fine])) == 0.0
    assert np.max(np.abs(fa[:, ~fine] - fb[:, ~fine])) > 1e-9


@pytest.mark.parametrize("eq", ALL)
def test_reconstructed_collision_conserves(eq):
    inst = W.random_smooth(9, eq, seed=80 + eq, eps=1e-3).with_(collision=W.COLLIDE_RECONSTRUCTED)
    o = oracle_of(inst)
    m0 = o.mass()
    o.step(20)
    assert np.allclose(o.mass(), m0, rtol=0, atol=1e-12)

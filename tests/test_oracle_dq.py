"""Pins of the oracle's D1Q3 and D1Q5 shallow water schemes (Section 5.2)
against facts the paper and the mathematics fix."""
import numpy as np
import pytest

import oracle as O
from oracle_helpers import oracle_of, params_of, random_graded_tree
from paper_2102_12163_gb300 import workloads as W

DQ = [W.EQ_SW_D1Q3, W.EQ_SW_D1Q5]
VEL = {W.EQ_SW_D1Q3: [0, 1, -1], W.EQ_SW_D1Q5: [0, 1, -1, 2, -2]}


def _params(eq, s=(1.3, 1.1, 0.9), J=6, bc=O.BC_PERIODIC, lam=2.0):
    return O.Params(Jmin=2, Jmax=J, eq=eq, lam=lam, eps=0.0, bc=bc, s=s, eqp=1.0)


def _moments_np(eq, lam, f):
    """All q moments m^i = sum_h (v^h)^i f^h, from the velocity set alone."""
    v = lam * np.array(VEL[eq], float)
    return np.stack([(v[:, None] ** i * f).sum(axis=0) for i in range(len(v))])


@pytest.mark.parametrize("eq", DQ)
def test_equilibrium_has_the_shallow_water_moments(eq):
    """f^eq(h, hu): m^0 = h, m^1 = hu, m^2 = h u^2 + g h^2 / 2 (the flux of
    hu), and for D1Q5 m^3 = lambda^2 hu, m^4 = lambda^2 m^{2,eq} (alpha = beta = 1)."""
    p = _params(eq)
    rng = np.random.default_rng(1)
    h = rng.uniform(0.5, 2.0, 64)
    hu = rng.uniform(-0.5, 0.5, 64)
    f = O.equilibrium(p, np.stack([h, hu]))
    m = _moments_np(eq, p.lam, f)
    flux = hu * hu / h + 0.5 * h * h
    assert np.allclose(m[0], h, rtol=1e-14) and np.allclose(m[1], hu, rtol=1e-13, atol=1e-14)
    assert np.allclose(m[2], flux, rtol=1e-13)
    if eq == W.EQ_SW_D1Q5:
        assert np.allclose(m[3], p.lam ** 2 * hu, rtol=1e-12, atol=1e-13)
        assert np.allclose(m[4], p.lam ** 2 * flux, rtol=1e-12)
    assert np.allclose(O.moments(p, f), np.stack([h, hu]), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("eq", DQ)
def test_zero_relaxation_is_pure_transport(eq):
    """s = 0 keeps every moment, so the collision is the identity (M^{-1} M = I)
    and one step shifts population h by w^h = v^h / lambda cells."""
    p = _params(eq, s=(0.0, 0.0, 0.0))
    rng = np.random.default_rng(2)
    f = rng.uniform(0.1, 1.0, (len(VEL[eq]), 1 << p.Jmax))
    g = O.uniform_step(p, f.copy())
    for h, w in enumerate(VEL[eq]):
        assert np.allclose(g[h], np.roll(f[h], w), rtol=1e-13, atol=1e-14), h


@pytest.mark.parametrize("eq", DQ)
def test_full_relaxation_lands_on_the_equilibrium(eq):
    """s = 1 for every relaxed moment: the post-collision state is f^eq of the
    conserved moments, which the collision keeps."""
    p = _params(eq, s=(1.0, 1.0, 1.0))
    rng = np.random.default_rng(3)
    f = rng.uniform(0.2, 1.0, (len(VEL[eq]), 1 << p.Jmax))
    m = O.moments(p, f)
    g = O.uniform_step(p, f.copy())
    feq = O.equilibrium(p, m)
    for h, w in enumerate(VEL[eq]):
        assert np.allclose(g[h], np.roll(feq[h], w), rtol=1e-12, atol=1e-14), h


@pytest.mark.parametrize("eq", DQ)
@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_COPY])
def test_zero_threshold_reproduces_the_uniform_scheme(eq, bc):
    inst = W.random_smooth(8, eq, seed=10 + eq, eps=0.0, bc=bc)
    p = params_of(inst)
    o = oracle_of(inst)
    F = O.equilibrium(p, inst.m0)
    for _ in range(12):
        o.step()
        F = O.uniform_step(p, F)
    lv, _, f = o.leaves()
    assert np.all(lv == inst.Jmax)
    assert np.max(np.abs(f - F)) < 1e-13


@pytest.mark.parametrize("eq", DQ)
@pytest.mark.parametrize("seed,bc", [(20, O.BC_PERIODIC), (21, O.BC_COPY)])
def test_compact_stream_equals_the_mean_of_shifted_finest_values(eq, seed, bc):
    """eq. AdaptiveStreamPhase with |w| = 2 (two eta terms per side) equals the
    mean over the leaf's finest cells of the reconstruction shifted by w^h."""
    rng = np.random.default_rng(seed)
    inst = W.random_smooth(9, eq, seed=seed, bc=bc)
    p = params_of(inst)
    o = O.Oracle(p)
    R = random_graded_tree(inst.Jmin, inst.Jmax, rng, density=0.3, bc=bc)
    base = O.equilibrium(p, np.array([[1.2], [0.1]]))[:, :1]
    vals = base + 0.02 * rng.normal(size=(p.q, o.S))
    o.set_state(R, vals)
    ref = o.lbm_step_uncompacted()
    o.lbm_step()
    _, v = o.get_state()
    lv, ix, _ = o.leaves()
    off = O.level_offsets(inst.Jmin, inst.Jmax)
    cells = np.array([off[l] for l in lv]) + ix
    assert np.max(np.abs(v[:, cells] - ref[:, cells])) < 1e-13


@pytest.mark.parametrize("eq", DQ)
def test_mass_and_momentum_conserved_with_periodic_boundaries(eq):
    inst = W.random_smooth(9, eq, seed=30 + eq, eps=1e-3)
    o = oracle_of(inst)
    m0 = o.mass()
    o.step(25)
    assert np.allclose(o.mass(), m0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["d1q3", "d1q5"])
def test_reference_scheme_converges_to_the_exact_dam_break(scheme):
    """The uniform reference scheme of each velocity set converges to the exact
    entropy solution of the dam break (left rarefaction, right shock) as the
    lattice is refined: a wrong equilibrium (a missing g h^2 / 2, a wrong
    sign) would converge to something else."""
    E = []
    for J in (8, 9, 10):
        inst = W.shallow_water_dq(scheme, Jmax=J, s2=1.6 if scheme == "d1q5" else 1.5)
        p = params_of(inst)
        F = O.equilibrium(p, inst.m0)
        for _ in range(inst.nsteps):
            F = O.uniform_step(p, F)
        ex = W.sw_riemann_exact(W.cell_edges(inst.a, inst.b, J), inst.nsteps * inst.dx / inst.lam)
        E.append(inst.dx * np.abs(O.moments(p, F) - ex).sum())
    assert E[1] < 0.85 * E[0] and E[2] < 0.85 * E[1], E
    assert E[2] < 0.02, E


@pytest.mark.parametrize("scheme", ["d1q3", "d1q5"])
def test_adaptive_dam_break_stays_close_to_the_reference(scheme):
    """Section 5.2: the perturbation error is several orders of magnitude below
    the reference scheme's discretisation error at eps = 1e-4."""
    inst = W.shallow_water_dq(scheme, Jmax=9, s2=1.6 if scheme == "d1q5" else 1.5)
    p = params_of(inst)
    o = oracle_of(inst)
    F = O.equilibrium(p, inst.m0)
    for _ in range(inst.nsteps):
        o.step()
        F = O.uniform_step(p, F)
    M = O.moments(p, F)
    ex = W.sw_riemann_exact(W.cell_edges(inst.a, inst.b, inst.Jmax), inst.nsteps * inst.dx / inst.lam)
    E = inst.dx * np.abs(M - ex).sum(axis=1)
    d = inst.dx * np.abs(M - o.finest_moments()).sum(axis=1)
    assert np.all(d < 1e-2 * E), (d, E)
    assert len(o.leaves()[0]) < 0.6 * (1 << inst.Jmax)

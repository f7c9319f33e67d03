"""Pins of the oracle's adaptive scheme against facts the paper fixes
(Sections 2, 4 and 5)."""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from oracle_helpers import is_graded, leaves_of, levels, oracle_of, params_of, random_graded_tree
from paper_2102_12163_gb300 import workloads as W

SCHEMES = [W.EQ_ADVECTION, W.EQ_BURGERS, W.EQ_SW, W.EQ_EULER]


def _uniform_state(p, m_cons):
    f = O.equilibrium(p, np.asarray(m_cons, float).reshape(p.nf, 1) * np.ones((1, 1 << p.Jmax)))
    return f


@pytest.mark.parametrize("s", [0.6, 1.0, 1.7])
def test_collision_closed_forms(s):
    """Relaxation of the non-conserved moment towards the paper's equilibria;
    Euler and shallow water equilibria equal the physical fluxes."""
    gg, g = 1.4, 1.0
    cases = [
        (W.EQ_ADVECTION, 0.7, [0.8], lambda m: [0.7 * m[0]]),
        (W.EQ_BURGERS, 0.0, [0.6], lambda m: [0.5 * m[0] ** 2]),
        # shallow water: (hu, hu^2/h + g h^2/2)
        (W.EQ_SW, g, [2.0, 1.0], lambda m: [m[1], m[1] ** 2 / m[0] + 0.5 * g * m[0] ** 2]),
        # Euler: (rho u, rho u^2 + p, u (E + p)), p = (gamma - 1)(E - rho u^2 / 2)
        (W.EQ_EULER, gg, [1.0, 0.5, 2.0],
         lambda m: [m[1], m[1] ** 2 / m[0] + (gg - 1) * (m[2] - 0.5 * m[1] ** 2 / m[0]),
                    m[1] / m[0] * (m[2] + (gg - 1) * (m[2] - 0.5 * m[1] ** 2 / m[0]))]),
    ]
    for eq, eqp, mc, flux in cases:
        lam = 3.0
        p = O.Params(Jmin=2, Jmax=4, eq=eq, lam=lam, s=(s, s, s), eqp=eqp)
        nf = p.nf
        # a uniform state off equilibrium: the stream of a constant field is the identity
        f = _uniform_state(p, mc)
        rng = np.random.default_rng(5)
        pert = rng.normal(size=nf) * 0.1
        for i in range(nf):
            f[2 * i] += pert[i]
            f[2 * i + 1] -= pert[i]
        m1 = [lam * (f[2 * i, 0] - f[2 * i + 1, 0]) for i in range(nf)]
        out = O.uniform_step(p, f)
        meq = flux(mc)
        for i in range(nf):
            assert out[2 * i, 0] + out[2 * i + 1, 0] == pytest.approx(mc[i], abs=1e-15)
            m1s = lam * (out[2 * i, 0] - out[2 * i + 1, 0])
            assert m1s == pytest.approx((1 - s) * m1[i] + s * meq[i], rel=1e-13, abs=1e-14)
    # hand values: rho = 1, rho u = 0.5, E = 2 -> (0.5, 1.0, 1.375)
    e = cases[3][3]([1.0, 0.5, 2.0])
    assert e == pytest.approx([0.5, 1.0, 1.375], abs=1e-15)


def test_equilibrium_moments_round_trip():
    rng = np.random.default_rng(1)
    for eq in SCHEMES:
        p = O.Params(Jmin=2, Jmax=5, eq=eq, lam=2.0, eqp=1.4 if eq == W.EQ_EULER else 0.6)
        m = rng.uniform(0.5, 1.5, size=(p.nf, 1 << 5))
        f = O.equilibrium(p, m)
        assert np.max(np.abs(O.moments(p, f) - m)) < 1e-15


def test_uniform_advection_at_lattice_speed_is_an_exact_shift():
    inst = W.advection(Jmax=8, c=1.0, s=1.0)
    p = params_of(inst)
    f = O.equilibrium(p, inst.m0)
    for n in range(1, 20):
        f = O.uniform_step(p, f)
        assert np.array_equal(O.moments(p, f)[0], np.roll(inst.m0[0], n))


@pytest.mark.parametrize("eq,bc", [(e, b) for e in SCHEMES for b in (W.BC_PERIODIC, W.BC_COPY)])
def test_zero_threshold_reproduces_the_uniform_scheme(eq, bc):
    """eps = 0: T keeps every pair (>=), the mesh stays the full tree and the
    adaptive scheme is the reference scheme on the finest lattice."""
    inst = W.random_smooth(7, eq, seed=10 + eq, eps=0.0, bc=bc)
    o = oracle_of(inst)
    p = params_of(inst)
    F = O.equilibrium(p, inst.m0)
    for n in range(25):
        o.step()
        F = O.uniform_step(p, F)
        lv, ix, f = o.leaves()
        assert np.all(lv == inst.Jmax) and len(lv) == 1 << inst.Jmax
        assert np.max(np.abs(f - F)) < 1e-14


@pytest.mark.parametrize("seed,bc,eq", [(1, O.BC_PERIODIC, W.EQ_BURGERS), (2, O.BC_COPY, W.EQ_EULER),
                                        (3, O.BC_COPY, W.EQ_SW), (4, O.BC_PERIODIC, W.EQ_ADVECTION)])
def test_compact_stream_equals_uncompacted_stream(seed, bc, eq):
    rng = np.random.default_rng(seed)
    Jmin, Jmax = 2, 8
    R = random_graded_tree(Jmin, Jmax, rng, density=0.25, bc=bc)
    inst = W.random_smooth(Jmax, eq, seed=seed, bc=bc)
    p = params_of(inst)
    o = O.Oracle(p)
    base = O.equilibrium(p, np.ones((p.nf, 1)) * np.array([[1.0], [0.2], [2.0]][:p.nf]))[:, :1]
    vals = base + 0.05 * rng.normal(size=(p.q, o.S))
    o.set_state(R, vals)
    unc = o.lbm_step_uncompacted()
    o.lbm_step()
    _, after = o.get_state()
    for l, k in leaves_of(Jmin, Jmax, R):
        c = O.level_offsets(Jmin, Jmax)[l] + k
        assert np.max(np.abs(after[:, c] - unc[:, c])) < 1e-14


def test_mass_is_conserved_with_periodic_boundaries():
    for eq in SCHEMES:
        inst = W.random_smooth(9, eq, seed=20 + eq, eps=1e-3)
        o = oracle_of(inst)
        m0 = o.mass()
        for n in range(40):
            o.step()
            assert np.max(np.abs(o.mass() - m0)) < 1e-13 * max(1.0, np.max(np.abs(m0)))


def test_copy_boundary_mass_change_is_the_boundary_flux():
    """Dam break at rest: until a wave reaches the walls the boundary cells stay
    at the constant states, and each step changes the momentum by
    dt (g h_L^2 / 2 - g h_R^2 / 2) and the height by nothing."""
    inst = W.shallow_water(Jmax=10, eps=1e-4)
    o = oracle_of(inst)
    dt = inst.dx / inst.lam
    m0 = o.mass()
    for n in range(1, 60):
        o.step()
        m = o.mass()
        assert abs(m[0] - m0[0]) < 1e-13
        assert m[1] - m0[1] == pytest.approx(n * dt * (0.5 * 4.0 - 0.5 * 1.0), rel=1e-12)


def test_meshes_stay_graded_partitions_holding_the_threshold_set():
    inst = W.burgers(Jmax=10)
    o = oracle_of(inst)
    for n in range(30):
        R_old, _ = o.get_state()
        o.adapt()
        D, T, H, G = o.trace()
        assert is_graded(inst.Jmin, inst.Jmax, 1, inst.bc, G)
        assert np.all(G >= T) and np.all(G >= H) and np.all(T <= R_old)  # T(L^n) in L^n and L^{n+1}
        cover = np.zeros(1 << inst.Jmax, int)
        for l, k in leaves_of(inst.Jmin, inst.Jmax, G):
            dj = inst.Jmax - l
            cover[k << dj:(k + 1) << dj] += 1
        assert np.all(cover == 1)
        o.lbm_step()


def test_threshold_on_a_dyadic_step():
    """A step aligned with cell boundaries at every level, jumps two coarse
    cells apart: the gamma = 1 detail has modulus 1/8 (times the population's
    jump) on the two pairs whose prediction stencil straddles each jump and is
    0 elsewhere (hand computation from the prediction formula)."""
    Jmin, Jmax = 2, 7
    N = 1 << Jmax
    m = np.zeros(N)
    m[N // 4: 3 * N // 4] = 1.0  # jumps at the level-2 boundaries 1 and 3
    p = O.Params(Jmin=Jmin, Jmax=Jmax, eq=O.EQ_ADVECTION, lam=1.0, eps=1e-3, eqp=0.5)
    o = O.Oracle(p)
    o.set_initial(m[None, :])
    o.adapt()
    D, T, H, G = o.trace()
    Dl, Tl = levels(Jmin, Jmax, D), levels(Jmin, Jmax, T)
    fmax = 0.5 * (1 + 0.5)  # largest population of the unit state (c = 0.5, lambda = 1)
    for l in range(Jmin + 1, Jmax + 1):
        n = 1 << l
        j1, j2 = n // 4, 3 * n // 4  # jump positions on level l (cell boundaries)
        expect = np.zeros(n)
        for j in (j1, j2):
            pj = j // 2  # jump between parent cells pj - 1 and pj
            for par in (pj - 1, pj):
                expect[2 * par] = expect[2 * par + 1] = 0.125 * fmax
        assert np.allclose(Dl[l], expect, atol=1e-15), l
        eps_l = 1e-3 * 2.0 ** (l - Jmax)
        assert np.array_equal(Tl[l].astype(bool), expect >= eps_l)


def _scalar_errors(test, s, J=9, eps=1e-4):
    """Test I-IV of Table 1: E = reference scheme vs exact solution, delta =
    adaptive vs reference scheme (weighted l1 of the conserved moment at the
    final step), and the compression factor CR."""
    inst = W.scalar_test(test, s=s, Jmax=J, eps=eps)
    p = params_of(inst)
    o = O.Oracle(p)
    o.set_initial(inst.m0)
    F = O.equilibrium(p, inst.m0)
    N = inst.nsteps
    for _ in range(N):
        o.step()
        F = O.uniform_step(p, F)
    M = O.moments(p, F)[0]
    dx = inst.dx
    exact = W.scalar_exact(test, W.cell_edges(inst.a, inst.b, J), N * dx / inst.lam)
    E = dx * np.abs(exact - M).sum()
    delta = dx * np.abs(M - o.finest_moments()[0]).sum()
    cr = 100.0 * (1.0 - len(o.leaves()[0]) / (1 << J))
    return E, delta, cr, N


def test_table2_error_ratios_order_of_magnitude():
    """Soft cross-check with Table 2 (Test I: smooth, nu = inf -> mu_bar = 3;
    Test II: indicator, nu = 0 -> mu_bar = 0): the perturbation error stays far
    below the reference discretisation error, within the paper's order of
    magnitude.  The paper's boundary treatment and implementation details are
    not given, so only the order of magnitude is checked."""
    rows = {float(r[0]): [float(x) for x in r[1:]] for r in read_golden("table2_error_ratios.txt")}
    for s in (0.75, 1.0, 1.75):
        E, d, cr, _ = _scalar_errors("I", s)
        assert rows[s][0] / 3 < E / d < rows[s][0] * 30, (s, E / d)
        assert cr > 70.0
        E, d, cr, _ = _scalar_errors("II", s)
        assert rows[s][1] / 3 < E / d < rows[s][1] * 30, (s, E / d)
        assert cr > 70.0


def test_burgers_tests_delta_is_far_below_the_discretisation_error():
    """Tests III and IV (Burgers) at eps = 1e-4, Jmax = 9: the paper fixes
    delta << E for every test (Section 5, choice of eps) and prints E / delta
    in Table 2.  Our delta is never more than 3x the paper's (E / delta at
    least a third of the printed ratio); it is often much smaller (more cells
    are kept), so only this side is checked."""
    rows = {float(r[0]): [float(x) for x in r[1:]] for r in read_golden("table2_error_ratios.txt")}
    for s in (0.75, 1.0, 1.25, 1.5, 1.75):
        for col, test in ((2, "III"), (3, "IV")):
            E, d, cr, _ = _scalar_errors(test, s)
            assert E / d > 5.0, (test, s, E / d)
            assert E / d > rows[s][col] / 3, (test, s, E / d, rows[s][col])
            assert cr > 60.0


@pytest.mark.parametrize("test", ["I", "III", "IV"])
def test_reference_scheme_converges_to_the_exact_solutions(test):
    """Pin of the exact solutions of Tests I, III, IV (cell averages of the
    entropy solution): the uniform reference scheme, first order, converges
    to them as the lattice is refined (a wrong exact solution would leave an
    O(1) error that does not shrink)."""
    Es = []
    for J in (9, 10, 11):
        inst = W.scalar_test(test, Jmax=J)
        p = params_of(inst)
        F = O.equilibrium(p, inst.m0)
        for _ in range(inst.nsteps):
            F = O.uniform_step(p, F)
        exact = W.scalar_exact(test, W.cell_edges(inst.a, inst.b, J), inst.nsteps * inst.dx / inst.lam)
        Es.append(inst.dx * np.abs(exact - O.moments(p, F)[0]).sum())
    assert Es[1] < 0.8 * Es[0] and Es[2] < 0.8 * Es[1], Es


def test_exact_burgers_solutions_conserve_mass_up_to_the_boundary_flux():
    """Test III (copy boundary): the total changes by the outflow phi(1) t = t / 2
    through x = 3; Test IV: the total is conserved; the shock of Test IV sits
    at x = 1/2 + t/2 (Rankine-Hugoniot speed (1 + 0) / 2)."""
    e = W.cell_edges(-3.0, 3.0, 12)
    dx = 6.0 / 4096
    for t in (0.1, 0.4):
        m0 = W.scalar_exact("III", e, 0.0).sum() * dx
        assert abs(W.scalar_exact("III", e, t).sum() * dx - (m0 - 0.5 * t)) < 1e-9
        assert abs(W.scalar_exact("IV", e, t).sum() * dx - 1.0) < 1e-12
        m = W.scalar_exact("IV", e, t)
        xs = 0.5 + 0.5 * t
        i = int((xs + 3.0) / dx)
        assert m[i - 2] == pytest.approx(1.0) and m[i + 2] == 0.0


def test_perturbation_error_is_linear_in_eps():
    """Prop. Additional error estimate with C_L = 1 (s = 1 <= 2 / (1 + c / lambda)
    for c = 0.75, Example of Section 5.1): delta <= C_MR eps (n + 1), and the
    observed delta decreases with eps with a slope close to one."""
    epss = [1e-2, 1e-3, 1e-4, 1e-5]
    ds = []
    for eps in epss:
        E, d, cr, N = _scalar_errors("II", 1.0, J=9, eps=eps)
        ds.append(d)
        assert d <= 10.0 * eps * (N + 1)
    slope = np.polyfit(np.log10(epss), np.log10(ds), 1)[0]
    assert 0.6 < slope < 1.4, slope


def test_adaptive_advection_at_lattice_speed_tracks_the_exact_shift():
    for eps in (1e-3, 1e-4):
        inst = W.advection(Jmax=9, c=1.0, s=1.0, eps=eps)
        o = oracle_of(inst)
        for n in range(1, 41):
            o.step()
            err = inst.dx * np.abs(o.finest_moments()[0] - np.roll(inst.m0[0], n)).sum()
            assert err <= 4.0 * eps * (n + 1)


def test_vectorial_shallow_water_converges_to_the_exact_dam_break():
    """Pin of the vectorial D1Q2^2 shallow-water equilibrium (m^1eq = m^2,
    m^3eq = (m^2)^2 / m^0 + g (m^0)^2 / 2; a scheme the paper does not print):
    the uniform reference scheme converges to the exact entropy solution of the
    dam break (rarefaction to the left, shock to the right, both exact from the
    Riemann invariants and the Rankine-Hugoniot relation) as the lattice is
    refined.  A dropped g h^2 / 2, a wrong sign or swapped moments would
    converge to another solution, and the error would stop shrinking."""
    Es = []
    for J in (8, 9, 10):
        inst = W.shallow_water(Jmax=J, T=0.2)
        p = params_of(inst)
        F = O.equilibrium(p, inst.m0)
        nsteps = int(round(0.2 / (inst.dx / inst.lam)))
        for _ in range(nsteps):
            F = O.uniform_step(p, F)
        ex = W.sw_riemann_exact(W.cell_edges(inst.a, inst.b, J), nsteps * inst.dx / inst.lam)
        Es.append(inst.dx * np.abs(O.moments(p, F) - ex).sum())
    assert Es[1] < 0.85 * Es[0] and Es[2] < 0.85 * Es[1], Es
    assert Es[2] < 0.05, Es


def test_exact_sod_solution_balances_and_star_state():
    """The exact Sod solution used as a pin: mass and energy conserved inside
    [-1, 1] before the waves reach the ends, momentum grown by the pressure
    difference (p_L - p_R) t, and star-region velocity and densities equal on
    both sides of the contact where the pressure and velocity must agree."""
    e = W.cell_edges(-1.0, 1.0, 7)
    dx = 2.0 / 128
    for t in (0.1, 0.2):
        ex = W.euler_riemann_exact(e, t, sub=16)
        assert abs(ex[0].sum() * dx - 1.125) < 1e-3
        assert abs(ex[2].sum() * dx - 2.75) < 1e-3
        assert abs(ex[1].sum() * dx - 0.9 * t) < 1e-3
    # two points in the star region, left and right of the contact
    l, r = (W.euler_riemann_exact(np.array([x, x + 1e-9]), 1.0, sub=1)[:, 0] for x in (0.5, 1.2))
    ul, ur = l[1] / l[0], r[1] / r[0]
    pl_, pr_ = [(W.GAMMA_GAS - 1.0) * (s[2] - 0.5 * s[1] ** 2 / s[0]) for s in (l, r)]
    assert abs(ul - ur) < 1e-9 and abs(pl_ - pr_) < 1e-9
    assert l[0] > r[0]  # the contact separates the denser expanded gas from the shocked gas


def test_vectorial_euler_converges_to_the_exact_sod_tube():
    """Pin of the vectorial D1Q2^3 Euler scheme of Section 5.3 beyond its
    closed-form flux: the uniform reference scheme converges to the exact Sod
    solution (rarefaction, contact, shock) as the lattice is refined; an error
    in the equilibrium would converge to something else."""
    Es = []
    for J in (8, 9, 10):
        inst = W.sod(Jmax=J, T=0.2)
        p = params_of(inst)
        F = O.equilibrium(p, inst.m0)
        nsteps = int(round(0.2 / (inst.dx / inst.lam)))
        for _ in range(nsteps):
            F = O.uniform_step(p, F)
        ex = W.euler_riemann_exact(W.cell_edges(inst.a, inst.b, J), nsteps * inst.dx / inst.lam, sub=8)
        Es.append(inst.dx * np.abs(O.moments(p, F) - ex).sum())
    assert Es[1] < 0.85 * Es[0] and Es[2] < 0.85 * Es[1], Es
    assert Es[2] < 0.08, Es

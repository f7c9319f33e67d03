"""Pins of the oracle's multiresolution operators against facts of the paper
and of the mathematics (Sections 3.1-3.4)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from oracle_helpers import is_graded, levels, poly_averages, random_graded_tree

RNG = np.random.default_rng(2102)


def test_prediction_coefficients_follow_the_paper():
    rows = read_golden("prediction_coefficients.txt")
    for g, a, num, den, sign in rows:
        g, a = int(g), int(a)
        printed = Fraction(int(num), int(den))
        c = O.prediction_coefficients(g)[a - 1]
        if (g, a) == (3, 3):
            # reading: the printed +5/1024 carries a sign typo
            assert Fraction(c) == -printed
        else:
            assert Fraction(c) == printed


def test_printed_gamma3_sign_is_not_exact_on_linear_averages():
    # exactness on averages of x over the children of cell k needs sum_a a c_a = -1/8
    printed = [Fraction(-201, 1024), Fraction(11, 256), Fraction(5, 1024)]
    corrected = printed[:2] + [-printed[2]]
    assert sum((i + 1) * c for i, c in enumerate(printed)) != Fraction(-1, 8)
    assert sum((i + 1) * c for i, c in enumerate(corrected)) == Fraction(-1, 8)
    for g in (1, 2, 3):
        c = [Fraction(x) for x in O.prediction_coefficients(g)]
        assert sum((i + 1) * ci for i, ci in enumerate(c)) == Fraction(-1, 8)


def test_prediction_weights_of_the_figure():
    rows = read_golden("prediction_figure_weights.txt")
    n, k = 16, 7
    for off, w in rows:
        e = np.zeros(n)
        e[k + int(off)] = 1.0
        fine = O.predict_level(1, O.BC_PERIODIC, e)
        assert fine[2 * k] == pytest.approx(float(w), abs=0)


@pytest.mark.parametrize("gamma", [1, 2, 3])
def test_prediction_exact_on_polynomials_up_to_degree_2gamma(gamma):
    n = 64
    coarse_edges = np.linspace(-1.0, 1.0, n + 1)
    fine_edges = np.linspace(-1.0, 1.0, 2 * n + 1)
    interior = slice(2 * (gamma + 1), 2 * (n - gamma - 1))
    for deg in range(0, 2 * gamma + 2):
        coef = RNG.uniform(-1, 1, deg + 1)
        coef[-1] = 1.0
        fine = O.predict_level(gamma, O.BC_COPY, poly_averages(coef, coarse_edges))
        exact = poly_averages(coef, fine_edges)
        err = np.max(np.abs(fine[interior] - exact[interior]))
        if deg <= 2 * gamma:
            assert err < 1e-13, (gamma, deg, err)
        else:
            assert err > 1e-11, (gamma, deg, err)  # order 2 gamma + 1 is tight


@pytest.mark.parametrize("gamma,bc", list(itertools.product([1, 2, 3], [O.BC_PERIODIC, O.BC_COPY])))
def test_projection_of_prediction_is_identity(gamma, bc):
    for n in (4, 8, 37 * 2, 256):
        f = RNG.normal(size=n)
        back = O.project_level(O.predict_level(gamma, bc, f))
        assert np.max(np.abs(back - f)) <= 4e-16 * max(1.0, np.max(np.abs(f)))


def test_projection_is_the_mean_of_the_children():
    edges = np.linspace(-2.0, 3.0, 65)
    coef = [0.3, -1.0, 2.0, 0.5]
    fine = poly_averages(coef, edges)
    coarse = O.project_level(fine)
    assert np.allclose(coarse, poly_averages(coef, edges[::2]), atol=1e-14, rtol=0)


@pytest.mark.parametrize("gamma", [1, 2, 3])
def test_details_of_siblings_are_opposite(gamma):
    f = RNG.normal(size=128)
    d = f - O.predict_level(gamma, O.BC_PERIODIC, O.project_level(f))
    assert np.max(np.abs(d[0::2] + d[1::2])) < 1e-15 * 8


@pytest.mark.parametrize("gamma,bc", list(itertools.product([1, 2, 3], [O.BC_PERIODIC, O.BC_COPY])))
def test_multiresolution_transform_round_trip(gamma, bc):
    Jmin, Jmax = 2, 9
    x = RNG.normal(size=1 << Jmax)
    packed = O.mr_encode(Jmin, Jmax, gamma, bc, x)
    back = O.mr_decode(Jmin, Jmax, gamma, bc, packed)
    assert np.max(np.abs(back - x)) < 1e-13
    # the packed vector has as many degrees of freedom as the input (odd details omitted)
    L = levels(Jmin, Jmax, packed)
    for l in range(Jmin + 1, Jmax + 1):
        assert np.all(L[l][1::2] == 0.0)


def test_details_vanish_on_quadratics_and_decay_like_the_regularity():
    Jmin, Jmax = 2, 10
    edges = np.linspace(-1.0, 1.0, (1 << Jmax) + 1)
    packed = O.mr_encode(Jmin, Jmax, 1, O.BC_COPY, poly_averages([0.2, -0.7, 1.3], edges))
    L = levels(Jmin, Jmax, packed)
    for l in range(Jmin + 1, Jmax + 1):
        n = 1 << l
        assert np.max(np.abs(L[l][4:n - 4]), initial=0.0) < 1e-13
    # smooth data: |d_l| ~ 2^{-3 l} (mu = 2 gamma + 1 = 3, Prop. Details decay)
    x = np.sin(3.0 * edges)
    avg = -np.diff(np.cos(3.0 * edges)) / 3.0 / np.diff(edges)
    L = levels(Jmin, Jmax, O.mr_encode(Jmin, Jmax, 1, O.BC_COPY, avg))
    dmax = [np.max(np.abs(L[l][8:(1 << l) - 8:2])) for l in range(6, Jmax + 1)]
    ratios = np.array(dmax[:-1]) / np.array(dmax[1:])
    assert np.all((ratios > 6.0) & (ratios < 10.0)), ratios
    del x


@pytest.mark.parametrize("seed,bc", [(1, O.BC_PERIODIC), (2, O.BC_COPY), (3, O.BC_PERIODIC)])
def test_reconstruction_is_the_zero_detail_completion(seed, bc):
    """Definition V: the finest reconstruction averages back to every leaf value
    and has no detail outside the tree (the two facts determine it)."""
    rng = np.random.default_rng(seed)
    Jmin, Jmax = 2, 8
    R = random_graded_tree(Jmin, Jmax, rng, density=0.3, bc=bc)
    p = O.Params(Jmin=Jmin, Jmax=Jmax, eq=O.EQ_BURGERS, lam=1.0, bc=bc)
    o = O.Oracle(p)
    vals = rng.normal(size=(p.q, o.S))
    o.set_state(R, vals)
    fin = o.finest()
    lv, ix, f = o.leaves()
    for h in range(p.q):
        for l, k, v in zip(lv, ix, f[h]):
            dj = Jmax - l
            assert abs(fin[h, k << dj:(k + 1) << dj].mean() - v) < 1e-13
        packed = O.mr_encode(Jmin, Jmax, 1, bc, fin[h])
        Lp, LR = levels(Jmin, Jmax, packed), levels(Jmin, Jmax, R)
        for l in range(Jmin + 1, Jmax + 1):
            outside = (LR[l] == 0) & (np.arange(1 << l) % 2 == 0)
            assert np.max(np.abs(Lp[l][outside]), initial=0.0) < 1e-12


def _all_trees_small(Jmin, Jmax, gamma, bc):
    """Every sibling-closed cell set of levels Jmin..Jmax holding level Jmin."""
    off = O.level_offsets(Jmin, Jmax)
    S = off[Jmax + 1]
    pairs = [(l, k) for l in range(Jmin + 1, Jmax + 1) for k in range(0, 1 << l, 2)]
    for bits in range(1 << len(pairs)):
        R = np.zeros(S, np.uint8)
        R[off[Jmin]:off[Jmin + 1]] = 1
        for i, (l, k) in enumerate(pairs):
            if bits >> i & 1:
                R[off[l] + k] = R[off[l] + k + 1] = 1
        yield R


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_COPY])
def test_grading_gives_the_smallest_graded_tree(bc):
    Jmin, Jmax, gamma = 2, 4, 1
    graded = [R for R in _all_trees_small(Jmin, Jmax, gamma, bc) if is_graded(Jmin, Jmax, gamma, bc, R)]
    assert len(graded) > 3
    rng = np.random.default_rng(7 + bc)
    sets = list(_all_trees_small(Jmin, Jmax, gamma, bc))
    for _ in range(60):
        H = sets[rng.integers(len(sets))]
        G = O.grade(Jmin, Jmax, gamma, bc, H)
        assert is_graded(Jmin, Jmax, gamma, bc, G)
        assert O.check_graded(Jmin, Jmax, gamma, bc, G) == 0
        sup = [R for R in graded if np.all(R >= H)]
        smallest = np.min(np.stack(sup), axis=0)
        assert np.array_equal(G, smallest)


def test_check_graded_rejects_each_violation():
    Jmin, Jmax = 2, 5
    R = random_graded_tree(Jmin, Jmax, np.random.default_rng(3), density=0.5)
    assert O.check_graded(Jmin, Jmax, 1, O.BC_PERIODIC, R) == 0
    off = O.level_offsets(Jmin, Jmax)
    bad = R.copy()
    bad[off[Jmin]] = 0
    assert O.check_graded(Jmin, Jmax, 1, O.BC_PERIODIC, bad) == -1
    l = Jmax
    k = int(np.nonzero(R[off[l]:off[l + 1]])[0][0])
    bad = R.copy()
    bad[off[l] + (k ^ 1)] = 0
    assert O.check_graded(Jmin, Jmax, 1, O.BC_PERIODIC, bad) == -2
    bad = R.copy()
    bad[off[l - 1] + (k >> 1)] = 0
    assert O.check_graded(Jmin, Jmax, 1, O.BC_PERIODIC, bad) < 0

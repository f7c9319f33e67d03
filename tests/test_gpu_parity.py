"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Meshes are compared bit for bit.  Values: every conserved moment on the
leaves of the FP64 path within 1e-12 of the oracle relative to its largest
magnitude over the leaves, and every population within 1e-12 relative to the
instance's largest population (no absolute floor); the
stream uses per-level-gap reconstruction tables while the oracle predicts
level by level, so the two differ by rounding only.  Lock-step tests re-seed the oracle with the GPU state before every
step, so each step's decisions are checked on identical inputs; free-running
tests compare whole trajectories.
"""
import numpy as np
import pytest

import oracle as O
from oracle_helpers import leaves_of, oracle_of, params_of, random_graded_tree
from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, MRError, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_12163_gb300 import capi

    capi.load()


def _solver(insts, precision=MR_FP64, block=None):
    from paper_2102_12163_gb300 import MRLBM

    s = MRLBM(insts, precision=precision, block=block)
    s.set_initial()
    return s


def gpu_state(s, i=0):
    """(R, values) of instance i in the oracle's dense layout."""
    inst = s.instances[i]
    R = s.tree(i)
    lv, ix, f = s.leaves(i)
    off = O.level_offsets(inst.Jmin, inst.Jmax)
    vals = np.zeros((inst.q, off[inst.Jmax + 1]))
    cells = np.array([off[l] for l in lv], dtype=np.int64) + ix
    vals[:, cells] = f
    return R, vals, (lv, ix, f)


def assert_same_leaves(gpu_leaves, o, tol=TOL):
    """Leaf sets equal; every conserved moment on the leaves within tol
    relative to its largest magnitude over the leaves, and every population
    within tol relative to the largest population of the instance (no absolute
    floor; a population that is near zero everywhere, such as the |v| = 2
    lambda populations of a D1Q5 state at rest, is measured against the
    populations that carry the solution)."""
    lv, ix, f = gpu_leaves
    olv, oix, of = o.leaves()
    assert np.array_equal(lv, olv) and np.array_equal(ix, oix), "leaf sets differ"
    if not f.size:
        return
    scale = float(np.max(np.abs(of)))
    err = float(np.max(np.abs(f - of)))
    assert err <= tol * scale, ("populations", err, scale)
    a, b = O.moments(o.p, f), O.moments(o.p, of)
    for j in range(b.shape[0]):
        scale = float(np.max(np.abs(b[j])))
        err = float(np.max(np.abs(a[j] - b[j])))
        assert err <= tol * scale, ("moment", j, err, scale)


def assert_finest_close(a, b, tol=TOL):
    """Reconstructed finest conserved moments: each field within tol relative
    to its largest magnitude."""
    for j in range(b.shape[0]):
        scale = float(np.max(np.abs(b[j])))
        err = float(np.max(np.abs(a[j] - b[j])))
        assert err <= tol * scale, (j, err, scale)


PARITY_CASES = [
    # (name, instance factory)
    ("adv-periodic-J9", lambda: W.random_smooth(9, W.EQ_ADVECTION, seed=1, eps=1e-3)),
    ("burgers-copy-J10", lambda: W.random_smooth(10, W.EQ_BURGERS, seed=2, eps=1e-4, bc=W.BC_COPY)),
    ("sw-copy-J9", lambda: W.random_smooth(9, W.EQ_SW, seed=3, eps=1e-4, bc=W.BC_COPY)),
    ("euler-periodic-J10", lambda: W.random_smooth(10, W.EQ_EULER, seed=4, eps=3e-4)),
    ("euler-copy-J11-jmin4", lambda: W.random_smooth(11, W.EQ_EULER, seed=5, eps=1e-4, bc=W.BC_COPY, Jmin=4)),
    ("adv-config", lambda: W.advection()),
    ("testI-s1.75", lambda: W.scalar_test("I", s=1.75)),
    ("testIII-copy", lambda: W.scalar_test("III", s=1.25)),
    ("testIV", lambda: W.scalar_test("IV", s=0.75)),
]


@pytest.mark.parametrize("name,make", PARITY_CASES, ids=[c[0] for c in PARITY_CASES])
def test_initial_state_matches(name, make):
    inst = make()
    s = _solver(inst)
    o = oracle_of(inst)
    R, _, lvs = gpu_state(s)
    Ro, _ = o.get_state()
    assert np.array_equal(R, Ro)
    assert_same_leaves(lvs, o, tol=0.0)  # same IEEE operations


@pytest.mark.parametrize("name,make", PARITY_CASES, ids=[c[0] for c in PARITY_CASES])
def test_lockstep_parity(name, make):
    inst = make()
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(12):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        Ro, _ = o.get_state()
        assert np.array_equal(R2, Ro), f"step {n}: mesh differs"
        assert_same_leaves(lvs, o)


@pytest.mark.parametrize("name,make", PARITY_CASES[:4], ids=[c[0] for c in PARITY_CASES[:4]])
def test_adapt_then_step_equals_advance(name, make):
    inst = make()
    a, b = _solver(inst), _solver(inst)
    for n in range(5):
        a.adapt()
        a.lbm_step()
        b.advance(1)
    ra, _, la = gpu_state(a)
    rb, _, lb = gpu_state(b)
    assert np.array_equal(ra, rb)
    assert np.array_equal(la[2], lb[2])


@pytest.mark.parametrize("name,make", PARITY_CASES, ids=[c[0] for c in PARITY_CASES])
def test_free_running_parity(name, make):
    inst = make()
    s = _solver(inst)
    o = oracle_of(inst)
    for n in range(40):
        o.step()
        s.advance(1)
        R, _, lvs = gpu_state(s)
        Ro, _ = o.get_state()
        assert np.array_equal(R, Ro), f"step {n}: mesh differs"
        assert_same_leaves(lvs, o)
    m, res = s.audit()
    assert np.allclose(m, o.mass(), rtol=1e-12, atol=1e-13)
    assert res < 1e-12


def test_many_steps_in_one_launch():
    inst = W.burgers(Jmax=11)
    s = _solver(inst)
    o = oracle_of(inst)
    s.advance(60)
    o.step(60)
    R, _, lvs = gpu_state(s)
    assert np.array_equal(R, o.get_state()[0])
    assert_same_leaves(lvs, o)
    upd, steps, leaves = s.stats()
    assert steps == 60 and leaves == len(lvs[0])


def test_finest_reconstruction_matches():
    inst = W.random_smooth(10, W.EQ_EULER, seed=8, eps=1e-4, bc=W.BC_COPY)
    s = _solver(inst)
    o = oracle_of(inst)
    s.advance(15)
    o.step(15)
    assert_finest_close(s.finest(), o.finest_moments())


@pytest.mark.parametrize("eq", [W.EQ_ADVECTION, W.EQ_BURGERS, W.EQ_SW, W.EQ_EULER])
def test_zero_threshold_is_the_uniform_scheme(eq):
    inst = W.random_smooth(8, eq, seed=30 + eq, eps=0.0, bc=W.BC_COPY)
    s = _solver(inst)
    p = params_of(inst)
    F = O.equilibrium(p, inst.m0)
    for n in range(10):
        s.advance(1)
        F = O.uniform_step(p, F)
    lv, ix, f = s.leaves()
    assert np.all(lv == inst.Jmax)
    assert np.max(np.abs(f - F)) < 1e-14


EDGE_CASES = [
    ("single-level", lambda: W.random_smooth(6, W.EQ_BURGERS, seed=11, Jmin=6)),
    ("two-levels", lambda: W.random_smooth(6, W.EQ_SW, seed=12, Jmin=5, bc=W.BC_COPY)),
    ("tiny-levels", lambda: W.random_smooth(4, W.EQ_EULER, seed=13, Jmin=2, eps=1e-5)),
    ("coarsen-all", lambda: W.random_smooth(9, W.EQ_BURGERS, seed=14, eps=10.0)),
    ("jmin5-copy", lambda: W.random_smooth(10, W.EQ_ADVECTION, seed=15, Jmin=5, bc=W.BC_COPY)),
    ("deep-J15", lambda: W.random_smooth(15, W.EQ_BURGERS, seed=16, eps=1e-5)),
]


@pytest.mark.parametrize("name,make", EDGE_CASES, ids=[c[0] for c in EDGE_CASES])
def test_edge_cases_lockstep(name, make):
    inst = make()
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(6):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0]), f"step {n}"
        assert_same_leaves(lvs, o)


@pytest.mark.parametrize("seed,bc", [(40, W.BC_PERIODIC), (41, W.BC_COPY)])
def test_arbitrary_graded_tree_lockstep(seed, bc):
    """Random graded trees (many level jumps, coarse and fine neighbours)."""
    rng = np.random.default_rng(seed)
    inst = W.random_smooth(10, W.EQ_EULER, seed=seed, bc=bc, eps=1e-4)
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    R = random_graded_tree(inst.Jmin, inst.Jmax, rng, density=0.3, bc=bc)
    base = O.equilibrium(params_of(inst), np.array([[1.0], [0.1], [2.0]]))[:, :1]
    vals = base + 0.02 * rng.normal(size=(inst.q, o.S))
    s.set_state(0, R, vals)
    o.set_state(R, vals)
    o.lbm_step()
    s.lbm_step()
    _, _, lvs = gpu_state(s)
    assert_same_leaves(lvs, o)
    for n in range(4):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0])
        assert_same_leaves(lvs, o)


def test_batch_matches_individual_oracles():
    insts = W.batch(n=48, seed=99, Jmax_range=(6, 10))
    s = _solver(insts, block=256)
    steps = 10
    s.advance(steps)
    for i in range(0, len(insts), 5):
        o = oracle_of(insts[i])
        o.step(steps)
        R, _, lvs = gpu_state(s, i)
        assert np.array_equal(R, o.get_state()[0]), i
        assert_same_leaves(lvs, o)
    upd, _, _ = s.stats()
    assert upd > 0


@pytest.mark.parametrize("precision", [MR_FP64, MR_FP32_MIXED])
def test_scalar_only_batch_runs_the_scalar_kernel(precision):
    """A batch of one-field instances alone runs in the scalar kernel variant
    (compiled for more resident blocks): FP64 trees and leaves equal the
    oracle's, FP32 within 1e-4 in L1 of the finest moments, and a captured
    launch replays to the same state."""
    import torch

    insts = [i for i in W.batch(n=64, seed=98, Jmax_range=(6, 10)) if i.eq in (W.EQ_ADVECTION, W.EQ_BURGERS)]
    s, t = _solver(insts, precision=precision), _solver(insts, precision=precision)
    l0 = s.launches()
    g = s.capture(4)
    assert s.launches() - l0 == 1
    with torch.cuda.stream(s.stream):
        for _ in range(3):
            g.replay()
    t.advance(12)
    s.sync()
    t.sync()
    for i in range(len(insts)):
        assert np.array_equal(s.tree(i), t.tree(i)), i
        assert np.array_equal(s.leaves(i)[2], t.leaves(i)[2]), i
    for i in range(0, len(insts), 4):
        o = oracle_of(insts[i])
        o.step(12)
        if precision == MR_FP64:
            R, _, lvs = gpu_state(s, i)
            assert np.array_equal(R, o.get_state()[0]), i
            assert_same_leaves(lvs, o)
        else:
            err = insts[i].dx * np.abs(s.finest(i) - o.finest_moments()).sum(axis=1)
            assert np.all(err < 1e-4), (i, err)


@pytest.mark.parametrize("block", [128, 256, 512, 1024])
def test_block_sizes_agree(block):
    insts = W.batch(n=9, seed=7, Jmax_range=(7, 11))
    ref = _solver(insts, block=256)
    s = _solver(insts, block=block)
    ref.advance(8)
    s.advance(8)
    for i in range(len(insts)):
        assert np.array_equal(ref.tree(i), s.tree(i))
        assert np.array_equal(ref.leaves(i)[2], s.leaves(i)[2])


def test_full_size_sod_lockstep_samples():
    """The largest single instance at its full size (Jmax = 18), in the launch
    configuration the benchmark uses, checked against the oracle on sampled steps."""
    inst = W.sod()
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(3):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0])
        assert_same_leaves(lvs, o)
    s.advance(50)
    R, vals, _ = gpu_state(s)
    o.set_state(R, vals)
    o.step()
    s.advance(1)
    R2, _, lvs = gpu_state(s)
    assert np.array_equal(R2, o.get_state()[0])
    assert_same_leaves(lvs, o)


def test_deepest_tree_lockstep():
    """Jmax = 24, the deepest tree the library takes (2^24 finest cells; the
    bitmasks no longer fit in shared memory and live in global memory): steps
    in lock-step with the oracle give the same tree and leaves; the FP32 path
    stays within 1e-4 (L1 of the finest moments) of the oracle."""
    inst = W.advection(Jmax=24)
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(2):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0]), n
        assert_same_leaves(lvs, o)
    s32 = _solver(inst, precision=MR_FP32_MIXED)
    o2 = O.Oracle(params_of(inst))
    o2.set_initial(inst.m0)
    s32.advance(2)
    o2.step(2)
    err = inst.dx * np.abs(s32.finest() - o2.finest_moments()).sum(axis=1)
    assert np.all(err < 1e-4), err


def test_fp32_path_tracks_the_fp64_oracle():
    inst = W.random_smooth(11, W.EQ_EULER, seed=50, eps=1e-4, bc=W.BC_COPY)
    s = _solver(inst, precision=MR_FP32_MIXED)
    o = oracle_of(inst)
    s.advance(40)
    o.step(40)
    err = inst.dx * np.abs(s.finest() - o.finest_moments()).sum(axis=1)
    assert np.all(err < 1e-4), err
    m, res = s.audit()
    assert np.allclose(m, o.mass(), rtol=1e-5)


def test_nonfinite_populations_are_reported():
    inst = W.random_smooth(8, W.EQ_BURGERS, seed=60)
    s = _solver(inst)
    R, vals, _ = gpu_state(s)
    off = O.level_offsets(inst.Jmin, inst.Jmax)
    vals[0, off[inst.Jmax] + 5] = np.nan
    s.set_state(0, R, vals)
    s.advance(1)
    with pytest.raises(MRError) as ei:
        s.sync()
    assert ei.value.code == -4


def test_autotune_leaves_the_state_and_results_unchanged():
    insts = W.batch(n=24, seed=31, Jmax_range=(6, 11))
    a, b = _solver(insts), _solver(insts)
    a.advance(3)
    b.advance(3)
    tune = a.autotune(2)
    assert tune["block"] in (128, 256, 512, 1024) and tune["ms_per_trial"] > 0.0
    assert a.stats()[0] == b.stats()[0]  # counters restored with the state
    a.advance(5)
    b.advance(5)
    for i in range(len(insts)):
        assert np.array_equal(a.tree(i), b.tree(i)), i
        assert np.array_equal(a.leaves(i)[2], b.leaves(i)[2]), i
    assert a.stats() == b.stats()


def test_graph_replay_equals_advance():
    import torch

    insts = W.batch(n=16, seed=32, Jmax_range=(6, 10))
    a, b = _solver(insts, precision=MR_FP32_MIXED), _solver(insts, precision=MR_FP32_MIXED)
    g = a.capture(4)
    with torch.cuda.stream(a.stream):
        for _ in range(3):
            g.replay()
    b.advance(12)
    a.sync()
    b.sync()
    for i in range(len(insts)):
        assert np.array_equal(a.tree(i), b.tree(i)), i
        assert np.array_equal(a.leaves(i)[2], b.leaves(i)[2]), i
    assert a.stats() == b.stats()


def test_graph_replay_of_every_kernel_variant_equals_advance():
    """A captured launch over a batch that needs three kernel variants (two
    streams forked and joined inside the capture) replays to the same state as
    plain launches."""
    import torch

    insts = _mixed_kinds_batch()
    for prec in (MR_FP64, MR_FP32_MIXED):
        a, b = _solver(insts, precision=prec), _solver(insts, precision=prec)
        assert a.launches() == b.launches()
        l0 = a.launches()
        g = a.capture(3)
        assert a.launches() - l0 == 3  # one kernel per group: gamma > 1, recollision, leaves collision
        with torch.cuda.stream(a.stream):
            for _ in range(4):
                g.replay()
        b.advance(12)
        a.sync()
        b.sync()
        for i in range(len(insts)):
            assert np.array_equal(a.tree(i), b.tree(i)), (prec, i)
            assert np.array_equal(a.leaves(i)[2], b.leaves(i)[2]), (prec, i)
        assert a.stats() == b.stats()


def test_queue_order_and_autotune_leave_results_unchanged_on_every_variant():
    """On a batch that needs three kernel variants (forked launches), the
    results do not depend on the queue order (by scheme or by size) nor on an
    autotuning pass (its trials run on a saved copy of the state)."""
    insts = _mixed_kinds_batch()
    for prec in (MR_FP64, MR_FP32_MIXED):
        a, b, c = (_solver(insts, precision=prec) for _ in range(3))
        b.set_order(False)
        a.advance(2)
        b.advance(2)
        c.advance(2)
        tune = c.autotune(2)
        assert tune["block"] in (128, 256, 512, 1024) and tune["order_by_fields"]
        for s in (a, b, c):
            s.advance(6)
            s.sync()
        for i in range(len(insts)):
            for s in (b, c):
                assert np.array_equal(a.tree(i), s.tree(i)), (prec, i)
                assert np.array_equal(a.leaves(i)[2], s.leaves(i)[2]), (prec, i)
        assert a.stats() == b.stats() == c.stats()


@pytest.mark.parametrize("test", ["I", "II", "III", "IV"])
def test_scalar_tests_full_run_errors(test):
    """Tests I-IV of Table 1 run to their final time on the GPU: the FP64 path's
    trajectory and delta equal the oracle's, and in both precisions delta stays
    far below the reference scheme's error E against the exact solution."""
    inst = W.scalar_test(test, s=1.0)
    N = inst.nsteps
    ref = _solver(inst.with_(eps=0.0))
    ref.advance(N)
    M = ref.finest()[0]
    exact = W.scalar_exact(test, W.cell_edges(inst.a, inst.b, inst.Jmax), N * inst.dx / inst.lam)
    E = inst.dx * np.abs(exact - M).sum()
    o = oracle_of(inst)
    o.step(N)
    d_oracle = inst.dx * np.abs(M - o.finest_moments()[0]).sum()
    for prec in (MR_FP64, MR_FP32_MIXED):
        s = _solver(inst, precision=prec)
        s.advance(N)
        d = inst.dx * np.abs(M - s.finest()[0]).sum()
        if prec == MR_FP64:
            R, _, lvs = gpu_state(s)
            assert np.array_equal(R, o.get_state()[0])
            assert_same_leaves(lvs, o)
            assert abs(d - d_oracle) <= 1e-10
        assert E / d > 5.0, (test, prec, E, d)


GAMMA_CASES = [
    ("g2-euler-periodic", lambda: W.random_smooth(10, W.EQ_EULER, seed=70, eps=3e-4).with_(gamma=2)),
    ("g2-burgers-copy", lambda: W.random_smooth(11, W.EQ_BURGERS, seed=71, eps=1e-4, bc=W.BC_COPY).with_(gamma=2)),
    ("g3-sw-copy", lambda: W.random_smooth(10, W.EQ_SW, seed=72, eps=1e-4, bc=W.BC_COPY).with_(gamma=3)),
    ("g3-adv-periodic", lambda: W.random_smooth(10, W.EQ_ADVECTION, seed=73, eps=1e-4).with_(gamma=3)),
    ("g3-euler-jmin4", lambda: W.random_smooth(9, W.EQ_EULER, seed=74, eps=1e-4, Jmin=4, bc=W.BC_COPY).with_(gamma=3)),
    ("g2-testIV", lambda: W.scalar_test("IV").with_(gamma=2)),
    # 4096 words per bitmask: a large instance in the general variant (every word visited)
    ("g2-burgers-J15", lambda: W.random_smooth(15, W.EQ_BURGERS, seed=76, eps=1e-4).with_(gamma=2)),
]


@pytest.mark.parametrize("name,make", GAMMA_CASES, ids=[c[0] for c in GAMMA_CASES])
def test_wide_stencil_lockstep_parity(name, make):
    """Prediction stencils gamma = 2, 3 (Section 3.1): meshes bit for bit and
    populations within 1e-12 of the oracle, step by step from identical states."""
    inst = make()
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(8):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0]), f"step {n}: mesh differs"
        assert_same_leaves(lvs, o)


@pytest.mark.parametrize("lam", [3.0 * 2.0 ** 14, 3.0 * 2.0 ** -15])
def test_extreme_lattice_velocity_lockstep_parity(lam):
    """A lattice velocity that is no power of two near either end of the
    accepted range [2^-16, 2^16]: the FP64 collision's division by lambda
    (Markstein's correction) gives the oracle's quotients, so meshes match bit
    for bit and populations within 1e-12, step by step from identical states."""
    inst = W.random_smooth(9, W.EQ_ADVECTION, seed=77, eps=1e-4).with_(lam=lam, eqp=0.25 * lam, s=(1.3,))
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(8):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0]), f"step {n}: mesh differs"
        assert_same_leaves(lvs, o)


@pytest.mark.parametrize("name,make", GAMMA_CASES, ids=[c[0] for c in GAMMA_CASES])
def test_wide_stencil_free_running_parity(name, make):
    inst = make()
    s = _solver(inst)
    o = oracle_of(inst)
    for n in range(30):
        o.step()
        s.advance(1)
    R, _, lvs = gpu_state(s)
    assert np.array_equal(R, o.get_state()[0])
    assert_same_leaves(lvs, o)
    assert_finest_close(s.finest(), o.finest_moments())
    m, res = s.audit()
    assert np.allclose(m, o.mass(), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("gamma,bc", [(2, W.BC_PERIODIC), (3, W.BC_COPY), (3, W.BC_PERIODIC)])
def test_wide_stencil_arbitrary_graded_trees(gamma, bc):
    """Random gamma-graded trees with many level jumps: the reconstruction walk,
    the ghost marks and the transfer against the oracle's Definition V."""
    rng = np.random.default_rng(80 + gamma + 3 * bc)
    inst = W.random_smooth(10, W.EQ_EULER, seed=81, bc=bc, eps=1e-4).with_(gamma=gamma)
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    R = random_graded_tree(inst.Jmin, inst.Jmax, rng, density=0.3, bc=bc, gamma=gamma)
    base = O.equilibrium(params_of(inst), np.array([[1.0], [0.1], [2.0]]))[:, :1]
    vals = base + 0.02 * rng.normal(size=(inst.q, o.S))
    s.set_state(0, R, vals)
    o.set_state(R, vals)
    o.lbm_step()
    s.lbm_step()
    _, _, lvs = gpu_state(s)
    assert_same_leaves(lvs, o)
    for n in range(4):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0])
        assert_same_leaves(lvs, o)


def test_wide_stencil_fp32_and_batch():
    insts = [i.with_(gamma=1 + (j % 3)) for j, i in enumerate(W.batch(n=18, seed=90, Jmax_range=(6, 10)))]
    for j, i in enumerate(W.batch(n=18, seed=90, Jmax_range=(6, 10))):
        insts[j].m0 = i.m0
    s64, s32 = _solver(insts), _solver(insts, precision=MR_FP32_MIXED)
    s64.advance(10)
    s32.advance(10)
    for i in range(len(insts)):
        o = oracle_of(insts[i])
        o.step(10)
        R, _, lvs = gpu_state(s64, i)
        assert np.array_equal(R, o.get_state()[0]), i
        assert_same_leaves(lvs, o)
        err = insts[i].dx * np.abs(s32.finest(i) - o.finest_moments()).sum(axis=1)
        assert np.all(err < 1e-4), (i, err)


DQ_CASES = [
    ("d1q3-copy-J9", lambda: W.random_smooth(9, W.EQ_SW_D1Q3, seed=100, eps=1e-4, bc=W.BC_COPY)),
    ("d1q3-periodic-J10", lambda: W.random_smooth(10, W.EQ_SW_D1Q3, seed=101, eps=3e-4)),
    ("d1q5-copy-J9", lambda: W.random_smooth(9, W.EQ_SW_D1Q5, seed=102, eps=1e-4, bc=W.BC_COPY)),
    ("d1q5-periodic-J10", lambda: W.random_smooth(10, W.EQ_SW_D1Q5, seed=103, eps=3e-4)),
    ("d1q5-jmin5", lambda: W.random_smooth(9, W.EQ_SW_D1Q5, seed=104, eps=1e-4, Jmin=5, bc=W.BC_COPY)),
    ("dam-break-d1q3", lambda: W.shallow_water_dq("d1q3")),
    ("dam-break-d1q5", lambda: W.shallow_water_dq("d1q5", s2=1.6)),
]


@pytest.mark.parametrize("name,make", DQ_CASES, ids=[c[0] for c in DQ_CASES])
def test_d1q3_d1q5_lockstep_parity(name, make):
    """Shallow water on one velocity set (Section 5.2): |v| = 2 lambda streams
    two finest cells per side, sigma = 2 enlargement (D1Q5)."""
    inst = make()
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(8):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0]), f"step {n}: mesh differs"
        assert_same_leaves(lvs, o)


@pytest.mark.parametrize("name,make", DQ_CASES, ids=[c[0] for c in DQ_CASES])
def test_d1q3_d1q5_free_running_parity(name, make):
    inst = make()
    s = _solver(inst)
    o = oracle_of(inst)
    for n in range(30):
        o.step()
        s.advance(1)
    R, _, lvs = gpu_state(s)
    assert np.array_equal(R, o.get_state()[0])
    assert_same_leaves(lvs, o)
    assert_finest_close(s.finest(), o.finest_moments())
    m, res = s.audit()
    assert np.allclose(m, o.mass(), rtol=1e-12, atol=1e-13)
    assert res < 1e-12


@pytest.mark.parametrize("eq,bc", [(W.EQ_SW_D1Q3, W.BC_PERIODIC), (W.EQ_SW_D1Q5, W.BC_COPY)])
def test_d1q3_d1q5_arbitrary_graded_trees(eq, bc):
    rng = np.random.default_rng(110 + eq + bc)
    inst = W.random_smooth(10, eq, seed=111, bc=bc, eps=1e-4)
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    R = random_graded_tree(inst.Jmin, inst.Jmax, rng, density=0.3, bc=bc)
    base = O.equilibrium(params_of(inst), np.array([[1.2], [0.1]]))[:, :1]
    vals = base + 0.02 * rng.normal(size=(inst.q, o.S))
    s.set_state(0, R, vals)
    o.set_state(R, vals)
    o.lbm_step()
    s.lbm_step()
    _, _, lvs = gpu_state(s)
    assert_same_leaves(lvs, o)
    for n in range(4):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0])
        assert_same_leaves(lvs, o)


def test_d1q3_d1q5_fp32_and_mixed_batch():
    """A batch mixing every scheme (D1Q2^n, D1Q3, D1Q5) in one context, both
    precisions: FP64 against the oracle, FP32 within 1e-4 in L1."""
    insts = [W.random_smooth(8 + (j % 3), eq, seed=120 + j, eps=1e-4, bc=j % 2)
             for j, eq in enumerate([W.EQ_SW_D1Q3, W.EQ_SW_D1Q5, W.EQ_EULER, W.EQ_BURGERS, W.EQ_SW_D1Q5,
                                     W.EQ_SW, W.EQ_SW_D1Q3, W.EQ_ADVECTION])]
    s64, s32 = _solver(insts), _solver(insts, precision=MR_FP32_MIXED)
    s64.advance(12)
    s32.advance(12)
    for i in range(len(insts)):
        o = oracle_of(insts[i])
        o.step(12)
        R, _, lvs = gpu_state(s64, i)
        assert np.array_equal(R, o.get_state()[0]), i
        assert_same_leaves(lvs, o)
        err = insts[i].dx * np.abs(s32.finest(i) - o.finest_moments()).sum(axis=1)
        assert np.all(err < 1e-4), (i, err)


RC = W.COLLIDE_RECONSTRUCTED
RECOLL_CASES = [
    ("rc-burgers-copy", lambda: W.random_smooth(10, W.EQ_BURGERS, seed=130, eps=1e-4, bc=W.BC_COPY).with_(collision=RC)),
    ("rc-euler-periodic", lambda: W.random_smooth(10, W.EQ_EULER, seed=131, eps=3e-4).with_(collision=RC)),
    ("rc-sw-copy", lambda: W.random_smooth(9, W.EQ_SW, seed=132, eps=1e-4, bc=W.BC_COPY).with_(collision=RC)),
    ("rc-d1q5-periodic", lambda: W.random_smooth(9, W.EQ_SW_D1Q5, seed=133, eps=1e-4).with_(collision=RC)),
    ("rc-d1q3-copy", lambda: W.random_smooth(9, W.EQ_SW_D1Q3, seed=134, eps=1e-4, bc=W.BC_COPY).with_(collision=RC)),
    ("rc-g2-euler", lambda: W.random_smooth(9, W.EQ_EULER, seed=135, eps=1e-4).with_(collision=RC, gamma=2)),
    ("rc-testIV", lambda: W.scalar_test("IV").with_(collision=RC)),
]


@pytest.mark.parametrize("name,make", RECOLL_CASES, ids=[c[0] for c in RECOLL_CASES])
def test_reconstructed_collision_lockstep_parity(name, make):
    """eq. reconstructedCollision (Section 4.5): equilibria averaged over each
    leaf's reconstructed finest cells; meshes bit for bit, values within 1e-12."""
    inst = make()
    s = _solver(inst)
    o = O.Oracle(params_of(inst))
    for n in range(8):
        R, vals, _ = gpu_state(s)
        o.set_state(R, vals)
        o.step()
        s.advance(1)
        R2, _, lvs = gpu_state(s)
        assert np.array_equal(R2, o.get_state()[0]), f"step {n}: mesh differs"
        assert_same_leaves(lvs, o)


@pytest.mark.parametrize("name,make", RECOLL_CASES, ids=[c[0] for c in RECOLL_CASES])
def test_reconstructed_collision_free_running_parity(name, make):
    inst = make()
    s = _solver(inst)
    o = oracle_of(inst)
    for n in range(25):
        o.step()
        s.advance(1)
    R, _, lvs = gpu_state(s)
    assert np.array_equal(R, o.get_state()[0])
    assert_same_leaves(lvs, o)
    m, res = s.audit()
    assert np.allclose(m, o.mass(), rtol=1e-12, atol=1e-13)


MIXED_KINDS = [(W.EQ_BURGERS, 1, RC), (W.EQ_EULER, 1, 0), (W.EQ_SW_D1Q5, 1, RC), (W.EQ_SW, 2, 0),
               (W.EQ_ADVECTION, 1, RC), (W.EQ_SW_D1Q3, 1, 0), (W.EQ_EULER, 3, RC), (W.EQ_BURGERS, 1, 0)]


def _mixed_kinds_batch():
    """Every kernel variant in one batch: fast (several fields), scalar, gamma =
    1 with the reconstructed collision, and gamma = 2, 3."""
    return [W.random_smooth(8 + (j % 3), eq, seed=140 + j, eps=1e-4, bc=j % 2).with_(gamma=g, collision=c)
            for j, (eq, g, c) in enumerate(MIXED_KINDS)]


def test_reconstructed_collision_fp32_and_mixed_batch():
    """Both collisions, all schemes and stencils in one context (four kernel
    variants, four launches on two streams), FP64 against the oracle and FP32
    within 1e-4."""
    insts = _mixed_kinds_batch()
    s64, s32 = _solver(insts), _solver(insts, precision=MR_FP32_MIXED)
    s64.advance(10)
    s32.advance(10)
    for i in range(len(insts)):
        o = oracle_of(insts[i])
        o.step(10)
        R, _, lvs = gpu_state(s64, i)
        assert np.array_equal(R, o.get_state()[0]), i
        assert_same_leaves(lvs, o)
        err = insts[i].dx * np.abs(s32.finest(i) - o.finest_moments()).sum(axis=1)
        assert np.all(err < 1e-4), (i, err)


@pytest.mark.parametrize("precision", [MR_FP64, MR_FP32_MIXED])
def test_full_batch_in_the_benchmark_launch_configuration(precision):
    """The 4096-instance batch at full size, in the benchmark's configuration
    (autotuned launch shape, a CUDA graph holding one 64-step persistent launch,
    replayed): sampled instances against the oracle after 64 steps — meshes bit
    for bit in FP64, FP32 within 1e-4 (L1) of the oracle's conserved moments."""
    import torch

    insts = W.batch(n=4096, seed=12163)
    from paper_2102_12163_gb300 import MRLBM

    s = MRLBM(insts, precision=precision)
    s.set_initial()
    s.autotune(8)
    g = s.capture(32)
    with torch.cuda.stream(s.stream):
        g.replay()
        g.replay()
    s.sync()
    for i in (0, 1365, 2730, 4095):
        o = oracle_of(insts[i])
        o.step(64)
        if precision == MR_FP64:
            R, _, lvs = gpu_state(s, i)
            assert np.array_equal(R, o.get_state()[0]), i
            assert_same_leaves(lvs, o)
        else:
            err = insts[i].dx * np.abs(s.finest(i) - o.finest_moments()).sum(axis=1)
            assert np.all(err < 1e-4), (i, err)
    upd, steps, _ = s.stats()
    assert steps == 64 and upd > 0

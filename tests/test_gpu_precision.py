"""Precision-specific parity of the CUDA path with the FP64 oracle.

FP32 path (populations, predictions, reconstruction and collide / stream in
float; threshold decisions re-checked in FP64 near the thresholds):
  - lock-step meshes: the oracle is fed the GPU's FP32 leaf values (as
    doubles) before every adaptation and the two trees are compared.  The GPU
    decides on its stored state, whose internal cells are FP32 projections of
    the leaves; the oracle projects the same leaves exactly.  The two differ
    by at most B_l = (2.25 (Jmax - l + 1) + 4) u max|f| in a detail of level l
    (u = 2^-24: one rounding per projection level on the four stencil values,
    weights 1, 1, 1/8, 1/8, plus the detail's own evaluation), so the trees
    must be equal unless some pair's exact detail lies within 2 B_l of its
    threshold eps_l or Harten level 2^(mu_bar + 1) eps_l;
  - one collide + stream from the same state, element by element: every leaf
    population within K u max|f| of the oracle, K = 64 + 8 (Jmax - Jmin)
    (collision, per-level FP32 projections feeding the reconstruction tables,
    compensated 4-term sums, the stream's difference of two edge values).
Both precisions:
  - a detail exactly equal to its threshold is kept (">=" as printed) and is
    counted by the near-tie log (mr_near_ties).
"""
import numpy as np
import pytest

import oracle as O
from oracle_helpers import oracle_of, params_of, prescribed_detail_state
from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_12163_gb300 import capi

    capi.load()


def _solver(insts, precision):
    from paper_2102_12163_gb300 import MRLBM

    s = MRLBM(insts, precision=precision)
    s.set_initial()
    return s


def _gpu_state(s, i=0):
    inst = s.instances[i]
    R = s.tree(i)
    lv, ix, f = s.leaves(i)
    off = O.level_offsets(inst.Jmin, inst.Jmax)
    vals = np.zeros((inst.q, off[inst.Jmax + 1]))
    vals[:, np.array([off[l] for l in lv], dtype=np.int64) + ix] = f
    return R, vals, (lv, ix, f)


CASES = [
    ("adv-periodic-J9", lambda: W.random_smooth(9, W.EQ_ADVECTION, seed=1, eps=1e-3)),
    ("burgers-copy-J10", lambda: W.random_smooth(10, W.EQ_BURGERS, seed=2, eps=1e-4, bc=W.BC_COPY)),
    ("sw-copy-J9", lambda: W.random_smooth(9, W.EQ_SW, seed=3, eps=1e-4, bc=W.BC_COPY)),
    ("euler-periodic-J10", lambda: W.random_smooth(10, W.EQ_EULER, seed=4, eps=3e-4)),
    ("euler-copy-J11-jmin4", lambda: W.random_smooth(11, W.EQ_EULER, seed=5, eps=1e-4, bc=W.BC_COPY, Jmin=4)),
    ("d1q3-copy-J9", lambda: W.shallow_water_dq("d1q3", Jmax=9)),
    ("d1q5-copy-J9", lambda: W.shallow_water_dq("d1q5", Jmax=9)),
    ("gamma2-burgers-J9", lambda: W.random_smooth(9, W.EQ_BURGERS, seed=6, eps=1e-4).with_(gamma=2)),
    ("testIV", lambda: W.scalar_test("IV", s=0.75)),
]


def _near_band_pairs(inst, D, M):
    """Pairs whose exact detail lies within 2 B_l of eps_l or of the Harten level."""
    off = O.level_offsets(inst.Jmin, inst.Jmax)
    n = 0
    for l in range(inst.Jmin + 1, inst.Jmax + 1):
        Dl = D[off[l]:off[l + 1]:2]
        B = 2.0 * (2.25 * (inst.Jmax - l + 1) + 4.0) * U32 * M
        eps_l = inst.eps * 2.0 ** (l - inst.Jmax)
        big = eps_l * 2.0 ** (inst.mu_bar + 1)
        n += int(np.sum(np.abs(Dl - eps_l) <= B)) + (int(np.sum(np.abs(Dl - big) <= B)) if l < inst.Jmax else 0)
    return n


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp32_lockstep_meshes(name, make):
    inst = make()
    s = _solver(inst, MR_FP32_MIXED)
    o = O.Oracle(params_of(inst))
    differ = 0
    for n in range(16):
        R, vals, (_, _, f) = _gpu_state(s)
        o.set_state(R, vals)
        o.adapt()
        s.adapt()
        Rg, Ro = s.tree(), o.get_state()[0]
        if not np.array_equal(Rg, Ro):
            D = o.trace()[0]
            assert _near_band_pairs(inst, D, float(np.max(np.abs(f)))) > 0, f"step {n}: meshes differ off the band"
            differ += 1
        s.lbm_step()
    assert differ <= 2, differ


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp32_collide_stream_elementwise(name, make):
    inst = make()
    s = _solver(inst, MR_FP32_MIXED)
    o = O.Oracle(params_of(inst))
    K = 64 + 8 * (inst.Jmax - inst.Jmin)
    worst = 0.0
    for n in range(10):
        s.adapt()
        R, vals, (_, _, f) = _gpu_state(s)
        o.set_state(R, vals)
        o.lbm_step()
        s.lbm_step()
        lv, ix, g = s.leaves()
        olv, oix, of = o.leaves()
        assert np.array_equal(lv, olv) and np.array_equal(ix, oix)
        M = max(float(np.max(np.abs(f))), float(np.max(np.abs(of))))
        err = float(np.max(np.abs(g - of)))
        worst = max(worst, err / (U32 * M))
        assert err <= K * U32 * M, (n, err / (U32 * M), K)
    assert worst > 0.0  # FP32 really ran


@pytest.mark.parametrize("precision", [MR_FP64, MR_FP32_MIXED])
@pytest.mark.parametrize("bc", [W.BC_PERIODIC, W.BC_COPY])
def test_exact_tie_is_kept_and_logged(precision, bc):
    """Population 0 of a full tree (levels 2..6, eps = 1/8, so eps_4 = 1/32)
    carries one detail exactly equal to eps_4 and one equal to the Harten level
    2 eps_5 = 1/8 (mu_bar = 0): both pairs are kept, the second refined, the
    tree equals the oracle's and both ties are in the log."""
    inst = W.random_smooth(6, W.EQ_BURGERS, seed=3, eps=0.125, bc=bc).with_(Jmin=2, mu_bar=0)
    R, vals = prescribed_detail_state(2, 6, bc, inst.q, {(4, 3): 1.0 / 32.0, (5, 10): 1.0 / 8.0})
    s = _solver(inst, precision)
    s.set_state(0, R, vals)
    o = O.Oracle(params_of(inst))
    o.set_state(R, vals)
    assert s.near_ties() == 0
    s.adapt()
    o.adapt()
    Rg, Ro = s.tree(), o.get_state()[0]
    assert np.array_equal(Rg, Ro)
    off = O.level_offsets(2, 6)
    assert Ro[off[4] + 6] and Ro[off[4] + 7]  # the tied pair is kept
    assert all(Ro[off[6] + c] for c in (40, 41, 42, 43))  # the Harten tie refines
    assert s.near_ties() >= 2


def test_no_ties_logged_away_from_thresholds():
    inst = W.random_smooth(6, W.EQ_BURGERS, seed=3, eps=0.125).with_(Jmin=2, mu_bar=0)
    R, vals = prescribed_detail_state(2, 6, W.BC_PERIODIC, inst.q, {(4, 3): 3.0 / 64.0})
    s = _solver(inst, MR_FP64)
    s.set_state(0, R, vals)
    s.adapt()
    assert s.near_ties() == 0

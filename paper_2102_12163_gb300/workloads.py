"""Seeded synthetic workloads shaped like the test cases of arXiv 2102.12163.

This module only describes problems: parameters, the exact cell averages of
the initial conserved moments on the finest lattice and, for the scalar test
cases of Table 1, the cell averages of the exact entropy solution of the PDE
at a later time.  It holds none of the method's arithmetic, and both the CUDA
path and the CPU oracle take their inputs from it.

Workloads (Section 5 of the paper for the shapes; the paper's own runs use
Jmax = 9 and unstated boundary conditions):
  advection  D1Q2, c = 0.75, lambda = 1, Omega = [-3, 3] periodic, indicator of
             [-1, 1], Jmax = 10, T = 0.4 (Table 1 style, Test II-like)
  burgers    D1Q2 Burgers, lambda = 1, Omega = [-3, 3] copy boundary, step of
             height 0.5 plus three seeded Gaussian bumps, Jmax = 13, T = 1.0
  shallow    vectorial D1Q2^2 shallow water, g = 1, lambda = 2, Omega = [-1, 1],
             dam break h = 2 | 1, u = 0, Jmax = 15, T = 0.4
  sod        vectorial D1Q2^3 Euler, gamma_gas = 1.4, lambda = 3, Omega = [-1, 1],
             Sod tube, Jmax = 18, T = 0.4
  batch      4096 seeded instances mixing the four families, Jmax in 8..14,
             eps log-uniform in [1e-5, 1e-2], piecewise-constant data with
             1..6 jumps, periodic.
  sw_d1q3/5  shallow water dam break with the D1Q3 / D1Q5 schemes (Section 5.2):
             (h, u) = (2, 0) | (1, 0), lambda 2, g 1, T 0.2, Jmax 9, copy boundary.
  test1..4   the scalar D1Q2 test cases I-IV of Table 1 (Section 5.1):
             Omega = [-3, 3], lambda = 1, Jmin 2, Jmax 9, gamma 1, eps 1e-4,
             with their exact solutions (scalar_test, scalar_exact).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

EQ_ADVECTION, EQ_BURGERS, EQ_SW, EQ_EULER = 0, 1, 2, 3
EQ_SW_D1Q3, EQ_SW_D1Q5 = 4, 5  # shallow water on one velocity set (Section 5.2)
COLLIDE_LEAVES, COLLIDE_RECONSTRUCTED = 0, 1
NFIELDS = {EQ_ADVECTION: 1, EQ_BURGERS: 1, EQ_SW: 2, EQ_EULER: 3, EQ_SW_D1Q3: 2, EQ_SW_D1Q5: 2}
NPOP = {EQ_ADVECTION: 2, EQ_BURGERS: 2, EQ_SW: 4, EQ_EULER: 6, EQ_SW_D1Q3: 3, EQ_SW_D1Q5: 5}
BC_PERIODIC, BC_COPY = 0, 1
GAMMA_GAS = 1.4


@dataclass
class Instance:
    """One 1D problem: scheme, multiresolution parameters and initial data."""

    name: str
    eq: int
    Jmin: int
    Jmax: int
    eps: float
    lam: float
    a: float
    b: float
    bc: int
    T: float
    gamma: int = 1
    mu_bar: int = 0
    s: tuple = (1.0, 1.0, 1.0)
    eqp: float = 0.0  # advection velocity | unused | gravity | gas constant | gravity (D1Q3, D1Q5)
    collision: int = 0  # 0: leaves collision, 1: reconstructed collision (Section 4.5)
    m0: np.ndarray = field(default=None, repr=False)  # (nf, 2^Jmax) cell averages

    @property
    def nf(self) -> int:
        return NFIELDS[self.eq]

    @property
    def q(self) -> int:
        return NPOP[self.eq]

    @property
    def dx(self) -> float:
        return (self.b - self.a) / (1 << self.Jmax)

    @property
    def nsteps(self) -> int:
        """N = T / dt with dt = dx / lambda (acoustic scaling), nearest integer."""
        return int(round(self.T * self.lam / self.dx))

    def with_(self, **kw) -> "Instance":
        return replace(self, **kw)


# exact cell averages ---------------------------------------------------------

def cell_edges(a: float, b: float, J: int) -> np.ndarray:
    n = 1 << J
    return a + (b - a) * np.arange(n + 1, dtype=np.float64) / n


def avg_indicator(edges: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Average of the indicator of [lo, hi] over each cell (overlap length / dx)."""
    left, right = edges[:-1], edges[1:]
    ov = np.clip(np.minimum(right, hi) - np.maximum(left, lo), 0.0, None)
    return ov / (right - left)


def avg_gaussian(edges: np.ndarray, amp: float, x0: float, w: float) -> np.ndarray:
    """Average of amp * exp(-(x - x0)^2 / (2 w^2)) over each cell, via erf."""
    from scipy.special import erf

    z = (edges - x0) / (math.sqrt(2.0) * w)
    prim = amp * w * math.sqrt(math.pi / 2.0) * erf(z)
    return np.diff(prim) / np.diff(edges)


def avg_piecewise(edges: np.ndarray, jumps: np.ndarray, values: np.ndarray) -> np.ndarray:
    """Average of a piecewise-constant function: values[i] on (jumps[i-1], jumps[i])."""
    bounds = np.concatenate([[edges[0]], np.sort(jumps), [edges[-1]]])
    out = np.zeros(edges.size - 1)
    for i, v in enumerate(values):
        out += v * avg_indicator(edges, bounds[i], bounds[i + 1])
    return out


# the named workloads ---------------------------------------------------------

def advection(Jmax: int = 10, eps: float = 1e-4, c: float = 0.75, s: float = 1.0,
              lo: float = -1.0, hi: float = 1.0, T: float = 0.4, Jmin: int = 2) -> Instance:
    inst = Instance("advection", EQ_ADVECTION, Jmin, Jmax, eps, 1.0, -3.0, 3.0, BC_PERIODIC, T,
                    s=(s,), eqp=c)
    inst.m0 = avg_indicator(cell_edges(inst.a, inst.b, Jmax), lo, hi)[None, :]
    return inst


def burgers(Jmax: int = 13, eps: float = 1e-4, seed: int = 2102, T: float = 1.0, s: float = 1.0,
            Jmin: int = 2) -> Instance:
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = rng.uniform(-0.5, 0.5)
    amp = rng.uniform(0.05, 0.15, 3)
    x0 = rng.uniform(-2.5, 2.5, 3)
    w = rng.uniform(0.05, 0.2, 3)
    inst = Instance("burgers", EQ_BURGERS, Jmin, Jmax, eps, 1.0, -3.0, 3.0, BC_COPY, T, s=(s,))
    e = cell_edges(inst.a, inst.b, Jmax)
    rho = 0.5 * avg_indicator(e, inst.a - 1.0, xs)
    for i in range(3):
        rho = rho + avg_gaussian(e, amp[i], x0[i], w[i])
    inst.m0 = rho[None, :]
    return inst


def shallow_water(Jmax: int = 15, eps: float = 1e-4, T: float = 0.4, g: float = 1.0,
                  s: float = 1.0, Jmin: int = 2) -> Instance:
    inst = Instance("shallow", EQ_SW, Jmin, Jmax, eps, 2.0, -1.0, 1.0, BC_COPY, T,
                    s=(s, s), eqp=g)
    e = cell_edges(inst.a, inst.b, Jmax)
    h = 2.0 * avg_indicator(e, -1.0, 0.0) + 1.0 * avg_indicator(e, 0.0, 1.0)
    inst.m0 = np.stack([h, np.zeros_like(h)])
    return inst


def sod(Jmax: int = 18, eps: float = 1e-4, T: float = 0.4, s: float = 1.0, Jmin: int = 2) -> Instance:
    inst = Instance("sod", EQ_EULER, Jmin, Jmax, eps, 3.0, -1.0, 1.0, BC_COPY, T,
                    s=(s, s, s), eqp=GAMMA_GAS)
    e = cell_edges(inst.a, inst.b, Jmax)
    left, right = avg_indicator(e, -1.0, 0.0), avg_indicator(e, 0.0, 1.0)
    rho = 1.0 * left + 0.125 * right
    E = 2.5 * left + 0.25 * right
    inst.m0 = np.stack([rho, np.zeros_like(rho), E])
    return inst


def batch(n: int = 4096, seed: int = 12163, Jmin: int = 2, Jmax_range=(8, 14),
          eps_log10=(-5.0, -2.0)) -> list[Instance]:
    """Mixed batch of independent periodic instances with piecewise-constant data."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        fam = int(rng.integers(0, 4))
        J = int(rng.integers(Jmax_range[0], Jmax_range[1] + 1))
        eps = float(10.0 ** rng.uniform(*eps_log10))
        nj = int(rng.integers(1, 7))
        jumps = np.sort(rng.uniform(-1.0, 1.0, nj))
        e = cell_edges(-1.0, 1.0, J)
        if fam == EQ_ADVECTION or fam == EQ_BURGERS:
            vals = rng.uniform(-0.9, 0.9, nj + 1)
            c = float(rng.uniform(-0.9, 0.9)) if fam == EQ_ADVECTION else 0.0
            inst = Instance(f"b{i}", fam, Jmin, J, eps, 1.0, -1.0, 1.0, BC_PERIODIC, 0.0,
                            s=(1.0,), eqp=c)
            inst.m0 = avg_piecewise(e, jumps, vals)[None, :]
        elif fam == EQ_SW:
            h = rng.uniform(0.5, 2.0, nj + 1)
            inst = Instance(f"b{i}", fam, Jmin, J, eps, 2.0, -1.0, 1.0, BC_PERIODIC, 0.0,
                            s=(1.0, 1.0), eqp=1.0)
            hh = avg_piecewise(e, jumps, h)
            inst.m0 = np.stack([hh, np.zeros_like(hh)])
        else:
            rho = rng.uniform(0.4, 1.0, nj + 1)
            p = rng.uniform(0.1, 1.0, nj + 1)
            inst = Instance(f"b{i}", fam, Jmin, J, eps, 3.0, -1.0, 1.0, BC_PERIODIC, 0.0,
                            s=(1.0, 1.0, 1.0), eqp=GAMMA_GAS)
            rr = avg_piecewise(e, jumps, rho)
            EE = avg_piecewise(e, jumps, p / (GAMMA_GAS - 1.0))
            inst.m0 = np.stack([rr, np.zeros_like(rr), EE])
        out.append(inst)
    return out


def batch_sw(n: int = 4096, seed: int = 5202, Jmin: int = 2, Jmax_range=(8, 14),
             eps_log10=(-5.0, -2.0)) -> list[Instance]:
    """Batch of shallow water instances on one velocity set, half D1Q3 (lambda 2)
    and half D1Q5 (lambda 3), periodic on [-1, 1], h piecewise constant in
    [0.5, 2] with 1..6 jumps, u = 0, g = 1, relaxation s^2 in [1, 1.6]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        eq = EQ_SW_D1Q3 if rng.random() < 0.5 else EQ_SW_D1Q5
        J = int(rng.integers(Jmax_range[0], Jmax_range[1] + 1))
        eps = float(10.0 ** rng.uniform(*eps_log10))
        nj = int(rng.integers(1, 7))
        jumps = np.sort(rng.uniform(-1.0, 1.0, nj))
        s2 = float(rng.uniform(1.0, 1.6))
        inst = Instance(f"w{i}", eq, Jmin, J, eps, 2.0 if eq == EQ_SW_D1Q3 else 3.0, -1.0, 1.0, BC_PERIODIC, 0.0,
                        s=(s2,) if eq == EQ_SW_D1Q3 else (s2, 1.0, 1.0), eqp=1.0)
        hh = avg_piecewise(cell_edges(-1.0, 1.0, J), jumps, rng.uniform(0.5, 2.0, nj + 1))
        inst.m0 = np.stack([hh, np.zeros_like(hh)])
        out.append(inst)
    return out


def random_smooth(Jmax: int, eq: int, seed: int, Jmin: int = 2, eps: float = 1e-3, bc: int = BC_PERIODIC,
                  nmodes: int = 3) -> Instance:
    """Small seeded instance with smooth plus step data, for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = {EQ_ADVECTION: 1.0, EQ_BURGERS: 1.0, EQ_SW: 2.0, EQ_EULER: 3.0, EQ_SW_D1Q3: 2.0, EQ_SW_D1Q5: 3.0}[eq]
    nf = NFIELDS[eq]
    inst = Instance(f"rand{seed}", eq, Jmin, Jmax, eps, lam, -1.0, 1.0, bc, 0.0,
                    s=tuple(float(v) for v in rng.uniform(0.8, 1.6, 3)),
                    eqp={EQ_ADVECTION: float(rng.uniform(-0.9, 0.9)), EQ_BURGERS: 0.0,
                         EQ_SW: 1.0, EQ_EULER: GAMMA_GAS, EQ_SW_D1Q3: 1.0, EQ_SW_D1Q5: 1.0}[eq])
    e = cell_edges(-1.0, 1.0, Jmax)
    xs = float(rng.uniform(-0.5, 0.5))
    base = avg_indicator(e, -1.0, xs)
    bumps = np.zeros(e.size - 1)
    for _ in range(nmodes):
        bumps = bumps + avg_gaussian(e, float(rng.uniform(0.02, 0.1)), float(rng.uniform(-0.8, 0.8)),
                                     float(rng.uniform(0.03, 0.2)))
    if eq in (EQ_ADVECTION, EQ_BURGERS):
        inst.m0 = (0.5 * base + bumps - 0.2)[None, :]
    elif eq in (EQ_SW, EQ_SW_D1Q3, EQ_SW_D1Q5):
        h = 1.0 + 0.8 * base + bumps
        inst.m0 = np.stack([h, 0.1 * bumps])
    else:
        rho = 0.5 + 0.4 * base + bumps
        p = 0.3 + 0.5 * base
        inst.m0 = np.stack([rho, 0.05 * bumps, p / (GAMMA_GAS - 1.0)])
    return inst


# shallow water with the D1Q3 / D1Q5 schemes (Section 5.2) ---------------------

def shallow_water_dq(scheme: str = "d1q3", Jmax: int = 9, eps: float = 1e-4, s2: float = 1.5, T: float = 0.2,
                     Jmin: int = 2) -> Instance:
    """Section 5.2: Riemann datum (h, u) = (2, 0) for x < 0, (1, 0) for x > 0 on
    [-1, 1], lambda = 2, g = 1, T = 0.2; relaxation s^2 (D1Q5: s^3 = s^4 = 1,
    alpha = beta = 1); copy boundary (no wave reaches it before T)."""
    eq = {"d1q3": EQ_SW_D1Q3, "d1q5": EQ_SW_D1Q5}[scheme]
    inst = Instance(f"sw_{scheme}", eq, Jmin, Jmax, eps, 2.0, -1.0, 1.0, BC_COPY, T,
                    s=(s2,) if eq == EQ_SW_D1Q3 else (s2, 1.0, 1.0), eqp=1.0)
    e = cell_edges(inst.a, inst.b, Jmax)
    h = 2.0 * avg_indicator(e, -1.0, 0.0) + 1.0 * avg_indicator(e, 0.0, 1.0)
    inst.m0 = np.stack([h, np.zeros_like(h)])
    return inst


def sw_riemann_exact(edges: np.ndarray, t: float, hl: float = 2.0, hr: float = 1.0, g: float = 1.0,
                     sub: int = 64) -> np.ndarray:
    """Cell averages of (h, h u) of the exact entropy solution of the shallow
    water Riemann problem with u = 0 on both sides and hl > hr (rarefaction to
    the left, shock to the right); the averages are midpoint sums over `sub`
    points per cell (the solution is piecewise smooth)."""
    cl, cr = math.sqrt(g * hl), math.sqrt(g * hr)

    def fL(h):  # rarefaction branch, h < hl
        return 2.0 * (math.sqrt(g * h) - cl)

    def fR(h):  # shock branch, h > hr
        return (h - hr) * math.sqrt(0.5 * g * (h + hr) / (h * hr))

    lo, hi = hr, hl
    for _ in range(200):  # fL + fR increasing in h; root between hr and hl
        mid = 0.5 * (lo + hi)
        if fL(mid) + fR(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    hs = 0.5 * (lo + hi)
    us = -fL(hs)
    cs = math.sqrt(g * hs)
    S = hs * us / (hs - hr)  # Rankine-Hugoniot speed of the shock
    x = np.asarray(edges, dtype=np.float64)
    n = x.size - 1
    pts = x[:-1, None] + (np.arange(sub)[None, :] + 0.5) / sub * np.diff(x)[:, None]
    xi = pts / t
    h = np.where(xi < -cl, hl, np.where(xi < us - cs, ((2.0 * cl - xi) / 3.0) ** 2 / g,
                                        np.where(xi < S, hs, hr)))
    u = np.where(xi < -cl, 0.0, np.where(xi < us - cs, (2.0 * cl + 2.0 * xi) / 3.0,
                                         np.where(xi < S, us, 0.0)))
    return np.stack([h.mean(axis=1), (h * u).mean(axis=1)]).reshape(2, n)


def euler_riemann_exact(edges: np.ndarray, t: float, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
                        gas: float = GAMMA_GAS, sub: int = 64) -> np.ndarray:
    """Cell averages of (rho, rho u, E) of the exact solution of the Euler
    Riemann problem with primitive states (rho, u, p) left and right of x = 0
    (defaults: the Sod tube), midpoint sums over `sub` points per cell.  The
    star pressure is the root of f_L(p) + f_R(p) + u_R - u_L, each f_K the
    shock (Rankine-Hugoniot) or rarefaction (Riemann invariant) branch, found by
    bisection; the solution is then sampled on x / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = math.sqrt(gas * pl / rl), math.sqrt(gas * pr / rr)

    def f(p, r, pk, ak):
        if p > pk:  # shock
            A, B = 2.0 / ((gas + 1.0) * r), (gas - 1.0) / (gas + 1.0) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2.0 * ak / (gas - 1.0) * ((p / pk) ** ((gas - 1.0) / (2.0 * gas)) - 1.0)

    lo, hi = 1e-12, 10.0 * max(pl, pr)
    for _ in range(200):  # f_L + f_R increasing in p
        mid = 0.5 * (lo + hi)
        if f(mid, rl, pl, al) + f(mid, rr, pr, ar) + (ur - ul) < 0.0:
            lo = mid
        else:
            hi = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, ar) - f(ps, rl, pl, al))
    gm = (gas - 1.0) / (gas + 1.0)

    def sample(xi):
        if xi < us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                S = ul - al * math.sqrt((gas + 1.0) / (2.0 * gas) * ps / pl + (gas - 1.0) / (2.0 * gas))
                return (rl, ul, pl) if xi < S else (rs, us, ps)
            rs = rl * (ps / pl) ** (1.0 / gas)
            head, tail = ul - al, us - al * (ps / pl) ** ((gas - 1.0) / (2.0 * gas))
            if xi < head:
                return rl, ul, pl
            if xi > tail:
                return rs, us, ps
            u = 2.0 / (gas + 1.0) * (al + 0.5 * (gas - 1.0) * ul + xi)
            c = 2.0 / (gas + 1.0) * (al + 0.5 * (gas - 1.0) * (ul - xi))
            r = rl * (c / al) ** (2.0 / (gas - 1.0))
            return r, u, pl * (c / al) ** (2.0 * gas / (gas - 1.0))
        if ps > pr:  # right shock
            rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
            S = ur + ar * math.sqrt((gas + 1.0) / (2.0 * gas) * ps / pr + (gas - 1.0) / (2.0 * gas))
            return (rs, us, ps) if xi < S else (rr, ur, pr)
        rs = rr * (ps / pr) ** (1.0 / gas)
        head, tail = ur + ar, us + ar * (ps / pr) ** ((gas - 1.0) / (2.0 * gas))
        if xi > head:
            return rr, ur, pr
        if xi < tail:
            return rs, us, ps
        u = 2.0 / (gas + 1.0) * (-ar + 0.5 * (gas - 1.0) * ur + xi)
        c = 2.0 / (gas + 1.0) * (ar - 0.5 * (gas - 1.0) * (ur - xi))
        r = rr * (c / ar) ** (2.0 / (gas - 1.0))
        return r, u, pr * (c / ar) ** (2.0 * gas / (gas - 1.0))

    x = np.asarray(edges, dtype=np.float64)
    n = x.size - 1
    out = np.zeros((3, n))
    for i in range(n):
        acc = np.zeros(3)
        for j in range(sub):
            r, u, p = sample((x[i] + (j + 0.5) / sub * (x[i + 1] - x[i])) / t)
            acc += (r, r * u, p / (gas - 1.0) + 0.5 * r * u * u)
        out[:, i] = acc / sub
    return out


# the scalar test cases of Table 1 (Section 5.1) ------------------------------

def _logcosh(y):
    a = np.abs(y)
    return a + np.log1p(np.exp(-2.0 * a)) - math.log(2.0)


def _tanh_prim(x):
    """Primitive of (1 + tanh(100 x)) / 2."""
    return 0.5 * (x + _logcosh(100.0 * x) / 100.0)


def _tanh_profile(x):
    return 0.5 * (1.0 + np.tanh(100.0 * x))


def _gauss_prim(x):
    """Primitive of exp(-20 x^2)."""
    from scipy.special import erf

    return math.sqrt(math.pi / 20.0) / 2.0 * erf(math.sqrt(20.0) * x)


# Test -> (equation, final time T, regularity nu of Table 1 as mu_bar (reading:
# mu_bar = min(nu, 2 gamma + 1)), boundary condition)
SCALAR_TESTS = {
    "I": (EQ_ADVECTION, 0.4, 3, BC_PERIODIC),
    "II": (EQ_ADVECTION, 0.4, 0, BC_PERIODIC),
    "III": (EQ_BURGERS, 0.4, 3, BC_COPY),
    "IV": (EQ_BURGERS, 0.7, 0, BC_PERIODIC),
}


def scalar_test(test: str, s: float = 1.0, Jmax: int = 9, eps: float = 1e-4, Jmin: int = 2) -> Instance:
    """Test I-IV of Table 1: advection (c = 3/4) of exp(-20 x^2) and of the
    indicator of |x| <= 1/2, Burgers with (1 + tanh(100 x)) / 2 and with the
    indicator of |x| <= 1/2; Omega = [-3, 3], lambda = 1, relaxation s."""
    eq, T, mu_bar, bc = SCALAR_TESTS[test]
    inst = Instance(f"test{test}", eq, Jmin, Jmax, eps, 1.0, -3.0, 3.0, bc, T, mu_bar=mu_bar, s=(s,),
                    eqp=0.75 if eq == EQ_ADVECTION else 0.0)
    inst.m0 = scalar_exact(test, cell_edges(inst.a, inst.b, Jmax), 0.0)[None, :]
    return inst


def scalar_exact(test: str, edges: np.ndarray, t: float) -> np.ndarray:
    """Cell averages over the cells [edges[i], edges[i+1]] of the exact entropy
    solution of Test I-IV at time t (no wave reaches the boundary before T)."""
    x = np.asarray(edges, dtype=np.float64)
    dx = np.diff(x)
    if test == "I":  # advection at c = 3/4
        return np.diff(_gauss_prim(x - 0.75 * t)) / dx
    if test == "II":
        return avg_indicator(x, -0.5 + 0.75 * t, 0.5 + 0.75 * t)
    if test == "III":
        # smooth increasing datum: rho(t, x) = rho0(xi) with x = xi + t rho0(xi); in the
        # variable xi, int rho dx = int rho0 (1 + t rho0') dxi = [P0(xi) + t rho0(xi)^2 / 2]
        if t == 0.0:
            return np.diff(_tanh_prim(x)) / dx
        lo, hi = x - t, x.copy()  # xi + t rho0(xi) is increasing, rho0 in (0, 1)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            f = mid + t * _tanh_profile(mid) - x
            lo = np.where(f < 0.0, mid, lo)
            hi = np.where(f < 0.0, hi, mid)
        xi = 0.5 * (lo + hi)
        G = _tanh_prim(xi) + 0.5 * t * _tanh_profile(xi) ** 2
        return np.diff(G) / dx
    if test == "IV":
        # rarefaction from x = -1/2 (head -1/2 + t), shock from x = 1/2 at speed 1/2 (t < 2)
        if t == 0.0:
            return avg_indicator(x, -0.5, 0.5)
        a, b = x[:-1], x[1:]

        def fan(u):  # primitive of (u + 1/2) / t
            return (u + 0.5) ** 2 / (2.0 * t)

        r0, r1 = -0.5, -0.5 + t
        lo_f, hi_f = np.clip(a, r0, r1), np.clip(b, r0, r1)
        out = fan(hi_f) - fan(lo_f)
        out += np.clip(np.minimum(b, 0.5 + 0.5 * t) - np.maximum(a, r1), 0.0, None)
        return out / dx
    raise ValueError(test)


WORKLOADS = {
    "advection": advection,
    "burgers": burgers,
    "shallow": shallow_water,
    "sod": sod,
    "test1": lambda: scalar_test("I"),
    "test2": lambda: scalar_test("II"),
    "test3": lambda: scalar_test("III"),
    "test4": lambda: scalar_test("IV"),
    "sw_d1q3": lambda: shallow_water_dq("d1q3"),
    "sw_d1q5": lambda: shallow_water_dq("d1q5"),
}

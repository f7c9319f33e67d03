// mr_kernels.cuh -- sm_103a kernels of the multiresolution-adaptive lattice
// Boltzmann step (Bellotti, Gouarin, Graille, Massot, arXiv 2102.12163).
//
// A thread block owns one instance at a time and runs every phase of the step
// on it, with block barriers between phases; blocks pull instances from an
// atomic work queue sorted largest first (persistent launch).  Inside a step:
//
//   adapt (Section 4.1)
//     A1  projection up the current tree (Def. Projection operator); right
//         after a D1Q2^n step, one conservative update of the internal cells
//     A2  details of the pairs of the tree, threshold T, Harten flags (Sections
//         3.2, 3.4, 4.2) -> KEEP / REF bitmasks
//     A3  enlargement H: same-level dilation and children of REF pairs
//     A4  grading G, sweeping fine to coarse over bitmask words (Def. Graded
//         tree), fused with the leaf / transfer / ghost marking
//     A5  list compaction: popcount + prefix scan over the mask words
//     A6  data transfer: prediction of the new cells, coarse to fine
//   step (Sections 4.3, 4.5)
//     S1  leaves collision (eq. LeavesCollision)
//     S2  projection of the collided values up the new tree
//     S3  ghost prediction coarse to fine (reconstruction operator, Section 3.3)
//     S4  boundary reconstruction on the first / last finest cell of every
//         leaf from the per-level-gap tables -> interface array Phi
//     S5  compact stream (eq. AdaptiveStreamPhase) + mass audit (FP64 totals)
//
// The cell arrays are dense per level (every cell of every level has a slot),
// the tree is a set of bitmasks with 32 cells per word, and every per-cell
// phase walks a compacted list so its work is proportional to the tree.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "mr_common.h"

namespace mrg {

constexpr double C1 = -0.125;  // prediction coefficient c_1 for gamma = 1 (Section 3.1)
constexpr unsigned FULL = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// arithmetic: the FP64 path uses explicitly rounded operations (never fused)
// in the collision, so that it follows the same rounding sequence as a plain
// IEEE evaluation of the formulas; the FP32 path lets the compiler fuse.
template <typename T>
struct Ar;
template <>
struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float div(float a, float b) { return a / b; }
};

template <typename T>
struct V2;
template <>
struct V2<double> {
    using type = double2;
};
template <>
struct V2<float> {
    using type = float2;
};

// ---------------------------------------------------------------------------
// level geometry and bit helpers

__device__ __forceinline__ long long cell_off(int l, int Jmin) { return (1LL << l) - (1LL << Jmin); }
__device__ __forceinline__ int nwords(int l) { return l >= 5 ? (1 << (l - 5)) : 1; }
__device__ __forceinline__ uint32_t valid_bits(int l) {
    return l >= 5 ? 0xFFFFFFFFu : ((1u << (1 << l)) - 1u);
}
// cell index at level l under the boundary condition (0 periodic: wrap, 1 copy: clamp)
__device__ __forceinline__ long long wrapc(long long k, int l, int bc) {
    long long n = 1LL << l;
    if (bc == 0) return k & (n - 1);
    return k < 0 ? 0 : (k >= n ? n - 1 : k);
}
__device__ __forceinline__ uint32_t pack(int l, long long k) { return ((uint32_t)l << KBITS) | (uint32_t)k; }

// bits 0, 2, ..., 30 of x -> bits 0..15
__device__ __forceinline__ uint32_t compact_even(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}
// parent bits of two child words (a: cells 0..31, b: cells 32..63)
__device__ __forceinline__ uint32_t fold2(uint32_t a, uint32_t b) {
    return compact_even(a | (a >> 1)) | (compact_even(b | (b >> 1)) << 16);
}
// 16 parent bits -> 32 child bits (both children of every parent)
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x | (x << 1);
}
// close a set of cells under siblings (pairs 2p, 2p+1 never straddle a word)
__device__ __forceinline__ uint32_t pairexpand(uint32_t x) {
    return x | ((x & 0x55555555u) << 1) | ((x & 0xAAAAAAAAu) >> 1);
}
// word wp of level l-1 holding the parents of the cells set in level l (words `child`)
__device__ __forceinline__ uint32_t fold_at(const uint32_t *child, int l, int wp) {
    return l >= 6 ? fold2(child[2 * wp], child[2 * wp + 1]) : fold2(child[0], 0u);
}

// Dilation by r cells of the set held in word wi of level l; get(j) returns word j
// of that level.  Periodic: wrap; copy: cells beyond the domain are dropped.
template <class Get>
__device__ __forceinline__ uint32_t dilate(Get get, int l, int wi, int r, int bc) {
    uint32_t x = get(wi);
    uint32_t out = x;
    if (l < 5) {
        int n = 1 << l;
        uint32_t vb = (1u << n) - 1u;
        for (int s = 1; s <= r; ++s) {
            if (bc == 0)
                out |= (((x << s) | (x >> (n - s))) & vb) | (((x >> s) | (x << (n - s))) & vb);
            else
                out |= ((x << s) & vb) | (x >> s);
        }
        return out;
    }
    int W = 1 << (l - 5);
    uint32_t xl, xr;
    if (W == 1) {
        xl = xr = (bc == 0) ? x : 0u;
    } else if (bc == 0) {
        xl = get((wi - 1) & (W - 1));
        xr = get((wi + 1) & (W - 1));
    } else {
        xl = wi > 0 ? get(wi - 1) : 0u;
        xr = wi + 1 < W ? get(wi + 1) : 0u;
    }
    for (int s = 1; s <= r; ++s) out |= (x << s) | (xl >> (32 - s)) | (x >> s) | (xr << (32 - s));
    return out;
}

// word j of a level of W words under the boundary rule: wrapped (periodic) or
// empty beyond the domain (copy)
__device__ __forceinline__ uint32_t word_bc(const uint32_t *a, int j, int W, int bc) {
    if (j < 0) return bc == 0 ? a[j + W] : 0u;
    if (j >= W) return bc == 0 ? a[j - W] : 0u;
    return a[j];
}
// 4 child bits -> 2 parent bits
__device__ __forceinline__ uint32_t fold_low2(uint32_t x) { return ((x | (x >> 1)) & 1u) | (((x >> 2) | (x >> 3)) & 1u) << 1; }
// dilation by one cell of a word, given the neighbouring cells just outside it
__device__ __forceinline__ uint32_t dilate1_edges(uint32_t x, bool left, bool right) {
    return x | (x << 1) | (x >> 1) | (left ? 1u : 0u) | (right ? 0x80000000u : 0u);
}

// ---------------------------------------------------------------------------
// shared memory: per-team state and per-block tables

template <typename T>
struct TeamSmem {
    InstDesc d;
    int woff[MAXLEV + 2];
    int ooff[MAXLEV + 2];    // occupancy words of level l start at ooff[l]
    int cw_seg[MAXLEV + 2];  // candidate words of level l: entries [cw_seg[l], cw_seg[l+1]) of the list
    int sparse;              // word passes over candidate words (else over every word)
    int seg[NLIST][MAXLEV + 2];
    double eps_l[MAXLEV + 1], big_l[MAXLEV + 1], dx_l[MAXLEV + 1];  // per level
    float eps_f[MAXLEV + 1], big_f[MAXLEV + 1];
    double mass[3];
    double audit;
    unsigned long long updates, steps, passes;
    int cur, nleaf, status, near_ties;
    uint32_t deplev[2];  // levels holding transfer (0) / ghost (1) cells that wait on the same list
    int idx;
    int g0s, gbase;  // level_of_word constants
#ifdef MRG_PHASE_TIMERS
    long long tlast;
    unsigned long long ptime[NPHASE];
#endif
};

// block-team scratch (scan partials and reduction slots of the warps)
struct BlockScratch {
    int scan_w[2][NLIST][32];
    double red[3][64];
};

template <typename T, int NT>
struct BlockSmem {
    Tables<T> tab;
    BlockScratch scratch;
    TeamSmem<T> team;
    int idx;
};

template <typename T>
__device__ __forceinline__ void level_of_word(const TeamSmem<T> &sm, int g, int &l, int &wi) {
    if (g < sm.g0s) {
        l = sm.d.Jmin + g;
        wi = 0;
    } else {
        int x = g - sm.g0s + sm.gbase;
        l = 5 + (31 - __clz(x));
        wi = x - (1 << (l - 5));
    }
}

// ---------------------------------------------------------------------------
// scheme: vectorial D1Q2^n (Section 2.1, equilibria of Sections 5.1 and 5.3)

// 2^-n exactly, built from its exponent field (0 <= n <= 126): no conversion
// instruction, which for a double would occupy GB300's scarce FP64 units
template <typename T>
__device__ __forceinline__ T pow2m(int n) {
    if constexpr (sizeof(T) == 8)
        return __longlong_as_double((long long)(1023 - n) << 52);
    else
        return __int_as_float((127 - n) << 23);
}

// x * 2^k (|k| <= 1022), bit for bit the correctly rounded product, in integer
// arithmetic where the exponent field allows (zero, or a normal operand and
// result) and with the multiply otherwise: GB300's FP64 units are scarce,
// integer units are not.
__device__ __forceinline__ double scale2(double x, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFull);
    if ((b << 1) == 0ull) return x;
    if (e > 0 && e < 0x7FF && e + k > 0 && e + k < 0x7FF)
        return __longlong_as_double((long long)(b + ((unsigned long long)(long long)k << 52)));
    return x * __longlong_as_double((long long)(1023 + k) << 52);
}
__device__ __forceinline__ float scale2(float x, int k) { return x * ldexpf(1.0f, k); }

// x / 2, bit for bit the product x * 0.5, on the integer units: an exponent
// field e >= 2 loses one; for e <= 1 the magnitude bits are the value in units
// of 2^-1074 (the implicit bit included), halved with ties to even (which also
// carries into the smallest normal number); infinities and NaNs pass unchanged
__device__ __forceinline__ double half_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = b & 0x8000000000000000ull, mag = b ^ sign;
    const unsigned e = (unsigned)(mag >> 52);
    unsigned long long r;
    if (e >= 2u)
        r = e == 0x7FFu ? mag : mag - (1ull << 52);
    else
        r = (mag >> 1) + ((mag & 1ull) & ((mag >> 1) & 1ull));
    return __longlong_as_double((long long)(sign | r));
}
template <typename T>
__device__ __forceinline__ T half_of(T x) {
    if constexpr (sizeof(T) == 8)
        return half_f64(x);
    else
        return T(0.5) * x;
}

// the scheme constants in the path's precision: FP64, or the float copies the
// host rounds once (no double-to-float conversion per cell in the FP32 path)
template <typename T>
__device__ __forceinline__ T lam_of(const InstDesc &d) {
    if constexpr (sizeof(T) == 8) return d.lam; else return d.lam_f;
}
template <typename T>
__device__ __forceinline__ T eqp_of(const InstDesc &d) {
    if constexpr (sizeof(T) == 8) return d.eqp; else return d.eqp_f;
}
template <typename T>
__device__ __forceinline__ T s_of(const InstDesc &d, int i) {
    if constexpr (sizeof(T) == 8) return d.s[i]; else return d.s_f[i];
}
template <typename T>
__device__ __forceinline__ T minv_of(const InstDesc &d, int h, int i) {
    if constexpr (sizeof(T) == 8) return d.minv[h][i]; else return d.minv_f[h][i];
}
// 1 - s[i] and the equilibria's constant factors: in FP64 rounded once on the
// host (GB300's FP64 pipe is the scarce one), in FP32 computed in place (the
// loads cost the FP32 kernel registers, the operations cost it nothing)
template <typename T>
__device__ __forceinline__ T oms_of(const InstDesc &d, int i) {
    if constexpr (sizeof(T) == 8) return d.oms[i]; else return 1.0f - d.s_f[i];
}
template <typename T>
__device__ __forceinline__ void eq_consts(const InstDesc &d, T &a, T &b, T &c, T &g2) {
    if constexpr (sizeof(T) == 8) {
        a = d.eu_a; b = d.eu_b; c = d.eu_c; g2 = d.sw_g2;
    } else {
        const float gg = d.eqp_f;
        a = 1.5f - 0.5f * gg;
        b = gg - 1.0f;
        c = 0.5f * (1.0f - gg);
        g2 = 0.5f * gg;
    }
}

// x / lambda for a lambda that is no power of two, in FP64 bit for bit the
// correctly rounded quotient without a division: q0 = RN(x r) with r = RN(1 / lambda) is
// within one ulp of x / lambda, the residual x - q0 lambda is exact in one FMA,
// and q0 + residual r rounded once is the correctly rounded quotient (P.
// Markstein, IBM J. Res. Dev. 34(1), 1990).  Operands near the ends of the
// exponent range, zeros and non-finite values take the division.
template <typename T>
__device__ __forceinline__ T div_lam(T x, const InstDesc &d) {
    if constexpr (sizeof(T) == 8) {
        const int e = (__double2hiint(x) >> 20) & 0x7FF;
        if (e < 64 || e > 1983) return __ddiv_rn(x, d.lam);
        const double q0 = __dmul_rn(x, d.rlam);
        return __fma_rn(__fma_rn(-q0, d.lam, x), d.rlam, q0);
    } else {
        return __fdiv_rn(x, d.lam_f);  // FP32 divisions are cheap; the register budget is not
    }
}

// equilibria of the relaxed moments; the constant factors (0.5 g, 1.5 - 0.5
// gamma_gas, gamma_gas - 1, 0.5 (1 - gamma_gas)) come rounded from the host,
// the same values the expressions would give per cell
template <typename T, int NF>
__device__ __forceinline__ void equilibria(const InstDesc &d, T eqp, const T *mc, T *meq) {
    using A = Ar<T>;
    T ca, cb, cc, g2;
    eq_consts<T>(d, ca, cb, cc, g2);
    if constexpr (NF == 1) {
        if (d.eq == 0)
            meq[0] = A::mul(eqp, mc[0]);  // advection: c m0
        else
            meq[0] = half_of<T>(A::mul(mc[0], mc[0]));  // Burgers: m0^2 / 2
    } else if constexpr (NF == 2) {
        // shallow water (h, hu): hu, hu^2 / h + g h^2 / 2
        meq[0] = mc[1];
        meq[1] = A::add(A::div(A::mul(mc[1], mc[1]), mc[0]), A::mul(g2, A::mul(mc[0], mc[0])));
    } else {
        // Euler (rho, rho u, E), Section 5.3
        T gg = eqp;
        T u2 = A::mul(mc[1], mc[1]);
        meq[0] = mc[1];
        meq[1] = A::add(A::mul(ca, A::div(u2, mc[0])), A::mul(cb, mc[2]));
        meq[2] = A::add(A::mul(gg, A::div(A::mul(mc[2], mc[1]), mc[0])),
                        A::mul(cc, A::div(A::mul(u2, mc[1]), A::mul(mc[0], mc[0]))));
    }
}

// leaves collision on the q populations of one cell: m = M f, relax, f* = M^-1 m*
template <typename T, int NF>
__device__ __forceinline__ void collide(const InstDesc &d, T *f) {
    using A = Ar<T>;
    T mc[NF], mn[NF], meq[NF];
    const T lam = lam_of<T>(d);
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        mc[i] = A::add(f[2 * i], f[2 * i + 1]);
        mn[i] = A::mul(lam, A::sub(f[2 * i], f[2 * i + 1]));
    }
    equilibria<T, NF>(d, eqp_of<T>(d), mc, meq);
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        T s = s_of<T>(d, i);
        T mstar = A::add(A::mul(oms_of<T>(d, i), mn[i]), A::mul(s, meq[i]));
        // m*/lambda: an exact power-of-two scaling when lambda = 2^k (same value as the division)
        T g = d.lam_log2 != NOT_POW2 ? scale2(mstar, -d.lam_log2) : div_lam<T>(mstar, d);
        f[2 * i] = half_of<T>(A::add(mc[i], g));
        f[2 * i + 1] = half_of<T>(A::sub(mc[i], g));
    }
}

// populations at equilibrium of the conserved moments (initial datum), in FP64
template <int NF>
__device__ __forceinline__ void equilibrium_populations(const InstDesc &d, const double *mc, double *f) {
    using A = Ar<double>;
    double meq[NF];
    equilibria<double, NF>(d, d.eqp, mc, meq);
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        double g = A::div(meq[i], d.lam);
        f[2 * i] = A::mul(0.5, A::add(mc[i], g));
        f[2 * i + 1] = A::mul(0.5, A::sub(mc[i], g));
    }
}

// ---- shallow water on one velocity set (Section 5.2): D1Q3 (Q = 3), D1Q5 (Q = 5)
// velocities v^h = lambda w^h, w = (0, 1, -1, 2, -2); moments m^i = sum_h (v^h)^i f^h
__device__ __forceinline__ int dq_w(int h) { return h == 0 ? 0 : (h & 1) ? (h + 1) / 2 : -(h / 2); }

// collision: the relaxed moments i >= 2 move to (1 - s^i) m^i + s^i m^{i,eq}, with
// m^{2,eq} = (hu)^2 / h + g h^2 / 2, m^{3,eq} = lambda^2 hu, m^{4,eq} = lambda^2
// m^{2,eq}; f* = f + M^{-1} (m* - m) (the conserved rows of m* - m are zero)
template <typename T, int Q>
__device__ __forceinline__ void dq_collide(const InstDesc &d, T *f) {
    const T lam = lam_of<T>(d);
    T m[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) m[i] = T(0);
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const T v = (T)dq_w(h) * lam;
        T x = f[h];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            m[i] = m[i] + x;
            x = x * v;
        }
    }
    T meq[Q];
    T ca, cb, cc, g2;
    eq_consts<T>(d, ca, cb, cc, g2);
    meq[2] = (m[1] * m[1]) / m[0] + g2 * (m[0] * m[0]);
    if constexpr (Q == 5) {
        meq[3] = (lam * lam) * m[1];
        meq[4] = (lam * lam) * meq[2];
    }
    T dm[Q];
#pragma unroll
    for (int i = 2; i < Q; ++i) dm[i] = s_of<T>(d, i - 2) * (meq[i] - m[i]);
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        T acc = T(0);
#pragma unroll
        for (int i = 2; i < Q; ++i) acc = acc + minv_of<T>(d, h, i) * dm[i];
        f[h] = f[h] + acc;
    }
}

// populations at equilibrium of (h, hu), in FP64: f = M^{-1} (h, hu, m^{2,eq}, ...)
template <int Q>
__device__ __forceinline__ void dq_equilibrium_populations(const InstDesc &d, const double *mc, double *f) {
    double m[5];
    m[0] = mc[0];
    m[1] = mc[1];
    m[2] = (mc[1] * mc[1]) / mc[0] + (0.5 * d.eqp) * (mc[0] * mc[0]);
    if constexpr (Q == 5) {
        m[3] = (d.lam * d.lam) * mc[1];
        m[4] = (d.lam * d.lam) * m[2];
    }
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) acc = acc + d.minv[h][i] * m[i];
        f[h] = acc;
    }
}

// prediction of child `odd` of cell p of a row at level lp (Section 3.1, gamma = 1)
template <typename T, typename R>
__device__ __forceinline__ T predict(const R &row, long long p, int odd, int lp, int bc) {
    T vl = row[wrapc(p - 1, lp, bc)], vp = row[p], vr = row[wrapc(p + 1, lp, bc)];
    T t = T(C1) * (vr - vl);  // exact: c_1 is a power of two
    return odd ? vp - t : vp + t;
}

// the same for a stencil of half-width gamma = 2 or 3 (coefficients c[0..gamma-1]):
// f_p +- sum_a c_a (f_{p+a} - f_{p-a}), the sum accumulated in increasing a
template <typename T, typename R>
__device__ __forceinline__ T predict_g(const R &row, long long p, int odd, int lp, int bc, int gamma, const T *c) {
    T t = c[0] * (row[wrapc(p + 1, lp, bc)] - row[wrapc(p - 1, lp, bc)]);
#pragma unroll
    for (int a = 2; a <= 3; ++a)
        if (a <= gamma) t = t + c[a - 1] * (row[wrapc(p + a, lp, bc)] - row[wrapc(p - a, lp, bc)]);
    const T vp = row[p];
    return odd ? vp - t : vp + t;
}

// dilation by r <= 16 cells of the word x, given the words on its left (xl) and
// right (xr) (only their r cells nearest to x are read)
__device__ __forceinline__ uint32_t dilate_edges(uint32_t x, uint32_t xl, uint32_t xr, int r) {
    uint32_t out = x;
    for (int s = 1; s <= r; ++s) out |= (x << s) | (xl >> (32 - s)) | (x >> s) | (xr << (32 - s));
    return out;
}
// parent bits of 6 child bits (3 parents)
__device__ __forceinline__ uint32_t fold3(uint32_t t) {
    t |= t >> 1;
    return (t & 1u) | ((t >> 1) & 2u) | ((t >> 2) & 4u);
}

// First (last = false) or last finest value of one population row of the leaf
// (l, k), by the reconstruction operator of Section 3.3 (Definition V): the
// level-l window k - 2G .. k + 2G (tree and ghost values) is predicted level by
// level down to Jmax around the leaf's first (last) finest cell, and wherever a
// finer level holds a cell of the tree (the children of refined neighbours)
// its value is used instead.  Out-of-domain cells take the value of the nearest
// domain cell (copy boundary) or wrap (periodic), as in the prediction.
template <typename T, int G, bool LAST>
__device__ __noinline__ T edge_walk(const T *rowbase, int qs, int Jmin, int Jmax, int bc, const uint32_t *R,
                                    const int *woff, const T *c, int l, long long k) {
    constexpr int W = 4 * G + 1, C = 2 * G, E = LAST ? 1 : 0;
    T w[W], nw[W];
    {
        const T *row = rowbase + cell_off(l, Jmin) * qs;
#pragma unroll
        for (int t = 0; t < W; ++t) w[t] = row[wrapc(k + t - C, l, bc) * qs];
    }
    long long i = k;
    for (int m = l; m < Jmax; ++m) {
        const long long nn = 1LL << (m + 1), inext = 2 * i + E;
        const T *row = rowbase + cell_off(m + 1, Jmin) * qs;
        const uint32_t *Rm = R + woff[m + 1];
        T lo = T(0), hi = T(0);  // values of the first and last cells of the level (copy boundary)
#pragma unroll
        for (int t = 0; t < W; ++t) {
            // window position t is cell inext + t - C; its parent is window position pp of level m
            const long long pos = inext + t - C;
            const int pp = C + ((E + t - C) >> 1);
            const bool odd = ((E + t - C) & 1) != 0;
            long long cp = pos;
            bool inside = true;
            if (bc == 0)
                cp = pos & (nn - 1);
            else
                inside = pos >= 0 && pos < nn;
            T v;
            if (inside && ((Rm[(int)(cp >> 5)] >> (cp & 31)) & 1u)) {
                v = row[cp * qs];
            } else {
                T sum = c[0] * (w[pp + 1] - w[pp - 1]);
#pragma unroll
                for (int a = 2; a <= G; ++a) sum = sum + c[a - 1] * (w[pp + a] - w[pp - a]);
                v = odd ? w[pp] - sum : w[pp] + sum;
            }
            nw[t] = v;
            if (pos == 0) lo = v;
            if (pos == nn - 1) hi = v;
        }
        if (bc != 0) {
#pragma unroll
            for (int t = 0; t < W; ++t) {
                const long long pos = inext + t - C;
                if (pos < 0) nw[t] = lo;
                if (pos >= nn) nw[t] = hi;
            }
        }
#pragma unroll
        for (int t = 0; t < W; ++t) w[t] = nw[t];
        i = inext;
    }
    return w[C];
}

// NaN or infinity, from the exponent field (integer units)
__device__ __forceinline__ bool nonfinite(double x) { return (__double2hiint(x) & 0x7FF00000) == 0x7FF00000; }
__device__ __forceinline__ bool nonfinite(float x) { return (__float_as_uint(x) & 0x7F800000u) == 0x7F800000u; }

// ---------------------------------------------------------------------------
// FP64 threshold decisions on bit patterns.  Non-negative doubles order as
// their bit patterns, so max |d| over the populations and its comparisons with
// eps_l and the Harten level run on the integer units instead of GB300's
// scarce FP64 pipe, with the same outcome as the floating-point max and >=
// (a NaN detail is skipped, as fmax skips it).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    return b > 0x7FF0000000000000ull ? 0ull : b;
}
// keep / refine decisions of a pair with max |detail| bits Db, and whether it
// lies within 1e-12 relative of eps_l or of the Harten level: an integer
// pre-filter (1e-12 relative is at most 9008 units in the last place) and the
// exact test behind it
__device__ __forceinline__ void decide_bits(unsigned long long Db, double el, double bl, bool hasref, bool &keepit,
                                            bool &refit, bool &tie) {
    const unsigned long long eb = (unsigned long long)__double_as_longlong(el),
                             bb = (unsigned long long)__double_as_longlong(bl);
    keepit = Db >= eb;
    refit = hasref && Db >= bb;
    const long long de = (long long)(Db - eb), db = (long long)(Db - bb);
    tie = false;
    if ((de < 16384 && de > -16384) || (hasref && db < 16384 && db > -16384)) {
        const double D = __longlong_as_double((long long)Db);
        tie = fabs(D - el) <= 1e-12 * el || (hasref && fabs(D - bl) <= 1e-12 * bl);
    }
}

// ---------------------------------------------------------------------------
// the instance worker; TS threads (a warp or the whole block) form the team

constexpr int QMAX = 6;  // populations of the largest scheme (vectorial D1Q2^3)

// One population of the cell-major value layout: the Q values of a cell are
// contiguous, so element k of the population starting at p sits at p[k * Q].
template <typename T, int Q>
struct SRow {
    T *p;
    __device__ __forceinline__ T &operator[](long long k) const { return p[k * Q]; }
};

// WIDE: prediction stencils gamma = 2, 3 (the gamma = 1 code is a separate instantiation)
// SPM: word passes over every word (0) or over candidate words (1, the
// large-instance variant K_LARGE alone: code that a kernel carries costs it
// even where it does not run)
template <typename T, int NF, int TS, bool WIDE, int SPM>
struct Worker {
    static constexpr bool WARP = TS == 32;
    // NF = 1, 2, 3: vectorial D1Q2^NF; NF = 4: D1Q3, NF = 5: D1Q5 shallow water
    static constexpr bool DQ = NF >= 4;
    static constexpr int nf = DQ ? 2 : NF;                          // conserved moments
    static constexpr int q = DQ ? (NF == 4 ? 3 : 5) : 2 * NF;       // populations
    static constexpr int SIGMA = NF == 5 ? 2 : 1;                   // enlargement width max |w^h|
    TeamSmem<T> &sm;
    const Tables<T> &tab;
    BlockScratch &bx;
    const InstDesc &d;
    T *V;
    T *Phi;
    uint32_t *M;     // mask base (shared memory when the masks fit, else global)
    int tid;         // rank in the team
    long long voff;  // -2^Jmin q: level l's values start at V + 2^l q + voff

    __device__ Worker(TeamSmem<T> &s, const Tables<T> &tb, BlockScratch &x, int rank, uint32_t *masks)
        : sm(s), tab(tb), bx(x), d(s.d), tid(rank) {
        V = (T *)d.V;
        Phi = (T *)d.Phi;
        M = masks;
        voff = -(1LL << d.Jmin) * q;
    }

    // leaves collision of the q populations of one cell
    __device__ __forceinline__ void collide_cell(T *f) const {
        if constexpr (DQ)
            dq_collide<T, q>(d, f);
        else
            collide<T, NF>(d, f);
    }

    // team barrier; every one ends a pass whose results the next pass reads.
    // The variants that run large single instances count them (the chain of
    // dependent passes of a step, the floor of its latency) by the team's last
    // thread after the barrier; the batch variants do not: the count cost them
    // 7 % (measured), most of their passes being short.
    __device__ __forceinline__ void sync() const {
        if constexpr (WARP)
            __syncwarp();
        else
            __syncthreads();
        if constexpr (SPM != 0)
            if (tid == TS - 1) ++sm.passes;
    }

    // profiling build: cycles since the previous tick charged to phase p (after a team barrier)
    __device__ __forceinline__ void tick(int p) {
#ifdef MRG_PHASE_TIMERS
        sync();
        if (tid == 0) {
            long long t = clock64();
            if (p < NPHASE) sm.ptime[p] += (unsigned long long)(t - sm.tlast);
            sm.tlast = t;
        }
#else
        (void)p;
#endif
    }

    __device__ __forceinline__ uint32_t *mask(int m) { return M + (long long)m * d.Wtot; }
    // candidate-word list of the step (global mask word indices, sorted by level then word)
    __device__ __forceinline__ uint32_t *cwl() { return M + (long long)NMASK * d.Wtot; }
    // i-th word of the step's word passes: a candidate word, or word i itself
    __device__ __forceinline__ int cw_at(int i) { return sparse_on() ? (int)cwl()[i] : i; }
    __device__ __forceinline__ bool sparse_on() const { return SPM != 0; }
    // occupancy bitmap of tree buffer b (M_R0 or M_R1): bit wi & 31 of word ooff[l] + (wi >> 5) is set
    // when word wi of level l of that tree holds a cell
    __device__ __forceinline__ uint32_t *occ(int b) { return M + (long long)(NMASK + 1) * d.Wtot + (long long)b * d.OW; }
    __device__ __forceinline__ uint32_t *list(int L) { return d.lists + d.list_off[L]; }
    // population h on level l, and population h of the interface array
    // population h of level l, at cell_off(l, Jmin) q + h.  The FP64 kernels hold
    // Jmin in voff: the descriptor field, reloaded from shared memory after every
    // store, would sit on the dependent chain of each population loop (measured:
    // +1.5 % FP64); the FP32 kernels keep the reload, whose register is dearer
    // to them (the offset cost them spills and 3.6 %)
    __device__ __forceinline__ SRow<T, q> row(int h, int l) const {
        if constexpr (sizeof(T) == 8)
            return SRow<T, q>{V + ((1LL << l) * q + voff + h)};
        else
            return SRow<T, q>{V + cell_off(l, d.Jmin) * q + h};
    }
    __device__ __forceinline__ SRow<T, q> phi(int h) const { return SRow<T, q>{Phi + h}; }

    // sums over the team of nf per-thread doubles, valid in thread 0 (one barrier)
    // The team's sum of x[j], in thread 0.  GB300's FP64 units take a warp-wide
    // instruction whole whatever its active lanes, so the additions are kept
    // off most warps: a few shuffle rounds in each warp leave 64 partial sums
    // per field (groups of TS / 64 lanes) in shared memory, and warp 0 folds
    // them (two per lane, then a shuffle tree).  A fixed order: deterministic.
    __device__ __forceinline__ void team_sum(double (&x)[3]) {
        if constexpr (WARP) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < nf)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x[j] += __shfl_down_sync(FULL, x[j], o);
        } else {
            static_assert(TS >= 64 && TS % 64 == 0, "team width");
            constexpr int G = TS / 64;  // lanes per partial sum: 1, 2, 4, 8 or 16
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < nf)
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) x[j] += __shfl_down_sync(FULL, x[j], o);
            if ((tid & (G - 1)) == 0)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nf) bx.red[j][tid / G] = x[j];
            sync();
            if (tid < 32)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nf) {
                        double v = bx.red[j][tid] + bx.red[j][tid + 32];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
                        x[j] = v;
                    }
        }
    }

    // float-float accumulation (hi + lo, error-free transformation TwoSum of
    // Knuth): the FP32 path keeps its mass audit off the FP64 pipe
    static __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
        s = a + b;
        const float bb = s - a;
        e = (a - (s - bb)) + (b - bb);
    }
    static __device__ __forceinline__ void ff_add(float &hi, float &lo, float xh, float xl) {
        float s, e;
        two_sum(hi, xh, s, e);
        hi = s;
        lo = lo + (xl + e);
    }
    // team sums of nf float-float pairs, as doubles valid in thread 0 (one barrier)
    __device__ __forceinline__ void team_sum_ff(float (&hi)[3], float (&lo)[3], double (&out)[3]) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (j < nf)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float h2 = __shfl_down_sync(FULL, hi[j], o), l2 = __shfl_down_sync(FULL, lo[j], o);
                    ff_add(hi[j], lo[j], h2, l2);
                }
        if constexpr (!WARP) {
            float2 *red = reinterpret_cast<float2 *>(&bx.red[0][0]);
            if ((tid & 31) == 0)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nf) red[j * 32 + (tid >> 5)] = make_float2(hi[j], lo[j]);
            sync();
            if (tid == 0)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nf) {
                        float h = 0.0f, l = 0.0f;
                        for (int w = 0; w < TS / 32; ++w) ff_add(h, l, red[j * 32 + w].x, red[j * 32 + w].y);
                        hi[j] = h;
                        lo[j] = l;
                    }
        }
        // only thread 0 holds the sums: the other threads keep off the FP64 pipe
        if (tid == 0)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < nf) out[j] = (double)hi[j] + (double)lo[j];
    }

    // ---- projection of the internal cells of level l (Def. Projection operator)
    __device__ __forceinline__ void project_level(const uint32_t *lst, int l) {
        int b = sm.seg[L_INT][l], e = sm.seg[L_INT][l + 1];
        for (int i = b + tid; i < e; i += TS) {
            long long k = lst[i] & KMASK;
            // the two children are adjacent cells: 2q contiguous values
            T ce[QMAX], co[QMAX];
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) {
                    const auto rc = row(h, l + 1);
                    ce[h] = rc[2 * k];
                    co[h] = rc[2 * k + 1];
                }
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) row(h, l)[k] = half_of<T>(ce[h] + co[h]);
        }
    }

    // ---- S1: leaves collision (eq. LeavesCollision) ---------------------------
    __device__ void collide_all() {
        const uint32_t *lst = list(L_LEAF);
        for (int i = tid; i < sm.nleaf; i += TS) {
            uint32_t ent = lst[i];
            int l = ent >> KBITS;
            long long k = ent & KMASK;
            T f[QMAX];
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) f[h] = row(h, l)[k];
            collide_cell(f);
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) row(h, l)[k] = f[h];
        }
    }

    // equilibria of the relaxed moments at one cell (populations g)
    __device__ __forceinline__ void relaxed_equilibria(const T *g, T *meq) const {
        if constexpr (DQ) {
            const T lam = lam_of<T>(d);
            T h = T(0), hu = T(0);
#pragma unroll
            for (int c = 0; c < q; ++c) {
                h = h + g[c];
                hu = hu + ((T)dq_w(c) * lam) * g[c];
            }
            T ca, cb, cc, g2;
            eq_consts<T>(d, ca, cb, cc, g2);
            meq[0] = (hu * hu) / h + g2 * (h * h);
            if constexpr (q == 5) {
                meq[1] = (lam * lam) * hu;
                meq[2] = (lam * lam) * meq[0];
            }
        } else {
            using A = Ar<T>;
            T mc[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) mc[i] = A::add(g[2 * i], g[2 * i + 1]);
            equilibria<T, NF>(d, eqp_of<T>(d), mc, meq);
        }
    }

    // S1 with the reconstructed collision (Section 4.5, eq. reconstructedCollision):
    // the pre-collision populations are reconstructed on every finest cell
    // (projection up the tree, prediction of every other cell level by level);
    // each warp averages, one leaf at a time, the equilibria of the relaxed
    // moments over the leaf's 2^dj finest cells (into the interface array, free
    // until S4); then every leaf relaxes towards those averages.
    __device__ __noinline__ void collide_reconstructed() {
        upsweep();
        sync();
        const uint32_t *R = mask(sm.cur);
        for (int l = d.Jmin + 1; l <= d.Jmax; ++l) {
            const long long n = 1LL << l;
            const uint32_t *rl = R + sm.woff[l];
            for (long long k = tid; k < n; k += TS)
                if (!((rl[k >> 5] >> (k & 31)) & 1u))
                    for (int h = 0; h < q; ++h)
                        row(h, l)[k] = predict_g<T>(row(h, l - 1), k >> 1, (int)(k & 1), l - 1, d.bc, d.gamma,
                                                    tab.pc[d.gamma]);
            sync();
        }
        constexpr int NR = DQ ? q - 2 : nf;  // relaxed moments
        constexpr int NWARP = TS / 32;
        const int lane = tid & 31, warp = tid >> 5;
        const uint32_t *leaves = list(L_LEAF);
        const long long stride = d.N + 1;
        for (int i = warp; i < sm.nleaf; i += NWARP) {
            const uint32_t ent = leaves[i];
            const int l = ent >> KBITS;
            const long long k = ent & KMASK;
            const int dj = d.Jmax - l;
            const long long first = k << dj, ncell = 1LL << dj;
            T acc[3] = {T(0), T(0), T(0)};
            for (long long c = first + lane; c < first + ncell; c += 32) {
                T g[QMAX], meq[3];
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q) g[h] = row(h, d.Jmax)[c];
                relaxed_equilibria(g, meq);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = acc[r] + meq[r];
            }
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[r] = acc[r] + __shfl_xor_sync(FULL, acc[r], o);
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < NR; ++r) Phi[r * stride + i] = acc[r] * pow2m<T>(dj);
        }
        sync();
        for (int i = tid; i < sm.nleaf; i += TS) {
            const uint32_t ent = leaves[i];
            const int l = ent >> KBITS;
            const long long k = ent & KMASK;
            T f[QMAX], mavg[3];
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) f[h] = row(h, l)[k];
#pragma unroll
            for (int r = 0; r < NR; ++r) mavg[r] = Phi[r * stride + i];
            if constexpr (DQ) {
                const T lam = lam_of<T>(d);
                T m[q];
#pragma unroll
                for (int r = 0; r < q; ++r) m[r] = T(0);
#pragma unroll
                for (int h = 0; h < q; ++h) {
                    const T v = (T)dq_w(h) * lam;
                    T x = f[h];
#pragma unroll
                    for (int r = 0; r < q; ++r) {
                        m[r] = m[r] + x;
                        x = x * v;
                    }
                }
                T dm[q];
#pragma unroll
                for (int r = 2; r < q; ++r) dm[r] = s_of<T>(d, r - 2) * (mavg[r - 2] - m[r]);
#pragma unroll
                for (int h = 0; h < q; ++h) {
                    T a = T(0);
#pragma unroll
                    for (int r = 2; r < q; ++r) a = a + minv_of<T>(d, h, r) * dm[r];
                    f[h] = f[h] + a;
                }
            } else {
                using A = Ar<T>;
                const T lam = lam_of<T>(d);
#pragma unroll
                for (int j = 0; j < NF; ++j) {
                    const T mc = A::add(f[2 * j], f[2 * j + 1]), mn = A::mul(lam, A::sub(f[2 * j], f[2 * j + 1]));
                    const T sj = s_of<T>(d, j);
                    const T mstar = A::add(A::mul(oms_of<T>(d, j), mn), A::mul(sj, mavg[j]));
                    const T g = d.lam_log2 != NOT_POW2 ? scale2(mstar, -d.lam_log2) : div_lam<T>(mstar, d);
                    f[2 * j] = half_of<T>(A::add(mc, g));
                    f[2 * j + 1] = half_of<T>(A::sub(mc, g));
                }
            }
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) row(h, l)[k] = f[h];
        }
        sync();
    }

    // ---- A1 / S2: projection sweep, fine to coarse ---------------------------
    __device__ void upsweep() {
        const uint32_t *li = list(L_INT);
        for (int l = d.Jmax - 1; l >= d.Jmin; --l) {
            if (sm.seg[L_INT][l] == sm.seg[L_INT][l + 1]) continue;
            project_level(li, l);
            sync();
        }
    }

    // A1 right after a step of a D1Q2^n scheme, by conservation.  The stream
    // (S5) moved every leaf by w (Phi[first] - Phi[next]) with w = +-2^-dj, one
    // value of Phi per interface shared by the two cells it separates, so the
    // size-weighted mean of the leaves under an internal cell moved by the same
    // expression at the cell's own two edges (the inner interfaces cancel), and
    // the internal cells still hold the projection of f* (S2; ghosts lie outside
    // the tree).  One update of every internal cell, all levels in one pass,
    // therefore equals the level-by-level projection of the streamed leaves up
    // to rounding, and replaces its Jmax - Jmin dependent passes.
    // The update runs in the stream's own pass (S5): it reads only Phi, which S4
    // completed, and the internal cells, which S5 does not touch; the next
    // adaptation then starts from projected internal cells (status ST_FLUXED).
    __device__ __forceinline__ void project_by_flux_pass() {
        const uint32_t *li = list(L_INT);
        const int b = sm.seg[L_INT][d.Jmin], e = sm.seg[L_INT][d.Jmax];
        for (int i = b + tid; i < e; i += TS) {
            const uint32_t ent = li[i];
            const int l = ent >> KBITS;
            const long long k = ent & KMASK;
            const int dj = d.Jmax - l;
            long long first = k << dj, next = (k + 1) << dj;
            if (d.bc == 0) next &= d.N - 1;
            const T w = pow2m<T>(dj);
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) {
                    const auto ph = phi(h);
                    const T coef = (h & 1) ? -w : w;
                    const auto r = row(h, l);
                    r[k] = r[k] + coef * (ph[first] - ph[next]);
                }
        }
    }

    // ---- A2: details of the pairs of the tree, threshold T, Harten flags ----
    // FP64: the detail of Section 3.2 in double.  FP32: the detail in float with
    // a rigorous bound on its rounding error; only when a threshold lies within
    // that bound is the detail recomputed in FP64 from the stored values, so
    // every decision equals the one the exact detail of the stored state gives.
    __device__ void details() {
        if constexpr (WIDE) {
            details_wide();
            return;
        }
        // the even cells of the tree above Jmin: first children 2p of the internal cells p
        const uint32_t *lst = list(L_INT);
        int b = sm.seg[L_INT][d.Jmin], e = sm.seg[L_INT][d.Jmax];
        uint32_t *keep = mask(M_KEEP), *ref = mask(M_REF);
        for (int i = b + tid; i < e; i += TS) {
            uint32_t ent = lst[i];
            int l = (int)(ent >> KBITS) + 1;
            const bool hasref = l < d.Jmax;
            long long p = ent & KMASK, k = 2 * p;
            long long pl = wrapc(p - 1, l - 1, d.bc), pr = wrapc(p + 1, l - 1, d.bc);
            bool keepit, refit, tie = false;
            if constexpr (sizeof(T) == 8) {
                unsigned long long Db = 0ull;
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q) {
                        const auto rc = row(h, l - 1);
                        const double dv = row(h, l)[k] - (rc[p] + C1 * (rc[pr] - rc[pl]));
                        const unsigned long long b = abs_bits(dv);
                        Db = b > Db ? b : Db;
                    }
                decide_bits(Db, sm.eps_l[l], sm.big_l[l], hasref, keepit, refit, tie);
            } else {
                float D = 0.0f, B = 0.0f;
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q) {
                        const auto rc = row(h, l - 1);
                        float vk = row(h, l)[k], vl = rc[pl], vp = rc[p], vr = rc[pr];
                        float dv = vk - (vp + float(C1) * (vr - vl));
                        D = fmaxf(D, fabsf(dv));
                        B = fmaxf(B, fabsf(vk) + fabsf(vp) + fabsf(vl) + fabsf(vr));
                    }
                B *= 0x1p-21f;  // 4 times the rounding bound of the detail evaluation
                float el = sm.eps_f[l], bl = sm.big_f[l];
                // the band also covers the rounding of the thresholds to float
                bool amb = fabsf(D - el) <= B + el * 0x1p-22f || (hasref && fabsf(D - bl) <= B + bl * 0x1p-22f);
                if (amb) {
                    double Dd = 0.0;
                    for (int h = 0; h < q; ++h) {
                        const auto rc = row(h, l - 1);
                        double dv = (double)row(h, l)[k] - ((double)rc[p] + C1 * ((double)rc[pr] - (double)rc[pl]));
                        Dd = fmax(Dd, fabs(dv));
                    }
                    double e64 = sm.eps_l[l], b64 = sm.big_l[l];
                    keepit = Dd >= e64;
                    refit = hasref && Dd >= b64;
                    tie = fabs(Dd - e64) <= 1e-12 * e64 || (hasref && fabs(Dd - b64) <= 1e-12 * b64);
                } else {
                    keepit = D >= el;
                    refit = hasref && D >= bl;
                }
            }
            if (tie) atomicAdd(&sm.near_ties, 1);
            if (keepit) {
                int w = (int)(k >> 5);
                uint32_t bits = 3u << (k & 31);
                atomicOr(&keep[sm.woff[l] + w], bits);
                if (refit) atomicOr(&ref[sm.woff[l] + w], bits);
            }
        }
    }

    // A2 with the stencil of half-width gamma = 2 or 3: the prediction sums
    // c_a (f_{p+a} - f_{p-a}) in increasing a; the FP32 rounding band grows with
    // the number of operations, (6 gamma + 2) u times the sum of |inputs|
    // (3 gamma + 1 roundings, each at most u times that sum, with a factor 2 margin)
    __device__ __noinline__ void details_wide() {
        const uint32_t *lst = list(L_INT);  // first children 2p of the internal cells p
        const int b = sm.seg[L_INT][d.Jmin], e = sm.seg[L_INT][d.Jmax], g = d.gamma;
        const T *c = tab.pc[g];
        uint32_t *keep = mask(M_KEEP), *ref = mask(M_REF);
        for (int i = b + tid; i < e; i += TS) {
            const uint32_t ent = lst[i];
            const int l = (int)(ent >> KBITS) + 1;
            const bool hasref = l < d.Jmax;
            const long long p = ent & KMASK, k = 2 * p;
            bool keepit, refit, tie = false;
            double Dd = 0.0;
            unsigned long long Db = 0ull;
            float Df = 0.0f, B = 0.0f;
            for (int h = 0; h < q; ++h) {
                const auto rc = row(h, l - 1);
                T sum = T(0);
                float mag = 0.0f;
                for (int a = 1; a <= g; ++a) {
                    const T vr = rc[wrapc(p + a, l - 1, d.bc)], vl = rc[wrapc(p - a, l - 1, d.bc)];
                    sum = a == 1 ? c[0] * (vr - vl) : sum + c[a - 1] * (vr - vl);
                    if constexpr (sizeof(T) == 4) mag = mag + fabsf(vr) + fabsf(vl);
                }
                const T vk = row(h, l)[k], vp = rc[p];
                if constexpr (sizeof(T) == 8) {
                    const unsigned long long b = abs_bits(vk - (vp + sum));
                    Db = b > Db ? b : Db;
                } else {
                    Df = fmaxf(Df, fabsf(vk - (vp + sum)));
                    B = fmaxf(B, fabsf(vk) + fabsf(vp) + mag);
                }
            }
            if constexpr (sizeof(T) == 8) {
                decide_bits(Db, sm.eps_l[l], sm.big_l[l], hasref, keepit, refit, tie);
            } else {
                B *= (float)(6 * g + 2) * 0x1p-24f;
                const float el = sm.eps_f[l], bl = sm.big_f[l];
                const bool amb = fabsf(Df - el) <= B + el * 0x1p-22f || (hasref && fabsf(Df - bl) <= B + bl * 0x1p-22f);
                if (amb) {
                    for (int h = 0; h < q; ++h) {
                        const auto rc = row(h, l - 1);
                        double sum = 0.0;
                        for (int a = 1; a <= g; ++a)
                            sum = a == 1 ? (double)c[0] * ((double)rc[wrapc(p + 1, l - 1, d.bc)] - (double)rc[wrapc(p - 1, l - 1, d.bc)])
                                         : sum + (double)c[a - 1] * ((double)rc[wrapc(p + a, l - 1, d.bc)] -
                                                                     (double)rc[wrapc(p - a, l - 1, d.bc)]);
                        Dd = fmax(Dd, fabs((double)row(h, l)[k] - ((double)rc[p] + sum)));
                    }
                    const double e64 = sm.eps_l[l], b64 = sm.big_l[l];
                    keepit = Dd >= e64;
                    refit = hasref && Dd >= b64;
                    tie = fabs(Dd - e64) <= 1e-12 * e64 || (hasref && fabs(Dd - b64) <= 1e-12 * b64);
                } else {
                    keepit = Df >= el;
                    refit = hasref && Df >= bl;
                }
            }
            if (tie) atomicAdd(&sm.near_ties, 1);
            if (keepit) {
                const int w = (int)(k >> 5);
                const uint32_t bits = 3u << (k & 31);
                atomicOr(&keep[sm.woff[l] + w], bits);
                if (refit) atomicOr(&ref[sm.woff[l] + w], bits);
            }
        }
    }

    // ---- candidate words of the step -----------------------------------------
    // Every cell of the new tree lies within 2 gamma + 4 cells of a cell of the
    // old tree on its level or of a child of one (the enlargement moves at most
    // sigma + 1 <= 3 cells from a kept cell and adds children of kept pairs;
    // grading from level l + 1 reaches gamma + 2 cells beyond half of that
    // level's distance), and every transfer or ghost mark lies within
    // 2 gamma + 10 <= 16 cells of one: inside the mask words next to (+-1 word)
    // a word that holds an old cell, or a child word of one.  Those words are
    // the step's candidates.  The word passes (enlargement, grading and
    // marking, list compaction, clearing) visit them only; every other word of
    // every mask stays zero.  The list is built from the occupancy bitmap of
    // the old tree (one bit per mask word) by a block scan.

    // level l and index j within the level of occupancy word og (levels up to 9
    // have one occupancy word, level l >= 10 has 2^(l - 10))
    __device__ __forceinline__ void level_of_occ(int og, int &l, int &j) const {
        const int nsmall = max(0, min(d.Jmax, 9) - d.Jmin + 1);
        if (og < nsmall) {
            l = d.Jmin + og;
            j = 0;
            return;
        }
        const int L0 = d.Jmin > 10 ? d.Jmin : 10;
        const int x = og - nsmall + (1 << (L0 - 10));
        l = 10 + (31 - __clz(x));
        j = x - (1 << (l - 10));
    }
    // candidate bits of occupancy word j of level l, from the old tree's occupancy oc
    __device__ __forceinline__ uint32_t cand_bits(const uint32_t *oc, int l, int j) const {
        const int Lo = l >= 5 ? l - 5 : 0;  // the level's mask words: 2^Lo
        const uint32_t vb = Lo >= 5 ? FULL : ((1u << (1 << Lo)) - 1u);
        if (l <= 6) return vb;  // levels of at most two words: every word
        const uint32_t *ol = oc + sm.ooff[l];
        uint32_t x = dilate([&](int q) { return ol[q]; }, Lo, j, 1, d.bc);
        if (l > d.Jmin) {
            // child words of the occupied words of level l - 1
            const uint32_t *op = oc + sm.ooff[l - 1];
            x |= dilate([&](int q) { return Lo > 5 ? spread16(op[q >> 1] >> (16 * (q & 1))) : (spread16(op[0]) & vb); },
                        Lo, j, 1, d.bc);
        }
        return x & vb;
    }

    __device__ void build_cw() {
        constexpr int NW = TS / 32;
        const int lane = tid & 31, warp = tid >> 5;
        const uint32_t *oc = occ(sm.cur);
        uint32_t *cw = cwl();
        const int OW = d.OW;
        int run = 0;
        for (int r = 0, base = 0; base < OW; ++r, base += TS) {
            const int og = base + tid;
            int l = d.Jmin, j = 0;
            uint32_t c = 0u;
            if (og < OW) {
                level_of_occ(og, l, j);
                c = cand_bits(oc, l, j);
            }
            const int cnt = __popc(c);
            int x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            int *sw = bx.scan_w[r & 1][0];  // alternate buffers: one barrier per round
            if (lane == 31) sw[warp] = x;
            sync();
            const int v = lane < NW ? sw[lane] : 0;
            const int before = __reduce_add_sync(FULL, lane < warp ? v : 0);
            const int tot = __reduce_add_sync(FULL, v);
            int off = run + before + x - cnt;
            if (og < OW && j == 0) sm.cw_seg[l] = off;
            const uint32_t g0 = (uint32_t)(sm.woff[l] + 32 * j);
            while (c) {
                const int b = __ffs(c) - 1;
                c &= c - 1u;
                cw[off++] = g0 + (uint32_t)b;
            }
            run += tot;
        }
        if (tid == 0) sm.cw_seg[d.Jmax + 1] = run;
        sync();
    }

    // ---- A3: R(H(T)) per candidate word --------------------------------------
    __device__ void enlarge(uint32_t *Rn) {
        const uint32_t *keep = mask(M_KEEP), *ref = mask(M_REF);
        const int ncw = sm.cw_seg[d.Jmax + 1];
        for (int i = tid; i < ncw; i += TS) {
            const int g = cw_at(i);
            int l, wi;
            level_of_word(sm, g, l, wi);
            uint32_t vb = valid_bits(l), rh;
            if (l == d.Jmin) {
                rh = vb;
            } else {
                const uint32_t *kl = keep + sm.woff[l];
                uint32_t rt = kl[wi];
                rh = rt | pairexpand(dilate([&](int j) { return kl[j]; }, l, wi, SIGMA, d.bc));
                if (l >= d.Jmin + 2) rh |= spread16(ref[sm.woff[l - 1] + (wi >> 1)] >> (16 * (wi & 1)));
            }
            Rn[g] = rh & vb;
        }
    }

    // ---- A4: grading sweep + leaf / transfer / ghost marking -----------------
    // Fine to coarse: the cells of level l require (l-1, floor(k/2) + delta),
    // |delta| <= gamma = 1, with siblings (Def. Graded tree); once level l is
    // final its leaves (no child in the tree), its transfer marks (new leaves
    // outside the old tree and the parent stencils of finer marks) and its ghost
    // marks (reconstruction windows k-2..k+2 of its leaves and the parent
    // stencils of finer ghosts, outside the tree) are written.  Levels of 64
    // cells or more work on whole words, with the neighbouring words' edge bits;
    // the smaller levels are done by one thread without barriers.
    // grade = false only re-derives the marks of a tree known to be graded.
    __device__ void grade_and_mark(uint32_t *Rn, const uint32_t *Ro, bool grade) {
        uint32_t *LF = mask(M_LEAF), *PR = mask(M_PRED), *GH = mask(M_GH);
        const int g = d.gamma;
        const int lbig = d.Jmin > 6 ? d.Jmin : 6;
        for (int l = d.Jmax; l >= lbig; --l) {
            const int Wl = 1 << (l - 5);
            const uint32_t *rl = Rn + sm.woff[l];
            if (grade && l > d.Jmin + 1) {
                uint32_t *rp = Rn + sm.woff[l - 1];
                if constexpr (!WIDE) {
                    for (int i = sm.cw_seg[l - 1] + tid; i < sm.cw_seg[l]; i += TS) {
                        const int wp = cw_at(i) - sm.woff[l - 1];
                        uint32_t x = fold2(rl[2 * wp], rl[2 * wp + 1]);
                        bool eL = (word_bc(rl, 2 * wp - 1, Wl, d.bc) >> 30) != 0u;  // children of parent 32 wp - 1
                        bool eR = (word_bc(rl, 2 * wp + 2, Wl, d.bc) & 3u) != 0u;   // children of parent 32 wp + 32
                        rp[wp] |= pairexpand(dilate1_edges(x, eL, eR));
                    }
                } else {
                    for (int i = sm.cw_seg[l - 1] + tid; i < sm.cw_seg[l]; i += TS) {
                        const int wp = cw_at(i) - sm.woff[l - 1];
                        const uint32_t x = fold2(rl[2 * wp], rl[2 * wp + 1]);
                        // parents 29..31 of the word on the left, 0..2 of the word on the right
                        const uint32_t xl = fold3(word_bc(rl, 2 * wp - 1, Wl, d.bc) >> 26) << 29;
                        const uint32_t xr = fold3(word_bc(rl, 2 * wp + 2, Wl, d.bc) & 63u);
                        rp[wp] |= pairexpand(dilate_edges(x, xl, xr, g));
                    }
                }
            }
            const uint32_t *rol = Ro + sm.woff[l];
            uint32_t *lfl = LF + sm.woff[l], *prl = PR + sm.woff[l], *ghl = GH + sm.woff[l];
            const int cb = sm.cw_seg[l], ce = sm.cw_seg[l + 1], wo = sm.woff[l];
            if (l == d.Jmax) {
                for (int i = cb + tid; i < ce; i += TS) {
                    const int wi = cw_at(i) - wo;
                    uint32_t r = rl[wi];
                    lfl[wi] = r;
                    prl[wi] = r & ~rol[wi];
                    ghl[wi] = 0u;
                }
            } else if constexpr (WIDE) {
                const int Wc = Wl << 1;
                const uint32_t *rc = Rn + sm.woff[l + 1], *pc = PR + sm.woff[l + 1], *gc = GH + sm.woff[l + 1];
                for (int i = cb + tid; i < ce; i += TS) {
                    const int wi = cw_at(i) - wo;
                    const uint32_t r = rl[wi], ro = rol[wi];
                    const uint32_t lf = r & ~fold2(rc[2 * wi], rc[2 * wi + 1]);
                    // leaf bits of the 16 cells of each neighbouring word next to this one
                    const uint32_t cL = word_bc(rc, 2 * wi - 1, Wc, d.bc), cR = word_bc(rc, 2 * wi + 2, Wc, d.bc);
                    const uint32_t lfL = word_bc(rl, wi - 1, Wl, d.bc) & ~(compact_even(cL | (cL >> 1)) << 16);
                    const uint32_t lfR = word_bc(rl, wi + 1, Wl, d.bc) & ~compact_even(cR | (cR >> 1));
                    const uint32_t gw = dilate_edges(lf, lfL, lfR, 2 * g);  // reconstruction windows
                    const uint32_t pd = dilate_edges(fold2(pc[2 * wi], pc[2 * wi + 1]),
                                                     fold3(word_bc(pc, 2 * wi - 1, Wc, d.bc) >> 26) << 29,
                                                     fold3(word_bc(pc, 2 * wi + 2, Wc, d.bc) & 63u), g);
                    const uint32_t gd = dilate_edges(fold2(gc[2 * wi], gc[2 * wi + 1]),
                                                     fold3(word_bc(gc, 2 * wi - 1, Wc, d.bc) >> 26) << 29,
                                                     fold3(word_bc(gc, 2 * wi + 2, Wc, d.bc) & 63u), g);
                    lfl[wi] = lf;
                    prl[wi] = (lf | pd) & ~ro;
                    ghl[wi] = (gw | gd) & ~r;
                }
            } else {
                const int Wc = Wl << 1;
                const uint32_t *rc = Rn + sm.woff[l + 1], *pc = PR + sm.woff[l + 1], *gc = GH + sm.woff[l + 1];
                for (int i = cb + tid; i < ce; i += TS) {
                    const int wi = cw_at(i) - wo;
                    uint32_t r = rl[wi], ro = rol[wi];
                    uint32_t lf = r & ~fold2(rc[2 * wi], rc[2 * wi + 1]);
                    // leaf bits of cells 30, 31 of the left word and 0, 1 of the right word
                    uint32_t lfL = (word_bc(rl, wi - 1, Wl, d.bc) >> 30) & ~fold_low2(word_bc(rc, 2 * wi - 1, Wc, d.bc) >> 28);
                    uint32_t lfR = (word_bc(rl, wi + 1, Wl, d.bc) & 3u) & ~fold_low2(word_bc(rc, 2 * wi + 2, Wc, d.bc) & 15u);
                    uint32_t gw = lf | (lf << 1) | (lf << 2) | (lf >> 1) | (lf >> 2);
                    gw |= (lfL ? 1u : 0u) | ((lfL & 2u) ? 2u : 0u);                    // from cells 30, 31 on the left
                    gw |= (lfR ? 0x80000000u : 0u) | ((lfR & 1u) ? 0x40000000u : 0u);  // from cells 0, 1 on the right
                    uint32_t p = fold2(pc[2 * wi], pc[2 * wi + 1]);
                    uint32_t pd = dilate1_edges(p, (word_bc(pc, 2 * wi - 1, Wc, d.bc) >> 30) != 0u,
                                                (word_bc(pc, 2 * wi + 2, Wc, d.bc) & 3u) != 0u);
                    uint32_t g = fold2(gc[2 * wi], gc[2 * wi + 1]);
                    uint32_t gd = dilate1_edges(g, (word_bc(gc, 2 * wi - 1, Wc, d.bc) >> 30) != 0u,
                                                (word_bc(gc, 2 * wi + 2, Wc, d.bc) & 3u) != 0u);
                    lfl[wi] = lf;
                    prl[wi] = (lf | pd) & ~ro;
                    ghl[wi] = (gw | gd) & ~r;
                }
            }
            sync();
        }
        tick(T_GRADE);
        if (tid == 0 && d.Jmin <= 5) small_levels(Rn, Ro, grade);
        sync();
    }

    // The levels of at most 32 cells (one word each), coarsest last, by one
    // thread: grading of level l-1 and the marks of level l as in the word-wise
    // sweep, with the words of the level below kept in registers rather than
    // reloaded after the previous level wrote them.
    __device__ void small_levels(uint32_t *Rn, const uint32_t *Ro, bool grade) {
        const int gam = WIDE ? d.gamma : 1;
        // the descriptor fields in registers: a store through a mask pointer
        // could otherwise force their reload from shared memory at every level
        const int Jmin = d.Jmin, Jmax = d.Jmax, bc = d.bc;
        uint32_t *LF = mask(M_LEAF), *PR = mask(M_PRED), *GH = mask(M_GH);
        const int ltop = Jmax < 5 ? Jmax : 5;
        // words of level ltop + 1 (two words when it has 64 cells, one when fewer)
        uint32_t rc0 = 0u, rc1 = 0u, pc0 = 0u, pc1 = 0u, gc0 = 0u, gc1 = 0u;
        if (ltop < Jmax) {
            const int oc = sm.woff[ltop + 1];
            rc0 = Rn[oc];
            pc0 = PR[oc];
            gc0 = GH[oc];
            if (ltop + 1 >= 6) {
                rc1 = Rn[oc + 1];
                pc1 = PR[oc + 1];
                gc1 = GH[oc + 1];
            }
        }
        uint32_t r = Rn[sm.woff[ltop]];
        int o = sm.woff[ltop];
        for (int l = ltop; l >= Jmin; --l) {
            const int n = 1 << l;
            const int op = l > Jmin ? sm.woff[l - 1] : 0;
            const uint32_t vb = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
            const uint32_t ro = Ro[o];
            uint32_t rp = l > Jmin ? Rn[op] : 0u;
            if (grade && l > Jmin + 1) {
                const int np = n >> 1;
                const uint32_t vbp = (1u << np) - 1u;
                rp |= pairexpand(dil_small(fold2(r, 0u), np, gam, bc)) & vbp;
            }
            uint32_t lf = r, pr, gh = 0u;
            if (l < Jmax) {
                lf = r & ~fold2(rc0, rc1);
                pr = (lf | dil_small(fold2(pc0, pc1), n, gam, bc)) & ~ro;
                gh = (dil_small(lf, n, 2 * gam, bc) | dil_small(fold2(gc0, gc1), n, gam, bc)) & ~r;
            } else {
                pr = lf & ~ro;
            }
            lf &= vb;
            pr &= vb;
            gh &= vb;
            LF[o] = lf;
            PR[o] = pr;
            GH[o] = gh;
            if (l > Jmin) Rn[op] = rp;
            rc0 = r;
            rc1 = 0u;
            pc0 = pr;
            pc1 = 0u;
            gc0 = gh;
            gc1 = 0u;
            r = rp;
            o = op;
        }
    }

    // dilation by r cells inside a level of n <= 32 cells held in one word
    __device__ __forceinline__ uint32_t dil_small(uint32_t x, int n, int r, int bc) const {
        const uint32_t vb = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
        uint32_t out = x;
        for (int s = 1; s <= r; ++s) {
            if (bc == 0) {
                // rotations within the level (a wide stencil's reach may exceed n)
                const int sm_ = WIDE ? s % n : s;
                if (sm_) out |= ((x << sm_) | (x >> (n - sm_)) | (x >> sm_) | (x << (n - sm_))) & vb;
            } else {
                out |= ((x << s) & vb) | (x >> s);
            }
        }
        return out;
    }
    // parent bits (n of them) of the child level l+1 of a level of n <= 32 cells
    __device__ __forceinline__ uint32_t fold_small(const uint32_t *child, int l) const {
        return l + 1 >= 6 ? fold2(child[0], child[1]) : fold2(child[0], 0u);
    }

    // ---- A5: list compaction -------------------------------------------------
    __device__ __forceinline__ void word_lists(const uint32_t *Rn, int g, int l, uint32_t (&m)[NLIST]) {
        uint32_t r = Rn[g], lf = mask(M_LEAF)[g];
        m[L_INT] = r & ~lf;
        m[L_LEAF] = lf;
        m[L_PRED] = mask(M_PRED)[g];
        m[L_GH] = mask(M_GH)[g];
    }

    // Rounds of TS consecutive candidate words, one word per thread; a block
    // scan of the per-word counts places each word's entries (the lists stay
    // sorted by level, then cell).  A dense word costs its owner at most 32
    // stores per list, and dense levels are spread over as many threads as they
    // have words.  The occupancy bitmap occn of the listed tree is set on the
    // way (it must start cleared).
    __device__ void build_lists(const uint32_t *Rn, uint32_t *occn) {
        constexpr int NW = TS / 32;
        const int lane = tid & 31, warp = tid >> 5;
        const int ncw = sm.cw_seg[d.Jmax + 1];
        const bool sparse = sparse_on();
        int run[NLIST] = {0, 0, 0, 0};
        if (tid == 0) sm.deplev[0] = sm.deplev[1] = 0u;  // new lists: gathered again by predict_fill
        for (int r = 0, base = 0; base < ncw; ++r, base += TS) {
            const int i = base + tid;
            const bool valid = i < ncw;
            int l = 0, wi = 0;
            uint32_t m[NLIST] = {0u, 0u, 0u, 0u};
            if (valid) {
                const int g = cw_at(i);
                level_of_word(sm, g, l, wi);
                word_lists(Rn, g, l, m);
                if (sparse && (m[L_INT] | m[L_LEAF])) atomicOr(&occn[sm.ooff[l] + (wi >> 5)], 1u << (wi & 31));
            }
            int inc[NLIST];
#pragma unroll
            for (int L = 0; L < NLIST; ++L) {
                int x = __popc(m[L]);
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += y;
                }
                inc[L] = x;
            }
            int(*sw)[32] = bx.scan_w[r & 1];  // alternate buffers: one barrier per round
            if (lane == 31)
#pragma unroll
                for (int L = 0; L < NLIST; ++L) sw[L][warp] = inc[L];
            sync();
            const uint32_t pk = pack(l, 32LL * wi);
#pragma unroll
            for (int L = 0; L < NLIST; ++L) {
                const int v = lane < NW ? sw[L][lane] : 0;
                const int before = __reduce_add_sync(FULL, lane < warp ? v : 0);
                const int tot = __reduce_add_sync(FULL, v);
                uint32_t x = m[L];
                int off = run[L] + before + inc[L] - __popc(x);
                if (valid && i == sm.cw_seg[l]) {
                    // first candidate word of level l; levels just below without
                    // candidate words hold no cell and start at the same place
                    sm.seg[L][l] = off;
                    for (int k = l - 1; k >= d.Jmin && sm.cw_seg[k] == sm.cw_seg[l]; --k) sm.seg[L][k] = off;
                }
                uint32_t *dst = list(L);
                while (x) {
                    const int bit = __ffs(x) - 1;
                    x &= x - 1u;
                    dst[off++] = pk + (uint32_t)bit;
                }
                run[L] += tot;
            }
        }
        if (tid == 0) {
#pragma unroll
            for (int L = 0; L < NLIST; ++L) sm.seg[L][d.Jmax + 1] = run[L];
            // the finest levels without candidate words are empty
            for (int k = d.Jmax; k >= d.Jmin && sm.cw_seg[k] == ncw; --k)
#pragma unroll
                for (int L = 0; L < NLIST; ++L) sm.seg[L][k] = run[L];
            sm.nleaf = run[L_LEAF];
        }
        sync();
    }

    // ---- the word passes over every word (instances without candidate words) ----
    __device__ void enlarge_dense(uint32_t *Rn) {
        const uint32_t *keep = mask(M_KEEP), *ref = mask(M_REF);
        for (int g = tid; g < d.Wtot; g += TS) {
            int l, wi;
            level_of_word(sm, g, l, wi);
            uint32_t vb = valid_bits(l), rh;
            if (l == d.Jmin) {
                rh = vb;
            } else {
                const uint32_t *kl = keep + sm.woff[l];
                uint32_t rt = kl[wi];
                rh = rt | pairexpand(dilate([&](int j) { return kl[j]; }, l, wi, SIGMA, d.bc));
                if (l >= d.Jmin + 2) rh |= spread16(ref[sm.woff[l - 1] + (wi >> 1)] >> (16 * (wi & 1)));
            }
            Rn[g] = rh & vb;
        }
    }

    __device__ void grade_and_mark_dense(uint32_t *Rn, const uint32_t *Ro, bool grade) {
        uint32_t *LF = mask(M_LEAF), *PR = mask(M_PRED), *GH = mask(M_GH);
        const int g = d.gamma;
        const int lbig = d.Jmin > 6 ? d.Jmin : 6;
        // gamma = 1: the levels of at most 32 words go to one warp (grade_warp)
        const int lwarp = WIDE ? lbig - 1 : (d.Jmax < 10 ? d.Jmax : 10);
        for (int l = d.Jmax; l >= lbig && l > lwarp; --l) {
            const int Wl = 1 << (l - 5);
            const uint32_t *rl = Rn + sm.woff[l];
            if (grade && l > d.Jmin + 1) {
                uint32_t *rp = Rn + sm.woff[l - 1];
                if constexpr (!WIDE) {
                    for (int wp = tid; wp < (Wl >> 1); wp += TS) {
                        uint32_t x = fold2(rl[2 * wp], rl[2 * wp + 1]);
                        bool eL = (word_bc(rl, 2 * wp - 1, Wl, d.bc) >> 30) != 0u;  // children of parent 32 wp - 1
                        bool eR = (word_bc(rl, 2 * wp + 2, Wl, d.bc) & 3u) != 0u;   // children of parent 32 wp + 32
                        rp[wp] |= pairexpand(dilate1_edges(x, eL, eR));
                    }
                } else {
                    for (int wp = tid; wp < (Wl >> 1); wp += TS) {
                        const uint32_t x = fold2(rl[2 * wp], rl[2 * wp + 1]);
                        // parents 29..31 of the word on the left, 0..2 of the word on the right
                        const uint32_t xl = fold3(word_bc(rl, 2 * wp - 1, Wl, d.bc) >> 26) << 29;
                        const uint32_t xr = fold3(word_bc(rl, 2 * wp + 2, Wl, d.bc) & 63u);
                        rp[wp] |= pairexpand(dilate_edges(x, xl, xr, g));
                    }
                }
            }
            const uint32_t *rol = Ro + sm.woff[l];
            uint32_t *lfl = LF + sm.woff[l], *prl = PR + sm.woff[l], *ghl = GH + sm.woff[l];
            if (l == d.Jmax) {
                for (int wi = tid; wi < Wl; wi += TS) {
                    uint32_t r = rl[wi];
                    lfl[wi] = r;
                    prl[wi] = r & ~rol[wi];
                    ghl[wi] = 0u;
                }
            } else if constexpr (WIDE) {
                const int Wc = Wl << 1;
                const uint32_t *rc = Rn + sm.woff[l + 1], *pc = PR + sm.woff[l + 1], *gc = GH + sm.woff[l + 1];
                for (int wi = tid; wi < Wl; wi += TS) {
                    const uint32_t r = rl[wi], ro = rol[wi];
                    const uint32_t lf = r & ~fold2(rc[2 * wi], rc[2 * wi + 1]);
                    // leaf bits of the 16 cells of each neighbouring word next to this one
                    const uint32_t cL = word_bc(rc, 2 * wi - 1, Wc, d.bc), cR = word_bc(rc, 2 * wi + 2, Wc, d.bc);
                    const uint32_t lfL = word_bc(rl, wi - 1, Wl, d.bc) & ~(compact_even(cL | (cL >> 1)) << 16);
                    const uint32_t lfR = word_bc(rl, wi + 1, Wl, d.bc) & ~compact_even(cR | (cR >> 1));
                    const uint32_t gw = dilate_edges(lf, lfL, lfR, 2 * g);  // reconstruction windows
                    const uint32_t pd = dilate_edges(fold2(pc[2 * wi], pc[2 * wi + 1]),
                                                     fold3(word_bc(pc, 2 * wi - 1, Wc, d.bc) >> 26) << 29,
                                                     fold3(word_bc(pc, 2 * wi + 2, Wc, d.bc) & 63u), g);
                    const uint32_t gd = dilate_edges(fold2(gc[2 * wi], gc[2 * wi + 1]),
                                                     fold3(word_bc(gc, 2 * wi - 1, Wc, d.bc) >> 26) << 29,
                                                     fold3(word_bc(gc, 2 * wi + 2, Wc, d.bc) & 63u), g);
                    lfl[wi] = lf;
                    prl[wi] = (lf | pd) & ~ro;
                    ghl[wi] = (gw | gd) & ~r;
                }
            } else {
                const int Wc = Wl << 1;
                const uint32_t *rc = Rn + sm.woff[l + 1], *pc = PR + sm.woff[l + 1], *gc = GH + sm.woff[l + 1];
                for (int wi = tid; wi < Wl; wi += TS) {
                    uint32_t r = rl[wi], ro = rol[wi];
                    uint32_t lf = r & ~fold2(rc[2 * wi], rc[2 * wi + 1]);
                    // leaf bits of cells 30, 31 of the left word and 0, 1 of the right word
                    uint32_t lfL = (word_bc(rl, wi - 1, Wl, d.bc) >> 30) & ~fold_low2(word_bc(rc, 2 * wi - 1, Wc, d.bc) >> 28);
                    uint32_t lfR = (word_bc(rl, wi + 1, Wl, d.bc) & 3u) & ~fold_low2(word_bc(rc, 2 * wi + 2, Wc, d.bc) & 15u);
                    uint32_t gw = lf | (lf << 1) | (lf << 2) | (lf >> 1) | (lf >> 2);
                    gw |= (lfL ? 1u : 0u) | ((lfL & 2u) ? 2u : 0u);                    // from cells 30, 31 on the left
                    gw |= (lfR ? 0x80000000u : 0u) | ((lfR & 1u) ? 0x40000000u : 0u);  // from cells 0, 1 on the right
                    uint32_t p = fold2(pc[2 * wi], pc[2 * wi + 1]);
                    uint32_t pd = dilate1_edges(p, (word_bc(pc, 2 * wi - 1, Wc, d.bc) >> 30) != 0u,
                                                (word_bc(pc, 2 * wi + 2, Wc, d.bc) & 3u) != 0u);
                    uint32_t g = fold2(gc[2 * wi], gc[2 * wi + 1]);
                    uint32_t gd = dilate1_edges(g, (word_bc(gc, 2 * wi - 1, Wc, d.bc) >> 30) != 0u,
                                                (word_bc(gc, 2 * wi + 2, Wc, d.bc) & 3u) != 0u);
                    lfl[wi] = lf;
                    prl[wi] = (lf | pd) & ~ro;
                    ghl[wi] = (gw | gd) & ~r;
                }
            }
            sync();
        }
        if constexpr (!WIDE)
            if (tid < 32 && lwarp >= lbig) grade_warp(Rn, Ro, grade, lwarp, lbig);
        tick(T_GRADE);
        if (tid == 0 && d.Jmin <= 5) small_levels(Rn, Ro, grade);
        sync();
    }

    // Grading and marking of the levels ltop .. lbot of at most 32 words each
    // (gamma = 1) by one warp, without block barriers: lane i holds word i of
    // the current level and words 2i, 2i + 1 of the level below it (R, PR, GH)
    // in registers, neighbouring and child words arrive by shuffles (wrapped
    // or empty beyond the domain, as word_bc), and the results are stored for
    // the list compaction and the small levels.  The same operations as the
    // block-wide sweep, level for level.
    __device__ __noinline__ void grade_warp(uint32_t *Rn, const uint32_t *Ro, bool grade, int ltop, int lbot) {
        uint32_t *LF = mask(M_LEAF), *PR = mask(M_PRED), *GH = mask(M_GH);
        const int lane = tid;  // tid < 32
        const int bc = d.bc;
        const int Wt = 1 << (ltop - 5);
        // words 2 lane, 2 lane + 1 of level ltop + 1 (final: graded and marked by the block)
        uint32_t rc0 = 0u, rc1 = 0u, pc0 = 0u, pc1 = 0u, gc0 = 0u, gc1 = 0u;
        if (ltop < d.Jmax && lane < Wt) {
            const int o = sm.woff[ltop + 1] + 2 * lane;
            rc0 = Rn[o];
            rc1 = Rn[o + 1];
            pc0 = PR[o];
            pc1 = PR[o + 1];
            gc0 = GH[o];
            gc1 = GH[o + 1];
        }
        uint32_t r = lane < Wt ? Rn[sm.woff[ltop] + lane] : 0u;  // level ltop, graded from ltop + 1
        for (int l = ltop; l >= lbot; --l) {
            const int Wl = 1 << (l - 5);  // 2 .. 32 words
            const bool act = lane < Wl;
            const uint32_t ro = act ? Ro[sm.woff[l] + lane] : 0u;
            // word j of a level of Wl words whose word q lane q holds in v
            auto word = [&](uint32_t v, int j) -> uint32_t {
                const bool out = j < 0 || j >= Wl;
                const int src = bc == 0 ? ((j + Wl) & (Wl - 1)) : (out ? 0 : j);
                const uint32_t x = __shfl_sync(FULL, v, src);
                return (bc != 0 && out) ? 0u : x;
            };
            // grading of level l - 1: parent word wp = lane from words 2wp - 1 .. 2wp + 2 of level l
            const uint32_t c0 = word(r, 2 * lane), c1 = word(r, 2 * lane + 1);
            const uint32_t cL = word(r, 2 * lane - 1), cR = word(r, 2 * lane + 2);
            uint32_t rpn = 0u;
            if (l > d.Jmin) {
                const int Wp = Wl >> 1;
                uint32_t hp = lane < Wp ? Rn[sm.woff[l - 1] + lane] : 0u;  // enlarged set of level l - 1
                if (grade && l > d.Jmin + 1 && lane < Wp)
                    hp |= pairexpand(dilate1_edges(fold2(c0, c1), (cL >> 30) != 0u, (cR & 3u) != 0u));
                if (lane < Wp) Rn[sm.woff[l - 1] + lane] = hp;
                rpn = lane < Wp ? hp : 0u;
            }
            // leaf, transfer and ghost marks of level l
            uint32_t lf, pr, gh = 0u;
            if (l == d.Jmax) {
                lf = r;
                pr = r & ~ro;
            } else {
                const uint32_t rl0 = word(r, lane - 1), rl1 = word(r, lane + 1);
                const uint32_t rcL = word(rc1, lane - 1), rcR = word(rc0, lane + 1);  // words 2 lane - 1, 2 lane + 2 below
                const uint32_t pcL = word(pc1, lane - 1), pcR = word(pc0, lane + 1);
                const uint32_t gcL = word(gc1, lane - 1), gcR = word(gc0, lane + 1);
                lf = r & ~fold2(rc0, rc1);
                const uint32_t lfL = (rl0 >> 30) & ~fold_low2(rcL >> 28);
                const uint32_t lfR = (rl1 & 3u) & ~fold_low2(rcR & 15u);
                uint32_t gw = lf | (lf << 1) | (lf << 2) | (lf >> 1) | (lf >> 2);
                gw |= (lfL ? 1u : 0u) | ((lfL & 2u) ? 2u : 0u);
                gw |= (lfR ? 0x80000000u : 0u) | ((lfR & 1u) ? 0x40000000u : 0u);
                const uint32_t pd = dilate1_edges(fold2(pc0, pc1), (pcL >> 30) != 0u, (pcR & 3u) != 0u);
                const uint32_t gd = dilate1_edges(fold2(gc0, gc1), (gcL >> 30) != 0u, (gcR & 3u) != 0u);
                pr = (lf | pd) & ~ro;
                gh = (gw | gd) & ~r;
            }
            if (act) {
                const int o = sm.woff[l] + lane;
                LF[o] = lf;
                PR[o] = pr;
                GH[o] = gh;
            }
            // the next level (l - 1): its lane i holds words 2i, 2i + 1 of level l
            rc0 = c0;
            rc1 = c1;
            pc0 = __shfl_sync(FULL, pr, (2 * lane) & 31);
            pc1 = __shfl_sync(FULL, pr, (2 * lane + 1) & 31);
            gc0 = __shfl_sync(FULL, gh, (2 * lane) & 31);
            gc1 = __shfl_sync(FULL, gh, (2 * lane + 1) & 31);
            r = rpn;
        }
        __syncwarp();
    }

    __device__ void build_lists_dense(const uint32_t *Rn) {
        constexpr int NW = TS / 32;
        const int lane = tid & 31, warp = tid >> 5;
        const int Wtot = d.Wtot;
        int run[NLIST] = {0, 0, 0, 0};
        if (tid == 0) sm.deplev[0] = sm.deplev[1] = 0u;  // new lists: gathered again by predict_fill
        for (int r = 0, base = 0; base < Wtot; ++r, base += TS) {
            const int g = base + tid;
            const bool valid = g < Wtot;
            int l = 0, wi = 0;
            uint32_t m[NLIST] = {0u, 0u, 0u, 0u};
            if (valid) {
                level_of_word(sm, g, l, wi);
                word_lists(Rn, g, l, m);
            }
            // the four lists' counts two per value, in 16-bit fields (a round's
            // totals are at most 1024 x 32 < 2^16): half the scan steps and reductions
            uint32_t x01 = (uint32_t)__popc(m[0]) | ((uint32_t)__popc(m[1]) << 16);
            uint32_t x23 = (uint32_t)__popc(m[2]) | ((uint32_t)__popc(m[3]) << 16);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y01 = __shfl_up_sync(FULL, x01, o), y23 = __shfl_up_sync(FULL, x23, o);
                if (lane >= o) {
                    x01 += y01;
                    x23 += y23;
                }
            }
            int(*sw)[32] = bx.scan_w[r & 1];  // alternate buffers: one barrier per round
            if (lane == 31) {
                sw[0][warp] = (int)x01;
                sw[1][warp] = (int)x23;
            }
            sync();
            const uint32_t v01 = lane < NW ? (uint32_t)sw[0][lane] : 0u, v23 = lane < NW ? (uint32_t)sw[1][lane] : 0u;
            const uint32_t b01 = __reduce_add_sync(FULL, lane < warp ? v01 : 0u);
            const uint32_t b23 = __reduce_add_sync(FULL, lane < warp ? v23 : 0u);
            const uint32_t t01 = __reduce_add_sync(FULL, v01), t23 = __reduce_add_sync(FULL, v23);
            const int inc[NLIST] = {(int)(x01 & 0xFFFFu), (int)(x01 >> 16), (int)(x23 & 0xFFFFu), (int)(x23 >> 16)};
            const int before[NLIST] = {(int)(b01 & 0xFFFFu), (int)(b01 >> 16), (int)(b23 & 0xFFFFu), (int)(b23 >> 16)};
            const int tot[NLIST] = {(int)(t01 & 0xFFFFu), (int)(t01 >> 16), (int)(t23 & 0xFFFFu), (int)(t23 >> 16)};
            const uint32_t pk = pack(l, 32LL * wi);
#pragma unroll
            for (int L = 0; L < NLIST; ++L) {
                uint32_t x = m[L];
                int off = run[L] + before[L] + inc[L] - __popc(x);
                if (valid && wi == 0) sm.seg[L][l] = off;
                uint32_t *dst = list(L);
                while (x) {
                    const int bit = __ffs(x) - 1;
                    x &= x - 1u;
                    dst[off++] = pk + (uint32_t)bit;
                }
                run[L] += tot[L];
            }
        }
        if (tid == 0) {
#pragma unroll
            for (int L = 0; L < NLIST; ++L) sm.seg[L][d.Jmax + 1] = run[L];
            sm.nleaf = run[L_LEAF];
        }
        sync();
    }

    // ---- A6 / S3: prediction of listed cells, coarse to fine -----------------
    // predicts the listed cell ent (level l) from level l - 1
    __device__ __forceinline__ void predict_entry(uint32_t ent, int l) {
        {
            const long long k = ent & KMASK;
            T v[QMAX];
            if constexpr (!WIDE) {
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q) v[h] = predict<T>(row(h, l - 1), k >> 1, (int)(k & 1), l - 1, d.bc);
            } else {
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q)
                        v[h] = predict_g<T>(row(h, l - 1), k >> 1, (int)(k & 1), l - 1, d.bc, d.gamma, tab.pc[d.gamma]);
            }
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) row(h, l)[k] = v[h];
        }
    }

    // whether the prediction stencil of cell (l, k) at level l - 1 (parent +-
    // gamma, wrapped or clamped as the prediction does) holds a cell marked in P
    __device__ __forceinline__ bool stencil_marked(const uint32_t *P, int l, long long k) const {
        const int gg = WIDE ? d.gamma : 1, lp = l - 1;
        const uint32_t *pl = P + sm.woff[lp];
        const long long p = k >> 1;
        bool hit = false;
        for (int a = -gg; a <= gg; ++a) {
            const long long c = wrapc(p + a, lp, d.bc);
            hit |= ((pl[c >> 5] >> (c & 31)) & 1u) != 0u;
        }
        return hit;
    }

    // A6 / S3.  A listed cell whose stencil holds no cell of the same list reads
    // only tree values (the old tree for the transfer, the current tree for the
    // ghosts: the marking closes both lists under prediction stencils), so those
    // cells go in one pass over all levels; the rest follow level by level,
    // coarse to fine, on the levels that have any.  The marks of both lists stay
    // in their masks until the next step's A2 clears them.
    __device__ void predict_fill(int L) {
        const uint32_t *lst = list(L);
        const uint32_t *P = mask(L == L_GH ? M_GH : M_PRED);
        const int slot = L == L_GH ? 1 : 0;
        const int b = sm.seg[L][d.Jmin + 1], e = sm.seg[L][d.Jmax + 1];
        for (int i = b + tid; i < e; i += TS) {
            const uint32_t ent = lst[i];
            const int l = (int)(ent >> KBITS);
            if (stencil_marked(P, l, ent & KMASK))
                atomicOr(&sm.deplev[slot], 1u << l);
            else
                predict_entry(ent, l);
        }
        sync();
        const uint32_t lv = sm.deplev[slot];
        for (int l = d.Jmin + 1; l <= d.Jmax; ++l) {
            if (!((lv >> l) & 1u)) continue;
            for (int i = sm.seg[L][l] + tid; i < sm.seg[L][l + 1]; i += TS) {
                const uint32_t ent = lst[i];
                if (stencil_marked(P, l, ent & KMASK)) predict_entry(ent, l);
            }
            sync();
        }
    }

    // ---- mesh adaptation ----------------------------------------------------
    __device__ void adapt() {
        uint32_t *Ro = mask(sm.cur), *Rn = mask(sm.cur ^ 1);
        tick(NPHASE);
        if (sparse_on()) build_cw();
        {
            // the transfer / ghost marks of the last list compaction share storage
            // with KEEP / REF, which A2 accumulates into: clear them (all of them
            // lie in candidate words; the barrier of A1 orders this before A2),
            // and the occupancy bitmap the list compaction will fill
            uint32_t *pr = mask(M_PRED), *gh = mask(M_GH);
            const int ncw = sm.cw_seg[d.Jmax + 1];
            for (int i = tid; i < ncw; i += TS) {
                const int g = cw_at(i);
                pr[g] = 0u;
                gh[g] = 0u;
            }
            if (sparse_on()) {
                uint32_t *on = occ(sm.cur ^ 1);
                for (int g = tid; g < d.OW; g += TS) on[g] = 0u;
            }
        }
        tick(T_CANDIDATES);
        // internal cells: already projected by the last stream (D1Q2^n), else level by level
        if (DQ || !(sm.status & ST_FLUXED)) upsweep();
        sync();
        tick(T_UPSWEEP_A);
        details();
        sync();
        tick(T_DETAILS);
        if (sparse_on()) enlarge(Rn); else enlarge_dense(Rn);
        sync();
        tick(T_ENLARGE);
        if (sparse_on()) grade_and_mark(Rn, Ro, true); else grade_and_mark_dense(Rn, Ro, true);
        tick(T_GRADE_SMALL);
        if (sparse_on()) build_lists(Rn, occ(sm.cur ^ 1)); else build_lists_dense(Rn);
        tick(T_LISTS);
        predict_fill(L_PRED);
        if (sparse_on()) {
            // the old tree's buffer holds the next step's new tree: clear it (its
            // cells lie in candidate words; nothing reads it after the grading);
            // without candidate words the enlargement writes every word
            const uint32_t *cw = cwl();
            const int ncw = sm.cw_seg[d.Jmax + 1];
            for (int i = tid; i < ncw; i += TS) Ro[cw[i]] = 0u;
        }
        tick(T_TRANSFER);
        if (tid == 0) {
            sm.cur ^= 1;
            sm.updates += (unsigned long long)sm.nleaf;
            sm.status &= ~(int)ST_FLUXED;  // new tree: its internal cells are projections of f
        }
        sync();
    }

    // ---- one step of the adaptive scheme on the current mesh -----------------
    __device__ void lbm_step() {
        tick(NPHASE);
        if constexpr (WIDE) {
            if (d.collision)
                collide_reconstructed();  // S1, eq. reconstructedCollision
            else
                collide_all();
        } else {
            collide_all();      // S1
        }
        sync();
        tick(T_COLLIDE);
        upsweep();              // S2
        tick(T_UPSWEEP_S);
        predict_fill(L_GH);     // S3
        tick(T_GHOSTS);
        reconstruct_edges();    // S4
        sync();
        tick(T_RECON);
        stream_and_audit();     // S5
        tick(T_STREAM);
    }

    // S4: first / last finest-cell values of every leaf -> Phi
    __device__ void reconstruct_edges() {
        if constexpr (DQ) {
            reconstruct_dq();  // gamma = 1 (the tables)
            return;
        }
        if constexpr (WIDE) {
            if (d.gamma > 1) {
                reconstruct_wide();
                return;
            }
        }
        const uint32_t *R = mask(sm.cur);
        const uint32_t *leaves = list(L_LEAF);
        for (int i = tid; i < sm.nleaf; i += TS) {
            uint32_t ent = leaves[i];
            int l = ent >> KBITS;
            long long k = ent & KMASK;
            const int dj = d.Jmax - l;
            const long long nl = 1LL << l;
            bool at_left = d.bc == 1 && k == 0, at_right = d.bc == 1 && k == nl - 1;
            bool fin_l = false, fin_r = false;
            if (dj > 0) {
                const uint32_t *rf = R + sm.woff[l + 1];
                if (!at_left) {
                    long long c = 2 * wrapc(k - 1, l, d.bc);
                    fin_l = (rf[c >> 5] >> (c & 31)) & 1u;
                }
                if (!at_right) {
                    long long c = 2 * wrapc(k + 1, l, d.bc);
                    fin_r = (rf[c >> 5] >> (c & 31)) & 1u;
                }
            }
            const T *cf = tab.cf[dj], *t1 = tab.t1[dj], *bf = tab.bf[dj];
#pragma unroll
            for (int h = 0; h < QMAX; ++h) {
                if (h >= q) break;
                const auto r = row(h, l);
                const bool plus = (h & 1) == 0;  // velocity +lambda
                bool need_first = !plus || at_left, need_last = plus || at_right;
                T rfirst = T(0), rlast = T(0);
                if (dj == 0) {
                    rfirst = rlast = r[k];
                } else {
                    T vm1 = r[wrapc(k - 1, l, d.bc)], v0 = r[k], vp1 = r[wrapc(k + 1, l, d.bc)];
                    const auto rf = row(h, l + 1);
                    // one sum of four products for both stencils, so that a warp whose
                    // leaves mix them evaluates it once: next to a finer neighbour the
                    // leaf's own children (predicted) enter with the weights t1, else
                    // the cells of level l with the weights cf
                    if (need_first) {
                        if (at_left) {
                            rfirst = bf[0] * v0 + bf[1] * vp1;
                        } else {
                            T x0, x1, x2, x3;
                            const T *wt;
                            if (fin_l) {
                                const T tt = T(C1) * (vp1 - vm1);
                                const long long c = 2 * wrapc(k - 1, l, d.bc);
                                x0 = rf[c];
                                x1 = rf[c + 1];
                                x2 = v0 + tt;
                                x3 = v0 - tt;
                                wt = t1;
                            } else {
                                x0 = r[wrapc(k - 2, l, d.bc)];
                                x1 = vm1;
                                x2 = v0;
                                x3 = vp1;
                                wt = cf;
                            }
                            rfirst = dot4(wt[0], x0, wt[1], x1, wt[2], x2, wt[3], x3);
                        }
                    }
                    if (need_last) {
                        if (at_right) {
                            rlast = bf[0] * v0 + bf[1] * vm1;
                        } else {
                            T x0, x1, x2, x3;
                            const T *wt;
                            if (fin_r) {
                                const T tt = T(C1) * (vp1 - vm1);
                                const long long c = 2 * wrapc(k + 1, l, d.bc);
                                x0 = v0 + tt;
                                x1 = v0 - tt;
                                x2 = rf[c];
                                x3 = rf[c + 1];
                                wt = t1;
                            } else {
                                x0 = vm1;
                                x1 = v0;
                                x2 = vp1;
                                x3 = r[wrapc(k + 2, l, d.bc)];
                                wt = cf;
                            }
                            rlast = dot4(wt[3], x0, wt[2], x1, wt[1], x2, wt[0], x3);
                        }
                    }
                }
                const auto ph = phi(h);
                if (plus) {
                    long long ix = (k + 1) << dj;
                    if (d.bc == 0) ix &= d.N - 1;
                    ph[ix] = rlast;
                    if (at_left) ph[0] = rfirst;
                } else {
                    ph[k << dj] = rfirst;
                    if (at_right) ph[d.N] = rlast;
                }
            }
        }
    }

    // S4 with the stencil of half-width gamma = 2 or 3: the first / last finest
    // values by the level-by-level reconstruction (edge_walk) instead of tables
    __device__ __noinline__ void reconstruct_wide() {
        const uint32_t *R = mask(sm.cur);
        const uint32_t *leaves = list(L_LEAF);
        const int g = d.gamma;
        const T *c = tab.pc[g];
        for (int i = tid; i < sm.nleaf; i += TS) {
            const uint32_t ent = leaves[i];
            const int l = ent >> KBITS;
            const long long k = ent & KMASK;
            const int dj = d.Jmax - l;
            const bool at_left = d.bc == 1 && k == 0, at_right = d.bc == 1 && k == (1LL << l) - 1;
            for (int h = 0; h < q; ++h) {
                const T *rb = V + h;
                const bool plus = (h & 1) == 0;  // velocity +lambda
                const bool need_first = !plus || at_left, need_last = plus || at_right;
                T rfirst = T(0), rlast = T(0);
                if (dj == 0) {
                    rfirst = rlast = row(h, l)[k];
                } else {
                    if (need_first)
                        rfirst = g == 2 ? edge_walk<T, 2, false>(rb, q, d.Jmin, d.Jmax, d.bc, R, sm.woff, c, l, k)
                                        : edge_walk<T, 3, false>(rb, q, d.Jmin, d.Jmax, d.bc, R, sm.woff, c, l, k);
                    if (need_last)
                        rlast = g == 2 ? edge_walk<T, 2, true>(rb, q, d.Jmin, d.Jmax, d.bc, R, sm.woff, c, l, k)
                                       : edge_walk<T, 3, true>(rb, q, d.Jmin, d.Jmax, d.bc, R, sm.woff, c, l, k);
                }
                const auto ph = phi(h);
                if (plus) {
                    long long ix = (k + 1) << dj;
                    if (d.bc == 0) ix &= d.N - 1;
                    ph[ix] = rlast;
                    if (at_left) ph[0] = rfirst;
                } else {
                    ph[k << dj] = rfirst;
                    if (at_right) ph[d.N] = rlast;
                }
            }
        }
    }

    // S4 for the D1Q3 / D1Q5 schemes: every leaf writes the reconstructed
    // finest values it holds within |w^h| cells of its edges, by finest
    // position: a +v population needs the cells left of each interface (the
    // last |w| cells of a leaf), a -v population the cells right of it (the
    // first |w|); at a copy boundary also the cell next to the boundary, which
    // the clamped out-of-domain cells copy.  Second cells from an edge use the
    // second-cell tables.
    __device__ __noinline__ void reconstruct_dq() {
        const uint32_t *R = mask(sm.cur);
        const uint32_t *leaves = list(L_LEAF);
        for (int i = tid; i < sm.nleaf; i += TS) {
            const uint32_t ent = leaves[i];
            const int l = ent >> KBITS;
            const long long k = ent & KMASK;
            const int dj = d.Jmax - l;
            const long long first = k << dj, last = ((k + 1) << dj) - 1;
            const bool at_left = d.bc == 1 && k == 0, at_right = d.bc == 1 && k == (1LL << l) - 1;
            bool fin_l = false, fin_r = false;
            long long cl = 0, cr = 0;
            if (dj > 0) {
                const uint32_t *rf = R + sm.woff[l + 1];
                cl = 2 * wrapc(k - 1, l, d.bc);
                cr = 2 * wrapc(k + 1, l, d.bc);
                if (!at_left) fin_l = (rf[cl >> 5] >> (cl & 31)) & 1u;
                if (!at_right) fin_r = (rf[cr >> 5] >> (cr & 31)) & 1u;
            }
            for (int h = 1; h < q; ++h) {
                const int w = dq_w(h), a = w < 0 ? -w : w;
                const auto r = row(h, l);
                const auto ph = phi(h);
                if (dj == 0) {
                    ph[first] = r[k];
                    continue;
                }
                const T vm1 = r[wrapc(k - 1, l, d.bc)], v0 = r[k], vp1 = r[wrapc(k + 1, l, d.bc)];
                const auto rf = row(h, l + 1);
                // cell `sec` (0: first / last, 1: second from that edge) next to the left or right
                // edge: one sum of four products for both stencils (as in reconstruct_edges), next
                // to a finer neighbour with the leaf's own (predicted) children and the weights t1
                auto from_left = [&](int sec) -> T {
                    const T *bf = sec ? tab.bf2[dj] : tab.bf[dj], *t1 = sec ? tab.t12[dj] : tab.t1[dj],
                            *cf = sec ? tab.cf2[dj] : tab.cf[dj];
                    if (at_left) return bf[0] * v0 + bf[1] * vp1;
                    T x0, x1, x2, x3;
                    const T *wt;
                    if (fin_l) {
                        const T tt = T(C1) * (vp1 - vm1);
                        x0 = rf[cl];
                        x1 = rf[cl + 1];
                        x2 = v0 + tt;
                        x3 = v0 - tt;
                        wt = t1;
                    } else {
                        x0 = r[wrapc(k - 2, l, d.bc)];
                        x1 = vm1;
                        x2 = v0;
                        x3 = vp1;
                        wt = cf;
                    }
                    return dot4(wt[0], x0, wt[1], x1, wt[2], x2, wt[3], x3);
                };
                auto from_right = [&](int sec) -> T {
                    const T *bf = sec ? tab.bf2[dj] : tab.bf[dj], *t1 = sec ? tab.t12[dj] : tab.t1[dj],
                            *cf = sec ? tab.cf2[dj] : tab.cf[dj];
                    if (at_right) return bf[0] * v0 + bf[1] * vm1;
                    T x0, x1, x2, x3;
                    const T *wt;
                    if (fin_r) {
                        const T tt = T(C1) * (vp1 - vm1);
                        x0 = v0 + tt;
                        x1 = v0 - tt;
                        x2 = rf[cr];
                        x3 = rf[cr + 1];
                        wt = t1;
                    } else {
                        x0 = vm1;
                        x1 = v0;
                        x2 = vp1;
                        x3 = r[wrapc(k + 2, l, d.bc)];
                        wt = cf;
                    }
                    return dot4(wt[3], x0, wt[2], x1, wt[1], x2, wt[0], x3);
                };
                if (w > 0) {
                    ph[last] = from_right(0);
                    if (a == 2) ph[last - 1] = from_right(1);
                    if (at_left) ph[first] = from_left(0);
                } else {
                    ph[first] = from_left(0);
                    if (a == 2) ph[first + 1] = from_left(1);
                    if (at_right) ph[last] = from_right(0);
                }
            }
        }
    }

    // S5 for the D1Q3 / D1Q5 schemes (eq. AdaptiveStreamPhase with |w| <= 2):
    // f^{n+1} = f* + sigma 2^-dj sum_{delta=1}^{|w|} (V[first + eta] - V[next + eta]),
    // eta = -delta (sigma > 0) or delta - 1 (sigma < 0), V the finest values of
    // reconstruct_dq (wrapped, or clamped at a copy boundary); audit of (h, hu)
    __device__ __noinline__ void stream_dq() {
        const uint32_t *leaves = list(L_LEAF);
        const long long N = d.N;
        auto at = [&](long long i) -> long long { return d.bc == 0 ? (i & (N - 1)) : (i < 0 ? 0 : (i >= N ? N - 1 : i)); };
        double macc[3] = {0.0, 0.0, 0.0};
        float fhi[3] = {0.0f, 0.0f, 0.0f}, flo[3] = {0.0f, 0.0f, 0.0f};
        bool bad = false;
        for (int i = tid; i < sm.nleaf; i += TS) {
            const uint32_t ent = leaves[i];
            const int l = ent >> KBITS;
            const long long k = ent & KMASK;
            const int dj = d.Jmax - l;
            const long long first = k << dj, next = (k + 1) << dj;
            const T wgt = pow2m<T>(dj);
            T fn[QMAX];
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) {
                    const int w = dq_w(h);
                    const auto r = row(h, l);
                    T v = r[k];
                    if (w != 0) {
                        const auto ph = phi(h);
                        const int a = w < 0 ? -w : w;
                        T acc = T(0);
                        for (int dl = 1; dl <= a; ++dl) {
                            const long long eta = w > 0 ? -dl : dl - 1;
                            acc = acc + (ph[at(first + eta)] - ph[at(next + eta)]);
                        }
                        v = v + (w > 0 ? wgt : -wgt) * acc;
                    }
                    bad |= nonfinite(v);
                    r[k] = v;
                    fn[h] = v;
                }
            if constexpr (sizeof(T) == 8) {
                double m0 = 0.0, m1 = 0.0;
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q) {
                        m0 += (double)fn[h];
                        m1 += (dq_w(h) * d.lam) * (double)fn[h];
                    }
                macc[0] += sm.dx_l[l] * m0;
                macc[1] += sm.dx_l[l] * m1;
            } else {
                // exact per-leaf sums of f and of w f in float-float, scaled by 2^-l
                const float sc = pow2m<float>(l);
                float a0 = 0.0f, e0 = 0.0f, a1 = 0.0f, e1 = 0.0f;
#pragma unroll
                for (int h = 0; h < QMAX; ++h)
                    if (h < q) {
                        ff_add(a0, e0, (float)fn[h], 0.0f);
                        ff_add(a1, e1, (float)(dq_w(h)) * (float)fn[h], 0.0f);
                    }
                ff_add(fhi[0], flo[0], a0 * sc, e0 * sc);
                ff_add(fhi[1], flo[1], a1 * sc, e1 * sc);
            }
        }
        if (bad) atomicOr(&sm.status, (int)ST_NONFINITE);
        if constexpr (sizeof(T) == 8) {
            team_sum(macc);
        } else {
            team_sum_ff(fhi, flo, macc);
            if (tid == 0) {
                macc[0] *= d.b - d.a;
                macc[1] *= (d.b - d.a) * d.lam;
            }
        }
        if (tid == 0) {
            // copy boundary: what leaves through x = a and x = b, sum over the
            // populations of sigma 2^-Jmax-weighted telescoped stream terms
            double flux[2] = {0.0, 0.0};
            if (d.bc == 1) {
                const double dxJ = sm.dx_l[d.Jmax];
                for (int h = 1; h < q; ++h) {
                    const int w = dq_w(h), a = w < 0 ? -w : w;
                    const auto ph = phi(h);
                    double t = 0.0;
                    for (int dl = 1; dl <= a; ++dl) {
                        const long long eta = w > 0 ? -dl : dl - 1;
                        t += (double)ph[at(eta)] - (double)ph[at(N + eta)];
                    }
                    t *= (w > 0 ? dxJ : -dxJ);
                    flux[0] += t;
                    flux[1] += (w * d.lam) * t;
                }
            }
            for (int j = 0; j < 2; ++j) {
                const double res = fabs(macc[j] - sm.mass[j] - flux[j]);
                sm.audit = fmax(sm.audit, res);
                sm.mass[j] = macc[j];
            }
            sm.steps += 1ULL;
        }
        sync();
    }

    // sum of four products; FP32: compensated (Kahan) accumulation
    static __device__ __forceinline__ T dot4(T c0, T x0, T c1, T x1, T c2, T x2, T c3, T x3) {
        if constexpr (sizeof(T) == 8) {
            return fma(c3, x3, fma(c2, x2, fma(c1, x1, c0 * x0)));
        } else {
            T p[4] = {c0 * x0, c1 * x1, c2 * x2, c3 * x3};
            T s = T(0), comp = T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                T y = p[j] - comp;
                T t = s + y;
                comp = (t - s) - y;
                s = t;
            }
            return s;
        }
    }

    // S5: f^{n+1} = f* + sigma 2^-dj (Phi[first] - Phi[next]); mass audit.
    // The totals sum dx_l (f+ + f-) over the leaves: FP64 in the FP64 path; in
    // the FP32 path 2^-l (f+ + f-) is summed exactly per leaf into float-float
    // partials (relative error near 2^-44) and scaled by b - a at the end.
    __device__ void stream_and_audit() {
        if constexpr (DQ) {
            stream_dq();
            return;
        }
        const uint32_t *leaves = list(L_LEAF);
        double macc[3] = {0.0, 0.0, 0.0};
        float fhi[3] = {0.0f, 0.0f, 0.0f}, flo[3] = {0.0f, 0.0f, 0.0f};
        bool bad = false;
        for (int i = tid; i < sm.nleaf; i += TS) {
            uint32_t ent = leaves[i];
            int l = ent >> KBITS;
            long long k = ent & KMASK;
            int dj = d.Jmax - l;
            long long first = k << dj, next = (k + 1) << dj;
            if (d.bc == 0) next &= d.N - 1;
            const T w = pow2m<T>(dj);
            T fn[QMAX];
#pragma unroll
            for (int h = 0; h < QMAX; ++h)
                if (h < q) {
                    const auto ph = phi(h);
                    T coef = (h & 1) ? -w : w;
                    const auto r = row(h, l);
                    T v = r[k] + coef * (ph[first] - ph[next]);
                    bad |= nonfinite(v);
                    r[k] = v;
                    fn[h] = v;
                }
            if constexpr (sizeof(T) == 8) {
                const double dx = sm.dx_l[l];
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nf) macc[j] += dx * ((double)fn[2 * j] + (double)fn[2 * j + 1]);
            } else {
                const float sc = pow2m<float>(l);
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nf) {
                        float sj, ej;
                        two_sum((float)fn[2 * j], (float)fn[2 * j + 1], sj, ej);
                        ff_add(fhi[j], flo[j], sj * sc, ej * sc);
                    }
            }
        }
        if (bad) atomicOr(&sm.status, (int)ST_NONFINITE);
        project_by_flux_pass();  // A1 of the next adaptation, same pass
        if constexpr (sizeof(T) == 8) {
            team_sum(macc);
        } else {
            team_sum_ff(fhi, flo, macc);
            if (tid == 0)
                for (int j = 0; j < nf; ++j) macc[j] *= d.b - d.a;
        }
        if (tid == 0) {
            double dxJ = sm.dx_l[d.Jmax];
            for (int j = 0; j < nf; ++j) {
                double flux = 0.0;
                if (d.bc == 1) {
                    const auto pp = phi(2 * j), pm = phi(2 * j + 1);
                    flux = dxJ * (((double)pp[0] - (double)pp[d.N]) - ((double)pm[0] - (double)pm[d.N]));
                }
                double res = fabs(macc[j] - sm.mass[j] - flux);
                sm.audit = fmax(sm.audit, res);
                sm.mass[j] = macc[j];
            }
            sm.steps += 1ULL;
            sm.status |= ST_FLUXED;  // before the barrier: every thread of the next adaptation sees it
        }
        sync();
    }

    // ---- initial state -------------------------------------------------------
    // full tree, populations at equilibrium of the conserved moments (staged m_cons)
    __device__ __noinline__ void init_full(const double *mcons) {
        uint32_t *R = mask(M_R0);
        for (int g = tid; g < d.Wtot; g += TS) {
            int l, wi;
            level_of_word(sm, g, l, wi);
            R[g] = valid_bits(l);
            mask(M_R1)[g] = 0u;
            mask(M_KEEP)[g] = 0u;
            mask(M_REF)[g] = 0u;
        }
        for (long long k = tid; k < d.N; k += TS) {
            double mc[3], f[QMAX];
            for (int j = 0; j < nf; ++j) mc[j] = mcons[j * d.N + k];
            if constexpr (DQ)
                dq_equilibrium_populations<q>(d, mc, f);
            else
                equilibrium_populations<NF>(d, mc, f);
            for (int h = 0; h < q; ++h) row(h, d.Jmax)[k] = (T)f[h];
        }
        if (tid == 0) sm.cur = M_R0;
        sync();
        finish_init();
    }

    // arbitrary graded tree (one byte per cell) and values
    __device__ __noinline__ void init_state(const unsigned char *Rb, const double *vals) {
        uint32_t *R = mask(M_R0);
        for (int g = tid; g < d.Wtot; g += TS) {
            int l, wi;
            level_of_word(sm, g, l, wi);
            long long base = cell_off(l, d.Jmin) + 32LL * wi;
            int nb = l >= 5 ? 32 : (1 << l);
            uint32_t w = 0;
            for (int b = 0; b < nb; ++b) w |= (Rb[base + b] ? 1u : 0u) << b;
            R[g] = w;
            mask(M_R1)[g] = 0u;
            mask(M_KEEP)[g] = 0u;
            mask(M_REF)[g] = 0u;
        }
        // population-major input to the cell-major layout
        for (long long c = tid; c < (long long)q * d.S; c += TS) {
            const long long hh = c / d.S, cell = c - hh * d.S;
            V[cell * q + hh] = (T)vals[c];
        }
        if (tid == 0) sm.cur = M_R0;
        sync();
        finish_init();
    }

    __device__ __noinline__ void finish_init() {
        uint32_t *R = mask(sm.cur);
        {
            // every mask word is a candidate of this first marking
            if (sparse_on()) {
                uint32_t *cw = cwl();
                for (int g = tid; g < d.Wtot; g += TS) cw[g] = (uint32_t)g;
                for (int g = tid; g < d.OW; g += TS) {
                    occ(M_R0)[g] = 0u;
                    occ(M_R1)[g] = 0u;
                }
            }
            for (int l = d.Jmin + tid; l <= d.Jmax + 1; l += TS) sm.cw_seg[l] = sm.woff[l];
        }
        sync();
        grade_and_mark(R, R, false);  // PRED empty: the tree is its own old tree
        build_lists(R, occ(sm.cur));
        // FP64 totals of the initial leaves
        const uint32_t *leaves = list(L_LEAF);
        double macc[3] = {0.0, 0.0, 0.0};
        for (int i = tid; i < sm.nleaf; i += TS) {
            uint32_t ent = leaves[i];
            int l = ent >> KBITS;
            long long k = ent & KMASK;
            double dx = sm.dx_l[l];
            if constexpr (DQ) {
                double m0 = 0.0, m1 = 0.0;
                for (int h = 0; h < q; ++h) {
                    const double f = (double)row(h, l)[k];
                    m0 += f;
                    m1 += (dq_w(h) * d.lam) * f;
                }
                macc[0] += dx * m0;
                macc[1] += dx * m1;
            } else {
                for (int j = 0; j < nf; ++j) macc[j] += dx * ((double)row(2 * j, l)[k] + (double)row(2 * j + 1, l)[k]);
            }
        }
        team_sum(macc);
        if (tid == 0) {
            for (int j = 0; j < nf; ++j) sm.mass[j] = macc[j];
            sm.audit = 0.0;
            sm.status = 0;
            sm.near_ties = 0;
            sm.updates = 0ULL;
            sm.steps = 0ULL;
        }
        if (tid == TS - 1) sm.passes = 0ULL;  // the thread that counts the barriers
        sync();
    }

    // ---- multiresolution reconstruction on the finest level (measurement) ----
    __device__ __noinline__ void finest(double *out) {
        upsweep();
        if (tid == 0) sm.status &= ~(int)ST_FLUXED;  // internal cells now project f, not f*
        sync();
        const uint32_t *R = mask(sm.cur);
        for (int l = d.Jmin + 1; l <= d.Jmax; ++l) {
            long long n = 1LL << l;
            const uint32_t *rl = R + sm.woff[l];
            for (long long k = tid; k < n; k += TS)
                if (!((rl[k >> 5] >> (k & 31)) & 1u))
                    for (int h = 0; h < q; ++h)
                        row(h, l)[k] = predict_g<T>(row(h, l - 1), k >> 1, (int)(k & 1), l - 1, d.bc, d.gamma,
                                                    tab.pc[d.gamma]);
            sync();
        }
        for (long long k = tid; k < d.N; k += TS) {
            if constexpr (DQ) {
                double m0 = 0.0, m1 = 0.0;
                for (int h = 0; h < q; ++h) {
                    const double f = (double)row(h, d.Jmax)[k];
                    m0 += f;
                    m1 += (dq_w(h) * d.lam) * f;
                }
                out[k] = m0;
                out[d.N + k] = m1;
            } else {
                for (int j = 0; j < nf; ++j) out[j * d.N + k] = (double)row(2 * j, d.Jmax)[k] + (double)row(2 * j + 1, d.Jmax)[k];
            }
        }
        sync();
    }
};

// ---------------------------------------------------------------------------
// instance state in and out of shared memory (TS threads of the team)

template <typename T, int TS, int SPM>
__device__ void load_instance(TeamSmem<T> &sm, const InstDesc &dg, int tid) {
    if (tid == 0) {
        sm.d = dg;
        const InstState &st = *dg.st;
        sm.cur = st.cur;
        sm.nleaf = st.nleaf;
        sm.status = st.status;
        sm.near_ties = st.near_ties;
        sm.deplev[0] = st.deplev[0];
        sm.deplev[1] = st.deplev[1];
        sm.updates = st.updates;
        sm.steps = st.steps;
        sm.passes = st.passes;
        sm.audit = st.audit;
        for (int j = 0; j < 3; ++j) sm.mass[j] = st.mass[j];
#ifdef MRG_PHASE_TIMERS
        for (int p = 0; p < NPHASE; ++p) sm.ptime[p] = st.ptime[p];
        sm.tlast = clock64();
#endif
        int Jmin = dg.Jmin, Jmax = dg.Jmax;
        int o = 0, oo = 0;
        for (int l = Jmin; l <= Jmax; ++l) {
            sm.woff[l] = o;
            sm.ooff[l] = oo;
            o += l >= 5 ? (1 << (l - 5)) : 1;
            oo += l >= 10 ? (1 << (l - 10)) : 1;
        }
        sm.woff[Jmax + 1] = o;
        sm.ooff[Jmax + 1] = oo;
        sm.sparse = SPM != 0 ? 1 : 0;
        // without candidate words every word of level l is visited
        if (!sm.sparse)
            for (int l = Jmin; l <= Jmax + 1; ++l) sm.cw_seg[l] = sm.woff[l];
        sm.g0s = Jmin < 5 ? 5 - Jmin : 0;
        sm.gbase = Jmin < 5 ? 1 : (1 << (Jmin - 5));
    }
    for (int l = tid; l <= MAXLEV; l += TS) {
        // eps_l = 2^{l - Jmax} eps (Prop. ErrorControl), Harten level 2^{mu_bar + 1} eps_l
        double el = ldexp(dg.eps, l - dg.Jmax);
        double bl = ldexp(el, dg.mu_bar + 1);
        sm.eps_l[l] = el;
        sm.big_l[l] = bl;
        sm.eps_f[l] = (float)el;
        sm.big_f[l] = (float)bl;
        sm.dx_l[l] = ldexp(dg.b - dg.a, -l);
    }
    for (int i = tid; i < NLIST * (MAXLEV + 2); i += TS) (&sm.seg[0][0])[i] = (&dg.st->seg[0][0])[i];
    if constexpr (TS == 32)
        __syncwarp();
    else
        __syncthreads();
}

template <typename T, int TS>
__device__ void store_instance(TeamSmem<T> &sm, int tid) {
    // the barrier count of the last pass is written after that pass's barrier
    if constexpr (TS == 32)
        __syncwarp();
    else
        __syncthreads();
    InstState &st = *sm.d.st;
    if (tid == 0) {
        st.cur = sm.cur;
        st.nleaf = sm.nleaf;
        st.status = sm.status;
        st.near_ties = sm.near_ties;
        st.deplev[0] = sm.deplev[0];
        st.deplev[1] = sm.deplev[1];
        st.updates = sm.updates;
        st.steps = sm.steps;
        st.passes = sm.passes;
        st.audit = sm.audit;
        for (int j = 0; j < 3; ++j) st.mass[j] = sm.mass[j];
#ifdef MRG_PHASE_TIMERS
        for (int p = 0; p < NPHASE; ++p) st.ptime[p] = sm.ptime[p];
#endif
    }
    for (int i = tid; i < NLIST * (MAXLEV + 2); i += TS) (&st.seg[0][0])[i] = (&sm.seg[0][0])[i];
    if constexpr (TS == 32)
        __syncwarp();
    else
        __syncthreads();
}

// one instance for the launch's steps
template <typename T, int NF, int TS, bool WIDE, int SPM>
__device__ __forceinline__ void run_instance(TeamSmem<T> &sm, const Tables<T> &tab, BlockScratch &bx, const LaunchArgs &a, int tid,
                             uint32_t *masks) {
    Worker<T, NF, TS, WIDE, SPM> w(sm, tab, bx, tid, masks);
    if (a.phases & PH_INIT_FULL) w.init_full((const double *)a.aux0 + sm.d.m_off);
    if (a.phases & PH_INIT_STATE) w.init_state((const unsigned char *)a.aux0, (const double *)a.aux1);
    for (int n = 0; n < a.nsteps; ++n) {
        if (a.phases & PH_ADAPT) w.adapt();
        if (a.phases & PH_STEP) w.lbm_step();
    }
    if (a.phases & PH_FINEST) w.finest((double *)a.aux0);
}

// Bitmasks live in shared memory (smask, room for `cap` words per mask) when the
// instance fits: the current tree and the transfer / ghost marks (which a later
// step's predictions read; KEEP / REF share their storage and A2 clears it) are
// copied in at the start and back at the end; the other masks are rebuilt by
// every step.
template <typename T, int TS, bool WIDE, bool SCALAR, int SPM>
__device__ void run_team(TeamSmem<T> &sm, const Tables<T> &tab, BlockScratch &bx, const LaunchArgs &a,
                         const InstDesc &dg, int tid, uint32_t *smask, int cap) {
    load_instance<T, TS, SPM>(sm, dg, tid);
    const int W = sm.d.Wtot, OW = sm.d.OW;
    const long long region = smem_region_words(W, OW);
    const bool local = smask != nullptr && region <= cap;
    uint32_t *masks = local ? smask : sm.d.masks;
    const long long oo = (long long)(NMASK + 1) * W + (long long)sm.cur * OW;  // occupancy of the current tree
    if constexpr (SPM != 0) {
        // the other tree buffer starts empty: a step writes its new tree there in candidate words only
        uint32_t *other = masks + (long long)(sm.cur ^ 1) * W;
        for (int g = tid; g < W; g += TS) other[g] = 0u;
    }
    if (local) {
        const uint32_t *gr = sm.d.masks + (long long)sm.cur * W;
        uint32_t *lr = smask + sm.cur * W;
        const uint32_t *gp = sm.d.masks + (long long)M_PRED * W, *gg = sm.d.masks + (long long)M_GH * W;
        for (int g = tid; g < W; g += TS) {
            lr[g] = gr[g];
            smask[M_PRED * W + g] = gp[g];
            smask[M_GH * W + g] = gg[g];
        }
        if constexpr (SPM != 0)
            for (int g = tid; g < OW; g += TS) smask[oo + g] = sm.d.masks[oo + g];
    }
    __syncthreads();
    if constexpr (SCALAR) {
        run_instance<T, 1, TS, WIDE, SPM>(sm, tab, bx, a, tid, masks);
    } else {
        // scheme variant: D1Q2^nf, or D1Q3 / D1Q5 shallow water (equilibria 4, 5)
        const int var = sm.d.eq == 4 ? 4 : sm.d.eq == 5 ? 5 : sm.d.nf;
        switch (var) {
        case 1: run_instance<T, 1, TS, WIDE, SPM>(sm, tab, bx, a, tid, masks); break;
        case 2: run_instance<T, 2, TS, WIDE, SPM>(sm, tab, bx, a, tid, masks); break;
        case 4: run_instance<T, 4, TS, WIDE, SPM>(sm, tab, bx, a, tid, masks); break;
        case 5: run_instance<T, 5, TS, WIDE, SPM>(sm, tab, bx, a, tid, masks); break;
        default: run_instance<T, 3, TS, WIDE, SPM>(sm, tab, bx, a, tid, masks); break;
        }
    }
    if (local) {
        uint32_t *gr = sm.d.masks + (long long)sm.cur * W;
        uint32_t *gp = sm.d.masks + (long long)M_PRED * W, *gg = sm.d.masks + (long long)M_GH * W;
        const uint32_t *lr = smask + sm.cur * W;
        for (int g = tid; g < W; g += TS) {
            gr[g] = lr[g];
            gp[g] = smask[M_PRED * W + g];
            gg[g] = smask[M_GH * W + g];
        }
        const long long oc = (long long)(NMASK + 1) * W + (long long)sm.cur * OW;
        if constexpr (SPM != 0)
            for (int g = tid; g < OW; g += TS) sm.d.masks[oc + g] = smask[oc + g];
    }
    store_instance<T, TS>(sm, tid);
}

// Persistent kernel: each block takes instances from the queue (largest first)
// and advances one at a time with all its threads.  KIND selects the code the
// kernel holds: K_FAST every scheme with gamma = 1 and the leaves collision;
// K_LARGE the same schemes with the word passes over candidate words, for
// instances of at least CW_MIN_WORDS words per bitmask; K_GENERAL and K_RECOLL
// wide prediction stencils (gamma = 2, 3) and the reconstructed collision, at
// any size with the word passes over every word; K_SCALAR the gamma = 1 code
// of the scalar D1Q2 scheme alone, whose smaller register footprint lets more
// blocks share an SM (a larger MINB).
template <typename T, int NT, int MINB, int KIND>
__global__ void __launch_bounds__(NT, MINB) mr_persistent(LaunchArgs a) {
    constexpr bool WIDE = KIND == K_GENERAL || KIND == K_RECOLL;
    constexpr int SPM = KIND == K_LARGE ? 1 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockSmem<T, NT> &bs = *reinterpret_cast<BlockSmem<T, NT> *>(smem_raw);
    uint32_t *smask = a.smem_mask_words > 0
                          ? reinterpret_cast<uint32_t *>(smem_raw + ((sizeof(BlockSmem<T, NT>) + 15) / 16) * 16)
                          : nullptr;
    {
        const uint32_t *src = (const uint32_t *)a.tables;
        uint32_t *dst = (uint32_t *)&bs.tab;
        for (int i = threadIdx.x; i < (int)(sizeof(Tables<T>) / 4); i += NT) dst[i] = src[i];
    }
    for (;;) {
        if (threadIdx.x == 0) bs.idx = atomicAdd(a.queue, 1);
        __syncthreads();
        const int idx = bs.idx;
        __syncthreads();
        if (idx >= a.n) return;
        run_team<T, NT, WIDE, KIND == K_SCALAR, SPM>(bs.team, bs.tab, bs.scratch, a, a.descs[a.order[idx]], threadIdx.x, smask,
                                                a.smem_mask_words);
    }
}

}  // namespace mrg

// One translation unit per (precision, block size) instantiation keeps the
// build parallel; mr_dispatch.cu routes a launch to the right one.  MINB,
// MINB_S, MINB_G and MINB_R are the resident blocks per SM the fast, scalar,
// general and reconstructed-collision kernels are compiled for: the scalar
// code fits in fewer registers, the wide-stencil code runs faster with more
// registers and fewer resident blocks.
#define MRG_INSTANTIATE(T, NT, MINB, MINB_S, MINB_G, MINB_R, TAG)                                  \
    static size_t mrg_dyn_##TAG(int mask_words) {                                                 \
        size_t base = (sizeof(mrg::BlockSmem<T, NT>) + 15) / 16 * 16;                              \
        return base + (size_t)mask_words * sizeof(uint32_t);                                       \
    }                                                                                             \
    template <int M, int K>                                                                       \
    static int mrg_allow_##TAG() {                                                                \
        return (int)cudaFuncSetAttribute(mrg::mr_persistent<T, NT, M, K>,                         \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); \
    }                                                                                             \
    /* the attribute belongs to the current device: raised once per device ordinal */             \
    static int mrg_attr_##TAG() {                                                                 \
        static std::atomic<int> done[64];                                                         \
        int dev = 0;                                                                              \
        if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;                \
        if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return 0;          \
        int rc = mrg_allow_##TAG<MINB, mrg::K_FAST>() | mrg_allow_##TAG<MINB_G, mrg::K_GENERAL>() | \
                 mrg_allow_##TAG<MINB_S, mrg::K_SCALAR>() | mrg_allow_##TAG<MINB_R, mrg::K_RECOLL>() | \
                 mrg_allow_##TAG<MINB, mrg::K_LARGE>();                                           \
        if (!rc && dev >= 0 && dev < 64) done[dev].store(1, std::memory_order_release);            \
        return rc;                                                                                \
    }                                                                                             \
    template <int M, int K>                                                                       \
    static int mrg_occ1_##TAG(size_t dyn, int *nb) {                                              \
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, mrg::mr_persistent<T, NT, M, K>, NT, dyn); \
    }                                                                                             \
    template <int M, int K>                                                                       \
    static int mrg_go_##TAG(int grid, const mrg::LaunchArgs &a, size_t dyn, cudaStream_t s, int prio) { \
        cudaLaunchConfig_t cfg = {};                                                              \
        cfg.gridDim = dim3((unsigned)grid);                                                       \
        cfg.blockDim = dim3(NT);                                                                  \
        cfg.dynamicSmemBytes = dyn;                                                               \
        cfg.stream = s;                                                                           \
        cudaLaunchAttribute at[1];                                                                \
        at[0].id = cudaLaunchAttributePriority;                                                   \
        at[0].val.priority = prio;                                                                \
        cfg.attrs = at;                                                                           \
        cfg.numAttrs = 1;                                                                         \
        return (int)cudaLaunchKernelEx(&cfg, mrg::mr_persistent<T, NT, M, K>, a);                 \
    }                                                                                             \
    int mrg_launch_##TAG(int grid, const mrg::LaunchArgs &a, cudaStream_t s, int prio) {           \
        int rc = mrg_attr_##TAG();                                                                \
        if (rc) return rc;                                                                        \
        const size_t dyn = mrg_dyn_##TAG(a.smem_mask_words);                                       \
        switch (a.kind) {                                                                         \
        case mrg::K_FAST: return mrg_go_##TAG<MINB, mrg::K_FAST>(grid, a, dyn, s, prio);           \
        case mrg::K_GENERAL: return mrg_go_##TAG<MINB_G, mrg::K_GENERAL>(grid, a, dyn, s, prio);   \
        case mrg::K_SCALAR: return mrg_go_##TAG<MINB_S, mrg::K_SCALAR>(grid, a, dyn, s, prio);     \
        case mrg::K_RECOLL: return mrg_go_##TAG<MINB_R, mrg::K_RECOLL>(grid, a, dyn, s, prio);     \
        case mrg::K_LARGE: return mrg_go_##TAG<MINB, mrg::K_LARGE>(grid, a, dyn, s, prio);         \
        }                                                                                         \
        return (int)cudaErrorInvalidValue;                                                        \
    }                                                                                             \
    int mrg_occ_##TAG(int kind, int mask_words, int *nb) {                                        \
        int rc = mrg_attr_##TAG();                                                                \
        if (rc) return rc;                                                                        \
        const size_t dyn = mrg_dyn_##TAG(mask_words);                                              \
        switch (kind) {                                                                           \
        case mrg::K_FAST: return mrg_occ1_##TAG<MINB, mrg::K_FAST>(dyn, nb);                       \
        case mrg::K_GENERAL: return mrg_occ1_##TAG<MINB_G, mrg::K_GENERAL>(dyn, nb);               \
        case mrg::K_SCALAR: return mrg_occ1_##TAG<MINB_S, mrg::K_SCALAR>(dyn, nb);                 \
        case mrg::K_RECOLL: return mrg_occ1_##TAG<MINB_R, mrg::K_RECOLL>(dyn, nb);                   \
        case mrg::K_LARGE: return mrg_occ1_##TAG<MINB, mrg::K_LARGE>(dyn, nb);                     \
        }                                                                                         \
        return (int)cudaErrorInvalidValue;                                                        \
    }                                                                                             \
    int mrg_minb_##TAG(int kind) {                                                                \
        return kind == mrg::K_SCALAR ? MINB_S : kind == mrg::K_GENERAL ? MINB_G                     \
             : kind == mrg::K_RECOLL ? MINB_R : MINB;                                             \
    }                                                                                             \
    size_t mrg_smem_##TAG(int mask_words) { return mrg_dyn_##TAG(mask_words); }

/*
 * mrlbm_oracle.c -- plain FP64 CPU oracle of the multiresolution-adaptive
 * lattice Boltzmann method of Bellotti, Gouarin, Graille and Massot
 * (arXiv 2102.12163).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA implementation.  Compile with -ffp-contract=off.
 *
 * The oracle follows the paper's definitions literally and densely: every
 * level keeps all of its cells, and the value of the solution on any cell of
 * any level is given by one function ("Definition V"):
 *   - a cell of the complete tree R(Lambda) holds its leaf value, or the
 *     projection of its two children (Def. Projection operator, Section 3.1);
 *   - any other cell holds the prediction from its parent level with zero
 *     detail (prediction formula of Section 3.1, reconstruction operator of
 *     Section 3.3).
 * This is M_R^{-1} T_Lambda M_R of Prop. ErrorControl applied to the leaf
 * data; the finest row of it is the reconstruction used by the stream.
 *
 * Readings of the paper taken here (the paper is silent or inconsistent):
 *   - gamma = 3: c3 = -5/1024 (the printed +5/1024 is not exact on linear
 *     averages, Section 3.1);
 *   - cells outside [0, 2^l) are wrapped (periodic) or clamped to the nearest
 *     in-domain cell of the same level (copy boundary), at every level and
 *     for the finest-level stream;
 *   - the trees are handled at cell level: a leaf is a cell of R(Lambda)
 *     without children in R(Lambda); siblings are always added together;
 *   - H is computed once from T(Lambda^n): rule (a) on every cell of
 *     R(T(Lambda^n)), rule (b) on every kept pair; thresholds compare with >=;
 *   - the vectorial D1Q2^n schemes number the moments of field i as
 *     (m^{2i} conserved, m^{2i+1} relaxed) and the populations as
 *     (f^{2i}: velocity +lambda, f^{2i+1}: velocity -lambda);
 *   - the D1Q3 / D1Q5 shallow water schemes (Section 5.2) number the
 *     populations as the paper's velocities (0, lambda, -lambda, 2 lambda,
 *     -2 lambda) and use its parameters alpha = beta = 1; the enlargement width
 *     sigma is the largest |v^h| / lambda of the scheme (2 for D1Q5).
 */
#include "mrlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_state {
    orc_params p;
    int nf, q;
    int w[ORC_MAXQ];           /* normalised velocities w^h = v^h / lambda */
    long S;                    /* cells over all levels */
    long off[ORC_MAXLEV + 2];  /* first cell of level l in cell arrays */
    unsigned char *R;          /* complete tree membership */
    double *V;                 /* values (population-major) */
    double *D;                 /* trace: max |detail| of the pair of a cell */
    unsigned char *T, *H;      /* trace: R(T(Lambda^n)), R(H(T(Lambda^n))) */
    double *tmp;               /* scratch values */
};

/* ------------------------------------------------------------------ */
/* small helpers                                                       */

int orc_nfields(int eq) {
    switch (eq) {
    case ORC_EQ_ADVECTION:
    case ORC_EQ_BURGERS: return 1;
    case ORC_EQ_SW: return 2;
    case ORC_EQ_EULER: return 3;
    case ORC_EQ_SW_D1Q3:
    case ORC_EQ_SW_D1Q5: return 2;
    default: return 0;
    }
}

int orc_npop(int eq) {
    switch (eq) {
    case ORC_EQ_SW_D1Q3: return 3;
    case ORC_EQ_SW_D1Q5: return 5;
    default: return 2 * orc_nfields(eq);
    }
}

/* normalised velocities w^h = v^h / lambda of the scheme; returns q */
static int velocities(int eq, int *w) {
    if (eq == ORC_EQ_SW_D1Q3 || eq == ORC_EQ_SW_D1Q5) {
        const int v[5] = {0, 1, -1, 2, -2};
        int q = orc_npop(eq);
        for (int h = 0; h < q; ++h) w[h] = v[h];
        return q;
    }
    int q = orc_npop(eq);
    for (int h = 0; h < q; ++h) w[h] = (h & 1) ? -1 : 1;
    return q;
}

static int is_dq(int eq) { return eq == ORC_EQ_SW_D1Q3 || eq == ORC_EQ_SW_D1Q5; }

static long ncells(int l) { return 1L << l; }

/* Index of cell k of a row of n cells under the boundary condition;
 * returns -1 when a copy boundary puts it outside and clip is requested. */
static long wrap_or_clamp(int bc, long k, long n) {
    if (bc == ORC_BC_PERIODIC) {
        long r = k % n;
        return r < 0 ? r + n : r;
    }
    if (k < 0) return 0;
    if (k >= n) return n - 1;
    return k;
}

static long wrap_or_clip(int bc, long k, long n) {
    if (bc == ORC_BC_PERIODIC) return wrap_or_clamp(bc, k, n);
    return (k < 0 || k >= n) ? -1 : k;
}

/* Prediction coefficients c_alpha of Section 3.1 (gamma = 3: c3 = -5/1024,
 * see the readings above). */
void orc_prediction_coefficients(int gamma, double *c) {
    if (gamma == 1) {
        c[0] = -1.0 / 8.0;
    } else if (gamma == 2) {
        c[0] = -22.0 / 128.0;
        c[1] = 3.0 / 128.0;
    } else if (gamma == 3) {
        c[0] = -201.0 / 1024.0;
        c[1] = 11.0 / 256.0;
        c[2] = -5.0 / 1024.0;
    }
}

/* Prediction of cell k of level l+1 from the row of level l (n cells):
 * f_{l+1,2p+delta} = f_{l,p} + (-1)^delta sum_alpha c_alpha (f_{l,p+alpha} - f_{l,p-alpha}). */
static double predict_child(const double *row, long n, int bc, int gamma, const double *c,
                            long k) {
    long p = k >> 1;
    double sum = 0.0;
    for (int a = 1; a <= gamma; ++a)
        sum = sum + c[a - 1] * (row[wrap_or_clamp(bc, p + a, n)] - row[wrap_or_clamp(bc, p - a, n)]);
    return (k & 1) ? row[p] - sum : row[p] + sum;
}

void orc_predict_level(int gamma, int bc, const double *coarse, long n, double *fine) {
    double c[3];
    orc_prediction_coefficients(gamma, c);
    for (long k = 0; k < 2 * n; ++k) fine[k] = predict_child(coarse, n, bc, gamma, c, k);
}

/* Projection (Def. Projection operator): mean of the two children. */
void orc_project_level(const double *fine, long n_coarse, double *coarse) {
    for (long k = 0; k < n_coarse; ++k) coarse[k] = 0.5 * (fine[2 * k] + fine[2 * k + 1]);
}

/* ------------------------------------------------------------------ */
/* trees                                                               */

#define CELL(st, l, k) ((st)->off[(l)] + (k))
#define VAL(st, arr, h, l, k) ((arr)[(long)(h) * (st)->S + (st)->off[(l)] + (k)])

static void level_offsets(int Jmin, int Jmax, long *off) {
    long o = 0;
    for (int l = Jmin; l <= Jmax; ++l) {
        off[l] = o;
        o += ncells(l);
    }
    off[Jmax + 1] = o;
}

/* add cell (l,k) together with its sibling (the complete tree always holds
 * both children of a kept pair); cells cut off by a copy boundary are skipped */
static void add_pair(unsigned char *R, const long *off, int Jmin, int bc, int l, long k) {
    long kk = wrap_or_clip(bc, k, ncells(l));
    if (kk < 0) return;
    R[off[l] + kk] = 1;
    if (l > Jmin) R[off[l] + (kk ^ 1)] = 1;
}

/* Grading operator G (Def. Graded tree): sweeping from the finest level down,
 * every cell (l,k) of the set brings (l-1, floor(k/2)+delta), |delta| <= gamma,
 * into the set.  Additions at level l-1 only create requirements at level l-2,
 * so one sweep gives the smallest graded tree holding the input. */
void orc_grade(int Jmin, int Jmax, int gamma, int bc, unsigned char *R) {
    long off[ORC_MAXLEV + 2];
    level_offsets(Jmin, Jmax, off);
    for (long k = 0; k < ncells(Jmin); ++k) R[off[Jmin] + k] = 1;
    for (int l = Jmax; l > Jmin; --l)
        for (long k = 0; k < ncells(l); ++k)
            if (R[off[l] + k])
                for (int d = -gamma; d <= gamma; ++d) add_pair(R, off, Jmin, bc, l - 1, (k >> 1) + d);
}

int orc_check_graded(int Jmin, int Jmax, int gamma, int bc, const unsigned char *R) {
    long off[ORC_MAXLEV + 2];
    level_offsets(Jmin, Jmax, off);
    for (long k = 0; k < ncells(Jmin); ++k)
        if (!R[off[Jmin] + k]) return -1; /* coarsest level must be whole */
    for (int l = Jmin + 1; l <= Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k) {
            if (!R[off[l] + k]) continue;
            if (!R[off[l] + (k ^ 1)]) return -2;      /* siblings together */
            if (!R[off[l - 1] + (k >> 1)]) return -3; /* no orphan */
            for (int d = -gamma; d <= gamma; ++d) {
                long kk = wrap_or_clip(bc, (k >> 1) + d, ncells(l - 1));
                if (kk >= 0 && !R[off[l - 1] + kk]) return -4; /* grading */
            }
        }
    return 0;
}

static int is_leaf(const orc_state *st, int l, long k) {
    if (!st->R[CELL(st, l, k)]) return 0;
    if (l == st->p.Jmax) return 1;
    return !st->R[CELL(st, l + 1, 2 * k)] && !st->R[CELL(st, l + 1, 2 * k + 1)];
}

/* Definition V: from the leaf values, projection up the tree, then prediction
 * (zero details) on every cell outside the tree, coarse to fine. */
static void fill_values(const orc_state *st, double *V) {
    const orc_params *p = &st->p;
    double c[3];
    orc_prediction_coefficients(p->gamma, c);
    for (int l = p->Jmax - 1; l >= p->Jmin; --l)
        for (long k = 0; k < ncells(l); ++k)
            if (st->R[CELL(st, l, k)] && !is_leaf(st, l, k))
                for (int h = 0; h < st->q; ++h)
                    VAL(st, V, h, l, k) = 0.5 * (VAL(st, V, h, l + 1, 2 * k) + VAL(st, V, h, l + 1, 2 * k + 1));
    for (int l = p->Jmin + 1; l <= p->Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k)
            if (!st->R[CELL(st, l, k)])
                for (int h = 0; h < st->q; ++h)
                    VAL(st, V, h, l, k) = predict_child(&VAL(st, V, h, l - 1, 0), ncells(l - 1), p->bc,
                                                        p->gamma, c, k);
}

/* ------------------------------------------------------------------ */
/* schemes: vectorial D1Q2^n, d'Humieres form (Section 2.1)            */

/* Equilibria of the relaxed moments (Sections 5.1, 5.3; shallow water:
 * D1Q2 per field with the flux of the shallow water system). */
static void equilibria(const orc_params *p, const double *mc, double *meq) {
    switch (p->eq) {
    case ORC_EQ_ADVECTION: meq[0] = p->eqp * mc[0]; break;
    case ORC_EQ_BURGERS: meq[0] = 0.5 * (mc[0] * mc[0]); break;
    case ORC_EQ_SW:
        meq[0] = mc[1];
        meq[1] = (mc[1] * mc[1]) / mc[0] + (0.5 * p->eqp) * (mc[0] * mc[0]);
        break;
    case ORC_EQ_EULER: {
        double gg = p->eqp;
        double u2 = mc[1] * mc[1];
        meq[0] = mc[1];
        meq[1] = (1.5 - 0.5 * gg) * (u2 / mc[0]) + (gg - 1.0) * mc[2];
        meq[2] = gg * ((mc[2] * mc[1]) / mc[0]) + (0.5 * (1.0 - gg)) * ((u2 * mc[1]) / (mc[0] * mc[0]));
        break;
    }
    default: break;
    }
}

/* D1Q3 / D1Q5 (Section 5.2): moment matrix M[i][h] = (v^h)^i, i = 0 .. q-1,
 * and its inverse by Gauss-Jordan elimination with partial pivoting. */
static void dq_matrices(const orc_params *p, int q, double M[5][5], double Mi[5][5]) {
    int w[ORC_MAXQ];
    velocities(p->eq, w);
    double A[5][10];
    for (int i = 0; i < q; ++i)
        for (int h = 0; h < q; ++h) {
            double v = w[h] * p->lambda, x = 1.0;
            for (int e = 0; e < i; ++e) x = x * v;
            M[i][h] = x;
            A[i][h] = x;
            A[i][q + h] = i == h ? 1.0 : 0.0;
        }
    for (int c = 0; c < q; ++c) {
        int piv = c;
        for (int r = c + 1; r < q; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int j = 0; j < 2 * q; ++j) {
            double t = A[c][j];
            A[c][j] = A[piv][j];
            A[piv][j] = t;
        }
        double d = A[c][c];
        for (int j = 0; j < 2 * q; ++j) A[c][j] = A[c][j] / d;
        for (int r = 0; r < q; ++r)
            if (r != c) {
                double fct = A[r][c];
                for (int j = 0; j < 2 * q; ++j) A[r][j] = A[r][j] - fct * A[c][j];
            }
    }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) Mi[i][j] = A[i][q + j];
}

/* equilibria of the relaxed moments m^2 (, m^3, m^4): h u^2 + g h^2 / 2 with
 * h = m^0, h u = m^1 (, alpha lambda^2 m^1, beta lambda^2 m^{2,eq}) */
static void dq_equilibria(const orc_params *p, int q, const double *m, double *meq) {
    meq[2] = (m[1] * m[1]) / m[0] + (0.5 * p->eqp) * (m[0] * m[0]);
    if (q == 5) {
        double l2 = p->lambda * p->lambda;
        meq[3] = 1.0 * l2 * m[1];
        meq[4] = 1.0 * l2 * meq[2];
    }
}

/* collision of one cell: m = M f, m^i* = (1 - s^i) m^i + s^i m^{i,eq} for
 * i >= 2, f* = M^{-1} m* */
static void dq_collide(const orc_params *p, double *f, long stride) {
    int q = orc_npop(p->eq);
    double M[5][5], Mi[5][5], m[5], meq[5];
    dq_matrices(p, q, M, Mi);
    for (int i = 0; i < q; ++i) {
        double acc = 0.0;
        for (int h = 0; h < q; ++h) acc = acc + M[i][h] * f[h * stride];
        m[i] = acc;
    }
    dq_equilibria(p, q, m, meq);
    for (int i = 2; i < q; ++i) m[i] = (1.0 - p->s[i - 2]) * m[i] + p->s[i - 2] * meq[i];
    for (int h = 0; h < q; ++h) {
        double acc = 0.0;
        for (int i = 0; i < q; ++i) acc = acc + Mi[h][i] * m[i];
        f[h * stride] = acc;
    }
}

/* Collision (Section 2.1.1; eq. LeavesCollision on a leaf): m = M f with
 * M = [[1, 1], [lambda, -lambda]] per field, relax the non-conserved moment,
 * f* = M^{-1} m*.  f holds the q populations of one cell with stride `stride`. */
static void collide_cell(const orc_params *p, double *f, long stride) {
    if (is_dq(p->eq)) {
        dq_collide(p, f, stride);
        return;
    }
    int nf = orc_nfields(p->eq);
    double mc[ORC_MAXFIELDS], mn[ORC_MAXFIELDS], meq[ORC_MAXFIELDS];
    for (int i = 0; i < nf; ++i) {
        double fp = f[(2 * i) * stride], fm = f[(2 * i + 1) * stride];
        mc[i] = fp + fm;
        mn[i] = p->lambda * (fp - fm);
    }
    equilibria(p, mc, meq);
    for (int i = 0; i < nf; ++i) {
        double s = p->s[i];
        double mstar = (1.0 - s) * mn[i] + s * meq[i];
        double g = mstar / p->lambda;
        f[(2 * i) * stride] = 0.5 * (mc[i] + g);
        f[(2 * i + 1) * stride] = 0.5 * (mc[i] - g);
    }
}

void orc_equilibrium_populations(const orc_params *p, const double *m_cons, double *f, long n) {
    if (is_dq(p->eq)) {
        int q = orc_npop(p->eq);
        double M[5][5], Mi[5][5], m[5];
        dq_matrices(p, q, M, Mi);
        for (long k = 0; k < n; ++k) {
            m[0] = m_cons[k];
            m[1] = m_cons[n + k];
            dq_equilibria(p, q, m, m);
            for (int h = 0; h < q; ++h) {
                double acc = 0.0;
                for (int i = 0; i < q; ++i) acc = acc + Mi[h][i] * m[i];
                f[h * n + k] = acc;
            }
        }
        return;
    }
    int nf = orc_nfields(p->eq);
    for (long k = 0; k < n; ++k) {
        double mc[ORC_MAXFIELDS], meq[ORC_MAXFIELDS];
        for (int i = 0; i < nf; ++i) mc[i] = m_cons[i * n + k];
        equilibria(p, mc, meq);
        for (int i = 0; i < nf; ++i) {
            double g = meq[i] / p->lambda;
            f[(2 * i) * n + k] = 0.5 * (mc[i] + g);
            f[(2 * i + 1) * n + k] = 0.5 * (mc[i] - g);
        }
    }
}

void orc_moments(const orc_params *p, const double *f, double *m_cons, long n) {
    if (is_dq(p->eq)) {
        int w[ORC_MAXQ], q = velocities(p->eq, w);
        for (long k = 0; k < n; ++k) {
            double m0 = 0.0, m1 = 0.0;
            for (int h = 0; h < q; ++h) {
                m0 = m0 + f[h * n + k];
                m1 = m1 + (w[h] * p->lambda) * f[h * n + k];
            }
            m_cons[k] = m0;
            m_cons[n + k] = m1;
        }
        return;
    }
    int nf = orc_nfields(p->eq);
    for (long k = 0; k < n; ++k)
        for (int i = 0; i < nf; ++i) m_cons[i * n + k] = f[(2 * i) * n + k] + f[(2 * i + 1) * n + k];
}

/* Reference scheme L on the uniform finest lattice: collision on every cell,
 * then f^{n+1}_k = f*_{k - w^h} (Section 2.1.2). */
void orc_uniform_step(const orc_params *p, double *f) {
    long n = ncells(p->Jmax);
    int wv[ORC_MAXQ], q = velocities(p->eq, wv);
    for (long k = 0; k < n; ++k) collide_cell(p, f + k, n);
    double *row = (double *)malloc(sizeof(double) * n);
    for (int h = 0; h < q; ++h) {
        int w = wv[h];
        memcpy(row, f + (long)h * n, sizeof(double) * n);
        for (long k = 0; k < n; ++k) f[(long)h * n + k] = row[wrap_or_clamp(p->bc, k - w, n)];
    }
    free(row);
}

/* ------------------------------------------------------------------ */
/* state                                                               */

orc_state *orc_create(const orc_params *p) {
    if (p->Jmin < 1 || p->Jmax < p->Jmin || p->Jmax > ORC_MAXLEV) return NULL;
    if (p->gamma < 1 || p->gamma > 3 || orc_nfields(p->eq) == 0) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    st->p = *p;
    st->nf = orc_nfields(p->eq);
    st->q = velocities(p->eq, st->w);
    level_offsets(p->Jmin, p->Jmax, st->off);
    st->S = st->off[p->Jmax + 1];
    st->R = (unsigned char *)calloc(st->S, 1);
    st->T = (unsigned char *)calloc(st->S, 1);
    st->H = (unsigned char *)calloc(st->S, 1);
    st->D = (double *)calloc(st->S, sizeof(double));
    st->V = (double *)calloc((size_t)st->S * st->q, sizeof(double));
    st->tmp = (double *)calloc((size_t)st->S * st->q, sizeof(double));
    return st;
}

void orc_free(orc_state *st) {
    if (!st) return;
    free(st->R);
    free(st->T);
    free(st->H);
    free(st->D);
    free(st->V);
    free(st->tmp);
    free(st);
}

long orc_total_cells(const orc_state *st) { return st->S; }

/* Lambda^0 is the full tree (Section 4.4), leaves on the finest level at
 * equilibrium of the given conserved moments. */
void orc_set_initial(orc_state *st, const double *m_cons) {
    long n = ncells(st->p.Jmax);
    memset(st->R, 1, st->S);
    memset(st->V, 0, sizeof(double) * st->S * st->q);
    double *f = (double *)malloc(sizeof(double) * n * st->q);
    orc_equilibrium_populations(&st->p, m_cons, f, n);
    for (int h = 0; h < st->q; ++h)
        for (long k = 0; k < n; ++k) VAL(st, st->V, h, st->p.Jmax, k) = f[h * n + k];
    free(f);
}

int orc_set_state(orc_state *st, const unsigned char *R, const double *values) {
    int rc = orc_check_graded(st->p.Jmin, st->p.Jmax, st->p.gamma, st->p.bc, R);
    if (rc) return rc;
    memcpy(st->R, R, st->S);
    memcpy(st->V, values, sizeof(double) * st->S * st->q);
    return 0;
}

void orc_get_state(const orc_state *st, unsigned char *R, double *values) {
    if (R) memcpy(R, st->R, st->S);
    if (values) {
        memcpy(values, st->V, sizeof(double) * st->S * st->q);
        fill_values(st, values);
    }
}

long orc_leaves(const orc_state *st, int *level, long *index, double *f, long cap) {
    long c = 0;
    for (int l = st->p.Jmin; l <= st->p.Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k)
            if (is_leaf(st, l, k)) {
                if (c < cap) {
                    if (level) level[c] = l;
                    if (index) index[c] = k;
                    if (f)
                        for (int h = 0; h < st->q; ++h) f[h * cap + c] = VAL(st, st->V, h, l, k);
                }
                ++c;
            }
    return c;
}

void orc_get_trace(const orc_state *st, double *D, unsigned char *T, unsigned char *H,
                   unsigned char *G) {
    if (D) memcpy(D, st->D, sizeof(double) * st->S);
    if (T) memcpy(T, st->T, st->S);
    if (H) memcpy(H, st->H, st->S);
    if (G) memcpy(G, st->R, st->S);
}

/* ------------------------------------------------------------------ */
/* mesh adaptation (Section 4.1, enlargement Section 4.2)              */

void orc_adapt(orc_state *st) {
    const orc_params *p = &st->p;
    double c[3];
    orc_prediction_coefficients(p->gamma, c);
    int sigma = 1; /* enlargement width: max |w^h| of the scheme */
    for (int h = 0; h < st->q; ++h) sigma = abs(st->w[h]) > sigma ? abs(st->w[h]) : sigma;

    /* multiresolution analysis of the current solution */
    fill_values(st, st->V);

    /* details d_{l,k} = f_{l,k} - prediction, on the pairs (even k) of the
     * tree above the coarsest level; max over the populations */
    memset(st->D, 0, sizeof(double) * st->S);
    for (int l = p->Jmin + 1; l <= p->Jmax; ++l)
        for (long k = 0; k < ncells(l); k += 2) {
            if (!st->R[CELL(st, l, k)]) continue;
            double dmax = 0.0;
            for (int h = 0; h < st->q; ++h) {
                double pred = predict_child(&VAL(st, st->V, h, l - 1, 0), ncells(l - 1), p->bc, p->gamma, c, k);
                double d = VAL(st, st->V, h, l, k) - pred;
                if (fabs(d) > dmax) dmax = fabs(d);
            }
            st->D[CELL(st, l, k)] = dmax;
            st->D[CELL(st, l, k + 1)] = dmax;
        }

    /* T: coarsest level, plus the pairs with max |d| >= eps_l = 2^{l-Jmax} eps */
    memset(st->T, 0, st->S);
    for (long k = 0; k < ncells(p->Jmin); ++k) st->T[CELL(st, p->Jmin, k)] = 1;
    for (int l = p->Jmin + 1; l <= p->Jmax; ++l) {
        double eps_l = ldexp(p->eps, l - p->Jmax);
        for (long k = 0; k < ncells(l); k += 2)
            if (st->R[CELL(st, l, k)] && st->D[CELL(st, l, k)] >= eps_l) {
                st->T[CELL(st, l, k)] = 1;
                st->T[CELL(st, l, k + 1)] = 1;
            }
    }

    /* H: (a) same-level neighbours within sigma of every cell of R(T);
     *    (b) the four children of a kept pair whose detail reaches
     *        2^{mu_bar+1} eps_l (eq. HartenLossOfRegularity) */
    memcpy(st->H, st->T, st->S);
    for (int l = p->Jmin; l <= p->Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k)
            if (st->T[CELL(st, l, k)])
                for (int d = -sigma; d <= sigma; ++d) add_pair(st->H, st->off, p->Jmin, p->bc, l, k + d);
    for (int l = p->Jmin + 1; l < p->Jmax; ++l) {
        double eps_l = ldexp(p->eps, l - p->Jmax);
        double big = ldexp(eps_l, p->mu_bar + 1);
        for (long k = 0; k < ncells(l); k += 2)
            if (st->T[CELL(st, l, k)] && st->D[CELL(st, l, k)] >= big)
                for (int d = 0; d < 4; ++d) st->H[CELL(st, l + 1, 2 * k + d)] = 1;
    }

    /* G: smallest graded tree holding H(T(Lambda^n)) */
    memcpy(st->R, st->H, st->S);
    orc_grade(p->Jmin, p->Jmax, p->gamma, p->bc, st->R);

    /* data transfer: every cell already holds the value of Definition V of the
     * old tree (projection where the mesh is coarsened, prediction where it
     * is refined), so the new leaves read it in place. */
}

/* ------------------------------------------------------------------ */
/* adaptive scheme L_A (Sections 4.3 and 4.5)                          */

/* eq. reconstructedCollision on one leaf: the conserved moments stay, each
 * relaxed moment becomes (1 - s) m + s times the mean over the leaf's 2^{Jmax-l}
 * finest cells of its equilibrium evaluated on the reconstructed conserved
 * moments there (fin: the reconstruction of every population on the finest
 * level, row length nJ). */
static void collide_reconstructed(const orc_params *p, double *f, long stride, const double *fin, long nJ,
                                  long first, long ncell) {
    int nf = orc_nfields(p->eq), q = orc_npop(p->eq);
    double acc[ORC_MAXQ] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long i = first; i < first + ncell; ++i) {
        double g[ORC_MAXQ], mc[ORC_MAXFIELDS], meq[ORC_MAXQ];
        for (int h = 0; h < q; ++h) g[h] = fin[h * nJ + i];
        orc_moments(p, g, mc, 1);
        if (is_dq(p->eq)) {
            double m[5] = {mc[0], mc[1], 0.0, 0.0, 0.0};
            dq_equilibria(p, q, m, meq);
            for (int r = 2; r < q; ++r) acc[r] = acc[r] + meq[r];
        } else {
            equilibria(p, mc, meq);
            for (int r = 0; r < nf; ++r) acc[r] = acc[r] + meq[r];
        }
    }
    double inv = 1.0 / (double)ncell;
    if (is_dq(p->eq)) {
        double M[5][5], Mi[5][5], m[5];
        dq_matrices(p, q, M, Mi);
        for (int i = 0; i < q; ++i) {
            double a = 0.0;
            for (int h = 0; h < q; ++h) a = a + M[i][h] * f[h * stride];
            m[i] = a;
        }
        for (int i = 2; i < q; ++i) m[i] = (1.0 - p->s[i - 2]) * m[i] + p->s[i - 2] * (acc[i] * inv);
        for (int h = 0; h < q; ++h) {
            double a = 0.0;
            for (int i = 0; i < q; ++i) a = a + Mi[h][i] * m[i];
            f[h * stride] = a;
        }
        return;
    }
    for (int i = 0; i < nf; ++i) {
        double fp = f[(2 * i) * stride], fm = f[(2 * i + 1) * stride];
        double mc = fp + fm, mn = p->lambda * (fp - fm);
        double mstar = (1.0 - p->s[i]) * mn + p->s[i] * (acc[i] * inv);
        double g = mstar / p->lambda;
        f[(2 * i) * stride] = 0.5 * (mc + g);
        f[(2 * i + 1) * stride] = 0.5 * (mc - g);
    }
}

static void collide_leaves(orc_state *st) {
    if (st->p.collision == ORC_COLLIDE_RECONSTRUCTED) {
        /* reconstruction of the pre-collision populations on every finest cell */
        long nJ = ncells(st->p.Jmax);
        memcpy(st->tmp, st->V, sizeof(double) * st->S * st->q);
        fill_values(st, st->tmp);
        double *fin = (double *)malloc(sizeof(double) * nJ * st->q);
        for (int h = 0; h < st->q; ++h)
            for (long i = 0; i < nJ; ++i) fin[h * nJ + i] = VAL(st, st->tmp, h, st->p.Jmax, i);
        for (int l = st->p.Jmin; l <= st->p.Jmax; ++l) {
            int dj = st->p.Jmax - l;
            for (long k = 0; k < ncells(l); ++k)
                if (is_leaf(st, l, k))
                    collide_reconstructed(&st->p, &VAL(st, st->V, 0, l, k), st->S, fin, nJ, k << dj, 1L << dj);
        }
        free(fin);
        return;
    }
    for (int l = st->p.Jmin; l <= st->p.Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k)
            if (is_leaf(st, l, k)) collide_cell(&st->p, &VAL(st, st->V, 0, l, k), st->S);
}

void orc_collide(orc_state *st) { collide_leaves(st); }

void orc_lbm_step(orc_state *st) {
    const orc_params *p = &st->p;
    long nJ = ncells(p->Jmax);
    collide_leaves(st);
    fill_values(st, st->V); /* reconstruction of f* on every cell */
    /* compact stream, eq. AdaptiveStreamPhase */
    for (int l = p->Jmin; l <= p->Jmax; ++l) {
        int dj = p->Jmax - l;
        for (long k = 0; k < ncells(l); ++k) {
            if (!is_leaf(st, l, k)) continue;
            long first = k << dj, next = (k + 1) << dj;
            for (int h = 0; h < st->q; ++h) {
                int w = st->w[h];
                const double *fin = &VAL(st, st->V, h, p->Jmax, 0);
                double fstar = VAL(st, st->V, h, l, k);
                if (w == 0) {
                    VAL(st, st->tmp, h, l, k) = fstar;
                    continue;
                }
                int sg = w > 0 ? 1 : -1, aw = w > 0 ? w : -w;
                double acc = 0.0;
                for (int d = 1; d <= aw; ++d) {
                    long eta = sg > 0 ? -d : d - 1;
                    acc = acc + (fin[wrap_or_clamp(p->bc, first + eta, nJ)] - fin[wrap_or_clamp(p->bc, next + eta, nJ)]);
                }
                VAL(st, st->tmp, h, l, k) = fstar + ldexp((double)sg, -dj) * acc;
            }
        }
    }
    for (int l = p->Jmin; l <= p->Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k)
            if (is_leaf(st, l, k))
                for (int h = 0; h < st->q; ++h) VAL(st, st->V, h, l, k) = VAL(st, st->tmp, h, l, k);
}

void orc_lbm_step_uncompacted(orc_state *st, double *out) {
    const orc_params *p = &st->p;
    long nJ = ncells(p->Jmax);
    double *save = (double *)malloc(sizeof(double) * st->S * st->q);
    memcpy(save, st->V, sizeof(double) * st->S * st->q);
    collide_leaves(st);
    fill_values(st, st->V);
    memcpy(out, st->V, sizeof(double) * st->S * st->q);
    for (int l = p->Jmin; l <= p->Jmax; ++l) {
        int dj = p->Jmax - l;
        for (long k = 0; k < ncells(l); ++k) {
            if (!is_leaf(st, l, k)) continue;
            for (int h = 0; h < st->q; ++h) {
                const double *fin = &VAL(st, st->V, h, p->Jmax, 0);
                double acc = 0.0;
                for (long d = 0; d < (1L << dj); ++d)
                    acc = acc + fin[wrap_or_clamp(p->bc, (k << dj) + d - st->w[h], nJ)];
                VAL(st, out, h, l, k) = ldexp(acc, -dj);
            }
        }
    }
    memcpy(st->V, save, sizeof(double) * st->S * st->q);
    free(save);
}

void orc_step(orc_state *st) {
    orc_adapt(st);
    orc_lbm_step(st);
}

/* ------------------------------------------------------------------ */
/* measurements                                                        */

void orc_reconstruct_finest(orc_state *st, double *f_finest) {
    long n = ncells(st->p.Jmax);
    memcpy(st->tmp, st->V, sizeof(double) * st->S * st->q);
    fill_values(st, st->tmp);
    for (int h = 0; h < st->q; ++h)
        for (long k = 0; k < n; ++k) f_finest[h * n + k] = VAL(st, st->tmp, h, st->p.Jmax, k);
}

void orc_reconstruct_moments(orc_state *st, double *m_finest) {
    long n = ncells(st->p.Jmax);
    double *f = (double *)malloc(sizeof(double) * n * st->q);
    orc_reconstruct_finest(st, f);
    orc_moments(&st->p, f, m_finest, n);
    free(f);
}

void orc_mass(const orc_state *st, double *mass) {
    for (int i = 0; i < st->nf; ++i) mass[i] = 0.0;
    for (int l = st->p.Jmin; l <= st->p.Jmax; ++l) {
        double dx = ldexp(st->p.b - st->p.a, -l);
        for (long k = 0; k < ncells(l); ++k)
            if (is_leaf(st, l, k)) {
                double f[ORC_MAXQ], m[ORC_MAXFIELDS];
                for (int h = 0; h < st->q; ++h) f[h] = VAL(st, st->V, h, l, k);
                orc_moments(&st->p, f, m, 1);
                for (int i = 0; i < st->nf; ++i) mass[i] += dx * m[i];
            }
    }
}

/* ------------------------------------------------------------------ */
/* multiresolution transform of one population (eq. actionMultiresolutionTransform) */

void orc_mr_encode(int Jmin, int Jmax, int gamma, int bc, const double *finest, double *packed) {
    long off[ORC_MAXLEV + 2];
    level_offsets(Jmin, Jmax, off);
    double c[3];
    orc_prediction_coefficients(gamma, c);
    double *avg = (double *)malloc(sizeof(double) * off[Jmax + 1]);
    memcpy(avg + off[Jmax], finest, sizeof(double) * ncells(Jmax));
    for (int l = Jmax - 1; l >= Jmin; --l) orc_project_level(avg + off[l + 1], ncells(l), avg + off[l]);
    memcpy(packed + off[Jmin], avg + off[Jmin], sizeof(double) * ncells(Jmin));
    for (int l = Jmin + 1; l <= Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k)
            packed[off[l] + k] = (k & 1) ? 0.0
                                         : avg[off[l] + k] - predict_child(avg + off[l - 1], ncells(l - 1), bc, gamma, c, k);
    free(avg);
}

void orc_mr_decode(int Jmin, int Jmax, int gamma, int bc, const double *packed, double *finest) {
    long off[ORC_MAXLEV + 2];
    level_offsets(Jmin, Jmax, off);
    double c[3];
    orc_prediction_coefficients(gamma, c);
    double *avg = (double *)malloc(sizeof(double) * off[Jmax + 1]);
    memcpy(avg + off[Jmin], packed + off[Jmin], sizeof(double) * ncells(Jmin));
    for (int l = Jmin + 1; l <= Jmax; ++l)
        for (long k = 0; k < ncells(l); ++k) {
            double d = packed[off[l] + (k & ~1L)]; /* redundancy: d_{2p+1} = -d_{2p} */
            double pred = predict_child(avg + off[l - 1], ncells(l - 1), bc, gamma, c, k);
            avg[off[l] + k] = (k & 1) ? pred - d : pred + d;
        }
    memcpy(finest, avg + off[Jmax], sizeof(double) * ncells(Jmax));
    free(avg);
}

/*
 * mrlbm_oracle.h -- plain, slow, single-threaded FP64 CPU oracle of the
 * multiresolution-adaptive lattice Boltzmann step (Bellotti, Gouarin,
 * Graille, Massot, arXiv 2102.12163).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path of the package.
 *
 * Everything is stored densely: for every level l in [Jmin, Jmax] the
 * arrays hold all 2^l cells, whether or not the cell belongs to the tree.
 * Concatenated per-level layouts used at the interface:
 *   cell array      : level l occupies [2^l - 2^Jmin, 2^(l+1) - 2^Jmin)
 *   value array     : population-major, value[h * S + cell], S = 2^(Jmax+1) - 2^Jmin
 */
#ifndef MRLBM_ORACLE_H
#define MRLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXLEV 26
#define ORC_MAXFIELDS 3
#define ORC_MAXQ (2 * ORC_MAXFIELDS)

/* boundary conditions */
#define ORC_BC_PERIODIC 0
#define ORC_BC_COPY 1

/* equilibria of the vectorial D1Q2^n schemes (Sections 5.1 and 5.3) */
#define ORC_EQ_ADVECTION 0 /* n = 1, m1eq = c m0                 */
#define ORC_EQ_BURGERS 1   /* n = 1, m1eq = m0^2 / 2             */
#define ORC_EQ_SW 2        /* n = 2, shallow water, gravity g    */
#define ORC_EQ_EULER 3     /* n = 3, Euler, gas constant gamma_g */
/* shallow water with one velocity set for both conserved moments (Section 5.2):
 * populations numbered as the paper's velocities, moments m^i = sum_h (v^h)^i f^h */
#define ORC_EQ_SW_D1Q3 4   /* v = 0, +lambda, -lambda; s[0] = s^2 */
#define ORC_EQ_SW_D1Q5 5   /* v = 0, +-lambda, +-2 lambda; s = (s^2, s^3, s^4), alpha = beta = 1 */

typedef struct {
    int Jmin, Jmax; /* levels, Jmin >= 1 */
    int gamma;      /* prediction stencil half width (1, 2 or 3) */
    int mu_bar;     /* regularity guess of the Harten enlargement */
    int bc;         /* ORC_BC_* */
    double eps;     /* threshold epsilon */
    double a, b;    /* domain [a, b] */
    int eq;         /* ORC_EQ_* */
    double lambda;  /* lattice velocity */
    double s[ORC_MAXFIELDS];   /* relaxation rate of the non-conserved moment of each field
                                  (D1Q3 / D1Q5: of the moments m^2, m^3, m^4) */
    double eqp;     /* advection velocity c | unused | gravity g | gas constant gamma_g */
    int collision;  /* ORC_COLLIDE_LEAVES or ORC_COLLIDE_RECONSTRUCTED */
} orc_params;

/* collision of the adaptive scheme (Section 4.5): on the leaf averages
 * (eq. LeavesCollision) or with the equilibria averaged over the leaf's
 * reconstructed finest cells (eq. reconstructedCollision) */
#define ORC_COLLIDE_LEAVES 0
#define ORC_COLLIDE_RECONSTRUCTED 1

typedef struct orc_state orc_state;

/* number of D1Q2 fields (conserved moments) and populations of a scheme */
int orc_nfields(int eq);
/* number of populations q of the scheme */
int orc_npop(int eq);

orc_state *orc_create(const orc_params *p);
void orc_free(orc_state *st);
long orc_total_cells(const orc_state *st); /* S = 2^(Jmax+1) - 2^Jmin */

/* Initial state: full tree, leaves at Jmax, populations at equilibrium of the
 * given conserved moments m_cons[i * 2^Jmax + k] (field i, finest cell k). */
void orc_set_initial(orc_state *st, const double *m_cons);

/* Arbitrary state: R is the complete-tree membership (cell array layout),
 * values holds at least the leaf values (value layout).  Returns 0 when the
 * tree is a valid graded tree, a negative code otherwise (state unchanged). */
int orc_set_state(orc_state *st, const unsigned char *R, const double *values);

/* Copies out the complete tree and the leaf values (non-leaf entries are the
 * values of the multiresolution reconstruction, see orc_fill_values). */
void orc_get_state(const orc_state *st, unsigned char *R, double *values);

/* Mesh adaptation (Section 4.1): Lambda^{n+1} = G(H(T(Lambda^n))) and data
 * transfer onto the new leaves. */
void orc_adapt(orc_state *st);
/* One application of the adaptive scheme on the current mesh: leaves
 * collision (eq. LeavesCollision) and compact stream (eq. AdaptiveStreamPhase). */
/* the collision phase alone (S1 of the adaptive scheme), for tests */
void orc_collide(orc_state *st);
void orc_lbm_step(orc_state *st);
/* orc_adapt followed by orc_lbm_step. */
void orc_step(orc_state *st);

/* Stream in the uncompacted form (eq. StreamUncompacted) applied to the
 * current post-collision leaf values; writes the would-be new leaf values into
 * out (value layout) without changing the state.  Cross-check only. */
void orc_lbm_step_uncompacted(orc_state *st, double *out);

/* Trace of the last orc_adapt: per cell (cell array layout)
 *   D     max over populations of |detail| of the pair holding the cell (0 if none)
 *   T     membership of R(T(Lambda^n)),  H  of R(H(T(Lambda^n))),  G  of the new tree */
void orc_get_trace(const orc_state *st, double *D, unsigned char *T, unsigned char *H,
                   unsigned char *G);

/* Leaves of the current tree, ordered by level then index.  Returns the count;
 * level/index/f may be NULL.  f is population-major with stride cap. */
long orc_leaves(const orc_state *st, int *level, long *index, double *f, long cap);

/* Multiresolution reconstruction on the finest level of the current leaf
 * values (populations, value[h * 2^Jmax + k]) and of the conserved moments. */
void orc_reconstruct_finest(orc_state *st, double *f_finest);
void orc_reconstruct_moments(orc_state *st, double *m_finest);

/* Conserved quantities sum_leaves dx_l m_cons (one per field). */
void orc_mass(const orc_state *st, double *mass);

/* Reference scheme on the uniform finest lattice (Section 2): f has q rows of
 * 2^Jmax cells, updated in place by one collision and one stream. */
void orc_uniform_step(const orc_params *p, double *f);
void orc_equilibrium_populations(const orc_params *p, const double *m_cons, double *f,
                                 long n); /* n cells, m_cons[i*n+k], f[h*n+k] */
void orc_moments(const orc_params *p, const double *f, double *m_cons, long n);

/* Operators exposed for unit tests. */
void orc_prediction_coefficients(int gamma, double *c); /* c[0..gamma-1] */
/* children (2k, 2k+1) of every cell of a coarse row of n cells */
void orc_predict_level(int gamma, int bc, const double *coarse, long n, double *fine);
void orc_project_level(const double *fine, long n_coarse, double *coarse);
/* multiresolution transform of one population: finest (2^Jmax values) to
 * (coarsest values, details of the even cells of every finer level) and back;
 * packed as the cell array layout (level Jmin: averages, finer levels: detail
 * stored at even k, odd entries zero). */
void orc_mr_encode(int Jmin, int Jmax, int gamma, int bc, const double *finest, double *packed);
void orc_mr_decode(int Jmin, int Jmax, int gamma, int bc, const double *packed, double *finest);
/* grading operator G applied in place to a complete-tree membership */
void orc_grade(int Jmin, int Jmax, int gamma, int bc, unsigned char *R);
/* 0 when R is a sibling-closed graded tree */
int orc_check_graded(int Jmin, int Jmax, int gamma, int bc, const unsigned char *R);

#ifdef __cplusplus
}
#endif
#endif

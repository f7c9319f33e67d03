/*
 * mrlbm.h -- C ABI of the GB300 implementation of the multiresolution-adaptive
 * lattice Boltzmann step of Bellotti, Gouarin, Graille and Massot
 * (arXiv 2102.12163).
 *
 * One context holds one or many independent 1D problems ("instances").  Each
 * instance lives on a dyadic cell tree with levels Jmin..Jmax (Section 3.1):
 * level l has 2^l cells of size (b - a) 2^-l.  One adaptive time step is
 *   mr_adapt : multiresolution analysis (projection, prediction, details,
 *              Sections 3.1-3.2), mesh update Lambda^{n+1} = G(H(T(Lambda^n)))
 *              (Section 4.1, enlargement Section 4.2) and data transfer;
 *   lbm_step : leaves collision (eq. LeavesCollision, Section 4.5) and stream
 *              with fluxes reconstructed on virtual finest cells
 *              (eq. AdaptiveStreamPhase, Section 4.3).
 *
 * Conventions
 *   - Every call returns an mr_status; nothing else crosses the ABI.
 *   - Device memory is owned by the caller: the library never allocates it.
 *     mr_workspace_size() gives the bytes one context needs and mr_bind()
 *     attaches a caller-allocated device buffer of at least that size (256-byte
 *     aligned) and the CUDA stream every later call is ordered on.  The buffer
 *     must outlive the context's use; mr_destroy() does not free it.
 *   - Calls that launch work are asynchronous on the bound stream.  Errors found
 *     on the device (non-finite values) are reported by the next call that
 *     synchronises: mr_sync(), the getters, mr_stats().  A batch whose
 *     instances need more than one kernel variant (see mr_set_order) forks
 *     part of a launch onto a stream the context owns and joins it back to
 *     the bound stream before the call returns, by events; the pattern is
 *     legal inside a stream capture, so a captured launch stays one graph.
 *   - Pointers marked "host or device" may be either (unified addressing);
 *     pointers marked "host" must be host memory.
 *   - The library is not thread-safe per context.
 *
 * Scope of this build: D = 1; vectorial D1Q2^n schemes, n = 1, 2, 3 (velocities
 * +-lambda per field, Sections 5.1 and 5.3), and the D1Q3 / D1Q5 shallow water
 * schemes (Section 5.2); prediction stencils gamma = 1, 2, 3 (Section 3.1: c1 =
 * -1/8; c1 = -22/128, c2 = 3/128; c1 = -201/1024, c2 = 11/256, c3 = -5/1024);
 * enlargement width sigma = max |w^h| (Section 4.2): 1 for D1Q2^n and D1Q3, 2
 * for D1Q5; leaves collision or reconstructed collision (Section 4.5).
 * Lattice velocities lambda in [2^-16, 2^16].
 */
#ifndef MRLBM_H
#define MRLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mr_ctx mr_ctx;

typedef enum {
    MR_OK = 0,
    MR_ERR_ARG = -1,       /* invalid argument (message via mr_last_error)      */
    MR_ERR_CUDA = -2,      /* a CUDA runtime call failed                        */
    MR_ERR_CAPACITY = -3,  /* a caller buffer or the workspace is too small     */
    MR_ERR_NONFINITE = -4, /* a population became NaN or infinite on the device */
    MR_ERR_TIMEOUT = -5,   /* reserved: a bounded device wait gave up           */
    MR_ERR_STATE = -6      /* call out of order (e.g. step before mr_bind)      */
} mr_status;

typedef enum { MR_FP64 = 0, MR_FP32_MIXED = 1 } mr_precision;
typedef enum { MR_BC_PERIODIC = 0, MR_BC_COPY = 1 } mr_bc;
/* Equilibria of the vectorial D1Q2^n schemes (Section 5):
 *   ADVECTION   n = 1, m1eq = c m0                         eq_param = c
 *   BURGERS     n = 1, m1eq = m0^2 / 2                     eq_param unused
 *   SW_VEC      n = 2, shallow water (h, hu), gravity g    eq_param = g
 *   EULER_VEC   n = 3, Euler (rho, rho u, E), Section 5.3  eq_param = gamma_gas
 * and of the shallow water schemes on one velocity set (Section 5.2), two
 * conserved moments (h, hu), populations in the order of the velocities:
 *   SW_D1Q3     q = 3, v = (0, lambda, -lambda), relaxed m^2 with s[0];
 *               m^{2,eq} = (hu)^2 / h + g h^2 / 2          eq_param = g
 *   SW_D1Q5     q = 5, v = (0, +-lambda, +-2 lambda), relaxed m^2, m^3, m^4
 *               with s[0..2]; m^{3,eq} = lambda^2 hu, m^{4,eq} = lambda^2
 *               m^{2,eq} (alpha = beta = 1), enlargement width sigma = 2;
 *               eq_param = g
 * (moments m^i = sum_h (v^h)^i f^h).  D1Q3 / D1Q5 need gamma = 1. */
typedef enum {
    MR_EQ_ADVECTION = 0, MR_EQ_BURGERS = 1, MR_EQ_SW_VEC = 2, MR_EQ_EULER_VEC = 3,
    MR_EQ_SW_D1Q3 = 4, MR_EQ_SW_D1Q5 = 5
} mr_equilibrium;

/* Per-instance description for the batched interface. */
typedef struct {
    int Jmin, Jmax;   /* 2 <= Jmin <= Jmax <= 24 */
    int gamma;        /* prediction stencil half-width: 1, 2 or 3 */
    int mu_bar;       /* Harten regularity guess, >= 0 (eq. HartenLossOfRegularity) */
    int bc;           /* mr_bc */
    int eq;           /* mr_equilibrium */
    double eps;       /* threshold epsilon (Prop. ErrorControl), >= 0 */
    double a, b;      /* domain [a, b] */
    double lambda;    /* lattice velocity, dt = dx_Jmax / lambda */
    double s[3];      /* relaxation rate of the non-conserved moment of each field */
    double eq_param;  /* see mr_equilibrium */
    int collision;    /* mr_collision */
} mr_instance_desc;

/* Collision of the adaptive scheme (Section 4.5): on the leaf values (eq.
 * LeavesCollision, the default), or with the equilibria of the relaxed moments
 * averaged over the leaf's 2^(Jmax-l) reconstructed finest cells (eq.
 * reconstructedCollision; costs a reconstruction of the whole finest level
 * per step). */
typedef enum { MR_COLLIDE_LEAVES = 0, MR_COLLIDE_RECONSTRUCTED = 1 } mr_collision;

/* ---- creation -------------------------------------------------------- */

/* Mesh part of the problem statement (Sections 3.1-3.4, 4.2): one instance.
 * precision: mr_precision.  The scheme is set by lbm_scheme() before mr_bind(). */
mr_status mr_mesh_init(mr_ctx **out, int Jmin, int Jmax, int gamma, double eps, double a,
                       double b, int bc, int mu_bar, int precision);

/* Scheme part (d'Humieres formalism, Section 2.1): DdQq with d = 1 and
 * q = 2 n, lattice velocity lambda, relaxation rates s[0..n-1] of the
 * non-conserved moments, equilibrium eq with parameter *eq_params. */
mr_status lbm_scheme(mr_ctx *ctx, int d, int q, double lambda, const double *s, int eq,
                     const double *eq_params);

/* Collision kind (mr_collision) of every instance of the context; before mr_bind. */
mr_status mr_set_collision(mr_ctx *ctx, int kind);

/* n independent instances in one context (batched persistent launch). */
mr_status mr_batch_create(mr_ctx **out, const mr_instance_desc *desc, int n, int precision);

/* Device bytes needed by the context (valid once every scheme is set). */
mr_status mr_workspace_size(const mr_ctx *ctx, size_t *bytes);

/* Attach the caller-owned device workspace and the CUDA stream (cudaStream_t,
 * NULL for the legacy default stream).  Uploads the reconstruction tables. */
mr_status mr_bind(mr_ctx *ctx, void *d_workspace, size_t bytes, void *stream);

/* ---- state ----------------------------------------------------------- */

/* Initial datum (Section 2.1, Lambda^0 = full tree, Section 4.4): cell averages
 * of the conserved moments on the finest lattice, for every instance in order,
 * field-major per instance: instance i occupies n_i * 2^Jmax_i doubles
 * (field j, cell k at j * 2^Jmax_i + k).  Populations start at equilibrium.
 * Host or device pointer; count = total number of doubles. */
mr_status mr_set_initial(mr_ctx *ctx, const double *m_cons, size_t count);

/* Arbitrary state of one instance (testing, restart): R[c] != 0 marks cell c of
 * the complete tree R(Lambda), values[h * S + c] the population h on cell c,
 * cells numbered level by level (level l: [2^l - 2^Jmin, 2^(l+1) - 2^Jmin)),
 * S = 2^(Jmax+1) - 2^Jmin.  Only leaf values are used.  Device pointers.
 * The tree is checked on the host first (coarsest level whole, siblings
 * together, graded for the instance's gamma); MR_ERR_ARG if it is not. */
mr_status mr_set_state(mr_ctx *ctx, int inst, const unsigned char *R, const double *values);

/* ---- the adaptive step ------------------------------------------------ */

mr_status mr_adapt(mr_ctx *ctx);              /* Section 4.1 on every instance      */
mr_status lbm_step(mr_ctx *ctx);              /* Sections 4.3, 4.5 on every instance */
mr_status mr_advance(mr_ctx *ctx, int nsteps); /* nsteps x (mr_adapt; lbm_step), one launch */

/* Waits for the bound stream and reports device-side errors. */
mr_status mr_sync(mr_ctx *ctx);

/* ---- results (synchronising; host output pointers) -------------------- */

/* Complete leaves S(Lambda) of instance inst (Section 3.3: the cells of the
 * complete tree without children, a multi-level partition of the domain),
 * ordered by level then index, with their q populations (f[h * cap + i]); any
 * output may be NULL.  level / index / f are host pointers of cap entries per
 * row; *count receives #S(Lambda).  MR_ERR_CAPACITY (nothing written) when an
 * output is given and cap < #S(Lambda); MR_ERR_NONFINITE when a population of
 * the instance became NaN or infinite. */
mr_status mr_get_leaves(mr_ctx *ctx, int inst, int *level, long *index, double *f, long cap,
                        long *count);

/* Conserved moments m^j = sum_h M_{jh} f^h on the leaves (Section 2.1, the
 * moment matrix of the d'Humieres formalism: per D1Q2 field f+ + f-, for
 * D1Q3 / D1Q5 the moments of order 0 and 1), host pointer m[j * cap + i],
 * same order, count and errors as mr_get_leaves. */
mr_status mr_get_moments(mr_ctx *ctx, int inst, double *m, long cap, long *count);

/* Conserved moments reconstructed on every finest cell (n * 2^Jmax values,
 * m[j * 2^Jmax + k]); the multiresolution reconstruction of Section 3.3.
 * Host or device pointer. */
mr_status mr_get_finest(mr_ctx *ctx, int inst, double *m_finest);

/* Complete tree membership R (S bytes, cell numbering of mr_set_state). */
mr_status mr_get_tree(mr_ctx *ctx, int inst, unsigned char *R);

/* Conservation audit.  The collision keeps the conserved moments of every
 * leaf (Section 2.1) and the stream of eq. AdaptiveStreamPhase (Section 4.3)
 * exchanges one reconstructed value per interface between the two leaves it
 * separates, so the totals sum_leaves dx_l m^j change only by what crosses a
 * copy boundary (periodic: not at all).  mass (host, n values) receives the
 * totals in FP64 (the FP32 path accumulates them in float-float, relative
 * error near 2^-44); residual (host) the largest per-step |change of the
 * totals - boundary flux| seen so far.  Either may be NULL. */
mr_status mr_audit(mr_ctx *ctx, int inst, double *mass, double *residual);

/* Per-instance summary in one copy: FP64 conserved totals (mass[3 * i + j],
 * zero past the instance's field count) and current leaf counts nleaf[i];
 * either output may be NULL.  Host pointers. */
mr_status mr_get_summary(mr_ctx *ctx, double *mass, int *nleaf);

/* Near ties of the threshold test (Section 3.4, Prop. ErrorControl, and the
 * Harten rule of eq. HartenLossOfRegularity): the number of keep / refine
 * decisions of instance inst, since its initial state, whose max |detail| lay
 * within 1e-12 relative of eps_l or of 2^(mu_bar + 1) eps_l.  Such decisions
 * are taken on ">=" exactly as printed, in FP64 (the FP32 path recomputes
 * them in FP64 from the stored values); the count tells a caller comparing
 * meshes produced elsewhere where a rounding difference could flip a cell.
 * Host output; synchronising. */
mr_status mr_near_ties(mr_ctx *ctx, int inst, long long *count);

/* Totals over the context: leaf-cell updates (sum over steps and instances of
 * #S(Lambda^{n+1})), steps taken by instance 0, current leaves over instances. */
mr_status mr_stats(mr_ctx *ctx, unsigned long long *updates, unsigned long long *steps,
                   long long *leaves);

/* Length of the dependent-pass chain (no counterpart in the paper): the team
 * barriers instance inst has executed since its initial state and the steps
 * it has taken.  Every barrier ends a pass over a level or a list whose
 * results the next pass reads, so passes / steps times the cost of one such
 * hand-over (mr_probe_latency) is a floor under the time of one step of a
 * lone instance.  Host outputs (either may be NULL); synchronising. */
mr_status mr_step_passes(mr_ctx *ctx, int inst, unsigned long long *steps, unsigned long long *passes);

/* Latency probe (no counterpart in the paper): one block hands a value from
 * one warp to another through memory and a block barrier, as consecutive
 * passes of the step do, and times it in SM clock cycles on the current
 * device: cycles[0] per hand-over through global memory (a line the block has
 * read before), cycles[1] through shared memory, cycles[2] per bare block
 * barrier, cycles[3] through a global line the block has not touched before
 * (0 unless scratch holds more than 4096 + 256 bytes: one 128-byte line per
 * hand-over after the first 4096 bytes, up to 4096 of them).  scratch:
 * caller-owned device memory of at least 4096 bytes (256-byte aligned), all
 * of it overwritten; cycles: 4 host doubles; synchronises the stream. */
mr_status mr_probe_latency(void *scratch, size_t bytes, void *stream, double *cycles);

/* Launch shape: threads per block (128, 256, 512 or 1024; one block advances
 * one instance at a time) and blocks (0 = one wave of resident blocks).
 * Takes effect at the next launch. */
mr_status mr_set_launch(mr_ctx *ctx, int block, int grid);

/* Order in which the persistent launches' work queues hand out the instances.
 * The instances always form up to three groups, each run by its own kernel
 * variant: gamma = 2, 3 (compiled for fewer resident blocks with more
 * registers), gamma = 1 with the reconstructed collision, and gamma = 1 with
 * the leaves collision (a kernel compiled for more resident blocks when every
 * instance of that group has one field).  Within a group, by_fields = 1
 * (default) orders by scheme, largest first within a scheme; 0 orders by size
 * (populations x 2^Jmax) alone.  Stream-ordered. */
mr_status mr_set_order(mr_ctx *ctx, int by_fields);

/* Autotuner of the batch driver (the paper has no counterpart).  Times nsteps
 * adaptive steps of the context's current state under each launch shape --
 * threads per block 128, 256, 512, 1024 (the cells of a level each block
 * sweeps per pass) with the queue order of mr_set_order -- and keeps the
 * fastest.  Before every trial, and once more at the end, the state is
 * restored from scratch: caller-owned device memory of at least
 * mr_workspace_size bytes, which receives a copy of the workspace.  The
 * results are unchanged by the launch shape (every shape computes the same
 * values), so the state after the call equals the state before it.
 * Synchronises the stream; not for use during stream capture.  best_block,
 * best_order (the order in use, as mr_set_order's by_fields) and best_ms (the
 * fastest trial in milliseconds) may be NULL. */
mr_status mr_autotune(mr_ctx *ctx, int nsteps, void *scratch, size_t scratch_bytes, int *best_block,
                      int *best_order, float *best_ms);

/* Reconstruction coefficients used by the stream (Section 3.3 with gamma = 1):
 * for a leaf at level gap dj = Jmax - l (0 <= dj <= 24), kind 0 gives the
 * 4 weights of the first finest cell on the level-l window (k-2, k-1, k, k+1),
 * kind 1 the 4 weights on the window (2k-2, 2k-1, 2k, 2k+1) of level l+1 (used
 * next to a finer neighbour), kind 2 the 2 weights on (0, 1) for the leaf
 * k = 0 at a copy boundary; kinds 3, 4, 5 the same for the second finest cell
 * from the edge (used by the populations with |v| = 2 lambda of D1Q5).  The
 * last (second-to-last) finest cell uses the mirrored weights.
 * Host-only query, no device needed. */
mr_status mr_reconstruction_coefficients(int dj, int kind, double *out);

/* Tracing: SM clock cycles spent by instance inst in each phase of the step,
 * accumulated since its initial state, in the order
 *   projection (adapt), details + threshold, enlargement, grading + marking,
 *   grading of the levels of at most 32 cells, candidate mask words, list
 *   compaction, data transfer, collision, projection (step), ghosts,
 *   reconstruction, stream + audit
 * (n >= 13 slots).  Only a library compiled with MRG_PHASE_TIMERS records
 * them; otherwise the cycles are zero and MR_ERR_STATE is returned. */
mr_status mr_phase_times(mr_ctx *ctx, int inst, unsigned long long *cycles, int n);

/* Number of instances, and the number of kernel launches issued so far. */
mr_status mr_info(const mr_ctx *ctx, int *n_instances, long long *launches);

/* Last error message of the context (or of the last failed creation if ctx is NULL). */
mr_status mr_last_error(const mr_ctx *ctx, char *buf, int len);

mr_status mr_destroy(mr_ctx *ctx);

/* ---- running without any device allocation ----------------------------- */

/* Size of the scratch area built into the library for mr_run_static. */
#define MR_STATIC_SCRATCH_BYTES (16u << 20)

/* The paper has no counterpart to this call; it is here for callers that
 * cannot allocate device memory when they need to run a problem: a host
 * program that forbids new device allocations after start-up, a plug-in whose
 * host application owns every device buffer, or code that must not risk the
 * blocking and device-wide synchronisation an allocation can cause.
 *
 * mr_run_static runs one instance (desc, precision) from its initial datum
 * for nsteps adaptive steps and writes the conserved moments reconstructed on
 * every finest cell, exactly as mr_set_initial + mr_advance + mr_get_finest
 * of a context would.  It allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.  Its working memory is a fixed area of
 * MR_STATIC_SCRATCH_BYTES that is part of the library's device image, held
 * by every GPU that loads the library until the process exits.
 *   m_cons    device-readable input, n * 2^Jmax doubles (layout of mr_set_initial)
 *   m_finest  device-writable output, n * 2^Jmax doubles (layout of mr_get_finest)
 *   updates   optional host output: leaf-cell updates over the run; when it is
 *             given the call waits for the stream and reports non-finite values
 *   stream    CUDA stream the work is ordered on (NULL: legacy default stream)
 * The first call on a device looks up the scratch area's device address (with
 * that device current) and keeps it; that set-up is done once per device even
 * when several host threads make their first call at the same time.  The call
 * uploads its descriptor from host memory and may wait for the stream, so it
 * must not be recorded into a CUDA graph: on a stream that is capturing it
 * returns MR_ERR_STATE and enqueues nothing.  An instance whose layout exceeds the area is rejected with
 * MR_ERR_CAPACITY (FP64 Euler fits up to Jmax = 16); the message is available
 * from mr_last_error(NULL, ...).  Every call uses the same area and leaves its
 * contents behind; each call re-initialises what it reads, but calls whose
 * work overlaps on the GPU (other streams, other host threads) race on it. */
mr_status mr_run_static(const mr_instance_desc *desc, int precision, const double *m_cons, int nsteps,
                        double *m_finest, unsigned long long *updates, void *stream);

#ifdef __cplusplus
}
#endif
#endif

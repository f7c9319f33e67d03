// mr_common.h -- data layout shared by the CUDA kernels and the host side of
// the C ABI (include/mrlbm.h).  Internal to the library.
//
// Per instance the device workspace holds (all 256-byte aligned):
//   V      S x q values, cell-major (the q populations of a cell contiguous),
//          level l at cells [2^l - 2^Jmin, ...) (dense level-wise arrays:
//          every cell of every level has a slot)
//   Phi    (2^Jmax + 1) x q reconstructed boundary values, interface-major,
//          indexed by the finest-lattice interface they belong to
//   masks  NMASK bitmasks over all cells of all levels, 32 cells per word,
//          level l at words [woff_l, woff_l + max(1, 2^l / 32)); then the
//          candidate-word list of the step (Wtot entries at most) and two
//          occupancy bitmaps (one per tree buffer) with one bit per mask
//          word, level l at occupancy words [ooff_l, ooff_l + max(1, W_l / 32))
//   lists  compacted cell lists (entry = level << KBITS | index), sorted by
//          level then index; per-level segments in InstState::seg
//   state  InstState
#pragma once
#include <cstddef>
#include <cstdint>

namespace mrg {

constexpr int MAXLEV = 24;  // Jmax <= 24
constexpr int MAXDJ = MAXLEV;
constexpr int KBITS = 27;
constexpr uint32_t KMASK = (1u << KBITS) - 1u;

constexpr int NOT_POW2 = 1 << 20;  // InstDesc::lam_log2 of a lattice velocity that is no power of two

// bitmasks; KEEP / REF (written by the details, read by the enlargement) share
// storage with PRED / GH (written by the grading sweep, read by the list
// compaction, which clears them for the next step)
enum { M_R0 = 0, M_R1 = 1, M_LEAF = 2, M_PRED = 3, M_GH = 4, NMASK = 5, M_KEEP = M_PRED, M_REF = M_GH };
// lists: internal cells of the tree, leaves, cells to predict in the transfer (A6)
// and ghosts (S3); the even cells of the tree, whose details A2 tests, are the
// first children of the internal cells
enum { L_INT = 0, L_LEAF = 1, L_PRED = 2, L_GH = 3, NLIST = 4 };
// phases of the persistent kernel
enum { PH_INIT_FULL = 1, PH_INIT_STATE = 2, PH_ADAPT = 4, PH_STEP = 8, PH_FINEST = 16 };
// device status bits
// ST_FLUXED: the last step streamed with interface values in Phi (D1Q2^n
// schemes) and, in the same pass, moved every internal cell by the flux through
// its own edges, so the internal cells hold the projection of the leaves and the
// next adaptation skips its projection (see the kernel).
enum { ST_NONFINITE = 1, ST_FLUXED = 2 };
// phases timed by the profiling build (MRG_PHASE_TIMERS)
enum {
    T_UPSWEEP_A = 0, T_DETAILS, T_ENLARGE, T_GRADE, T_GRADE_SMALL, T_CANDIDATES, T_LISTS, T_TRANSFER,
    T_COLLIDE, T_UPSWEEP_S, T_GHOSTS, T_RECON, T_STREAM, NPHASE
};

struct InstState {
    int cur;                      // mask (M_R0 or M_R1) holding the current tree
    int nleaf;                    // #S(Lambda) of the current tree
    int seg[NLIST][MAXLEV + 2];   // list segments: level l at [seg[l], seg[l+1])
    int status;                   // ST_* bits
    int near_ties;                // threshold decisions within 1e-12 relative of the threshold
    unsigned deplev[2];           // levels holding transfer / ghost cells that wait on the same list
    unsigned long long updates;   // sum over steps of #S(Lambda^{n+1})
    unsigned long long steps;
    unsigned long long passes;    // team barriers since the initial state (dependent passes)
    double mass[3];               // FP64 totals sum_leaves dx_l m_j
    double audit;                 // max over steps of |mass change - boundary flux|
    unsigned long long ptime[NPHASE];  // SM clock cycles per phase (profiling build only)
};

struct InstDesc {
    int Jmin, Jmax, bc, eq, nf, mu_bar;
    int gamma;             // prediction stencil half-width (1, 2 or 3)
    int collision;         // 0: leaves collision, 1: reconstructed collision (Section 4.5)
    int lam_log2;          // k when lambda = 2^k exactly (|k| <= 16), else NOT_POW2
    int Wtot;              // mask words over all levels
    int OW;                // occupancy words over all levels (one bit per mask word)
    double eps, a, b, lam, eqp;
    double s[3];
    long long S;           // cells over all levels
    long long N;           // 2^Jmax
    long long m_off;       // offset of this instance's initial data in the input array
    void *V;
    void *Phi;
    uint32_t *masks;
    uint32_t *lists;
    long long list_off[NLIST];
    InstState *st;
    double minv[5][5];     // D1Q3 / D1Q5: inverse of the moment matrix (v^h)^i
    // the scheme constants rounded to float once, for the FP32 path
    float lam_f, eqp_f, s_f[3];
    float minv_f[5][5];
    // correctly rounded reciprocal of lambda, for the FP64 division by lambda
    // with one correction step (see the kernel's div_lam)
    double rlam;
    // constant factors of the FP64 collision, rounded once exactly as the
    // per-cell expressions would round them: 1 - s[j]; Euler 1.5 - 0.5 gamma_gas,
    // gamma_gas - 1, 0.5 (1 - gamma_gas); shallow water 0.5 g
    double oms[3], eu_a, eu_b, eu_c, sw_g2;
};

// words of the mask region of an instance: NMASK bitmasks, the candidate-word
// list and two occupancy bitmaps
inline long long mask_region_words(int Wtot, int OW) { return (long long)(NMASK + 1) * Wtot + 2LL * OW; }
// gamma = 1 instances with the leaves collision and at least this many mask
// words per bitmask run their word passes over the step's candidate words
// (K_LARGE); smaller ones visit every word, which costs less than building the
// candidate list (measured on the Jmax 8..14 batch and the single instances).
// The wide-stencil and reconstructed-collision variants visit every word at
// any size.
constexpr int CW_MIN_WORDS = 2048;
// words of the mask region a block keeps in shared memory: without candidate
// words the list and the occupancy bitmaps are not used
#ifdef __CUDACC__
__host__ __device__
#endif
inline long long smem_region_words(int Wtot, int OW) {
    return Wtot >= CW_MIN_WORDS ? (long long)(NMASK + 1) * Wtot + 2LL * OW : (long long)NMASK * Wtot;
}
// occupancy words of one level: one bit per mask word of the level
inline int occ_words_of(int l) { return l >= 10 ? (1 << (l - 10)) : 1; }

// fills InstDesc's float copies of lam, eqp, s and minv (host side, after those are set)
inline void fill_float_constants(InstDesc &h) {
    h.lam_f = (float)h.lam;
    h.eqp_f = (float)h.eqp;
    for (int j = 0; j < 3; ++j) h.s_f[j] = (float)h.s[j];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) h.minv_f[i][j] = (float)h.minv[i][j];
    h.rlam = 1.0 / h.lam;  // IEEE division: correctly rounded
    for (int j = 0; j < 3; ++j) h.oms[j] = 1.0 - h.s[j];
    h.eu_a = 1.5 - 0.5 * h.eqp;
    h.eu_b = h.eqp - 1.0;
    h.eu_c = 0.5 * (1.0 - h.eqp);
    h.sw_g2 = 0.5 * h.eqp;
}

// Reconstruction tables for gamma = 1, indexed by the level gap dj = Jmax - l
// (exact dyadic rationals, generated by integer recursion on the host):
//   cf[dj]  first finest cell of a leaf from its level window (k-2, k-1, k, k+1)
//   t1[dj]  same from the window (2k-2, 2k-1, 2k, 2k+1) one level finer
//   bf[dj]  first finest cell of the leaf k = 0 under a copy boundary, from (0, 1)
// The last finest cell uses the mirrored coefficients.
//   cf2, t12, bf2  the same for the second finest cell from the edge (the
//           populations with |v| = 2 lambda stream two cells per step)
//   pc[g]   the prediction coefficients c_1..c_g of the stencil gamma = g
//           (Section 3.1; gamma = 3 with c_3 = -5/1024)
template <typename T>
struct Tables {
    T cf[MAXDJ + 1][4];
    T t1[MAXDJ + 1][4];
    T bf[MAXDJ + 1][2];
    T cf2[MAXDJ + 1][4];
    T t12[MAXDJ + 1][4];
    T bf2[MAXDJ + 1][2];
    T pc[4][3];
};

struct LaunchArgs {
    const InstDesc *descs;
    const int *order;     // instance processing order (longest first)
    int n;                // instances in this launch
    int nsteps;
    int phases;           // PH_* bits
    int *queue;           // work-queue counter, zero at launch
    const void *aux0;     // phase input / output (see the kernel)
    const void *aux1;
    const void *tables;   // Tables<T> in device memory
    int smem_mask_words;  // block teams keep their mask region in shared memory when it has at most this many words
    int kind;             // kernel variant (K_*) the launch runs
};

// Kernel variants.  K_FAST: every scheme with gamma = 1 and the leaves collision;
// K_GENERAL: gamma = 2 or 3 (either collision); K_SCALAR: the instances of
// K_FAST with one conserved field (D1Q2), compiled on their own for a higher
// residency; K_RECOLL: gamma = 1 with the reconstructed collision, the code of
// K_GENERAL compiled for a residency of its own (its dense reconstruction gains
// from blocks in flight, the wide stencils from registers); K_LARGE: the code of
// K_FAST for the instances with at least CW_MIN_WORDS mask words per bitmask,
// whose word passes visit the step's candidate words (the code that builds
// them stays out of the other variants, which it slowed down).
constexpr int K_FAST = 0, K_GENERAL = 1, K_SCALAR = 2, K_RECOLL = 3, K_LARGE = 4, NKIND = 5;

}  // namespace mrg

// launchers (mr_dispatch.cu)
extern "C++" {
// priority: the launch's scheduling priority (cudaLaunchAttributePriority; 0 is
// the default, lower values are scheduled first when launches compete for SMs)
int mrg_launch(bool fp32, int block, int grid, const mrg::LaunchArgs &a, void *stream, int priority);
int mrg_occupancy(bool fp32, int block, int kind, int mask_words, int *blocks_per_sm);
int mrg_min_blocks(bool fp32, int block, int kind);  // residency the variant is compiled for
size_t mrg_smem_bytes(bool fp32, int block, int mask_words);
void mrg_tables(mrg::Tables<double> *td, mrg::Tables<float> *tf);
void mrg_set_error(const char *msg);
// scheme shape (mr_api.cu): conserved fields, populations, relaxation rates of
// an mr_equilibrium, and the inverse moment matrix of the D1Q3 / D1Q5 schemes
int mrg_nfields(int eq);
int mrg_npop(int eq);
int mrg_nrates(int eq);
void mrg_dq_inverse(int eq, double lambda, double inv[5][5]);
}

// mr_api.cu -- host implementation of the C ABI declared in include/mrlbm.h.
//
// The library never allocates device memory: the caller hands over one device
// buffer (mr_bind) that is carved into the per-context header (descriptors,
// per-instance state, work queue, reconstruction tables, input staging) and the
// per-instance regions described in mr_common.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mrlbm.h"
#include "mr_common.h"

using namespace mrg;

namespace {

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

int nfields_of(int eq) {
    switch (eq) {
    case MR_EQ_ADVECTION:
    case MR_EQ_BURGERS: return 1;
    case MR_EQ_SW_VEC: return 2;
    case MR_EQ_EULER_VEC: return 3;
    case MR_EQ_SW_D1Q3:
    case MR_EQ_SW_D1Q5: return 2;
    default: return 0;
    }
}
// populations q and relaxation rates of a scheme
int npop_of(int eq) { return eq == MR_EQ_SW_D1Q3 ? 3 : eq == MR_EQ_SW_D1Q5 ? 5 : 2 * nfields_of(eq); }
int nrates_of(int eq) { return eq == MR_EQ_SW_D1Q3 ? 1 : eq == MR_EQ_SW_D1Q5 ? 3 : nfields_of(eq); }

// D1Q3 / D1Q5: inverse of the moment matrix M[i][h] = (v^h)^i, v = lambda (0, 1, -1, 2, -2),
// by Gauss-Jordan elimination with partial pivoting
void dq_inverse(int eq, double lambda, double inv[5][5]) {
    const int q = npop_of(eq);
    const double w[5] = {0.0, 1.0, -1.0, 2.0, -2.0};
    double A[5][10];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) inv[i][j] = 0.0;
    for (int i = 0; i < q; ++i)
        for (int h = 0; h < q; ++h) {
            double x = 1.0;
            for (int e = 0; e < i; ++e) x *= w[h] * lambda;
            A[i][h] = x;
            A[i][q + h] = i == h ? 1.0 : 0.0;
        }
    for (int col = 0; col < q; ++col) {
        int piv = col;
        for (int r = col + 1; r < q; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        for (int j = 0; j < 2 * q; ++j) std::swap(A[col][j], A[piv][j]);
        const double dv = A[col][col];
        for (int j = 0; j < 2 * q; ++j) A[col][j] /= dv;
        for (int r = 0; r < q; ++r)
            if (r != col) {
                const double f = A[r][col];
                for (int j = 0; j < 2 * q; ++j) A[r][j] -= f * A[col][j];
            }
    }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) inv[i][j] = A[i][q + j];
}

int nwords_h(int l) { return l >= 5 ? (1 << (l - 5)) : 1; }
// compiled scheme variant of the kernels: D1Q2^n by field count, D1Q3, D1Q5
int variant_of(int eq) { return eq == MR_EQ_SW_D1Q3 ? 4 : eq == MR_EQ_SW_D1Q5 ? 5 : nfields_of(eq); }
// Group of the queue order an instance belongs to, most work per instance
// first: gamma = 2, 3 (general kernel); gamma = 1 with the reconstructed
// collision; gamma = 1 with the leaves collision and at least CW_MIN_WORDS
// mask words per bitmask (the fast code with candidate words); the other
// gamma = 1 instances with the leaves collision (fast kernel, or the scalar
// kernel when every instance of the group has one field).
constexpr int NGROUP = 4;
int group_of(const InstDesc &h) {
    return h.gamma > 1 ? 0 : h.collision != 0 ? 1 : h.Wtot >= CW_MIN_WORDS ? 2 : 3;
}
// kernel variant of a lone instance
int kind_of(const InstDesc &h) {
    return h.gamma > 1 ? K_GENERAL : h.collision != 0 ? K_RECOLL : h.Wtot >= CW_MIN_WORDS ? K_LARGE : K_FAST;
}

thread_local std::string g_create_error;


// Latency probe: warps 0 and 1 of one block alternately read the value the
// other wrote and write the next one, with a block barrier after every
// hand-over; through global memory (buf[0..63], lines the block has read
// before), through shared memory, bare barriers, and through global memory
// where every hand-over uses a line no thread of the block has touched
// (fresh[i * 32], i < nfresh, one 128-byte line each).  Every index stays
// inside buf[0..63], fresh[0 .. 32 nfresh) and the shared array.
constexpr int kProbeIters = 4096;
constexpr size_t kProbeFreshOff = 4096;  // bytes of scratch before the fresh lines
__global__ void mrg_probe(int *buf, unsigned long long *res, int iters, int *fresh, int nfresh) {
    __shared__ int sh[64];
    if (threadIdx.x < 64) sh[threadIdx.x] = 0;
    __syncthreads();
    const int me = threadIdx.x;
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        if (me == ((i & 1) ? 32 : 0)) buf[(i + 1) & 63] = buf[i & 63] + 1;
        __syncthreads();
    }
    long long t1 = clock64();
    for (int i = 0; i < iters; ++i) {
        if (me == ((i & 1) ? 32 : 0)) sh[(i + 1) & 63] = sh[i & 63] + 1;
        __syncthreads();
    }
    long long t2 = clock64();
    for (int i = 0; i < iters; ++i) __syncthreads();
    long long t3 = clock64();
    // fresh lines: hand-over i writes line i + 1 after reading line i
    for (int i = 0; i + 1 < nfresh; ++i) {
        if (me == ((i & 1) ? 32 : 0)) fresh[(i + 1) * 32] = fresh[i * 32] + 1;
        __syncthreads();
    }
    long long t4 = clock64();
    if (me == 0) {
        res[0] = (unsigned long long)(t1 - t0);
        res[1] = (unsigned long long)(t2 - t1) + (unsigned long long)(sh[iters & 63] & 0);
        res[2] = (unsigned long long)(t3 - t2);
        res[3] = nfresh > 1 ? (unsigned long long)(t4 - t3) / (unsigned long long)(nfresh - 1) : 0ull;
    }
}

}  // namespace

struct mr_ctx {
    std::vector<mr_instance_desc> desc;
    std::vector<bool> scheme_set;
    int precision = MR_FP64;
    // layout (bytes from the workspace base)
    size_t off_desc = 0, off_state = 0, off_order = 0, off_ident = 0, off_queue = 0, off_tab = 0,
           off_stage = 0, total = 0;
    std::vector<size_t> inst_off;  // per instance region start
    std::vector<InstDesc> hdesc;   // host copy of the device descriptors
    std::vector<long long> m_off;  // per instance offset in the initial-data array
    size_t stage_doubles = 0;
    // binding
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    bool bound = false, initialised = false;
    int block = 0, grid_req = 0, sms = 0;
    int grid[NKIND] = {};      // blocks per launch, by kernel variant (K_*)
    int mask_cap[NKIND] = {};  // mask-region words a block team keeps in shared memory, by variant
    int wmax = 0;              // mask-region words of the largest instance
    int n_group[NGROUP] = {};  // instances per group of the queue order (group_of)
    int group_kind[NGROUP] = {K_GENERAL, K_RECOLL, K_LARGE, K_FAST};  // kernel variant of each group
    // The groups run as separate kernels; a second stream lets one group's
    // kernel fill the SMs that another's tail leaves idle (fork and join by events).
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int prio_least = 0, prio_greatest = 0;  // the device's launch priority range
    bool order_by_fields = true;
    std::vector<int> order_host;  // staging of the queue order (kept alive for the async copy)
    long long launches = 0;
    std::string err;

    int fail(int code, const char *fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return MR_OK;
        return fail(MR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    bool fp32() const { return precision == MR_FP32_MIXED; }
    size_t vbytes() const { return fp32() ? 4 : 8; }
    int n() const { return (int)desc.size(); }
    ~mr_ctx() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
    }
};

// ---------------------------------------------------------------------------
// validation and layout

static int check_desc(mr_ctx *c, const mr_instance_desc &d, int i) {
    if (d.Jmin < 2 || d.Jmax < d.Jmin || d.Jmax > MAXLEV)
        return c->fail(MR_ERR_ARG, "instance %d: need 2 <= Jmin <= Jmax <= %d (got %d, %d)", i, MAXLEV, d.Jmin, d.Jmax);
    if (d.gamma < 1 || d.gamma > 3) return c->fail(MR_ERR_ARG, "instance %d: gamma must be 1, 2 or 3", i);
    if (d.mu_bar < 0 || d.mu_bar > 30) return c->fail(MR_ERR_ARG, "instance %d: mu_bar out of range", i);
    if (d.collision != MR_COLLIDE_LEAVES && d.collision != MR_COLLIDE_RECONSTRUCTED)
        return c->fail(MR_ERR_ARG, "instance %d: collision must be 0 (leaves) or 1 (reconstructed)", i);
    if (d.bc != MR_BC_PERIODIC && d.bc != MR_BC_COPY) return c->fail(MR_ERR_ARG, "instance %d: bad boundary", i);
    if (nfields_of(d.eq) == 0) return c->fail(MR_ERR_ARG, "instance %d: bad equilibrium", i);
    if (!(d.eps >= 0.0) || !(d.b > d.a) || !(d.lambda >= 0x1p-16 && d.lambda <= 0x1p16))
        return c->fail(MR_ERR_ARG, "instance %d: need eps >= 0, b > a, 2^-16 <= lambda <= 2^16", i);
    for (int j = 0; j < nrates_of(d.eq); ++j)
        if (!(d.s[j] > 0.0 && d.s[j] <= 2.0)) return c->fail(MR_ERR_ARG, "instance %d: relaxation rate outside (0, 2]", i);
    if ((d.eq == MR_EQ_SW_D1Q3 || d.eq == MR_EQ_SW_D1Q5) && d.gamma != 1)
        return c->fail(MR_ERR_ARG, "instance %d: the D1Q3 / D1Q5 schemes are built with gamma = 1", i);
    return MR_OK;
}

static void layout(mr_ctx *c) {
    int n = c->n();
    size_t o = 0;
    c->off_desc = o;
    o = align_up(o + sizeof(InstDesc) * n);
    c->off_state = o;
    o = align_up(o + sizeof(InstState) * n);
    c->off_order = o;
    o = align_up(o + sizeof(int) * n);
    c->off_ident = o;
    o = align_up(o + sizeof(int) * n);
    c->off_queue = o;
    o = align_up(o + sizeof(int) * 16 * NKIND);  // one queue counter per kernel variant, 64 bytes apart
    c->off_tab = o;
    o = align_up(o + sizeof(Tables<double>) + sizeof(Tables<float>));
    c->m_off.assign(n, 0);
    size_t st = 0;
    for (int i = 0; i < n; ++i) {
        c->m_off[i] = (long long)st;
        st += (size_t)nfields_of(c->desc[i].eq) << c->desc[i].Jmax;
    }
    c->stage_doubles = st;
    c->off_stage = o;
    o = align_up(o + st * sizeof(double));
    c->inst_off.assign(n, 0);
    c->hdesc.assign(n, InstDesc{});
    for (int i = 0; i < n; ++i) {
        const mr_instance_desc &d = c->desc[i];
        InstDesc &h = c->hdesc[i];
        int nf = nfields_of(d.eq), q = npop_of(d.eq);
        long long S = (1LL << (d.Jmax + 1)) - (1LL << d.Jmin), N = 1LL << d.Jmax;
        int W = 0, OW = 0;
        for (int l = d.Jmin; l <= d.Jmax; ++l) {
            W += nwords_h(l);
            OW += occ_words_of(l);
        }
        h.Jmin = d.Jmin;
        h.Jmax = d.Jmax;
        h.bc = d.bc;
        h.eq = d.eq;
        h.nf = nf;
        if (d.eq == MR_EQ_SW_D1Q3 || d.eq == MR_EQ_SW_D1Q5) dq_inverse(d.eq, d.lambda, h.minv);
        h.mu_bar = d.mu_bar;
        h.gamma = d.gamma;
        h.collision = d.collision;
        h.lam_log2 = NOT_POW2;
        {
            int e2 = 0;
            const double fr = std::frexp(d.lambda, &e2);  // lambda = fr 2^e2, fr in [0.5, 1)
            if (fr == 0.5 && e2 - 1 >= -16 && e2 - 1 <= 16) h.lam_log2 = e2 - 1;
        }
        h.Wtot = W;
        h.OW = OW;
        h.eps = d.eps;
        h.a = d.a;
        h.b = d.b;
        h.lam = d.lambda;
        h.eqp = d.eq_param;
        for (int j = 0; j < 3; ++j) h.s[j] = d.s[j];
        fill_float_constants(h);
        h.S = S;
        h.N = N;
        h.m_off = c->m_off[i];
        c->inst_off[i] = o;
        size_t vb = c->vbytes();
        size_t oV = 0, oPhi = align_up(oV + vb * q * S), oM = align_up(oPhi + vb * q * (N + 1));
        size_t oL = align_up(oM + sizeof(uint32_t) * (size_t)mask_region_words(W, OW));
        // every list holds distinct cells of the instance, so S entries always suffice
        long long caps[NLIST] = {S, S, S, S};
        long long lo = 0;
        for (int L = 0; L < NLIST; ++L) {
            h.list_off[L] = lo;
            lo += (caps[L] + 63) / 64 * 64;
        }
        size_t end = align_up(oL + sizeof(uint32_t) * lo);
        // pointers are filled at bind time; keep relative offsets for now
        h.V = (void *)oV;
        h.Phi = (void *)oPhi;
        h.masks = (uint32_t *)oM;
        h.lists = (uint32_t *)oL;
        o += end;
    }
    c->total = align_up(o);
}

// Reconstruction tables for gamma = 1 (c1 = -1/8), by exact integer recursion.
// Window recursion one level down (level m -> m+1) on the 4 cells
// (p-2, p-1, p, p+1) around the first cell p of a leaf, times 8:
//   rows (2p-2, 2p-1, 2p, 2p+1) = [1 8 -1 0], [-1 8 1 0], [0 1 8 -1], [0 -1 8 1].
// The first finest cell after dj levels is row 2 of the dj-th power.  At a copy
// boundary (left edge of cell 0 clamped to itself) the window is (0, 1) and
// the recursion is [9 -1], [7 1] (times 8).
static void make_tables(Tables<double> &td, Tables<float> &tf) {
    typedef __int128 i128;
    const i128 A[4][4] = {{1, 8, -1, 0}, {-1, 8, 1, 0}, {0, 1, 8, -1}, {0, -1, 8, 1}};
    const i128 B[2][2] = {{9, -1}, {7, 1}};
    // first cell: window position 2 (the cell p itself, even children all the way);
    // second cell (v2, u2): window position 3, the odd child at the last level
    i128 v[4] = {0, 0, 1, 0}, u[2] = {1, 0}, v2[4] = {0, 0, 0, 1}, u2[2] = {0, 1};
    std::memset(&td, 0, sizeof td);
    std::memset(&tf, 0, sizeof tf);
    for (int dj = 0; dj <= MAXDJ; ++dj) {
        for (int j = 0; j < 4; ++j) td.cf[dj][j] = std::ldexp((double)v[j], -3 * dj);
        for (int j = 0; j < 2; ++j) td.bf[dj][j] = std::ldexp((double)u[j], -3 * dj);
        for (int j = 0; j < 4; ++j) td.cf2[dj][j] = std::ldexp((double)v2[j], -3 * dj);
        for (int j = 0; j < 2; ++j) td.bf2[dj][j] = std::ldexp((double)u2[j], -3 * dj);
        if (dj > 0)
            for (int j = 0; j < 4; ++j) {
                td.t1[dj][j] = td.cf[dj - 1][j];
                td.t12[dj][j] = td.cf2[dj - 1][j];
            }
        i128 nv[4] = {0, 0, 0, 0}, nu[2] = {0, 0}, nv2[4] = {0, 0, 0, 0}, nu2[2] = {0, 0};
        for (int r = 0; r < 4; ++r)
            for (int j = 0; j < 4; ++j) {
                nv[j] += v[r] * A[r][j];
                nv2[j] += v2[r] * A[r][j];
            }
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < 2; ++j) {
                nu[j] += u[r] * B[r][j];
                nu2[j] += u2[r] * B[r][j];
            }
        std::memcpy(v, nv, sizeof v);
        std::memcpy(u, nu, sizeof u);
        std::memcpy(v2, nv2, sizeof v2);
        std::memcpy(u2, nu2, sizeof u2);
    }
    for (int dj = 0; dj <= MAXDJ; ++dj) {
        for (int j = 0; j < 4; ++j) {
            tf.cf[dj][j] = (float)td.cf[dj][j];
            tf.t1[dj][j] = (float)td.t1[dj][j];
            tf.cf2[dj][j] = (float)td.cf2[dj][j];
            tf.t12[dj][j] = (float)td.t12[dj][j];
        }
        for (int j = 0; j < 2; ++j) {
            tf.bf[dj][j] = (float)td.bf[dj][j];
            tf.bf2[dj][j] = (float)td.bf2[dj][j];
        }
    }
    // prediction coefficients c_1..c_gamma (Section 3.1; gamma = 3 with c_3 = -5/1024,
    // the sign that makes the stencil exact on polynomials of degree 5); all dyadic
    const double pc[4][3] = {{0.0, 0.0, 0.0},
                             {-1.0 / 8.0, 0.0, 0.0},
                             {-22.0 / 128.0, 3.0 / 128.0, 0.0},
                             {-201.0 / 1024.0, 11.0 / 256.0, -5.0 / 1024.0}};
    for (int g = 0; g < 4; ++g)
        for (int j = 0; j < 3; ++j) {
            td.pc[g][j] = pc[g][j];
            tf.pc[g][j] = (float)pc[g][j];
        }
}

static int launch_group(mr_ctx *c, int phases, int nsteps, const int *order, int n, int kind, const void *aux0,
                        const void *aux1, cudaStream_t stream, int priority) {
    LaunchArgs a{};
    a.descs = (const InstDesc *)(c->ws + c->off_desc);
    a.order = order;
    a.n = n;
    a.kind = kind;
    a.nsteps = nsteps;
    a.phases = phases;
    a.queue = (int *)(c->ws + c->off_queue) + 16 * kind;  // one counter per variant, 64 bytes apart
    a.aux0 = aux0;
    a.aux1 = aux1;
    a.tables = c->ws + c->off_tab + (c->fp32() ? sizeof(Tables<double>) : 0);
    a.smem_mask_words = c->mask_cap[kind];
    int rc = c->cuda(cudaMemsetAsync(a.queue, 0, sizeof(int), stream), "cudaMemsetAsync");
    if (rc) return rc;
    int grid = std::min(a.n, c->grid[kind]);
    int e = mrg_launch(c->fp32(), c->block, std::max(grid, 1), a, stream, priority);
    ++c->launches;
    if (e) return c->cuda((cudaError_t)e, "kernel launch");
    return MR_OK;
}

// A launch over the instances.  The queue order holds up to three groups, each
// run by its own kernel variant: the general kernel (gamma = 2, 3), the
// reconstructed-collision kernel (gamma = 1) and the fast kernel (gamma = 1,
// leaves collision; the scalar kernel when all of them have one field).  With
// more than one group the groups alternate between the context's stream and a
// side stream that forks from it and joins it again, so a group's kernel can
// fill the SMs the previous one's tail leaves idle.  Launch priorities (earlier
// groups first, the last at the default) ask the block scheduler to place the
// group with the most work per instance first when both kernels wait for SMs;
// a kernel that reached the SMs first keeps them until its queue runs dry.
static int launch(mr_ctx *c, int phases, int nsteps, int only_inst, const void *aux0, const void *aux1) {
    if (!c->bound) return c->fail(MR_ERR_STATE, "context not bound to a workspace");
    if (only_inst >= 0) {
        const InstDesc &h = c->hdesc[only_inst];
        const int kind = kind_of(h);
        return launch_group(c, phases, nsteps, (const int *)(c->ws + c->off_ident) + only_inst, 1, kind, aux0, aux1,
                            c->stream, c->prio_least);
    }
    const int *order = (const int *)(c->ws + c->off_order);
    int groups = 0;
    for (int g = 0; g < NGROUP; ++g) groups += c->n_group[g] > 0;
    const bool fork = groups > 1;
    int rc = MR_OK;
    if (fork) {
        if ((rc = c->cuda(cudaEventRecord(c->ev_fork, c->stream), "cudaEventRecord"))) return rc;
        if ((rc = c->cuda(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "cudaStreamWaitEvent"))) return rc;
    }
    int first = 0, k = 0;
    for (int g = 0; g < NGROUP && !rc; ++g) {
        if (c->n_group[g] == 0) continue;
        cudaStream_t st = (fork && (k & 1)) ? c->side : c->stream;
        const int prio = std::max(c->prio_greatest, c->prio_least - (groups - 1 - k));
        rc = launch_group(c, phases, nsteps, order + first, c->n_group[g], c->group_kind[g], aux0, aux1, st, prio);
        first += c->n_group[g];
        ++k;
    }
    if (fork) {
        // join even after a failed launch, so the side stream never outlives the caller's order
        int rj = c->cuda(cudaEventRecord(c->ev_join, c->side), "cudaEventRecord");
        if (!rj) rj = c->cuda(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "cudaStreamWaitEvent");
        if (!rc) rc = rj;
    }
    return rc;
}

static int read_state(mr_ctx *c, int inst, InstState *st) {
    int rc = c->cuda(cudaMemcpyAsync(st, c->ws + c->off_state + sizeof(InstState) * inst, sizeof(InstState),
                                     cudaMemcpyDeviceToHost, c->stream),
                     "cudaMemcpyAsync");
    if (rc) return rc;
    return c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

mr_status mr_mesh_init(mr_ctx **out, int Jmin, int Jmax, int gamma, double eps, double a, double b, int bc,
                       int mu_bar, int precision) {
    if (!out) return MR_ERR_ARG;
    *out = nullptr;
    if (precision != MR_FP64 && precision != MR_FP32_MIXED) {
        g_create_error = "bad precision";
        return MR_ERR_ARG;
    }
    mr_ctx *c = new mr_ctx;
    c->precision = precision;
    mr_instance_desc d{};
    d.Jmin = Jmin;
    d.Jmax = Jmax;
    d.gamma = gamma;
    d.mu_bar = mu_bar;
    d.bc = bc;
    d.eq = MR_EQ_ADVECTION;
    d.eps = eps;
    d.a = a;
    d.b = b;
    d.lambda = 1.0;
    d.s[0] = d.s[1] = d.s[2] = 1.0;
    int rc = check_desc(c, d, 0);
    if (rc) {
        g_create_error = c->err;
        delete c;
        return (mr_status)rc;
    }
    c->desc.push_back(d);
    c->scheme_set.push_back(false);
    *out = c;
    return MR_OK;
}

mr_status lbm_scheme(mr_ctx *c, int d, int q, double lambda, const double *s, int eq, const double *eq_params) {
    if (!c) return MR_ERR_ARG;
    if (c->bound) return (mr_status)c->fail(MR_ERR_STATE, "lbm_scheme after mr_bind");
    if (d != 1) return (mr_status)c->fail(MR_ERR_ARG, "only D = 1 is built");
    int nf = nfields_of(eq);
    if (nf == 0 || q != npop_of(eq))
        return (mr_status)c->fail(MR_ERR_ARG, "equilibrium %d needs q = %d (got %d)", eq, npop_of(eq), q);
    if (!s) return (mr_status)c->fail(MR_ERR_ARG, "relaxation rates missing");
    mr_instance_desc dd = c->desc[0];
    dd.eq = eq;
    dd.lambda = lambda;
    for (int j = 0; j < 3; ++j) dd.s[j] = j < nrates_of(eq) ? s[j] : 1.0;
    dd.eq_param = eq_params ? eq_params[0] : 0.0;
    if ((eq == MR_EQ_ADVECTION || eq == MR_EQ_SW_VEC || eq == MR_EQ_EULER_VEC || eq == MR_EQ_SW_D1Q3 ||
         eq == MR_EQ_SW_D1Q5) && !eq_params)
        return (mr_status)c->fail(MR_ERR_ARG, "equilibrium parameter missing");
    int rc = check_desc(c, dd, 0);
    if (rc) return (mr_status)rc;
    c->desc[0] = dd;
    c->scheme_set[0] = true;
    return MR_OK;
}

mr_status mr_batch_create(mr_ctx **out, const mr_instance_desc *desc, int n, int precision) {
    if (!out) return MR_ERR_ARG;
    *out = nullptr;
    if (!desc || n <= 0 || (precision != MR_FP64 && precision != MR_FP32_MIXED)) {
        g_create_error = "need n > 0 descriptors and a valid precision";
        return MR_ERR_ARG;
    }
    mr_ctx *c = new mr_ctx;
    c->precision = precision;
    for (int i = 0; i < n; ++i) {
        int rc = check_desc(c, desc[i], i);
        if (rc) {
            g_create_error = c->err;
            delete c;
            return (mr_status)rc;
        }
        c->desc.push_back(desc[i]);
        c->scheme_set.push_back(true);
    }
    *out = c;
    return MR_OK;
}

mr_status mr_workspace_size(const mr_ctx *cc, size_t *bytes) {
    mr_ctx *c = const_cast<mr_ctx *>(cc);
    if (!c || !bytes) return MR_ERR_ARG;
    for (int i = 0; i < c->n(); ++i)
        if (!c->scheme_set[i]) return (mr_status)c->fail(MR_ERR_STATE, "scheme of instance %d not set (lbm_scheme)", i);
    layout(c);
    *bytes = c->total;
    return MR_OK;
}

// Launch shape for the context's block size: shared-memory bitmasks of as many
// words as the largest instance needs, within a per-block budget (a lone
// instance may use most of the SM; a batch keeps several blocks resident), and
// one wave of resident blocks unless the caller fixed the grid.
static int configure(mr_ctx *c) {
    const size_t base = mrg_smem_bytes(c->fp32(), c->block, 0);
    for (int kind = 0; kind < NKIND; ++kind) {
        // the resident blocks a variant is compiled for share the SM's 227 KB
        const int minb = std::max(1, mrg_min_blocks(c->fp32(), c->block, kind));
        size_t budget = c->n() == 1 ? 220u * 1024u : (227u * 1024u) / (size_t)minb - 1024u;
        int fit = budget > base ? (int)((budget - base) / sizeof(uint32_t)) : 0;
        // the mask region of the largest instance when it fits (a batch keeps the
        // area for the instances that fit); a lone instance that does not fit
        // leaves it empty: shared memory is carved out of the SM's L1, which
        // keeps the population values between passes
        int mc = std::min(c->wmax, fit);
        if (c->n() == 1 && c->wmax > fit) mc = 0;
        c->mask_cap[kind] = mc;
        int nb = 0;
        int rc = c->cuda((cudaError_t)mrg_occupancy(c->fp32(), c->block, kind, mc, &nb), "occupancy");
        if (rc) return rc;
        c->grid[kind] = c->grid_req > 0 ? c->grid_req : std::max(1, nb) * c->sms;
    }
    return MR_OK;
}

// Processing order of the work queue: by kernel variant group (fast, scalar,
// general), then by field count (blocks resident together then run the same
// scheme's code, which keeps the instruction cache warm) unless disabled, then
// largest first (populations x 2^Jmax as the cost estimate).
static int upload_order(mr_ctx *c) {
    const int n = c->n();
    const std::vector<InstDesc> &dd = c->hdesc;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int gx = group_of(dd[x]), gy = group_of(dd[y]);
        if (gx != gy) return gx < gy;  // kernel variant groups
        const int vx = variant_of(dd[x].eq), vy = variant_of(dd[y].eq);
        if (c->order_by_fields && vx != vy) return vx > vy;
        double cx = (double)npop_of(dd[x].eq) * std::ldexp(1.0, dd[x].Jmax);
        double cy = (double)npop_of(dd[y].eq) * std::ldexp(1.0, dd[y].Jmax);
        return cx > cy;
    });
    c->order_host = order;
    for (int g = 0; g < NGROUP; ++g) c->n_group[g] = 0;
    bool scalar_only = true;  // every gamma = 1 leaves-collision instance has one field
    for (int i = 0; i < n; ++i) {
        ++c->n_group[group_of(dd[i])];
        if (group_of(dd[i]) == 3 && variant_of(dd[i].eq) != 1) scalar_only = false;
    }
    // A mixed group stays in one fast kernel: split into fast and scalar
    // kernels on two streams it ran 2 % faster or 5 % slower than one kernel,
    // depending on which kernel's blocks reached the SMs first.
    c->group_kind[3] = scalar_only ? K_SCALAR : K_FAST;
    return c->cuda(cudaMemcpyAsync(c->ws + c->off_order, c->order_host.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                                   c->stream),
                   "upload");
}

mr_status mr_bind(mr_ctx *c, void *ws, size_t bytes, void *stream) {
    if (!c || !ws) return MR_ERR_ARG;
    size_t need = 0;
    int rc = mr_workspace_size(c, &need);
    if (rc) return (mr_status)rc;
    if (bytes < need) return (mr_status)c->fail(MR_ERR_CAPACITY, "workspace of %zu bytes, need %zu", bytes, need);
    if (((uintptr_t)ws & 255u) != 0) return (mr_status)c->fail(MR_ERR_ARG, "workspace must be 256-byte aligned");
    c->ws = (unsigned char *)ws;
    c->ws_bytes = bytes;
    c->stream = (cudaStream_t)stream;
    int dev = 0;
    if ((rc = c->cuda(cudaGetDevice(&dev), "cudaGetDevice"))) return (mr_status)rc;
    if ((rc = c->cuda(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev), "attribute"))) return (mr_status)rc;
    if (!c->side) {
        if ((rc = c->cuda(cudaDeviceGetStreamPriorityRange(&c->prio_least, &c->prio_greatest),
                          "cudaDeviceGetStreamPriorityRange")) ||
            (rc = c->cuda(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "cudaStreamCreateWithFlags")) ||
            (rc = c->cuda(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "cudaEventCreateWithFlags")) ||
            (rc = c->cuda(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "cudaEventCreateWithFlags")))
            return (mr_status)rc;
    }
    // descriptors with absolute pointers
    int n = c->n();
    std::vector<InstDesc> dd = c->hdesc;
    for (int i = 0; i < n; ++i) {
        unsigned char *base = c->ws + c->inst_off[i];
        dd[i].V = base + (size_t)dd[i].V;
        dd[i].Phi = base + (size_t)dd[i].Phi;
        dd[i].masks = (uint32_t *)(base + (size_t)dd[i].masks);
        dd[i].lists = (uint32_t *)(base + (size_t)dd[i].lists);
        dd[i].st = (InstState *)(c->ws + c->off_state) + i;
    }
    // launch shape: one block per instance; 1024 threads for a lone large instance
    if (c->block == 0) {
        int jmax = 0;
        for (auto &d : c->desc) jmax = std::max(jmax, d.Jmax);
        c->block = n == 1 ? (jmax >= 12 ? 1024 : 512) : 256;
    }
    c->hdesc = dd;
    Tables<double> td;
    Tables<float> tf;
    make_tables(td, tf);
    cudaStream_t s = c->stream;
    if ((rc = c->cuda(cudaMemcpyAsync(c->ws + c->off_desc, dd.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, s), "upload")))
        return (mr_status)rc;
    if ((rc = c->cuda(cudaMemsetAsync(c->ws + c->off_state, 0, sizeof(InstState) * n, s), "memset"))) return (mr_status)rc;
    if ((rc = upload_order(c))) return (mr_status)rc;
    std::vector<int> ident(n);
    for (int i = 0; i < n; ++i) ident[i] = i;
    if ((rc = c->cuda(cudaMemcpyAsync(c->ws + c->off_ident, ident.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s), "upload")))
        return (mr_status)rc;
    if ((rc = c->cuda(cudaMemcpyAsync(c->ws + c->off_tab, &td, sizeof td, cudaMemcpyHostToDevice, s), "upload"))) return (mr_status)rc;
    if ((rc = c->cuda(cudaMemcpyAsync(c->ws + c->off_tab + sizeof td, &tf, sizeof tf, cudaMemcpyHostToDevice, s), "upload")))
        return (mr_status)rc;
    if ((rc = c->cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize"))) return (mr_status)rc;
    c->wmax = 0;
    for (int i = 0; i < n; ++i) c->wmax = std::max(c->wmax, (int)smem_region_words(dd[i].Wtot, dd[i].OW));
    if ((rc = configure(c))) return (mr_status)rc;
    c->bound = true;
    c->initialised = false;
    return MR_OK;
}

mr_status mr_set_initial(mr_ctx *c, const double *m, size_t count) {
    if (!c || !m) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "mr_set_initial before mr_bind");
    if (count != c->stage_doubles)
        return (mr_status)c->fail(MR_ERR_CAPACITY, "initial data has %zu values, expected %zu", count, c->stage_doubles);
    const void *src = m;
    if (!is_device_ptr(m)) {
        int rc = c->cuda(cudaMemcpyAsync(c->ws + c->off_stage, m, count * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                         "cudaMemcpyAsync");
        if (rc) return (mr_status)rc;
        src = c->ws + c->off_stage;
    }
    int rc = launch(c, PH_INIT_FULL, 0, -1, src, nullptr);
    if (rc) return (mr_status)rc;
    c->initialised = true;
    return MR_OK;
}

// Host-side check that a complete-tree membership is a sibling-closed graded
// tree (Def. Tree and Def. Graded tree with the instance's gamma) before a kernel reads it.
static int check_tree(mr_ctx *c, int inst, const unsigned char *Rd) {
    const mr_instance_desc &d = c->desc[inst];
    const InstDesc &h = c->hdesc[inst];
    std::vector<unsigned char> R(h.S);
    int rc = c->cuda(cudaMemcpy(R.data(), Rd, h.S, cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (rc) return rc;
    auto at = [&](int l, long long k) { return R[((1LL << l) - (1LL << d.Jmin)) + k] != 0; };
    for (long long k = 0; k < (1LL << d.Jmin); ++k)
        if (!at(d.Jmin, k)) return c->fail(MR_ERR_ARG, "tree: coarsest level must be whole");
    for (int l = d.Jmin + 1; l <= d.Jmax; ++l) {
        long long np = 1LL << (l - 1);
        for (long long k = 0; k < (1LL << l); ++k) {
            if (!at(l, k)) continue;
            if (!at(l, k ^ 1)) return c->fail(MR_ERR_ARG, "tree: cell (%d,%lld) without its sibling", l, k);
            for (int dd = -d.gamma; dd <= d.gamma; ++dd) {
                long long p = (k >> 1) + dd;
                if (d.bc == MR_BC_PERIODIC)
                    p = (p + np) % np;
                else if (p < 0 || p >= np)
                    continue;
                if (!at(l - 1, p)) return c->fail(MR_ERR_ARG, "tree: cell (%d,%lld) is not graded", l, k);
            }
        }
    }
    return MR_OK;
}

mr_status mr_set_state(mr_ctx *c, int inst, const unsigned char *R, const double *values) {
    if (!c || !R || !values || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "mr_set_state before mr_bind");
    int rc = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (rc) return (mr_status)rc;
    if ((rc = check_tree(c, inst, R))) return (mr_status)rc;
    rc = launch(c, PH_INIT_STATE, 0, inst, R, values);
    if (rc) return (mr_status)rc;
    c->initialised = true;
    return MR_OK;
}

mr_status mr_adapt(mr_ctx *c) {
    if (!c) return MR_ERR_ARG;
    if (!c->initialised) return (mr_status)c->fail(MR_ERR_STATE, "no initial state");
    return (mr_status)launch(c, PH_ADAPT, 1, -1, nullptr, nullptr);
}

mr_status lbm_step(mr_ctx *c) {
    if (!c) return MR_ERR_ARG;
    if (!c->initialised) return (mr_status)c->fail(MR_ERR_STATE, "no initial state");
    return (mr_status)launch(c, PH_STEP, 1, -1, nullptr, nullptr);
}

mr_status mr_advance(mr_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return MR_ERR_ARG;
    if (!c->initialised) return (mr_status)c->fail(MR_ERR_STATE, "no initial state");
    if (nsteps == 0) return MR_OK;
    return (mr_status)launch(c, PH_ADAPT | PH_STEP, nsteps, -1, nullptr, nullptr);
}

mr_status mr_sync(mr_ctx *c) {
    if (!c) return MR_ERR_ARG;
    int rc = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (rc) return (mr_status)rc;
    if (!c->bound) return MR_OK;
    std::vector<InstState> st(c->n());
    rc = c->cuda(cudaMemcpy(st.data(), c->ws + c->off_state, sizeof(InstState) * c->n(), cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (rc) return (mr_status)rc;
    for (int i = 0; i < c->n(); ++i)
        if (st[i].status & ST_NONFINITE) return (mr_status)c->fail(MR_ERR_NONFINITE, "instance %d: non-finite population", i);
    return MR_OK;
}

static int fetch_leaves(mr_ctx *c, int inst, std::vector<uint32_t> &ent, std::vector<double> &vals, InstState &st) {
    int rc = read_state(c, inst, &st);
    if (rc) return rc;
    if (st.status & ST_NONFINITE) return c->fail(MR_ERR_NONFINITE, "instance %d: non-finite population", inst);
    const InstDesc &h = c->hdesc[inst];
    int q = npop_of(h.eq);
    ent.resize(st.nleaf);
    if (st.nleaf)
        if ((rc = c->cuda(cudaMemcpy(ent.data(), h.lists + h.list_off[L_LEAF], sizeof(uint32_t) * st.nleaf, cudaMemcpyDeviceToHost), "copy")))
            return rc;
    size_t nv = (size_t)q * h.S;
    vals.resize(nv);
    if (c->fp32()) {
        std::vector<float> tmp(nv);
        if ((rc = c->cuda(cudaMemcpy(tmp.data(), h.V, sizeof(float) * nv, cudaMemcpyDeviceToHost), "copy"))) return rc;
        for (size_t i = 0; i < nv; ++i) vals[i] = tmp[i];
    } else {
        if ((rc = c->cuda(cudaMemcpy(vals.data(), h.V, sizeof(double) * nv, cudaMemcpyDeviceToHost), "copy"))) return rc;
    }
    return MR_OK;
}

mr_status mr_get_leaves(mr_ctx *c, int inst, int *level, long *index, double *f, long cap, long *count) {
    if (!c || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    std::vector<uint32_t> ent;
    std::vector<double> vals;
    InstState st;
    int rc = fetch_leaves(c, inst, ent, vals, st);
    if (rc) return (mr_status)rc;
    if (count) *count = st.nleaf;
    if ((level || index || f) && cap < st.nleaf) return (mr_status)c->fail(MR_ERR_CAPACITY, "need %d leaf slots", st.nleaf);
    const InstDesc &h = c->hdesc[inst];
    int q = npop_of(h.eq);
    for (int i = 0; i < st.nleaf; ++i) {
        int l = (int)(ent[i] >> KBITS);
        long k = (long)(ent[i] & KMASK);
        if (level) level[i] = l;
        if (index) index[i] = k;
        if (f) {
            long long cell = ((1LL << l) - (1LL << h.Jmin)) + k;
            for (int hh = 0; hh < q; ++hh) f[(long)hh * cap + i] = vals[(size_t)cell * q + hh];
        }
    }
    return MR_OK;
}

mr_status mr_get_moments(mr_ctx *c, int inst, double *m, long cap, long *count) {
    if (!c || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    std::vector<uint32_t> ent;
    std::vector<double> vals;
    InstState st;
    int rc = fetch_leaves(c, inst, ent, vals, st);
    if (rc) return (mr_status)rc;
    if (count) *count = st.nleaf;
    if (m && cap < st.nleaf) return (mr_status)c->fail(MR_ERR_CAPACITY, "need %d leaf slots", st.nleaf);
    const InstDesc &h = c->hdesc[inst];
    if (m)
        for (int i = 0; i < st.nleaf; ++i) {
            int l = (int)(ent[i] >> KBITS);
            long long cell = ((1LL << l) - (1LL << h.Jmin)) + (ent[i] & KMASK);
            if (h.eq == MR_EQ_SW_D1Q3 || h.eq == MR_EQ_SW_D1Q5) {
                const double w[5] = {0.0, 1.0, -1.0, 2.0, -2.0};
                double m0 = 0.0, m1 = 0.0;
                for (int hh = 0; hh < npop_of(h.eq); ++hh) {
                    const double f = vals[(size_t)cell * npop_of(h.eq) + hh];
                    m0 += f;
                    m1 += (w[hh] * h.lam) * f;
                }
                m[i] = m0;
                m[(long)cap + i] = m1;
            } else {
                for (int j = 0; j < h.nf; ++j)
                    m[(long)j * cap + i] = vals[(size_t)cell * npop_of(h.eq) + 2 * j] + vals[(size_t)cell * npop_of(h.eq) + 2 * j + 1];
            }
        }
    return MR_OK;
}

mr_status mr_get_finest(mr_ctx *c, int inst, double *out) {
    if (!c || !out || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    const InstDesc &h = c->hdesc[inst];
    bool dev = is_device_ptr(out);
    void *dst = dev ? (void *)out : (void *)(c->ws + c->off_stage);
    int rc = launch(c, PH_FINEST, 0, inst, dst, nullptr);
    if (rc) return (mr_status)rc;
    if (!dev) {
        rc = c->cuda(cudaMemcpyAsync(out, dst, sizeof(double) * h.nf * h.N, cudaMemcpyDeviceToHost, c->stream), "copy");
        if (rc) return (mr_status)rc;
    }
    rc = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return (mr_status)rc;
}

mr_status mr_get_tree(mr_ctx *c, int inst, unsigned char *R) {
    if (!c || !R || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    InstState st;
    int rc = read_state(c, inst, &st);
    if (rc) return (mr_status)rc;
    const InstDesc &h = c->hdesc[inst];
    std::vector<uint32_t> w(h.Wtot);
    if ((rc = c->cuda(cudaMemcpy(w.data(), h.masks + (size_t)st.cur * h.Wtot, sizeof(uint32_t) * h.Wtot, cudaMemcpyDeviceToHost), "copy")))
        return (mr_status)rc;
    int g = 0;
    for (int l = h.Jmin; l <= h.Jmax; ++l) {
        long long n = 1LL << l, base = (1LL << l) - (1LL << h.Jmin);
        for (long long k = 0; k < n; ++k) R[base + k] = (w[g + (k >> 5)] >> (k & 31)) & 1u;
        g += nwords_h(l);
    }
    return MR_OK;
}

mr_status mr_audit(mr_ctx *c, int inst, double *mass, double *residual) {
    if (!c || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    InstState st;
    int rc = read_state(c, inst, &st);
    if (rc) return (mr_status)rc;
    if (mass)
        for (int j = 0; j < c->hdesc[inst].nf; ++j) mass[j] = st.mass[j];
    if (residual) *residual = st.audit;
    return MR_OK;
}

mr_status mr_get_summary(mr_ctx *c, double *mass, int *nleaf) {
    if (!c) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    const unsigned char *base = c->ws + c->off_state;
    int rc;
    if (mass &&
        (rc = c->cuda(cudaMemcpy2DAsync(mass, 3 * sizeof(double), base + offsetof(InstState, mass), sizeof(InstState),
                                        3 * sizeof(double), c->n(), cudaMemcpyDeviceToHost, c->stream),
                      "cudaMemcpy2DAsync")))
        return (mr_status)rc;
    if (nleaf &&
        (rc = c->cuda(cudaMemcpy2DAsync(nleaf, sizeof(int), base + offsetof(InstState, nleaf), sizeof(InstState), sizeof(int),
                                        c->n(), cudaMemcpyDeviceToHost, c->stream),
                      "cudaMemcpy2DAsync")))
        return (mr_status)rc;
    return (mr_status)c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
}

mr_status mr_near_ties(mr_ctx *c, int inst, long long *count) {
    if (!c || !count || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    InstState st;
    int rc = read_state(c, inst, &st);
    if (rc) return (mr_status)rc;
    *count = st.near_ties;
    return MR_OK;
}

mr_status mr_step_passes(mr_ctx *c, int inst, unsigned long long *steps, unsigned long long *passes) {
    if (!c || inst < 0 || inst >= c->n()) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    InstState st;
    int rc = read_state(c, inst, &st);
    if (rc) return (mr_status)rc;
    if (steps) *steps = st.steps;
    if (passes) *passes = st.passes;
    return MR_OK;
}

mr_status mr_probe_latency(void *scratch, size_t bytes, void *stream, double *cycles) {
    if (!scratch || !cycles || bytes < 4096 || ((uintptr_t)scratch & 255u) != 0) {
        mrg_set_error("mr_probe_latency: need a 256-byte aligned scratch of at least 4096 bytes and an output");
        return MR_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long out[4] = {0, 0, 0, 0};
    int *buf = (int *)scratch;
    unsigned long long *res = (unsigned long long *)((unsigned char *)scratch + 2048);
    // fresh 128-byte lines after the first 4096 bytes, as many as fit (at most kProbeIters)
    const size_t nlines = bytes > kProbeFreshOff ? (bytes - kProbeFreshOff) / 128 : 0;
    const int nfresh = (int)(nlines < (size_t)kProbeIters ? nlines : (size_t)kProbeIters);
    int *fresh = (int *)((unsigned char *)scratch + kProbeFreshOff);
    cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, s);
    if (e == cudaSuccess) {
        mrg_probe<<<1, 256, 0, s>>>(buf, res, kProbeIters, fresh, nfresh);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, sizeof out, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        mrg_set_error(cudaGetErrorString(e));
        return MR_ERR_CUDA;
    }
    for (int i = 0; i < 3; ++i) cycles[i] = (double)out[i] / kProbeIters;
    cycles[3] = (double)out[3];
    return MR_OK;
}

mr_status mr_stats(mr_ctx *c, unsigned long long *updates, unsigned long long *steps, long long *leaves) {
    if (!c) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    int rc = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (rc) return (mr_status)rc;
    std::vector<InstState> st(c->n());
    rc = c->cuda(cudaMemcpy(st.data(), c->ws + c->off_state, sizeof(InstState) * c->n(), cudaMemcpyDeviceToHost), "copy");
    if (rc) return (mr_status)rc;
    unsigned long long u = 0;
    long long lv = 0;
    for (auto &s : st) {
        u += s.updates;
        lv += s.nleaf;
    }
    if (updates) *updates = u;
    if (steps) *steps = st[0].steps;
    if (leaves) *leaves = lv;
    return MR_OK;
}

mr_status mr_set_launch(mr_ctx *c, int block, int grid) {
    if (!c) return MR_ERR_ARG;
    if (block != 128 && block != 256 && block != 512 && block != 1024)
        return (mr_status)c->fail(MR_ERR_ARG, "block must be 128, 256, 512 or 1024");
    if (grid < 0) return (mr_status)c->fail(MR_ERR_ARG, "grid must be >= 0");
    c->block = block;
    c->grid_req = grid;
    if (c->bound) return (mr_status)configure(c);
    return MR_OK;
}

mr_status mr_set_collision(mr_ctx *c, int kind) {
    if (!c || (kind != MR_COLLIDE_LEAVES && kind != MR_COLLIDE_RECONSTRUCTED)) return MR_ERR_ARG;
    if (c->bound) return (mr_status)c->fail(MR_ERR_STATE, "mr_set_collision after mr_bind");
    for (auto &d : c->desc) d.collision = kind;
    return MR_OK;
}

mr_status mr_set_order(mr_ctx *c, int by_fields) {
    if (!c || (by_fields != 0 && by_fields != 1)) return MR_ERR_ARG;
    c->order_by_fields = by_fields != 0;
    if (c->bound) return (mr_status)upload_order(c);
    return MR_OK;
}

mr_status mr_autotune(mr_ctx *c, int nsteps, void *scratch, size_t scratch_bytes, int *best_block, int *best_order,
                      float *best_ms) {
    if (!c || nsteps < 1 || !scratch) return MR_ERR_ARG;
    if (!c->initialised) return (mr_status)c->fail(MR_ERR_STATE, "mr_autotune needs an initial state");
    if (scratch_bytes < c->total)
        return (mr_status)c->fail(MR_ERR_CAPACITY, "autotune scratch of %zu bytes, need %zu", scratch_bytes, c->total);
    cudaStream_t s = c->stream;
    int rc = c->cuda(cudaMemcpyAsync(scratch, c->ws, c->total, cudaMemcpyDeviceToDevice, s), "save state");
    if (rc) return (mr_status)rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = c->cuda(cudaEventCreate(&e0), "cudaEventCreate"))) return (mr_status)rc;
    if ((rc = c->cuda(cudaEventCreate(&e1), "cudaEventCreate"))) {
        cudaEventDestroy(e0);
        return (mr_status)rc;
    }
    // Only the block size is tuned.  The queue order is not: a trial's 64 steps
    // right after the initial state timed both orders alike on the mixed batch,
    // while over a thousand steps the order by scheme ran 7 % faster.
    const int blocks[4] = {128, 256, 512, 1024};
    const int block0 = c->block, grid0 = c->grid_req;
    int bb = block0;
    float bt = -1.0f;
    auto restore = [&]() { return c->cuda(cudaMemcpyAsync(c->ws, scratch, c->total, cudaMemcpyDeviceToDevice, s), "restore"); };
    for (int ib = 0; ib < 4 && !rc; ++ib) {
        c->block = blocks[ib];
        c->grid_req = 0;
        if ((rc = configure(c))) break;
        // untimed step first (first launch of a block size sets its attributes), then the trial
        if ((rc = restore()) || (rc = launch(c, PH_ADAPT | PH_STEP, 1, -1, nullptr, nullptr)) || (rc = restore())) break;
        if ((rc = c->cuda(cudaEventRecord(e0, s), "cudaEventRecord"))) break;
        if ((rc = launch(c, PH_ADAPT | PH_STEP, nsteps, -1, nullptr, nullptr))) break;
        if ((rc = c->cuda(cudaEventRecord(e1, s), "cudaEventRecord"))) break;
        if ((rc = c->cuda(cudaEventSynchronize(e1), "cudaEventSynchronize"))) break;
        float ms = 0.0f;
        if ((rc = c->cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime"))) break;
        if (bt < 0.0f || ms < bt) {
            bt = ms;
            bb = c->block;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the fastest shape (the caller's on failure) and the saved state
    c->block = rc ? block0 : bb;
    c->grid_req = rc ? grid0 : 0;
    int rc2 = configure(c);
    if (!rc2) rc2 = restore();
    if (!rc2) rc2 = c->cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (rc) return (mr_status)rc;
    if (rc2) return (mr_status)rc2;
    if (best_block) *best_block = bb;
    if (best_order) *best_order = c->order_by_fields ? 1 : 0;
    if (best_ms) *best_ms = bt;
    return MR_OK;
}

mr_status mr_reconstruction_coefficients(int dj, int kind, double *out) {
    if (!out || dj < 0 || dj > MAXDJ || kind < 0 || kind > 5) return MR_ERR_ARG;
    static Tables<double> td;
    static Tables<float> tf;
    static bool made = false;
    if (!made) {
        make_tables(td, tf);
        made = true;
    }
    const double *src = kind == 0 ? td.cf[dj] : kind == 1 ? td.t1[dj] : kind == 2 ? td.bf[dj]
                      : kind == 3 ? td.cf2[dj] : kind == 4 ? td.t12[dj] : td.bf2[dj];
    int n = (kind == 2 || kind == 5) ? 2 : 4;
    for (int j = 0; j < n; ++j) out[j] = src[j];
    return MR_OK;
}

mr_status mr_phase_times(mr_ctx *c, int inst, unsigned long long *cycles, int n) {
    if (!c || !cycles || inst < 0 || inst >= c->n() || n < NPHASE) return MR_ERR_ARG;
    if (!c->bound) return (mr_status)c->fail(MR_ERR_STATE, "not bound");
    InstState st;
    int rc = read_state(c, inst, &st);
    if (rc) return (mr_status)rc;
    for (int p = 0; p < NPHASE; ++p) cycles[p] = st.ptime[p];
#ifdef MRG_PHASE_TIMERS
    return MR_OK;
#else
    return (mr_status)c->fail(MR_ERR_STATE, "library built without phase timers (zeros returned)");
#endif
}

mr_status mr_info(const mr_ctx *c, int *n, long long *launches) {
    if (!c) return MR_ERR_ARG;
    if (n) *n = (int)c->desc.size();
    if (launches) *launches = c->launches;
    return MR_OK;
}

mr_status mr_last_error(const mr_ctx *c, char *buf, int len) {
    if (!buf || len <= 0) return MR_ERR_ARG;
    const std::string &s = c ? c->err : g_create_error;
    std::snprintf(buf, (size_t)len, "%s", s.c_str());
    return MR_OK;
}

mr_status mr_destroy(mr_ctx *c) {
    delete c;
    return MR_OK;
}

}  // extern "C"

// Reconstruction tables for other translation units of the library.
void mrg_tables(Tables<double> *td, Tables<float> *tf) { make_tables(*td, *tf); }
int mrg_nfields(int eq) { return nfields_of(eq); }
int mrg_npop(int eq) { return npop_of(eq); }
int mrg_nrates(int eq) { return nrates_of(eq); }
void mrg_dq_inverse(int eq, double lambda, double inv[5][5]) { dq_inverse(eq, lambda, inv); }

// Message reported by mr_last_error(NULL, ...) for calls without a context.
void mrg_set_error(const char *msg) { g_create_error = msg ? msg : ""; }

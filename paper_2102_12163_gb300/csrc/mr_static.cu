// mr_static.cu -- an entry point that needs no device allocation at all.
//
// Some callers cannot call cudaMalloc (or a framework allocator) at the point
// where they want to advance a problem: code running inside a memory budget
// that forbids new device allocations, plug-ins whose host application owns
// every device buffer, or runtimes where an allocation could block or trigger
// a device-wide synchronisation.  mr_run_static serves them: it runs one
// instance entirely inside a fixed scratch area that is part of the library
// image (a file-scope __device__ array), so the only device memory it touches
// is that area plus the caller's input and output buffers.  The paper has no
// counterpart; it is a deployment convenience.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mrlbm.h"
#include "mr_common.h"

using namespace mrg;

namespace {

// The scratch area.  Every GPU that loads the library keeps these bytes until
// the process exits; all calls share them (see mr_run_static in mrlbm.h).
static __device__ __align__(256) unsigned char g_scratch[MR_STATIC_SCRATCH_BYTES];

// Device address of g_scratch per device ordinal, looked up once per device
// with that device current.  In host code `g_scratch` only names a host-side
// stand-in, never the device memory, so it is never passed to a kernel.  The
// look-up is guarded by a mutex: host threads making their first call on a
// device at the same time see one look-up and the same address.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_scratch_dev[dev] = (unsigned char *)p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

// Host copies of the reconstruction tables, built on first use (a function-local
// static: its initialisation is thread-safe).
struct HostTables {
    Tables<double> td;
    Tables<float> tf;
    HostTables() { mrg_tables(&td, &tf); }
};
const HostTables &host_tables() {
    static const HostTables t;
    return t;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int nfields(int eq) { return mrg_nfields(eq); }

mr_status fail(mr_status code, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, b);
    mrg_set_error(buf);
    return code;
}

}  // namespace

extern "C" mr_status mr_run_static(const mr_instance_desc *desc, int precision, const double *m_cons, int nsteps,
                                   double *m_finest, unsigned long long *updates, void *stream) {
    if (!desc || !m_cons || !m_finest || nsteps < 0 || (precision != MR_FP64 && precision != MR_FP32_MIXED))
        return fail(MR_ERR_ARG, "mr_run_static: need a descriptor, input and output pointers, nsteps >= 0");
    const mr_instance_desc &d = *desc;
    const int nf = nfields(d.eq);
    if (d.Jmin < 2 || d.Jmax < d.Jmin || d.Jmax > MAXLEV || d.gamma < 1 || d.gamma > 3 || nf == 0 || d.mu_bar < 0 ||
        (d.bc != MR_BC_PERIODIC && d.bc != MR_BC_COPY) || !(d.eps >= 0.0) || !(d.b > d.a) || !(d.lambda >= 0x1p-16 && d.lambda <= 0x1p16))
        return fail(MR_ERR_ARG, "mr_run_static: invalid instance description");
    for (int j = 0; j < mrg_nrates(d.eq); ++j)
        if (!(d.s[j] > 0.0 && d.s[j] <= 2.0)) return fail(MR_ERR_ARG, "mr_run_static: relaxation rate outside (0, 2]");
    if (d.collision != MR_COLLIDE_LEAVES && d.collision != MR_COLLIDE_RECONSTRUCTED)
        return fail(MR_ERR_ARG, "mr_run_static: collision must be 0 or 1");
    if ((d.eq == MR_EQ_SW_D1Q3 || d.eq == MR_EQ_SW_D1Q5) && d.gamma != 1)
        return fail(MR_ERR_ARG, "mr_run_static: the D1Q3 / D1Q5 schemes are built with gamma = 1");
    const bool fp32 = precision == MR_FP32_MIXED;
    cudaStream_t s = (cudaStream_t)stream;
    // The descriptor is uploaded from host memory that does not outlive this
    // call, and `updates` waits for the stream: neither belongs in a graph.
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess) return fail(MR_ERR_CUDA, "mr_run_static: cudaStreamIsCapturing failed (%lld)", (long long)e);
        if (cs != cudaStreamCaptureStatusNone)
            return fail(MR_ERR_STATE, "mr_run_static: the stream is capturing; this call cannot be recorded in a graph");
    }

    // layout of the scratch area for this instance (same regions as a bound context)
    const int q = mrg_npop(d.eq);
    const long long S = (1LL << (d.Jmax + 1)) - (1LL << d.Jmin), N = 1LL << d.Jmax;
    int W = 0, OW = 0;
    for (int l = d.Jmin; l <= d.Jmax; ++l) {
        W += l >= 5 ? (1 << (l - 5)) : 1;
        OW += occ_words_of(l);
    }
    const long long region = mask_region_words(W, OW);
    const size_t vb = fp32 ? 4 : 8;
    size_t o = 0;
    const size_t oDesc = o;
    o = align256(o + sizeof(InstDesc));
    const size_t oState = o;
    o = align256(o + sizeof(InstState));
    const size_t oQueue = o;  // queue counter, then the processing order
    o = align256(o + 2 * sizeof(int));
    const size_t oTab = o;
    o = align256(o + sizeof(Tables<double>) + sizeof(Tables<float>));
    const size_t oV = o;
    o = align256(o + vb * q * S);
    const size_t oPhi = o;
    o = align256(o + vb * q * (N + 1));
    const size_t oM = o;
    o = align256(o + sizeof(uint32_t) * (size_t)region);
    const size_t oL = o;
    long long lo = 0, list_off[NLIST];
    for (int L = 0; L < NLIST; ++L) {
        list_off[L] = lo;
        lo += (S + 63) / 64 * 64;
    }
    o = align256(o + sizeof(uint32_t) * lo);
    if (o > (size_t)MR_STATIC_SCRATCH_BYTES)
        return fail(MR_ERR_CAPACITY, "mr_run_static: instance needs %lld scratch bytes, the static area holds %lld",
                    (long long)o, (long long)MR_STATIC_SCRATCH_BYTES);

    // set-up, once per device with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(MR_ERR_CUDA, "mr_run_static: no usable current device");
    unsigned char *base = nullptr;
    {
        const cudaError_t e = scratch_address(dev, &base);
        if (e != cudaSuccess) return fail(MR_ERR_CUDA, "mr_run_static: cudaGetSymbolAddress failed (%lld)", (long long)e);
    }

    // descriptor with absolute pointers into the scratch area
    InstDesc h;
    std::memset(&h, 0, sizeof h);
    h.Jmin = d.Jmin;
    h.Jmax = d.Jmax;
    h.bc = d.bc;
    h.eq = d.eq;
    h.nf = nf;
    if (d.eq == MR_EQ_SW_D1Q3 || d.eq == MR_EQ_SW_D1Q5) mrg_dq_inverse(d.eq, d.lambda, h.minv);
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
    h.m_off = 0;
    h.V = base + oV;
    h.Phi = base + oPhi;
    h.masks = (uint32_t *)(base + oM);
    h.lists = (uint32_t *)(base + oL);
    for (int L = 0; L < NLIST; ++L) h.list_off[L] = list_off[L];
    h.st = (InstState *)(base + oState);
    const Tables<double> &td = host_tables().td;
    const Tables<float> &tf = host_tables().tf;
    // Pageable host sources: cudaMemcpyAsync returns once they are staged, so
    // the stack copies may go out of scope afterwards.  The state and the queue
    // must start at zero; every other byte the kernel reads it writes first.
    int zero2[2] = {0, 0};
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + oDesc, &h, sizeof h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + oState, 0, sizeof(InstState), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + oQueue, zero2, sizeof zero2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + oTab, &td, sizeof td, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + oTab + sizeof td, &tf, sizeof tf, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(MR_ERR_CUDA, "mr_run_static: upload failed (%lld)", (long long)e);

    // one block for the instance, bitmasks in shared memory when they fit
    const int block = d.Jmax >= 12 ? 1024 : 512;
    size_t sbase = mrg_smem_bytes(fp32, block, 0), limit = 220u * 1024u;
    long long fit = limit > sbase ? (long long)((limit - sbase) / sizeof(uint32_t)) : 0;
    LaunchArgs a;
    std::memset(&a, 0, sizeof a);
    a.descs = (const InstDesc *)(base + oDesc);
    a.order = (const int *)(base + oQueue) + 1;  // the single instance, index 0
    a.n = 1;
    a.queue = (int *)(base + oQueue);
    a.tables = base + oTab + (fp32 ? sizeof(Tables<double>) : 0);
    const long long sregion = smem_region_words(W, OW);
    a.smem_mask_words = sregion <= fit ? (int)sregion : 0;
    a.kind = d.gamma > 1 ? K_GENERAL : d.collision != 0 ? K_RECOLL : W >= CW_MIN_WORDS ? K_LARGE : K_FAST;
    const int phases[3] = {PH_INIT_FULL, PH_ADAPT | PH_STEP, PH_FINEST};
    const int steps[3] = {0, nsteps, 0};
    for (int i = 0; i < 3; ++i) {
        if (i == 1 && nsteps == 0) continue;
        a.phases = phases[i];
        a.nsteps = steps[i];
        a.aux0 = i == 0 ? (const void *)m_cons : i == 2 ? (const void *)m_finest : nullptr;
        if ((e = cudaMemsetAsync(a.queue, 0, sizeof(int), s)) != cudaSuccess)
            return fail(MR_ERR_CUDA, "mr_run_static: queue reset failed (%lld)", (long long)e);
        int rc = mrg_launch(fp32, block, 1, a, s, 0);
        if (rc) return fail(MR_ERR_CUDA, "mr_run_static: kernel launch failed (%lld)", (long long)rc);
    }
    if (updates) {
        InstState st;
        if ((e = cudaMemcpyAsync(&st, base + oState, sizeof st, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(MR_ERR_CUDA, "mr_run_static: reading the counters failed (%lld)", (long long)e);
        if (st.status & ST_NONFINITE) return fail(MR_ERR_NONFINITE, "mr_run_static: non-finite population");
        *updates = st.updates;
    }
    return MR_OK;
}

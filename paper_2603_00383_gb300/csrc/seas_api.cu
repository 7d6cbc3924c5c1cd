// Host side of the C ABI (include/seas.h): handles, validation, network geometry, fault-wise cluster trees and the
// dual-tree traversal of the selective H-matrix (Sec. 2.3.2), causal windows, the device build of the operator, and
// the per-step call sequence.
#include "seas.h"
#include "seas_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

using namespace seas;

namespace {

thread_local std::string g_err;

seas_status fail(seas_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return fail(SEAS_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));          \
        }                                                                                     \
    } while (0)

#define SEAS_TRY(expr)                 \
    do {                               \
        seas_status s_ = (expr);       \
        if (s_ != SEAS_OK) return s_;  \
    } while (0)

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int64_t kChunkEntries = 48 << 20;   // kernel entries materialised per build chunk
constexpr int kDefaultMaxBlock = 64;          // largest side of an admissible block when hp->max_block == 0

}  // namespace

// ------------------------------------------------------------------------------------------------------------
// handles
// ------------------------------------------------------------------------------------------------------------

struct seas_ctx {
    int device = 0;
    int n_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    size_t used = 0;
    int children = 0;
};

namespace {

seas_status dev_alloc(seas_ctx *c, size_t bytes, void **p) {
    *p = nullptr;
    if (bytes == 0) return SEAS_OK;
    if (c->budget && c->used + bytes > c->budget)
        return fail(SEAS_ENOMEM, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu used)", bytes, c->used,
                    c->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SEAS_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->used += bytes;
    return SEAS_OK;
}

void dev_free(seas_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->used -= bytes;
}

// Device array owned by a context.
template <class T>
struct DArr {
    seas_ctx *ctx = nullptr;
    T *p = nullptr;
    size_t n = 0;
    DArr() = default;
    DArr(const DArr &) = delete;
    DArr &operator=(const DArr &) = delete;
    ~DArr() { release(); }
    seas_status alloc(seas_ctx *c, size_t count) {
        release();
        ctx = c;
        void *q = nullptr;
        SEAS_TRY(dev_alloc(c, count * sizeof(T), &q));
        p = static_cast<T *>(q);
        n = count;
        return SEAS_OK;
    }
    seas_status upload(seas_ctx *c, const std::vector<T> &v) {
        SEAS_TRY(alloc(c, v.size()));
        if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return SEAS_OK;
    }
    seas_status zero(cudaStream_t s) {
        if (n) CUDA_TRY(cudaMemsetAsync(p, 0, n * sizeof(T), s));
        return SEAS_OK;
    }
    void release() {
        if (p && ctx) dev_free(ctx, p, n * sizeof(T));
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// Pinned host buffer.
struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~HostBuf() {
        if (p) cudaFreeHost(p);
    }
    seas_status alloc(size_t b) {
        if (b == 0) return SEAS_OK;
        CUDA_TRY(cudaMallocHost(&p, b));
        bytes = b;
        return SEAS_OK;
    }
};

// Fault sizes the FFT handles: products of the radices 2, 3, 5, 7, 11, 13, 17, 19 and 23.
bool is_fft_size(int n) {
    if (n < 1) return false;
    for (int f : {2, 3, 5, 7, 11, 13, 17, 19, 23})
        while (n % f == 0) n /= f;
    return n == 1;
}

bool is_fin(double v) { return std::isfinite(v); }

}  // namespace

struct seas_net {
    seas_ctx *ctx = nullptr;
    std::vector<seas_fault> faults;
    seas_medium med{};
    double dt = 0.0;
    int N = 0, F = 0;
    // SEAS_FAULT_SURFACE_START (method of images): the network holds the doubled faults; the caller's vectors hold
    // the N_io real elements, io_map[i] = the real element of element i (-1 - j where i is the image of j)
    bool images = false;
    int N_io = 0;
    std::vector<int32_t> io_map;
    DArr<int32_t> d_io_map;
    std::vector<int> off;                       // F + 1
    std::vector<double> x, y, e1x, e1y, nx, ny, ds;
    std::vector<int> fault_of;
    DArr<double2> d_x, d_e1, d_n;
    DArr<double> d_ds;
    int children = 0;
};

struct StoredSlice {                 // one nonzero (block, lag) slice of the operator
    int32_t block, T, k;             // k < 0 dense, k > 0 rank
    const double *data;
};

struct seas_op {
    seas_net *net = nullptr;
    seas_hparams hp{};
    int children = 0;
    // spectral self effect
    std::vector<char> owned;         // per fault: 1 if its receivers belong to this operator (all unless partial)
    std::vector<FaultDev> faults_h;  // the owned faults (the spectral self effect runs on these)
    std::vector<ModeDev> modes_h;
    std::vector<int32_t> mode_W;     // per fault, modes 0..N_f
    DArr<FaultDev> d_faults;
    DArr<int32_t> d_big;             // owned faults whose FFTs run on a thread-block cluster
    int n_big = 0;
    DArr<ModeDev> d_modes;
    DArr<double> d_w;
    DArr<double2> d_tw;
    int n_modes_total = 0, max_nf = 0;
    // space-time interaction
    std::vector<BlockDev> blocks_h;
    std::vector<int32_t> block_far, block_pair;
    DArr<BlockDev> d_blocks;
    std::vector<std::unique_ptr<DArr<unsigned char>>> arena;
    DArr<ItemDev> d_items;
    DArr<TaskDev> d_tasks;
    std::vector<int32_t> task_T;     // T_start of each task (ascending)
    // pass 1 (source side of the far blocks)
    DArr<unsigned char> d_varena;    // V^T rows, source cluster-major
    DArr<RunDev> d_runs;
    DArr<TaskDev> d_ztasks;
    DArr<SrcDev> d_srcs;
    DArr<int32_t> d_zmap;
    DArr<float> d_zscale;
    std::vector<int32_t> ztask_T;    // T_start of each pass-1 task (ascending)
    int64_t z_rows = 0;              // rows of the z buffer (rows of the receiver-side arena)
    int64_t n_partial = 0;           // partial-sum slots (rows) over all tasks
    int max_q = 0;                   // widest block (source columns)
    DArr<int32_t> d_cover_ptr, d_cover_blk, d_blk_task_ptr, d_blk_task_T;
    DArr<int64_t> d_blk_part;
    std::vector<int32_t> pair_last;  // [F][F]
    std::vector<int32_t> block_lo, block_hi;  // window of each block (first and last lag)
    std::vector<int64_t> bytes_upto; // stored interaction bytes with lag <= T
    int ring = 1;
    // static tail (SEAS_FLAG_STATIC_TAIL)
    bool tail = false;
    DArr<double> d_smat;             // [N][N] -(mu / 2 c_s) A^static
    DArr<int32_t> d_block_last;      // with cluster-level windows: each block's last lag
    DArr<int32_t> d_pair_last;
    seas_op_stats stats{};
};

struct seas_scn {
    seas_op *op = nullptr;
    int B = 0;
    int64_t n = 0;                   // pushes so far (ticks)
    std::vector<int64_t> start;      // per member: tick of its first push (0 unless admitted later)
    std::vector<char> active;        // per member: 1 while admitted
    int64_t horizon = -1;            // largest lag the interaction has switched on (non-decreasing)
    int last_gamma = 1;              // lattice steps of the last push (seas_push_slip_rate_steps)
    // captured step (seas_scenario_graph_create): the graph, its per-step values on the device, and a pinned ring
    // of host copies the asynchronous uploads read from
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    DArr<DynDev> d_dyn;
    HostBuf h_dyn;
    int64_t dyn_used = 0;
    cudaEvent_t dyn_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    DArr<unsigned char> zbuf;        // pass-1 output: [z rows][batch] in the dot type of the precision
    DArr<double> vring, slip, slip_prev, fint, d_V, d_slip, d_tau, d_parts, partial;
    DArr<double> sring;              // static tail: slip after each push, [op->ring + 1][N][B]
    DArr<unsigned char> xring;       // history in the operator's arithmetic (DF64: float2, BF16/FP16: float)
    DArr<double2> dring, fmodes;
    DArr<int> counter_err;           // [0], [2]: task counters of the two interaction passes, [1]: device error word
    uint64_t wait_ns = 2000000000ull;   // bound of one device wait (seas_scenario_set_wait_limit)
    int cw[2] = {0, 0};              // consumer warps of the interaction passes (seas_scenario_autotune; 0: default)
    // side stream of the self-term convolution, forked from and joined back to the step's stream
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    int64_t ring_stride = 0;
    DArr<FaultDev> faults;           // fault table with spectral-ring offsets for this batch size
    int64_t dring_len = 0;
    HostBuf h_in, h_out;
    // kernel timing (seas_scenario_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev;     // pairs (start, stop)
    std::vector<int> ev_class;
    size_t ev_used = 0;
    seas_timing acc{};
    ~seas_scn() {
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (join_ev) cudaEventDestroy(join_ev);
        if (side) cudaStreamDestroy(side);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaEvent_t e : dyn_ev)
            if (e) cudaEventDestroy(e);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
    }
};

// ------------------------------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------------------------------

extern "C" seas_status seas_create(seas_ctx **out, int device, size_t hbm_budget, void *cuda_stream) {
    if (!out) return fail(SEAS_EINVAL, "ctx pointer is NULL");
    *out = nullptr;
    int count = 0;
    CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(SEAS_EINVAL, "device %d out of range (%d devices)", device, count);
    CUDA_TRY(cudaSetDevice(device));
    auto c = std::make_unique<seas_ctx>();
    c->device = device;
    c->budget = hbm_budget;
    CUDA_TRY(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device));
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    *out = c.release();
    return SEAS_OK;
}

extern "C" seas_status seas_ctx_get_memory(const seas_ctx *c, size_t *used, size_t *budget) {
    if (!c) return fail(SEAS_EINVAL, "ctx is NULL");
    if (used) *used = c->used;
    if (budget) *budget = c->budget;
    return SEAS_OK;
}

extern "C" seas_status seas_sync(seas_ctx *c) {
    if (!c) return fail(SEAS_EINVAL, "ctx is NULL");
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SEAS_OK;
}

// Status of the device error word: 1 = a bounded wait ran out, 2 = the interaction kernel was launched with less
// shared memory than its layout needs (an internal error; the kernel returned before touching shared memory).
static seas_status device_error_status(int err) {
    if (err == 1) return fail(SEAS_ETIMEOUT, "a bounded device wait ran out in the interaction kernel");
    if (err == 3) return fail(SEAS_ECUDA, "interaction unit larger than a pipeline stage (internal error)");
    if (err) return fail(SEAS_ECUDA, "interaction kernel launched with too little shared memory (error word %d)", err);
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_check(seas_scn *s) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    CUDA_TRY(cudaSetDevice(s->op->net->ctx->device));
    CUDA_TRY(cudaStreamSynchronize(s->op->net->ctx->stream));
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, s->counter_err.p + 1, sizeof(int), cudaMemcpyDeviceToHost));
    return device_error_status(err);
}

extern "C" seas_status seas_destroy_ctx(seas_ctx *c) {
    if (!c) return SEAS_OK;
    if (c->children) return fail(SEAS_EBUSY, "context has %d live networks", c->children);
    cudaSetDevice(c->device);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return SEAS_OK;
}

extern "C" const char *seas_strerror(seas_status s) {
    switch (s) {
        case SEAS_OK: return "ok";
        case SEAS_EINVAL: return "invalid argument";
        case SEAS_ENOMEM: return "out of device memory or over the HBM budget";
        case SEAS_ECUDA: return "CUDA error";
        case SEAS_ESTATE: return "call out of order";
        case SEAS_EBUSY: return "handle has live children";
        case SEAS_ETIMEOUT: return "device wait timed out";
        case SEAS_EIO: return "checkpoint I/O error";
        default: return "unknown status";
    }
}

extern "C" const char *seas_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------------------------------------------------
// network (Sec. 3.1 frames, Sec. 2.3.1 discretisation)
// ------------------------------------------------------------------------------------------------------------

namespace {

double seg_point_dist(double px, double py, double ax, double ay, double bx, double by) {
    const double ux = bx - ax, uy = by - ay;
    const double L2 = ux * ux + uy * uy;
    double t = L2 > 0 ? ((px - ax) * ux + (py - ay) * uy) / L2 : 0.0;
    t = std::min(1.0, std::max(0.0, t));
    return std::hypot(ax + t * ux - px, ay + t * uy - py);
}

}  // namespace

namespace {

// Method of images (App. B): every fault's start end lies on one traction-free surface normal to the parallel
// faults.  Each fault is replaced by its continuation across the surface, centred at the start end, of twice the
// length and element count; element N_f + j of the doubled fault is real element j, element N_f - 1 - j its image.
seas_status image_faults(const seas_fault *faults, int n_faults, std::vector<seas_fault> &doubled) {
    int flagged = 0;
    for (int f = 0; f < n_faults; ++f) {
        if (faults[f].flags & ~SEAS_FAULT_SURFACE_START)
            return fail(SEAS_EINVAL, "fault %d: unknown flags 0x%x", f, faults[f].flags);
        flagged += (faults[f].flags & SEAS_FAULT_SURFACE_START) ? 1 : 0;
    }
    if (flagged == 0) return SEAS_OK;
    if (flagged != n_faults)
        return fail(SEAS_EINVAL, "%d of %d faults on the free surface: with images every fault starts on it", flagged,
                    n_faults);
    const double c0 = std::cos(faults[0].strike_rad), s0 = std::sin(faults[0].strike_rad);
    double scale = 0.0;
    for (int f = 0; f < n_faults; ++f) scale = std::max(scale, std::fabs(faults[f].length));
    const double x0 = faults[0].cx - 0.5 * faults[0].length * c0, y0 = faults[0].cy - 0.5 * faults[0].length * s0;
    doubled.assign(faults, faults + n_faults);
    for (int f = 0; f < n_faults; ++f) {
        const seas_fault &F = faults[f];
        const double c1 = std::cos(F.strike_rad), s1 = std::sin(F.strike_rad);
        if (c1 * c0 + s1 * s0 < 1.0 - 1e-12)
            return fail(SEAS_EINVAL, "fault %d is not parallel to fault 0 with the same orientation (images)", f);
        const double xs = F.cx - 0.5 * F.length * c1, ys = F.cy - 0.5 * F.length * s1;
        if (std::fabs((xs - x0) * c0 + (ys - y0) * s0) > 1e-9 * scale)
            return fail(SEAS_EINVAL, "fault %d: its start end is off the free surface through fault 0's", f);
        if (F.n_elem > (1 << 30)) return fail(SEAS_EINVAL, "fault %d: n_elem too large", f);
        doubled[f].cx = xs;
        doubled[f].cy = ys;
        doubled[f].length = 2.0 * F.length;
        doubled[f].n_elem = 2 * F.n_elem;
        doubled[f].flags = 0;
    }
    return SEAS_OK;
}

// Host geometry of a network (validation, centroids, frames, dt); no device work.
seas_status make_geometry(const seas_fault *faults_in, int n_faults, const seas_medium *med, seas_net &net) {
    if (!faults_in || !med) return fail(SEAS_EINVAL, "NULL argument");
    if (n_faults < 1) return fail(SEAS_EINVAL, "n_faults must be >= 1");
    if (!(is_fin(med->mu) && med->mu > 0 && is_fin(med->cs) && med->cs > 0 && is_fin(med->beta) && med->beta > 0 &&
          is_fin(med->cp)))
        return fail(SEAS_EINVAL, "medium: mu, cs, beta must be finite and > 0");
    for (int f = 0; f < n_faults; ++f) {
        const seas_fault &F = faults_in[f];
        if (!(is_fin(F.cx) && is_fin(F.cy) && is_fin(F.strike_rad) && is_fin(F.length) && F.length > 0))
            return fail(SEAS_EINVAL, "fault %d: non-finite or non-positive geometry", f);
        if (F.n_elem < 1) return fail(SEAS_EINVAL, "fault %d: n_elem %d < 1", f, F.n_elem);
    }
    std::vector<seas_fault> doubled;
    SEAS_TRY(image_faults(faults_in, n_faults, doubled));
    net.images = !doubled.empty();
    const seas_fault *faults = net.images ? doubled.data() : faults_in;
    int64_t N = 0;
    for (int f = 0; f < n_faults; ++f) {
        const seas_fault &F = faults[f];
        if (!(is_fin(F.cx) && is_fin(F.cy) && is_fin(F.strike_rad) && is_fin(F.length) && F.length > 0))
            return fail(SEAS_EINVAL, "fault %d: non-finite or non-positive geometry", f);
        const char *with = net.images ? " (with its image across the free surface)" : "";
        if (F.n_elem < 1 || F.n_elem > kMaxFFT)
            return fail(SEAS_EINVAL, "fault %d: n_elem %d%s outside [1, %d]", f, F.n_elem, with, kMaxFFT);
        if (!is_fft_size(F.n_elem))
            return fail(SEAS_EINVAL, "fault %d: n_elem %d%s has a prime factor > 23 (FFT radices are the primes <= 23)",
                        f, F.n_elem, with);
        N += F.n_elem;
    }
    if (N > (1 << 24)) return fail(SEAS_EINVAL, "too many elements (%lld)", (long long)N);
    net.faults.assign(faults, faults + n_faults);
    net.med = *med;
    net.F = n_faults;
    net.N = (int)N;
    net.off.assign(n_faults + 1, 0);
    double min_ds = INFINITY;
    for (int f = 0; f < n_faults; ++f) {
        const seas_fault &F = faults[f];
        const double ds = F.length / F.n_elem;
        min_ds = std::min(min_ds, ds);
        const double c1 = std::cos(F.strike_rad), s1 = std::sin(F.strike_rad);
        for (int j = 0; j < F.n_elem; ++j) {
            const double s = -0.5 * F.length + (j + 0.5) * ds;
            net.x.push_back(F.cx + s * c1);
            net.y.push_back(F.cy + s * s1);
            net.e1x.push_back(c1);
            net.e1y.push_back(s1);
            net.nx.push_back(s1);
            net.ny.push_back(-c1);
            net.ds.push_back(ds);
            net.fault_of.push_back(f);
        }
        net.off[f + 1] = net.off[f] + F.n_elem;
    }
    net.dt = med->beta * min_ds / med->cs;
    net.N_io = net.images ? net.N / 2 : net.N;
    if (net.images) {
        net.io_map.resize((size_t)net.N);
        for (int f = 0; f < n_faults; ++f) {
            const int n = faults_in[f].n_elem, o = net.off[f], o_io = net.off[f] / 2;
            for (int j = 0; j < n; ++j) {
                net.io_map[(size_t)(o + n + j)] = o_io + j;
                net.io_map[(size_t)(o + n - 1 - j)] = -1 - (o_io + j);
            }
        }
    }
    // A receiver centroid on (or numerically at) another fault's element makes the kernel singular.
    for (int a = 0; a < n_faults; ++a) {
        for (int b = 0; b < n_faults; ++b) {
            if (a == b) continue;
            const seas_fault &Fb = faults[b];
            const double hx = 0.5 * Fb.length * std::cos(Fb.strike_rad), hy = 0.5 * Fb.length * std::sin(Fb.strike_rad);
            const double dsb = Fb.length / Fb.n_elem;
            for (int i = net.off[a]; i < net.off[a + 1]; ++i) {
                const double d = seg_point_dist(net.x[i], net.y[i], Fb.cx - hx, Fb.cy - hy, Fb.cx + hx, Fb.cy + hy);
                if (d < 1e-6 * dsb)
                    return fail(SEAS_EINVAL, "element %d of fault %d lies on fault %d (distance %g m)", i - net.off[a],
                                a, b, d);
            }
        }
    }
    return SEAS_OK;
}

}  // namespace

extern "C" seas_status seas_build_network(seas_ctx *c, const seas_fault *faults, int n_faults,
                                          const seas_medium *med, seas_net **out) {
    if (!c || !out) return fail(SEAS_EINVAL, "NULL argument");
    *out = nullptr;
    auto net = std::make_unique<seas_net>();
    SEAS_TRY(make_geometry(faults, n_faults, med, *net));
    CUDA_TRY(cudaSetDevice(c->device));
    net->ctx = c;
    const int64_t N = net->N;
    std::vector<double2> hx(N), he(N), hn(N);
    for (int64_t i = 0; i < N; ++i) {
        hx[i] = make_double2(net->x[i], net->y[i]);
        he[i] = make_double2(net->e1x[i], net->e1y[i]);
        hn[i] = make_double2(net->nx[i], net->ny[i]);
    }
    SEAS_TRY(net->d_x.upload(c, hx));
    SEAS_TRY(net->d_e1.upload(c, he));
    SEAS_TRY(net->d_n.upload(c, hn));
    SEAS_TRY(net->d_ds.upload(c, net->ds));
    if (net->images) SEAS_TRY(net->d_io_map.upload(c, net->io_map));
    c->children++;
    *out = net.release();
    return SEAS_OK;
}

extern "C" seas_status seas_net_get_info(const seas_net *net, seas_net_info *info) {
    if (!net || !info) return fail(SEAS_EINVAL, "NULL argument");
    info->dt = net->dt;
    info->n_faults = net->F;
    info->n_elem = net->N_io;
    return SEAS_OK;
}

extern "C" seas_status seas_net_get_elements(const seas_net *net, double *centroids, double *normals) {
    if (!net) return fail(SEAS_EINVAL, "NULL network");
    for (int k = 0; k < net->N; ++k) {
        const int i = net->images ? net->io_map[(size_t)k] : k;   // the caller's real elements only
        if (i < 0) continue;
        if (centroids) {
            centroids[2 * i] = net->x[k];
            centroids[2 * i + 1] = net->y[k];
        }
        if (normals) {
            normals[2 * i] = net->nx[k];
            normals[2 * i + 1] = net->ny[k];
        }
    }
    return SEAS_OK;
}

extern "C" seas_status seas_destroy_net(seas_net *net) {
    if (!net) return SEAS_OK;
    if (net->children) return fail(SEAS_EBUSY, "network has %d live operators", net->children);
    cudaSetDevice(net->ctx->device);
    net->ctx->children--;
    delete net;
    return SEAS_OK;
}

// ------------------------------------------------------------------------------------------------------------
// operator build
// ------------------------------------------------------------------------------------------------------------

namespace {

// Cluster of one fault-wise binary tree (Sec. 2.3.2): elements [a, b), bounding circle of centre c (mean of
// the centroids) and radius max ||x - c|| + ds / 2.
struct Cluster {
    int a, b;
    double cx, cy, r;
    int left = -1, right = -1;
    bool leaf() const { return left < 0; }
};

int build_tree(const seas_net &net, int f, int lo, int hi, int leaf, std::vector<Cluster> &t) {
    Cluster c;
    c.a = lo;
    c.b = hi;
    double sx = 0, sy = 0;
    for (int i = lo; i < hi; ++i) {
        sx += net.x[i];
        sy += net.y[i];
    }
    c.cx = sx / (hi - lo);
    c.cy = sy / (hi - lo);
    double r = 0;
    for (int i = lo; i < hi; ++i) r = std::max(r, std::hypot(net.x[i] - c.cx, net.y[i] - c.cy) + 0.5 * net.ds[i]);
    c.r = r;
    const int idx = (int)t.size();
    t.push_back(c);
    if (hi - lo > leaf) {
        const int mid = lo + (hi - lo + 1) / 2;     // odd counts: the left child takes the extra element
        const int l = build_tree(net, f, lo, mid, leaf, t);
        const int rr = build_tree(net, f, mid, hi, leaf, t);
        t[idx].left = l;
        t[idx].right = rr;
    }
    return idx;
}

// Dual-tree traversal (Sec. 2.3.2): admissible pairs become far blocks; inadmissible leaf pairs near blocks;
// otherwise the cluster with the larger radius is split (the other one if it is a leaf; the receiver on a tie).
void traverse(const std::vector<Cluster> &ta, const std::vector<Cluster> &tb, double eta, bool dense, int max_block,
              int pair, std::vector<BlockDev> &blocks, std::vector<int32_t> &far, std::vector<int32_t> &pairs) {
    std::vector<std::pair<int, int>> st{{0, 0}};
    while (!st.empty()) {
        auto [i, j] = st.back();
        st.pop_back();
        const Cluster &A = ta[i], &B = tb[j];
        const int p = A.b - A.a, q = B.b - B.a;
        const double d = std::hypot(A.cx - B.cx, A.cy - B.cy);
        const bool adm = !dense && d > eta * (A.r + B.r) && p <= max_block && q <= max_block;
        if (adm || (A.leaf() && B.leaf())) {
            blocks.push_back(BlockDev{A.a, p, B.a, q});
            far.push_back(adm ? 1 : 0);
            pairs.push_back(pair);
            continue;
        }
        bool split_recv;
        if (A.leaf()) split_recv = false;
        else if (B.leaf()) split_recv = true;
        else if (std::fabs(A.r - B.r) <= 1e-12 * std::max(A.r, B.r)) split_recv = true;
        else split_recv = A.r > B.r;
        if (split_recv) {
            st.push_back({A.right, j});
            st.push_back({A.left, j});
        } else {
            st.push_back({i, B.right});
            st.push_back({i, B.left});
        }
    }
}

// Points of one fault pair (receiver a, source b): last lag of the window.  T_max is the largest distance from the
// far ends of the source elements to the two receiver-fault endpoints over c_s; T_end = (1 + eta_Tmax) T_max
// (Sec. 2.3.2); last lag = ceil(T_end / dt - 1e-9), at most max_steps - 1.
int32_t pair_last_lag(const seas_net &net, int a, int b, double eta_tmax, int max_steps, bool no_trunc) {
    if (no_trunc) return max_steps - 1;
    const seas_fault &Fa = net.faults[a];
    const double c1 = std::cos(Fa.strike_rad), s1 = std::sin(Fa.strike_rad);
    const double h = 0.5 * Fa.length;
    const double ex[2] = {Fa.cx - h * c1, Fa.cx + h * c1}, ey[2] = {Fa.cy - h * s1, Fa.cy + h * s1};
    double dmax = 0.0;
    for (int j = net.off[b]; j < net.off[b + 1]; ++j) {
        const double hb = 0.5 * net.ds[j];
        const double sx[2] = {net.x[j] - hb * net.e1x[j], net.x[j] + hb * net.e1x[j]};
        const double sy[2] = {net.y[j] - hb * net.e1y[j], net.y[j] + hb * net.e1y[j]};
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v) dmax = std::max(dmax, std::hypot(ex[u] - sx[v], ey[u] - sy[v]));
    }
    const double tmax = dmax / net.med.cs;
    const double tend = (1.0 + eta_tmax) * tmax;
    const double lag = std::ceil(tend / net.dt - 1e-9);
    return (int32_t)std::min<double>(lag, max_steps - 1);
}

// Cluster-level end truncation (Sec. 4.3): the fault-pair criterion above applied to one block.  The receiver and
// source clusters are straight runs of consecutive elements, so the largest distance between a point of one and a
// point of the other is reached between segment ends: T_max^AB = the largest of the four distances between the
// outer ends of the block's first and last receiver elements and of its first and last source elements, over c_s.
int32_t cluster_last_lag(const seas_net &net, const BlockDev &b, double eta_tmax, int max_steps) {
    auto ends = [&](int first, int last, double *ex, double *ey) {
        const double h0 = 0.5 * net.ds[first], h1 = 0.5 * net.ds[last];
        ex[0] = net.x[first] - h0 * net.e1x[first];
        ey[0] = net.y[first] - h0 * net.e1y[first];
        ex[1] = net.x[last] + h1 * net.e1x[last];
        ey[1] = net.y[last] + h1 * net.e1y[last];
    };
    double rx[2], ry[2], sx[2], sy[2];
    ends(b.r0, b.r0 + b.p - 1, rx, ry);
    ends(b.c0, b.c0 + b.q - 1, sx, sy);
    double dmax = 0.0;
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) dmax = std::max(dmax, std::hypot(rx[u] - sx[v], ry[u] - sy[v]));
    const double lag = std::ceil((1.0 + eta_tmax) * (dmax / net.med.cs) / net.dt - 1e-9);
    return (int32_t)std::min<double>(lag, max_steps - 1);
}

// Conservative first lag of a block: one less than floor(min segment distance / (c_s dt)).  Exactly-zero slices
// found while building are dropped as well, so the stored window starts at the exact first nonzero lag.
int32_t block_first_lag(const seas_net &net, const BlockDev &b) {
    double dmin = INFINITY;
    for (int i = b.r0; i < b.r0 + b.p; ++i)
        for (int j = b.c0; j < b.c0 + b.q; ++j) {
            const double dx = net.x[i] - net.x[j], dy = net.y[i] - net.y[j];
            const double r1 = dx * net.e1x[j] + dy * net.e1y[j];
            const double r2 = dx * net.nx[j] + dy * net.ny[j];
            const double h = 0.5 * net.ds[j];
            const double d = std::fabs(r1) <= h ? std::fabs(r2) : std::hypot(std::fabs(r1) - h, r2);
            dmin = std::min(dmin, d);
        }
    const double lag = std::floor(dmin / (net.med.cs * net.dt)) - 1.0;
    return (int32_t)std::max(0.0, lag);
}

// Last lag W_f(n) of the spectral window of mode n >= 1 (Eq. mode_dependent_truncation):
// T_end(n) = eta_w L / c_s * Lcal(n), Lcal(n) = 1/n + (q_w - 1)/(n_max - 1) (1 - 1/n), n_max = N_f.
int32_t mode_window(const seas_net &net, int f, int n, const seas_hparams &hp, bool no_trunc) {
    if (no_trunc) return hp.max_steps - 1;
    const int nf = net.faults[f].n_elem;
    const double qw = hp.q_w <= 0 ? (double)nf : (double)hp.q_w;
    const double lcal = nf == 1 ? 1.0 : 1.0 / n + (qw - 1.0) / (nf - 1.0) * (1.0 - 1.0 / n);
    const double tend = hp.eta_w * net.faults[f].length / net.med.cs * lcal;
    const double lag = std::ceil(tend / net.dt - 1e-9);
    return (int32_t)std::min<double>(lag, hp.max_steps - 1);
}

std::vector<int> radix_plan(int n) {
    std::vector<int> r;
    for (int R : {4, 2, 3, 5, 7, 11, 13, 17, 19, 23})
        while (n % R == 0 && !(R == 2 && n % 4 == 0)) {
            r.push_back(R);
            n /= R;
        }
    return r;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n (in long double).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = cosl(pi * (i + 0.75L) / (n + 0.5L)), pp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pp = n * (z * p1 - p0) / (z * z - 1);
            const long double dz = p1 / pp;
            z -= dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        x[i] = (double)z;
        w[i] = (double)(2 / ((1 - z * z) * pp * pp));
    }
}

std::vector<double> static_mode_limits(int max_n);

seas_status build_self(seas_op &op) {
    seas_net &net = *op.net;
    seas_ctx *c = net.ctx;
    const bool no_trunc = op.hp.flags & SEAS_FLAG_NO_TRUNC;
    std::vector<double2> tw;
    std::vector<int64_t> g_prefix;
    std::vector<double> mode_L;
    int64_t w_total = 0, g_total = 0, dring = 0;
    op.n_modes_total = 0;
    op.max_nf = 0;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int f = 0; f < net.F; ++f) {
        const int nf = net.faults[f].n_elem;
        if (!op.owned[f]) {                    // another operator's fault: no self effect here
            op.mode_W.insert(op.mode_W.end(), (size_t)nf + 1, 0);
            continue;
        }
        FaultDev fd{};
        fd.off = net.off[f];
        fd.nf = nf;
        fd.mode_off = op.n_modes_total;
        std::vector<int> rp = radix_plan(nf);
        if ((int)rp.size() > kMaxStages) return fail(SEAS_EINVAL, "fault %d: FFT plan too deep", f);
        fd.nstages = (int)rp.size();
        for (size_t s = 0; s < rp.size(); ++s) fd.radix[s] = rp[s];
        // large faults: a four-step factorisation N_f = n1 n2 with both factors multiples of the cluster size,
        // n1 the one nearest sqrt(N_f) (the FFT then spreads over kFftCluster SMs)
        if (nf >= kFftClusterMin) {
            int best = 0;
            for (int n1 = kFftCluster; n1 <= nf / kFftCluster; n1 += kFftCluster)
                if (nf % n1 == 0 && (nf / n1) % kFftCluster == 0 &&
                    (best == 0 || std::fabs(n1 - std::sqrt((double)nf)) < std::fabs(best - std::sqrt((double)nf))))
                    best = n1;
            if (best > 0) {
                const std::vector<int> p1 = radix_plan(best), p2 = radix_plan(nf / best);
                if ((int)p1.size() <= kMaxStages && (int)p2.size() <= kMaxStages) {
                    fd.n1 = best;
                    fd.n2 = nf / best;
                    fd.nst1 = (int)p1.size();
                    fd.nst2 = (int)p2.size();
                    for (size_t s = 0; s < p1.size(); ++s) fd.radix1[s] = p1[s];
                    for (size_t s = 0; s < p2.size(); ++s) fd.radix2[s] = p2[s];
                }
            }
        }
        fd.tw_off = (int64_t)tw.size();
        for (int k = 0; k < nf; ++k) {
            const long double ang = -2 * pi * k / nf;
            tw.push_back(make_double2((double)cosl(ang), (double)sinl(ang)));
        }
        for (int k = 0; k <= nf; ++k) {
            const long double ang = -pi * k / nf;
            tw.push_back(make_double2((double)cosl(ang), (double)sinl(ang)));
        }
        fd.kfac = -(net.med.mu / 2.0) * kPi / net.faults[f].length;
        int32_t wmax = 0;
        op.mode_W.push_back(0);
        for (int n = 1; n <= nf; ++n) {
            const int32_t W = mode_window(net, f, n, op.hp, no_trunc);
            op.mode_W.push_back(W);
            wmax = std::max(wmax, W);
            ModeDev md{};
            md.w_off = w_total;
            md.W = W;
            md.fault = (int32_t)op.faults_h.size();
            md.n = n;
            op.modes_h.push_back(md);
            g_prefix.push_back(g_total);
            mode_L.push_back(net.faults[f].length);
            w_total += W + 1;
            g_total += W + 2;
        }
        fd.ring = wmax + (op.tail ? 2 : 1);    // the static tail reads D one step past the longest window
        fd.dring_off = dring;        // batch-1 layout; scenarios derive their own table
        dring += (int64_t)(nf + 1) * fd.ring;
        op.faults_h.push_back(fd);
        op.n_modes_total += nf + 1;
        op.max_nf = std::max(op.max_nf, nf);
    }
    SEAS_TRY(op.d_faults.upload(c, op.faults_h));
    std::vector<int32_t> big;
    for (size_t k = 0; k < op.faults_h.size(); ++k)
        if (op.faults_h[k].n1 > 0) big.push_back((int32_t)k);
    op.n_big = (int)big.size();
    if (!big.empty()) SEAS_TRY(op.d_big.upload(c, big));
    SEAS_TRY(op.d_modes.upload(c, op.modes_h));
    SEAS_TRY(op.d_tw.upload(c, tw));
    SEAS_TRY(op.d_w.alloc(c, (size_t)w_total));
    DArr<int64_t> d_gp;
    DArr<double> d_L, d_G, d_glx, d_glw;
    std::vector<double> glx, glw;
    gauss_legendre(10, glx, glw);
    SEAS_TRY(d_gp.upload(c, g_prefix));
    SEAS_TRY(d_L.upload(c, mode_L));
    SEAS_TRY(d_glx.upload(c, glx));
    SEAS_TRY(d_glw.upload(c, glw));
    SEAS_TRY(d_G.alloc(c, (size_t)g_total));
    CUDA_TRY(launch_spectral_tables(op.d_modes.p, (int)op.modes_h.size(), d_gp.p, g_total, d_L.p,
                                    net.med.cs * net.dt, d_glx.p, d_glw.p, (int)glx.size(), d_G.p, op.d_w.p,
                                    c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    op.stats.bytes_self = w_total * (int64_t)sizeof(double);
    if (op.tail) {
        // weight mass beyond each window: S_n - sum_{T <= W} w_n^T, S_n = (2/pi) Si(n pi)
        std::vector<double> w((size_t)w_total);
        CUDA_TRY(cudaMemcpy(w.data(), op.d_w.p, (size_t)w_total * sizeof(double), cudaMemcpyDeviceToHost));
        int max_n = 0;
        for (const ModeDev &m : op.modes_h) max_n = std::max(max_n, m.n);
        const std::vector<double> S = static_mode_limits(max_n);
        for (ModeDev &m : op.modes_h) {
            double sum = 0.0;
            for (int T = 0; T <= m.W; ++T) sum += w[(size_t)(m.w_off + T)];
            m.tailc = S[(size_t)m.n] - sum;
        }
        SEAS_TRY(op.d_modes.upload(c, op.modes_h));
    }
    return SEAS_OK;
}

// Static limits S_n = sum_{T >= 0} w_n^T = (2/pi) Si(n pi), n = 0..max_n: Si(n pi) accumulated one half period at
// a time, each by 20-point Gauss-Legendre (sin t / t is smooth on every [k pi, (k + 1) pi]).
std::vector<double> static_mode_limits(int max_n) {
    std::vector<double> gx, gw;
    gauss_legendre(20, gx, gw);
    std::vector<double> S((size_t)max_n + 1, 0.0);
    long double si = 0.0L;
    for (int k = 0; k < max_n; ++k) {
        const long double a = (long double)kPi * k, h = 0.5L * (long double)kPi;
        long double part = 0.0L;
        for (size_t i = 0; i < gx.size(); ++i) {
            const long double t = a + h * (1.0L + gx[i]);
            part += gw[i] * sinl(t) / t;
        }
        si += h * part;
        S[(size_t)k + 1] = (double)(2.0L / (long double)kPi * si);
    }
    return S;
}

// The elastostatic operator of the static tail: smat[i][j] = -(mu / 2 c_s) (n'_1 S_31 + n'_2 S_32) for receivers i
// and sources j on different faults, S_3l the t -> inf limit of K_3l / dt (Eq. primitives differenced over the
// source element as in Eq. kernel_interactions): S_31 = -(c_s/pi)(r2/rho_+^2 - r2/rho_-^2),
// S_32 = (c_s/pi)(r1_+/rho_+^2 - r1_-/rho_-^2), r1_+- = r1 +- ds_j/2, in the source element's frame.
seas_status build_static(seas_op &op) {
    seas_net &net = *op.net;
    seas_ctx *c = net.ctx;
    const int64_t N = net.N;
    std::vector<double> m((size_t)(N * N), 0.0);
    const double cpi = net.med.cs / kPi, rad = -net.med.mu / (2.0 * net.med.cs);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            if (net.fault_of[i] == net.fault_of[j]) continue;
            const double dx = net.x[i] - net.x[j], dy = net.y[i] - net.y[j];
            const double r1 = dx * net.e1x[j] + dy * net.e1y[j], r2 = dx * net.nx[j] + dy * net.ny[j];
            const double n1 = net.nx[i] * net.e1x[j] + net.ny[i] * net.e1y[j];
            const double n2 = net.nx[i] * net.nx[j] + net.ny[i] * net.ny[j];
            const double h = 0.5 * net.ds[j], rp = r1 + h, rm = r1 - h;
            const double pp = rp * rp + r2 * r2, pm = rm * rm + r2 * r2;
            const double s31 = -cpi * (r2 / pp - r2 / pm), s32 = cpi * (rp / pp - rm / pm);
            m[(size_t)(i * N + j)] = rad * (n1 * s31 + n2 * s32);
        }
    SEAS_TRY(op.d_smat.upload(c, m));
    SEAS_TRY(op.d_pair_last.upload(c, op.pair_last));
    if (op.hp.flags & SEAS_FLAG_CLUSTER_TRUNC) SEAS_TRY(op.d_block_last.upload(c, op.block_hi));
    return SEAS_OK;
}

seas_status build_interaction(seas_op &op) {
    seas_net &net = *op.net;
    seas_ctx *c = net.ctx;
    const seas_hparams &hp = op.hp;
    const bool dense = hp.flags & SEAS_FLAG_DENSE;
    const bool no_trunc = hp.flags & SEAS_FLAG_NO_TRUNC;
    const int max_block = hp.max_block > 0 ? std::min(hp.max_block, kMaxBlockSide) : kDefaultMaxBlock;

    // fault-wise cluster trees and per-pair block partitions
    std::vector<std::vector<Cluster>> trees(net.F);
    for (int f = 0; f < net.F; ++f) build_tree(net, f, net.off[f], net.off[f + 1], hp.leaf, trees[f]);
    op.pair_last.assign((size_t)net.F * net.F, -1);
    for (int a = 0; a < net.F; ++a)
        for (int b = 0; b < net.F; ++b) {
            if (a == b) continue;
            op.pair_last[(size_t)a * net.F + b] = pair_last_lag(net, a, b, hp.eta_tmax, hp.max_steps, no_trunc);
            if (!op.owned[a]) continue;        // rows of another operator
            traverse(trees[a], trees[b], hp.eta_h, dense, max_block, a * net.F + b, op.blocks_h, op.block_far,
                     op.block_pair);
        }
    const int nb = (int)op.blocks_h.size();
    std::vector<int32_t> lo(nb), hi(nb);
    int32_t Tmin = INT32_MAX, Tmax = -1;
    const bool cluster_trunc = (hp.flags & SEAS_FLAG_CLUSTER_TRUNC) && !no_trunc;
    for (int b = 0; b < nb; ++b) {
        lo[b] = block_first_lag(net, op.blocks_h[b]);
        hi[b] = op.pair_last[op.block_pair[b]];
        if (cluster_trunc) hi[b] = std::min(hi[b], cluster_last_lag(net, op.blocks_h[b], hp.eta_tmax, hp.max_steps));
        if (lo[b] <= hi[b]) {
            Tmin = std::min(Tmin, lo[b]);
            Tmax = std::max(Tmax, hi[b]);
        }
        if (op.block_far[b]) op.stats.n_blocks_far++;
        else op.stats.n_blocks_near++;
    }
    op.ring = std::max<int32_t>(1, Tmax + 1);
    op.block_lo = lo;
    op.block_hi = hi;
    SEAS_TRY(op.d_blocks.upload(c, op.blocks_h));

    GeomDev g{net.d_x.p, net.d_e1.p, net.d_n.p, net.d_ds.p, net.med.cs, net.dt, -net.med.mu / (2.0 * net.med.cs)};
    int64_t max_block_entries = 1;
    for (auto &b : op.blocks_h) {
        max_block_entries = std::max<int64_t>(max_block_entries, (int64_t)b.p * b.q);
        op.max_q = std::max(op.max_q, b.q);
    }
    // rows per dense item of each block (items of at most kItemBytes and kItemRows rows)
    const int prec = hp.precision;
    const int eb = elem_bytes(prec);
    std::vector<int32_t> drows(nb);
    for (int b = 0; b < nb; ++b) {
        const int p2 = pad_row(op.blocks_h[b].p, prec);
        drows[b] = (int32_t)std::min<int64_t>(kItemRows, std::max<int64_t>(1, kItemBytes / (eb * p2)));
    }
    const int64_t cap = std::max(kChunkEntries, max_block_entries);
    bool any_far = false;
    for (int b = 0; b < nb; ++b) any_far |= op.block_far[b] != 0;
    DArr<double> scratch, resid, factors;
    if (Tmax >= 0) {
        SEAS_TRY(scratch.alloc(c, (size_t)cap));
        if (any_far) {
            SEAS_TRY(resid.alloc(c, (size_t)cap));
            SEAS_TRY(factors.alloc(c, (size_t)cap));
        }
    }
    // Slices in block-major, lag-minor order, so that each block's slices are adjacent in the receiver-side arena.
    // Far slices' V^T rows go to a block-major staging buffer first and are gathered into the source-major
    // arena of pass 1 once every rank is known.
    struct Stored {
        int32_t block, T, k;
        const unsigned char *u, *v;
        float scale;
        int chunk;
    };
    std::vector<Stored> stored;
    std::vector<std::unique_ptr<DArr<unsigned char>>> vstage;
    int64_t bytes_dense = 0, bytes_stored = 0, rank_sum = 0;
    int cb = 0;
    int32_t cT = nb ? lo[0] : 0;
    auto advance = [&]() {            // next (block, lag) of the cursor
        ++cT;
        while (cb < nb && cT > hi[cb]) {
            ++cb;
            if (cb < nb) cT = lo[cb];
        }
    };
    while (cb < nb && cT > hi[cb]) {
        ++cb;
        if (cb < nb) cT = lo[cb];
    }
    int chunk_id = 0;
    while (cb < nb) {
        std::vector<SliceGen> sl;
        std::vector<int64_t> prefix;
        int64_t entries = 0;
        while (cb < nb) {
            const int64_t pq = (int64_t)op.blocks_h[cb].p * op.blocks_h[cb].q;
            if (entries + pq > cap) break;
            sl.push_back(SliceGen{cb, cT, op.block_far[cb], 0, entries});
            prefix.push_back(entries);
            entries += pq;
            advance();
        }
        DArr<SliceGen> d_sl;
        DArr<int64_t> d_pref, d_off, d_voff;
        DArr<SliceOut> d_out;
        SEAS_TRY(d_sl.upload(c, sl));
        SEAS_TRY(d_pref.upload(c, prefix));
        SEAS_TRY(d_out.alloc(c, sl.size()));
        CUDA_TRY(launch_gen_slices(g, op.d_blocks.p, d_sl.p, (int)sl.size(), d_pref.p, entries, scratch.p,
                                   c->stream));
        CUDA_TRY(launch_compress(op.d_blocks.p, d_sl.p, (int)sl.size(), scratch.p, resid.p, factors.p, d_out.p,
                                 hp.aca_tol, c->stream));
        std::vector<SliceOut> so(sl.size());
        CUDA_TRY(cudaMemcpyAsync(so.data(), d_out.p, so.size() * sizeof(SliceOut), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        std::vector<int64_t> dst(sl.size()), vdst(sl.size());
        int64_t total = 0, vtotal = 0;
        for (size_t k = 0; k < sl.size(); ++k) {
            const BlockDev &b = op.blocks_h[sl[k].block];
            dst[k] = total;
            vdst[k] = vtotal;
            if (so[k].k == 0) {
                op.stats.n_slices_zero++;
                continue;
            }
            const int p2 = pad_row(b.p, prec), q2 = pad_row(b.q, prec);
            bytes_dense += (int64_t)b.p * b.q * 8;
            if (so[k].k < 0) {
                op.stats.n_slices_dense++;
                total += (int64_t)b.q * p2;
            } else {
                op.stats.n_slices_lowrank++;
                rank_sum += so[k].k;
                op.stats.max_rank = std::max(op.stats.max_rank, so[k].k);
                total += (int64_t)so[k].k * p2;
                vtotal += (int64_t)so[k].k * q2;
            }
        }
        if (total > 0) {
            auto buf = std::make_unique<DArr<unsigned char>>();
            auto vbuf = std::make_unique<DArr<unsigned char>>();
            SEAS_TRY(buf->alloc(c, (size_t)(total * eb)));
            SEAS_TRY(vbuf->alloc(c, (size_t)std::max<int64_t>(16, vtotal * eb)));
            SEAS_TRY(d_off.upload(c, dst));
            SEAS_TRY(d_voff.upload(c, vdst));
            DArr<float> d_scale;
            SEAS_TRY(d_scale.alloc(c, sl.size()));
            CUDA_TRY(launch_pack(op.d_blocks.p, d_sl.p, d_out.p, (int)sl.size(), scratch.p, factors.p, d_off.p,
                                 buf->p, d_voff.p, vbuf->p, d_scale.p, prec, c->stream));
            std::vector<float> scl(sl.size());
            CUDA_TRY(cudaMemcpyAsync(scl.data(), d_scale.p, scl.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                     c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (size_t k = 0; k < sl.size(); ++k)
                if (so[k].k != 0)
                    stored.push_back(Stored{sl[k].block, sl[k].T, so[k].k, buf->p + dst[k] * eb,
                                            vbuf->p + vdst[k] * eb, scl[k], chunk_id});
            bytes_stored += (total + vtotal) * eb;
            op.arena.push_back(std::move(buf));
            vstage.push_back(std::move(vbuf));
        }
        ++chunk_id;
    }
    scratch.release();
    resid.release();
    factors.release();

    // z rows: one per row of the receiver-side arena, in its order (dense slices' rows unused)
    std::vector<int64_t> zrow0(stored.size());
    int64_t zrows = 0;
    for (size_t i = 0; i < stored.size(); ++i) {
        zrow0[i] = zrows;
        zrows += stored[i].k < 0 ? op.blocks_h[stored[i].block].q : stored[i].k;
    }
    if (zrows >= ((int64_t)1 << 31)) return fail(SEAS_EINVAL, "operator too large (%lld z rows)", (long long)zrows);
    op.z_rows = zrows;

    // ---- pass 1: far slices grouped by source cluster, then lag, then block (stable), V^T rows gathered into one
    // source-major arena; runs of one (source cluster, lag) split so that a run and its history slice fit a stage
    std::vector<int32_t> src_of(nb, -1);
    std::vector<SrcDev> srcs;
    {
        std::vector<std::pair<std::pair<int, int>, int>> keys;
        for (int b = 0; b < nb; ++b)
            if (op.block_far[b]) keys.push_back({{op.blocks_h[b].c0, op.blocks_h[b].q}, b});
        std::sort(keys.begin(), keys.end());
        for (size_t k = 0; k < keys.size(); ++k) {
            if (k == 0 || keys[k].first != keys[k - 1].first)
                srcs.push_back(SrcDev{keys[k].first.first, keys[k].first.second});
            src_of[keys[k].second] = (int32_t)srcs.size() - 1;
        }
    }
    std::vector<size_t> far_ix;
    for (size_t i = 0; i < stored.size(); ++i)
        if (stored[i].k > 0) far_ix.push_back(i);
    std::stable_sort(far_ix.begin(), far_ix.end(), [&](size_t x, size_t y) {
        const int sx = src_of[stored[x].block], sy = src_of[stored[y].block];
        return sx != sy ? sx < sy : stored[x].T < stored[y].T;
    });
    int64_t vbytes = 0;
    for (size_t i : far_ix) vbytes += (int64_t)stored[i].k * pad_row(op.blocks_h[stored[i].block].q, prec) * eb;
    SEAS_TRY(op.d_varena.alloc(c, (size_t)std::max<int64_t>(16, vbytes)));
    std::vector<RunDev> runs;
    std::vector<int32_t> zmap;
    std::vector<float> zscale;
    std::vector<TaskDev> ztasks;
    {
        std::vector<const void *> gsrc;
        std::vector<void *> gdst;
        std::vector<int32_t> gbytes;
        int64_t off = 0;
        const int64_t x_cap = (int64_t)kMaxBatch * 8;          // history bytes per source column, worst case
        TaskDev zt{-1, 0, 0, 0, 0};
        int64_t zt_bytes = 0;
        for (size_t n = 0; n < far_ix.size(); ++n) {
            const Stored &x = stored[far_ix[n]];
            const int sidx = src_of[x.block];
            const int q2 = pad_row(srcs[sidx].q, prec);
            const int64_t row_bytes = (int64_t)q2 * eb;
            // a run's rows, their z-row map (4 bytes a row) and its history slice fit one stage
            const int64_t max_rows =
                std::max<int64_t>(1, (kStageBytes - 64 - (int64_t)q2 * x_cap) / (row_bytes + 4));
            unsigned char *d = op.d_varena.p + off;
            gsrc.push_back(x.v);
            gdst.push_back(d);
            gbytes.push_back((int32_t)(x.k * row_bytes));
            for (int l = 0; l < x.k; ++l) {
                zmap.push_back((int32_t)(zrow0[far_ix[n]] + l));
                zscale.push_back(x.scale);
            }
            for (int l = 0; l < x.k;) {
                const bool extend = !runs.empty() && zt.block == sidx && runs.back().T == x.T &&
                                    runs.back().rows < max_rows;
                if (!extend) {
                    // a new run; a new task when the source cluster changes or the task is full
                    if (zt.block != sidx || zt_bytes >= kTaskBytes) {
                        if (zt.block >= 0) {
                            zt.item_end = (int32_t)runs.size();
                            ztasks.push_back(zt);
                        }
                        zt = TaskDev{sidx, (int32_t)runs.size(), 0, x.T, 0};
                        zt_bytes = 0;
                    }
                    runs.push_back(RunDev{x.T, 0, d + (int64_t)l * row_bytes, (int64_t)zmap.size() - x.k + l});
                }
                const int take = (int)std::min<int64_t>(x.k - l, max_rows - runs.back().rows);
                runs.back().rows += take;
                zt_bytes += take * row_bytes;
                l += take;
            }
            off += x.k * row_bytes;
        }
        if (zt.block >= 0) {
            zt.item_end = (int32_t)runs.size();
            ztasks.push_back(zt);
        }
        DArr<const void *> d_gs;
        DArr<void *> d_gd;
        DArr<int32_t> d_gb;
        SEAS_TRY(d_gs.upload(c, gsrc));
        SEAS_TRY(d_gd.upload(c, gdst));
        SEAS_TRY(d_gb.upload(c, gbytes));
        CUDA_TRY(launch_gather(d_gs.p, d_gd.p, d_gb.p, (int)gsrc.size(), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    vstage.clear();
    std::stable_sort(ztasks.begin(), ztasks.end(),
                     [](const TaskDev &x, const TaskDev &y) { return x.T_start < y.T_start; });
    for (auto &t : ztasks) op.ztask_T.push_back(t.T_start);
    SEAS_TRY(op.d_runs.upload(c, runs));
    SEAS_TRY(op.d_ztasks.upload(c, ztasks));
    SEAS_TRY(op.d_srcs.upload(c, srcs));
    zmap.resize(zmap.size() + 4, 0);             // the bulk copies of a run's map round up to 16 bytes
    SEAS_TRY(op.d_zmap.upload(c, zmap));
    if (prec == kPrecFP16) SEAS_TRY(op.d_zscale.upload(c, zscale));

    // ---- pass 2: work items (<= kItemBytes and kItemRows rows, adjacent in memory) and tasks (runs of items of one
    // block within one arena chunk, <= kTaskBytes); consecutive far slices of a block merge into one item; each
    // task owns p partial-sum rows, the k-th task of block b at blk_part[b] + k * p.
    std::vector<ItemDev> items;
    std::vector<TaskDev> tasks;
    size_t s = 0;
    while (s < stored.size()) {
        const int blk = stored[s].block;
        const BlockDev &b = op.blocks_h[blk];
        const int p2 = pad_row(b.p, prec);
        const int64_t row_bytes = (int64_t)p2 * eb;
        TaskDev task{blk, (int32_t)items.size(), 0, stored[s].T, 0};
        int64_t task_bytes = 0;
        int chunk = stored[s].chunk;
        bool open_far = false;                 // the last item is a far item that may take more rows
        for (; s < stored.size() && stored[s].block == blk; ++s) {
            const Stored &x = stored[s];
            if (task_bytes >= kTaskBytes || x.chunk != chunk) {
                task.item_end = (int32_t)items.size();
                tasks.push_back(task);
                task = TaskDev{blk, (int32_t)items.size(), 0, x.T, 0};
                task_bytes = 0;
                chunk = x.chunk;
                open_far = false;
            }
            if (x.k < 0) {
                for (int j = 0; j < b.q; j += drows[blk]) {
                    const int j1 = std::min(b.q, j + drows[blk]);
                    items.push_back(ItemDev{x.T, -1, j, j1, x.u + (int64_t)j * row_bytes, x.scale, 0, -1});
                }
                task_bytes += (int64_t)b.q * row_bytes;
                open_far = false;
            } else {
                for (int l = 0; l < x.k;) {
                    if (open_far) {
                        ItemDev &it = items.back();
                        const int room = (int)std::min<int64_t>(kItemRows - it.k, kItemBytes / row_bytes - it.k);
                        if (room > 0) {
                            const int take = std::min(room, x.k - l);
                            it.k += take;
                            it.i1 = it.k;
                            l += take;
                            continue;
                        }
                    }
                    const int take = (int)std::min<int64_t>(
                        x.k - l, std::max<int64_t>(1, std::min<int64_t>(kItemRows, kItemBytes / row_bytes)));
                    items.push_back(ItemDev{x.T, take, 0, take, x.u + (int64_t)l * row_bytes, 1.0f, 0, zrow0[s] + l});
                    open_far = true;
                    l += take;
                }
                task_bytes += (int64_t)x.k * row_bytes;
            }
        }
        task.item_end = (int32_t)items.size();
        tasks.push_back(task);
    }
    // per-block task lists (in lag order) and partial-sum slots
    std::vector<int32_t> blk_task_ptr(nb + 1, 0), blk_task_T;
    std::vector<int64_t> blk_part(nb, 0);
    for (const TaskDev &t : tasks) blk_task_ptr[t.block + 1]++;
    for (int b = 0; b < nb; ++b) blk_task_ptr[b + 1] += blk_task_ptr[b];
    blk_task_T.assign(tasks.size(), 0);
    {
        int64_t part = 0;
        for (int b = 0; b < nb; ++b) {
            blk_part[b] = part;
            part += (int64_t)(blk_task_ptr[b + 1] - blk_task_ptr[b]) * op.blocks_h[b].p;
        }
        op.n_partial = part;
        std::vector<int32_t> fill(nb, 0);
        for (TaskDev &t : tasks) {            // tasks are in block order, lag order within a block
            const int k = fill[t.block]++;
            blk_task_T[blk_task_ptr[t.block] + k] = t.T_start;
            t.part_off = blk_part[t.block] + (int64_t)k * op.blocks_h[t.block].p;
        }
    }
    // receiver cover lists: for each element, the blocks whose rows contain it
    std::vector<int32_t> cover_ptr(net.N + 1, 0), cover_blk;
    for (int b = 0; b < nb; ++b)
        for (int i = op.blocks_h[b].r0; i < op.blocks_h[b].r0 + op.blocks_h[b].p; ++i) cover_ptr[i + 1]++;
    for (int i = 0; i < net.N; ++i) cover_ptr[i + 1] += cover_ptr[i];
    cover_blk.assign(cover_ptr[net.N], 0);
    {
        std::vector<int32_t> fill(cover_ptr.begin(), cover_ptr.end() - 1);
        for (int b = 0; b < nb; ++b)
            for (int i = op.blocks_h[b].r0; i < op.blocks_h[b].r0 + op.blocks_h[b].p; ++i) cover_blk[fill[i]++] = b;
    }
    std::stable_sort(tasks.begin(), tasks.end(), [](const TaskDev &x, const TaskDev &y) { return x.T_start < y.T_start; });
    for (auto &t : tasks) op.task_T.push_back(t.T_start);
    // algorithmic bytes: the values each stored slice holds (p q near, k (p + q) far), row padding not counted
    op.bytes_upto.assign((size_t)op.ring, 0);
    for (const Stored &x : stored) {
        const BlockDev &b = op.blocks_h[x.block];
        op.bytes_upto[x.T] += eb * (x.k < 0 ? (int64_t)b.q * b.p : (int64_t)x.k * (b.p + b.q));
    }
    for (size_t T = 1; T < op.bytes_upto.size(); ++T) op.bytes_upto[T] += op.bytes_upto[T - 1];
    if (eb == 2) {
        // 2-byte arenas: each unit's row chunks rotated once (chunk_at), for conflict-free shared-memory reads
        std::vector<UnitRows> units;
        units.reserve(items.size() + runs.size());
        for (const TaskDev &t : tasks) {
            const int nch = pad_row(op.blocks_h[t.block].p, prec) / 8;
            for (int i = t.item_begin; i < t.item_end; ++i) {
                const ItemDev &it = items[(size_t)i];
                units.push_back(UnitRows{const_cast<void *>(it.a), it.k < 0 ? it.i1 - it.i0 : it.k, nch});
            }
        }
        for (const TaskDev &t : ztasks) {
            const int nch = pad_row(srcs[(size_t)t.block].q, prec) / 8;
            for (int i = t.item_begin; i < t.item_end; ++i)
                units.push_back(UnitRows{const_cast<void *>(runs[(size_t)i].v), runs[(size_t)i].rows, nch});
        }
        DArr<UnitRows> d_units;
        SEAS_TRY(d_units.upload(c, units));
        CUDA_TRY(launch_rotate_rows(d_units.p, (int)units.size(), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    SEAS_TRY(op.d_items.upload(c, items));
    SEAS_TRY(op.d_tasks.upload(c, tasks));
    SEAS_TRY(op.d_cover_ptr.upload(c, cover_ptr));
    SEAS_TRY(op.d_cover_blk.upload(c, cover_blk));
    SEAS_TRY(op.d_blk_task_ptr.upload(c, blk_task_ptr));
    SEAS_TRY(op.d_blk_task_T.upload(c, blk_task_T));
    SEAS_TRY(op.d_blk_part.upload(c, blk_part));
    op.stats.n_tasks = (int64_t)tasks.size();
    op.stats.bytes_interaction = bytes_stored;
    op.stats.bytes_dense_causal = bytes_dense;
    op.stats.compression_ratio = bytes_dense ? 100.0 * (double)bytes_stored / (double)bytes_dense : 0.0;
    op.stats.mean_rank = op.stats.n_slices_lowrank ? (double)rank_sum / op.stats.n_slices_lowrank : 0.0;
    op.stats.ring_depth = op.ring;
    return SEAS_OK;
}

}  // namespace

extern "C" seas_status seas_build_hmatrix(seas_net *net, const seas_hparams *hp, seas_op **out,
                                          seas_op_stats *stats) {
    return seas_build_hmatrix_part(net, hp, nullptr, 0, out, stats);
}

extern "C" seas_status seas_build_hmatrix_part(seas_net *net, const seas_hparams *hp, const int32_t *faults,
                                               int n_faults, seas_op **out, seas_op_stats *stats) {
    if (!net || !hp || !out) return fail(SEAS_EINVAL, "NULL argument");
    std::vector<char> owned((size_t)net->F, faults ? 0 : 1);
    if (faults) {
        if (n_faults < 1) return fail(SEAS_EINVAL, "no owned faults");
        for (int k = 0; k < n_faults; ++k) {
            if (faults[k] < 0 || faults[k] >= net->F) return fail(SEAS_EINVAL, "fault %d out of range", faults[k]);
            owned[(size_t)faults[k]] = 1;
        }
        if (hp->flags & SEAS_FLAG_STATIC_TAIL)
            return fail(SEAS_EINVAL, "the static tail needs every fault's rows (no partial operator)");
    }
    *out = nullptr;
    if (hp->leaf < 1 || hp->leaf > kMaxBlockSide) return fail(SEAS_EINVAL, "leaf must be in [1, %d]", kMaxBlockSide);
    if (!(hp->eta_h > 0)) return fail(SEAS_EINVAL, "eta_h must be > 0");
    if (!(is_fin(hp->aca_tol) && hp->aca_tol >= 0 && hp->aca_tol < 1)) return fail(SEAS_EINVAL, "aca_tol in [0, 1)");
    if (!(is_fin(hp->eta_tmax) && hp->eta_tmax >= 0)) return fail(SEAS_EINVAL, "eta_tmax must be >= 0");
    if (!(is_fin(hp->eta_w) && hp->eta_w > 0)) return fail(SEAS_EINVAL, "eta_w must be > 0");
    if (hp->max_steps < 1 || hp->max_steps > (1 << 22)) return fail(SEAS_EINVAL, "max_steps in [1, 2^22]");
    if (hp->precision < kPrecFP64 || hp->precision > kPrecDF64)
        return fail(SEAS_EINVAL, "precision %d not available", hp->precision);
    if (hp->flags & ~(SEAS_FLAG_DENSE | SEAS_FLAG_NO_TRUNC | SEAS_FLAG_STATIC_TAIL | SEAS_FLAG_LAG_CAP |
                      SEAS_FLAG_CLUSTER_TRUNC))
        return fail(SEAS_EINVAL, "unsupported flags 0x%x", hp->flags);
    if (hp->max_block != 0 && hp->max_block < hp->leaf) return fail(SEAS_EINVAL, "max_block must be >= leaf");
    seas_ctx *c = net->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    const auto t0 = std::chrono::steady_clock::now();
    auto op = std::make_unique<seas_op>();
    op->net = net;
    op->hp = *hp;
    op->tail = (hp->flags & SEAS_FLAG_STATIC_TAIL) && !(hp->flags & SEAS_FLAG_NO_TRUNC);
    op->owned = owned;
    SEAS_TRY(build_self(*op));
    SEAS_TRY(build_interaction(*op));
    if (op->tail) SEAS_TRY(build_static(*op));
    op->stats.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = op->stats;
    net->children++;
    *out = op.release();
    return SEAS_OK;
}


extern "C" seas_status seas_plan_hmatrix(const seas_fault *faults, int n_faults, const seas_medium *med,
                                         const seas_hparams *hp, int32_t *blocks, int64_t cap, int64_t *n_blocks,
                                         int32_t *pair_last, int32_t *mode_windows, double *dt) {
    if (!hp) return fail(SEAS_EINVAL, "NULL hparams");
    seas_net net;
    SEAS_TRY(make_geometry(faults, n_faults, med, net));
    if (hp->leaf < 1 || hp->leaf > kMaxBlockSide) return fail(SEAS_EINVAL, "leaf must be in [1, %d]", kMaxBlockSide);
    if (hp->max_steps < 1) return fail(SEAS_EINVAL, "max_steps must be >= 1");
    const bool dense = hp->flags & SEAS_FLAG_DENSE;
    const bool no_trunc = hp->flags & SEAS_FLAG_NO_TRUNC;
    const int max_block = hp->max_block > 0 ? std::min(hp->max_block, kMaxBlockSide) : kDefaultMaxBlock;
    std::vector<std::vector<Cluster>> trees(net.F);
    for (int f = 0; f < net.F; ++f) build_tree(net, f, net.off[f], net.off[f + 1], hp->leaf, trees[f]);
    std::vector<BlockDev> bl;
    std::vector<int32_t> far, pairs, pl((size_t)net.F * net.F, -1);
    for (int a = 0; a < net.F; ++a)
        for (int b = 0; b < net.F; ++b) {
            if (a == b) continue;
            pl[(size_t)a * net.F + b] = pair_last_lag(net, a, b, hp->eta_tmax, hp->max_steps, no_trunc);
            if (pair_last) pair_last[a * net.F + b] = pl[(size_t)a * net.F + b];
            traverse(trees[a], trees[b], hp->eta_h, dense, max_block, a * net.F + b, bl, far, pairs);
        }
    const bool cluster_trunc = (hp->flags & SEAS_FLAG_CLUSTER_TRUNC) && !no_trunc;
    if (pair_last)
        for (int a = 0; a < net.F; ++a) pair_last[a * net.F + a] = -1;
    if (n_blocks) *n_blocks = (int64_t)bl.size();
    if (blocks)
        for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)bl.size()); ++i) {
            int32_t *r = blocks + 7 * i;
            r[0] = bl[i].r0;
            r[1] = bl[i].p;
            r[2] = bl[i].c0;
            r[3] = bl[i].q;
            r[4] = far[i];
            r[5] = block_first_lag(net, bl[i]);
            r[6] = pl[(size_t)pairs[i]];
            if (cluster_trunc) r[6] = std::min(r[6], cluster_last_lag(net, bl[i], hp->eta_tmax, hp->max_steps));
        }
    if (mode_windows) {
        int64_t o = 0;
        for (int f = 0; f < net.F; ++f) {
            mode_windows[o++] = 0;
            for (int n = 1; n <= net.faults[f].n_elem; ++n) mode_windows[o++] = mode_window(net, f, n, *hp, no_trunc);
        }
    }
    if (dt) *dt = net.dt;
    return SEAS_OK;
}

extern "C" seas_status seas_op_pair_windows(const seas_op *op, int32_t *last_lag) {
    if (!op || !last_lag) return fail(SEAS_EINVAL, "NULL argument");
    std::copy(op->pair_last.begin(), op->pair_last.end(), last_lag);
    return SEAS_OK;
}

extern "C" seas_status seas_op_blocks(const seas_op *op, int32_t *blocks, int64_t cap, int64_t *n_blocks) {
    if (!op || (!blocks && cap > 0)) return fail(SEAS_EINVAL, "NULL argument");
    const int64_t nb = (int64_t)op->blocks_h.size();
    if (n_blocks) *n_blocks = nb;
    for (int64_t i = 0; i < std::min(cap, nb); ++i) {
        const BlockDev &b = op->blocks_h[(size_t)i];
        int32_t *r = blocks + 7 * i;
        r[0] = b.r0;
        r[1] = b.p;
        r[2] = b.c0;
        r[3] = b.q;
        r[4] = op->block_far[(size_t)i];
        r[5] = op->block_lo[(size_t)i];
        r[6] = op->block_hi[(size_t)i];
    }
    return SEAS_OK;
}

extern "C" seas_status seas_op_mode_windows(const seas_op *op, int32_t *w) {
    if (!op || !w) return fail(SEAS_EINVAL, "NULL argument");
    std::copy(op->mode_W.begin(), op->mode_W.end(), w);
    return SEAS_OK;
}

extern "C" seas_status seas_destroy_op(seas_op *op) {
    if (!op) return SEAS_OK;
    if (op->children) return fail(SEAS_EBUSY, "operator has %d live scenarios", op->children);
    cudaSetDevice(op->net->ctx->device);
    op->net->children--;
    delete op;
    return SEAS_OK;
}

// ------------------------------------------------------------------------------------------------------------
// scenarios and the per-step calls
// ------------------------------------------------------------------------------------------------------------

namespace {

StepArgs step_args(seas_scn &s, int64_t step) {
    seas_op &op = *s.op;
    seas_net &net = *op.net;
    StepArgs a{};
    a.N = net.N;
    a.io_map = net.images ? net.d_io_map.p : nullptr;
    a.N_io = net.N_io;
    a.F = net.F;
    a.n_self = (int)op.faults_h.size();
    a.big = op.d_big.p;
    a.n_big = op.n_big;
    a.n_small = a.n_self - op.n_big;
    a.B = s.B;
    a.n_modes_total = op.n_modes_total;
    a.max_nf = op.max_nf;
    a.step = step;
    a.cw[0] = s.cw[0];
    a.cw[1] = s.cw[1];
    int64_t lag_max = -1;            // the oldest active member's step
    for (int b = 0; b < s.B; ++b)
        if (s.active[b]) lag_max = std::max<int64_t>(lag_max, step - s.start[b]);
    // the interaction's horizon never shrinks (its z rows beyond the horizon must stay as they were: zero)
    if (lag_max > s.horizon && step == s.n - 1) s.horizon = lag_max;
    lag_max = std::max(lag_max, std::min<int64_t>(s.horizon, step));
    a.lag_max = lag_max;
    a.ring = op.ring;
    a.ring_stride = s.ring_stride;
    a.dt = net.dt;
    a.rad = -net.med.mu / (2.0 * net.med.cs);
    a.faults = s.faults.p;
    a.modes = op.d_modes.p;
    a.n_modes = (int)op.modes_h.size();
    a.w = op.d_w.p;
    a.tw = op.d_tw.p;
    a.vring = s.vring.p;
    a.xring = s.xring.p;
    a.prec = op.hp.precision;
    a.xsplit = xsplit_of(op.hp.precision, s.B) ? 1 : 0;
    a.slip = s.slip.p;
    a.slip_prev = s.slip_prev.p;
    a.dring = s.dring.p;
    a.fmodes = s.fmodes.p;
    a.fint = s.fint.p;
    a.blocks = op.d_blocks.p;
    a.items = op.d_items.p;
    a.tasks = op.d_tasks.p;
    a.n_tasks_active =
        lag_max < 0 ? 0
                    : (int)(std::upper_bound(op.task_T.begin(), op.task_T.end(),
                                             (int32_t)std::min<int64_t>(lag_max, INT32_MAX)) -
                            op.task_T.begin());
    a.runs = op.d_runs.p;
    a.ztasks = op.d_ztasks.p;
    a.srcs = op.d_srcs.p;
    a.zmap = op.d_zmap.p;
    a.zscale = op.d_zscale.p;
    a.n_ztasks_active =
        lag_max < 0 ? 0
                    : (int)(std::upper_bound(op.ztask_T.begin(), op.ztask_T.end(),
                                             (int32_t)std::min<int64_t>(lag_max, INT32_MAX)) -
                            op.ztask_T.begin());
    a.zbuf = s.zbuf.p;
    a.pass = 2;
    a.partial = s.partial.p;
    a.n_partial = op.n_partial;
    a.counter = s.counter_err.p;
    a.err = s.counter_err.p + 1;
    a.wait_ns = s.wait_ns;
    a.cover_ptr = op.d_cover_ptr.p;
    a.cover_blk = op.d_cover_blk.p;
    a.blk_task_ptr = op.d_blk_task_ptr.p;
    a.blk_task_T = op.d_blk_task_T.p;
    a.blk_part = op.d_blk_part.p;
    a.n_sms = net.ctx->n_sms > 0 ? net.ctx->n_sms : 1;
    a.tail = op.tail ? 1 : 0;
    a.sring_depth = op.ring + 1;
    a.sring = s.sring.p;
    a.smat = op.d_smat.p;
    a.pair_last = op.d_pair_last.p;
    a.block_last = op.d_block_last.p;
    return a;
}

seas_status scenario_alloc(seas_op *op, int batch, std::unique_ptr<seas_scn> &s) {
    seas_ctx *c = op->net->ctx;
    const int64_t N = op->net->N;
    s = std::make_unique<seas_scn>();
    s->op = op;
    s->B = batch;
    s->start.assign(batch, 0);
    s->active.assign(batch, 1);
    const int64_t BN = N * batch;
    // spectral rings: per fault [batch][N_f + 1][R_f], faults one after the other
    std::vector<FaultDev> ft = op->faults_h;
    int64_t dr = 0;
    for (auto &f : ft) {
        f.dring_off = dr;
        dr += (int64_t)batch * (f.nf + 1) * f.ring;
    }
    s->dring_len = dr;
    SEAS_TRY(s->faults.upload(c, ft));
    // a multiple of 4 elements (16-byte rows for 4- and 8-byte elements) with room for the 16-byte round-up of
    // history slices
    // (the split history of the tensor-core consumers is 8 scenarios wide whatever the batch)
    const bool xsplit = xsplit_of(op->hp.precision, batch);
    s->ring_stride = (std::max<int64_t>(BN, xsplit ? N * 8 : 0) + 3) / 4 * 4 + 4;
    // the interaction kernel's bulk copies of history slices are widened to 16-byte bounds and to the padded
    // column count of a block (at most 7 columns of 8 scenarios past the slice): a tail of kCopyTail bytes keeps
    // the last slot's copies inside the allocation
    SEAS_TRY(s->vring.alloc(c, (size_t)(op->ring * s->ring_stride + kCopyTail / 8)));
    if (op->hp.precision != kPrecFP64) {
        const int xb = op->hp.precision == kPrecDF64 ? 8 : 4;
        SEAS_TRY(s->xring.alloc(c, (size_t)(op->ring * s->ring_stride * xb + kCopyTail)));
        SEAS_TRY(s->xring.zero(c->stream));
    }
    SEAS_TRY(s->partial.alloc(c, (size_t)(op->n_partial * batch)));
    {
        const int zb = op->hp.precision == kPrecBF16 || op->hp.precision == kPrecFP16 ? 4 : 8;
        const int64_t zw = xsplit ? 8 : batch;        // z rows of the split layout: 8 (high, low) pairs
        SEAS_TRY(s->zbuf.alloc(c, (size_t)(op->z_rows * zw * zb + kCopyTail)));   // widened copies, as above
        SEAS_TRY(s->zbuf.zero(c->stream));
    }
    SEAS_TRY(s->counter_err.alloc(c, 4));
    {
        int least = 0, greatest = 0;                  // numerically greatest = lowest priority
        CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CUDA_TRY(cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, least));
    }
    CUDA_TRY(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming));
    SEAS_TRY(s->counter_err.zero(c->stream));
    SEAS_TRY(s->slip.alloc(c, (size_t)BN));
    SEAS_TRY(s->slip_prev.alloc(c, (size_t)BN));
    SEAS_TRY(s->fint.alloc(c, (size_t)BN));
    SEAS_TRY(s->d_V.alloc(c, (size_t)BN));
    SEAS_TRY(s->d_slip.alloc(c, (size_t)BN));
    SEAS_TRY(s->d_tau.alloc(c, (size_t)BN));
    SEAS_TRY(s->d_parts.alloc(c, (size_t)(3 * BN)));
    SEAS_TRY(s->dring.alloc(c, (size_t)s->dring_len));
    SEAS_TRY(s->fmodes.alloc(c, (size_t)(op->n_modes_total * (int64_t)batch)));
    SEAS_TRY(s->h_in.alloc((size_t)(2 * BN) * sizeof(double)));
    SEAS_TRY(s->h_out.alloc((size_t)(4 * BN) * sizeof(double)));
    if (op->tail) {
        SEAS_TRY(s->sring.alloc(c, (size_t)((op->ring + 1) * BN)));
        SEAS_TRY(s->sring.zero(c->stream));
    }
    for (DArr<double> *d : {&s->vring, &s->slip, &s->slip_prev, &s->fint}) SEAS_TRY(d->zero(c->stream));
    SEAS_TRY(s->dring.zero(c->stream));
    SEAS_TRY(s->fmodes.zero(c->stream));
    return SEAS_OK;
}

}  // namespace

extern "C" seas_status seas_scenario_create(seas_op *op, int batch, seas_scn **out) {
    if (!op || !out) return fail(SEAS_EINVAL, "NULL argument");
    *out = nullptr;
    if (batch < 1 || batch > kMaxBatch) return fail(SEAS_EINVAL, "batch must be in [1, %d]", kMaxBatch);
    const int xb = op->hp.precision == kPrecBF16 || op->hp.precision == kPrecFP16 ? 4 : 8;
    if (op->hp.precision == kPrecBF16 && batch > 4) {
        // the tensor-core consumers of BF16 batches of 5..8 tile at most 128 receivers of a block
        int max_p = 0;
        for (const BlockDev &b : op->blocks_h) max_p = std::max(max_p, b.p);
        if (pad_row(max_p, kPrecBF16) > 128)
            return fail(SEAS_EINVAL, "BF16 batches of 5..8 need blocks of at most 128 receivers (widest: %d)", max_p);
    }
    {
        // one row of a pass-1 run plus its history slice must fit a pipeline stage (pass-2 items always do)
        const int eb = elem_bytes(op->hp.precision);
        for (size_t b = 0; b < op->blocks_h.size(); ++b) {
            if (!op->block_far[b]) continue;
            const int64_t q2 = pad_row(op->blocks_h[b].q, op->hp.precision);
            const int xw = xsplit_of(op->hp.precision, batch) ? 8 : batch;
            if (q2 * eb + (q2 * xw * xb + 15) / 16 * 16 + 16 + 48 > kStageBytes)
                return fail(SEAS_EINVAL, "batch %d too large for blocks of %d columns (stage of %d bytes)", batch,
                            op->blocks_h[b].q, kStageBytes);
        }
    }
    CUDA_TRY(cudaSetDevice(op->net->ctx->device));
    std::unique_ptr<seas_scn> s;
    SEAS_TRY(scenario_alloc(op, batch, s));
    CUDA_TRY(cudaStreamSynchronize(op->net->ctx->stream));
    op->children++;
    *out = s.release();
    return SEAS_OK;
}



namespace {

// Reads the device error word (set by a bounded wait that ran out); the stream must be synchronised.
seas_status check_device_error(seas_scn &s) {
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, s.counter_err.p + 1, sizeof(int), cudaMemcpyDeviceToHost));
    return device_error_status(err);
}

constexpr size_t kEventPairs = 8192;

seas_status timing_resolve(seas_scn &s) {
    if (s.ev_used == 0) return SEAS_OK;
    CUDA_TRY(cudaEventSynchronize(s.ev[2 * s.ev_used - 1]));
    for (size_t i = 0; i < s.ev_used; ++i) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, s.ev[2 * i], s.ev[2 * i + 1]));
        s.acc.ms[s.ev_class[i]] += ms;
        s.acc.launches[s.ev_class[i]] += 1;
    }
    s.ev_used = 0;
    return SEAS_OK;
}

// Runs one launch, bracketed by an event pair of class `cls` when timing is on.
template <class F>
seas_status timed(seas_scn &s, int cls, F &&launch) {
    cudaStream_t st = s.op->net->ctx->stream;
    if (!s.timing) {
        CUDA_TRY(launch());
        return SEAS_OK;
    }
    if (s.ev_used == kEventPairs) SEAS_TRY(timing_resolve(s));
    CUDA_TRY(cudaEventRecord(s.ev[2 * s.ev_used], st));
    CUDA_TRY(launch());
    CUDA_TRY(cudaEventRecord(s.ev[2 * s.ev_used + 1], st));
    s.ev_class[s.ev_used++] = cls;
    return SEAS_OK;
}

}  // namespace

extern "C" seas_status seas_scenario_set_timing(seas_scn *s, int enable) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    CUDA_TRY(cudaSetDevice(s->op->net->ctx->device));
    CUDA_TRY(cudaStreamSynchronize(s->op->net->ctx->stream));
    s->ev_used = 0;
    s->acc = seas_timing{};
    s->timing = enable != 0;
    if (s->timing && s->ev.empty()) {
        // events are created here, not by the first timed launch, so that timing adds no creation cost to a step
        s->ev.resize(2 * kEventPairs);
        s->ev_class.resize(kEventPairs);
        for (cudaEvent_t &e : s->ev) CUDA_TRY(cudaEventCreate(&e));
    }
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_get_timing(seas_scn *s, seas_timing *out) {
    if (!s || !out) return fail(SEAS_EINVAL, "NULL argument");
    CUDA_TRY(cudaSetDevice(s->op->net->ctx->device));
    SEAS_TRY(timing_resolve(*s));
    *out = s->acc;
    return SEAS_OK;
}

extern "C" seas_status seas_op_step_bytes(const seas_op *op, int64_t step, int64_t *bytes) {
    if (!op || !bytes || step < 0) return fail(SEAS_EINVAL, "bad argument");
    if (op->bytes_upto.empty()) {
        *bytes = 0;
        return SEAS_OK;
    }
    *bytes = op->bytes_upto[(size_t)std::min<int64_t>(step, (int64_t)op->bytes_upto.size() - 1)];
    return SEAS_OK;
}

extern "C" seas_status seas_push_slip_rate(seas_scn *s, const double *V, const double *slip, int mem,
                                           int replace_last) {
    return seas_push_slip_rate_steps(s, V, slip, mem, 1, replace_last);
}

extern "C" seas_status seas_push_slip_rate_steps(seas_scn *s, const double *V, const double *slip, int mem, int gamma,
                                                 int replace_last) {
    if (!s || !V) return fail(SEAS_EINVAL, "NULL argument");
    if (mem != SEAS_MEM_HOST && mem != SEAS_MEM_DEVICE) return fail(SEAS_EINVAL, "mem must be HOST or DEVICE");
    if (gamma < 1) return fail(SEAS_EINVAL, "gamma must be >= 1");
    seas_op &op = *s->op;
    seas_ctx *c = op.net->ctx;
    if (replace_last && s->n == 0) return fail(SEAS_ESTATE, "replace_last before the first push");
    if (replace_last && gamma != s->last_gamma)
        return fail(SEAS_EINVAL, "replace_last with gamma %d: the last push held %d steps", gamma, s->last_gamma);
    if (!replace_last && !(op.hp.flags & SEAS_FLAG_LAG_CAP))
        for (int b = 0; b < s->B; ++b)
            if (s->active[b] && s->n - s->start[b] + gamma > op.hp.max_steps)
                return fail(SEAS_ESTATE, "push %lld of member %d beyond max_steps %d",
                            (long long)(s->n - s->start[b] + gamma - 1), b, op.hp.max_steps);
    CUDA_TRY(cudaSetDevice(c->device));
    const int64_t BN = (int64_t)s->B * op.net->N_io;     // the caller's elements
    const double *dV = V, *dS = slip;
    if (mem == SEAS_MEM_HOST) {
        for (int64_t i = 0; i < BN; ++i)
            if (!std::isfinite(V[i])) return fail(SEAS_EINVAL, "non-finite slip rate at index %lld", (long long)i);
        if (slip)
            for (int64_t i = 0; i < BN; ++i)
                if (!std::isfinite(slip[i])) return fail(SEAS_EINVAL, "non-finite slip at index %lld", (long long)i);
        double *hin = static_cast<double *>(s->h_in.p);
        CUDA_TRY(cudaStreamSynchronize(c->stream));   // the staging buffer may still feed a previous copy
        std::memcpy(hin, V, BN * sizeof(double));
        CUDA_TRY(cudaMemcpyAsync(s->d_V.p, hin, BN * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        dV = s->d_V.p;
        if (slip) {
            std::memcpy(hin + BN, slip, BN * sizeof(double));
            CUDA_TRY(cudaMemcpyAsync(s->d_slip.p, hin + BN, BN * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            dS = s->d_slip.p;
        }
    }
    const int64_t tick0 = replace_last ? s->n - gamma : s->n;
    for (int j = 1; j <= gamma; ++j) {
        StepArgs a = step_args(*s, tick0 + j - 1);
        SEAS_TRY(timed(*s, 0, [&] { return launch_push(a, dV, dS, replace_last, j, gamma, c->stream); }));
        SEAS_TRY(timed(*s, 1, [&] { return launch_fft_forward(a, c->stream); }));
    }
    if (!replace_last) s->n += gamma;
    s->last_gamma = gamma;
    return SEAS_OK;
}

// The step's kernels after the push.  The self-term mode convolution depends on neither interaction pass, and its
// blocks use no shared memory, so they run beside the persistent interaction CTAs: it goes to the scenario's side
// stream between a fork event on `st` and a join before the assembly, which needs both.
static cudaError_t launch_step_kernels(seas_scn &s, const StepArgs &a, double *tau, double *parts, cudaStream_t st) {
    // the source pass is enqueued first, so the persistent interaction CTAs take their SMs first and the
    // convolution's blocks fill what is left beside them (the side stream has the lowest priority)
    cudaError_t e = cudaEventRecord(s.fork_ev, st);
    if (e == cudaSuccess) e = launch_interaction(a, 1, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s.side, s.fork_ev, 0);
    if (e == cudaSuccess) e = launch_modeconv(a, s.side);
    if (e == cudaSuccess) e = cudaEventRecord(s.join_ev, s.side);
    if (e == cudaSuccess) e = launch_interaction(a, 2, st);
    if (e == cudaSuccess) e = launch_reduce(a, st);
    if (e == cudaSuccess) e = launch_static_tail(a, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s.join_ev, 0);
    if (e == cudaSuccess) e = launch_ifft_assemble(a, tau, parts, st);
    return e;
}

extern "C" seas_status seas_stress_step(seas_scn *s, double *tau, double *sigma_n, double *parts, int mem) {
    if (!s || !tau) return fail(SEAS_EINVAL, "NULL argument");
    if (mem != SEAS_MEM_HOST && mem != SEAS_MEM_DEVICE) return fail(SEAS_EINVAL, "mem must be HOST or DEVICE");
    if (s->n == 0) return fail(SEAS_ESTATE, "stress_step before the first push");
    seas_op &op = *s->op;
    seas_ctx *c = op.net->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    const int64_t BN = (int64_t)s->B * op.net->N_io;     // the caller's elements
    StepArgs a = step_args(*s, s->n - 1);
    double *dtau = mem == SEAS_MEM_DEVICE ? tau : s->d_tau.p;
    double *dparts = parts ? (mem == SEAS_MEM_DEVICE ? parts : s->d_parts.p) : nullptr;
    if (!s->timing) {
        CUDA_TRY(launch_step_kernels(*s, a, dtau, dparts, c->stream));
    } else {
        // per-kernel events: the kernels one after another on the step's stream
        SEAS_TRY(timed(*s, 2, [&] { return launch_modeconv(a, c->stream); }));
        SEAS_TRY(timed(*s, 6, [&] { return launch_interaction(a, 1, c->stream); }));
        SEAS_TRY(timed(*s, 3, [&] { return launch_interaction(a, 2, c->stream); }));
        SEAS_TRY(timed(*s, 4, [&] {
            const cudaError_t e = launch_reduce(a, c->stream);
            return e != cudaSuccess ? e : launch_static_tail(a, c->stream);
        }));
        SEAS_TRY(timed(*s, 5, [&] { return launch_ifft_assemble(a, dtau, dparts, c->stream); }));
    }
    if (s->timing) {
        int64_t b = 0;
        SEAS_TRY(seas_op_step_bytes(&op, s->n - 1, &b));
        s->acc.interaction_bytes += b;
        s->acc.steps += 1;
    }
    if (mem == SEAS_MEM_DEVICE) {
        if (sigma_n) CUDA_TRY(cudaMemsetAsync(sigma_n, 0, BN * sizeof(double), c->stream));
        return SEAS_OK;
    }
    double *hout = static_cast<double *>(s->h_out.p);
    CUDA_TRY(cudaMemcpyAsync(hout, dtau, BN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (parts)
        CUDA_TRY(cudaMemcpyAsync(hout + BN, dparts, 3 * BN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    SEAS_TRY(check_device_error(*s));
    std::memcpy(tau, hout, BN * sizeof(double));
    if (parts) std::memcpy(parts, hout + BN, 3 * BN * sizeof(double));
    if (sigma_n) std::memset(sigma_n, 0, BN * sizeof(double));
    return SEAS_OK;
}

extern "C" seas_status seas_stress_step_static(seas_scn *s, double *tau, double *parts) {
    // Same computation as seas_stress_step with device outputs, but nothing is allocated: the per-call scratch
    // (partial sums of the interaction tasks and the summed interaction term) is a static device array.
    if (!s || !tau) return fail(SEAS_EINVAL, "NULL argument");
    if (s->n == 0) return fail(SEAS_ESTATE, "stress_step before the first push");
    seas_op &op = *s->op;
    seas_ctx *c = op.net->ctx;
    const int64_t need = op.n_partial * s->B + (int64_t)s->B * op.net->N;
    if (need > kStaticScratchDoubles)
        return fail(SEAS_EINVAL, "static scratch too small: this scenario needs %lld doubles, the limit is %lld",
                    (long long)need, (long long)kStaticScratchDoubles);
    CUDA_TRY(cudaSetDevice(c->device));
    double *scratch = nullptr;
    CUDA_TRY(static_scratch(&scratch));               // first call on a device: symbol lookup (no allocation)
    StepArgs a = step_args(*s, s->n - 1);
    a.partial = scratch;
    a.fint = scratch + op.n_partial * s->B;
    CUDA_TRY(launch_step_kernels(*s, a, tau, parts, c->stream));
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_admit(seas_scn *s, int member) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    if (member < 0 || member >= s->B) return fail(SEAS_EINVAL, "member %d outside [0, %d)", member, s->B);
    seas_ctx *c = s->op->net->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    const StepArgs a = step_args(*s, s->n);
    CUDA_TRY(launch_reset_member(a, member, c->stream));
    s->start[member] = s->n;
    s->active[member] = 1;
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_retire(seas_scn *s, int member) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    if (member < 0 || member >= s->B) return fail(SEAS_EINVAL, "member %d outside [0, %d)", member, s->B);
    s->active[member] = 0;
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_member_step(const seas_scn *s, int member, int64_t *n) {
    if (!s || !n) return fail(SEAS_EINVAL, "NULL argument");
    if (member < 0 || member >= s->B) return fail(SEAS_EINVAL, "member %d outside [0, %d)", member, s->B);
    *n = s->active[member] ? s->n - s->start[member] : -1;
    return SEAS_OK;
}

namespace seas {

int scenario_view(const seas_scn *s, ScnView *v) {
    if (!s || !v) return fail(SEAS_EINVAL, "NULL argument");
    const seas_op &op = *s->op;
    v->stream = op.net->ctx->stream;
    v->device = op.net->ctx->device;
    v->B = s->B;
    v->N = op.net->N_io;
    v->dt = op.net->dt;
    v->rad = op.net->med.mu / (2.0 * op.net->med.cs);
    v->n = s->n;
    v->first_lag = op.task_T.empty() ? INT32_MAX : op.task_T.front();
    return SEAS_OK;
}

int scn_alloc(seas_scn *s, size_t bytes, void **p) { return dev_alloc(s->op->net->ctx, bytes, p); }

void scn_free(seas_scn *s, void *p, size_t bytes) { dev_free(s->op->net->ctx, p, bytes); }

}  // namespace seas

extern "C" seas_status seas_scenario_set_wait_limit(seas_scn *s, double seconds) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    if (!(std::isfinite(seconds) && seconds >= 1e-6 && seconds <= 60.0))
        return fail(SEAS_EINVAL, "wait limit %g s outside [1e-6, 60]", seconds);
    s->wait_ns = (uint64_t)(seconds * 1e9);
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_probe_wait(seas_scn *s) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    seas_ctx *c = s->op->net->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    const StepArgs a = step_args(*s, s->n > 0 ? s->n - 1 : 0);
    CUDA_TRY(launch_wait_probe(a, c->stream));
    return SEAS_OK;
}

// ------------------------------------------------------------------------------------------------------------
// autotuner: the consumer warp count of each interaction pass, by measurement
// ------------------------------------------------------------------------------------------------------------

namespace {

// Key of a tuning choice: the device, the precision and batch, and the shape of the operator's work (units, tasks
// and bytes of both passes), so that a cached choice is reused only for the same work on the same kind of GPU.
std::string tune_key(const seas_scn &s) {
    const seas_op &op = *s.op;
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, op.net->ctx->device);
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == ' ' || ch == '|') ch = '_';
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d|prec%d|B%d|tasks%zu|ztasks%zu|items%zu|runs%zu|bytes%lld|steps%d", name.c_str(),
             op.net->ctx->n_sms, op.hp.precision, s.B, op.task_T.size(), op.ztask_T.size(), op.d_items.n,
             op.d_runs.n, (long long)op.stats.bytes_interaction, op.hp.max_steps);
    return buf;
}

bool tune_lookup(const char *path, const std::string &key, int *cw) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool hit = false;
    while (fgets(line, sizeof line, f)) {
        const size_t n = key.size();
        if (strncmp(line, key.c_str(), n) == 0 && line[n] == ' ') {
            int a = 0, b = 0;
            if (sscanf(line + n + 1, "%d %d", &a, &b) == 2 && (a == 8 || a == 16) && (b == 8 || b == 16)) {
                cw[0] = a;                 // the last matching line wins
                cw[1] = b;
                hit = true;
            }
        }
    }
    fclose(f);
    return hit;
}

}  // namespace

extern "C" seas_status seas_scenario_autotune(seas_scn *s, const char *cache_path, int reps, seas_tune *out) {
    if (!s || !out) return fail(SEAS_EINVAL, "NULL argument");
    if (reps < 1 || reps > 100) return fail(SEAS_EINVAL, "reps %d outside [1, 100]", reps);
    if (s->gexec) return fail(SEAS_ESTATE, "the scenario has a captured step: its kernels are fixed");
    if (s->timing) return fail(SEAS_ESTATE, "kernel timing is on");
    seas_op &op = *s->op;
    seas_ctx *c = op.net->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    *out = seas_tune{};
    for (int p = 0; p < 2; ++p) {
        int opts[2] = {0, 0};
        const int n = interaction_options(op.hp.precision, s->B, p + 1, opts);
        for (int k = 0; k < n; ++k) out->candidates[p][k] = opts[k];
    }
    const std::string key = tune_key(*s);
    int cached[2] = {0, 0};
    if (cache_path && tune_lookup(cache_path, key, cached)) {
        for (int p = 0; p < 2; ++p) {
            const bool ok = cached[p] == out->candidates[p][0] || cached[p] == out->candidates[p][1];
            s->cw[p] = ok ? cached[p] : 0;
            out->consumer_warps[p] = ok ? cached[p] : out->candidates[p][0];
        }
        out->from_cache = 1;
        return SEAS_OK;
    }
    // every task active at the deepest lag: the passes' work does not depend on the history's values, and their
    // scratch (z rows, partial sums) is recomputed by the next step
    StepArgs a = step_args(*s, s->n > 0 ? s->n - 1 : 0);
    a.lag_max = op.ring - 1;
    a.n_tasks_active = (int)op.task_T.size();
    a.n_ztasks_active = (int)op.ztask_T.size();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        CUDA_TRY(ce);
    }
    for (int p = 0; p < 2 && ce == cudaSuccess; ++p) {
        double best = 0;
        for (int k = 0; k < 2 && ce == cudaSuccess; ++k) {
            const int cw = out->candidates[p][k];
            if (!cw) continue;
            a.cw[p] = cw;
            std::vector<float> t;
            for (int r = 0; r <= reps && ce == cudaSuccess; ++r) {      // launch 0 is untimed
                ce = cudaMemsetAsync(s->counter_err.p + (p == 0 ? 2 : 0), 0, sizeof(int), c->stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(e0, c->stream);
                if (ce == cudaSuccess) ce = launch_interaction(a, p + 1, c->stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
                if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                float ms = 0;
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) t.push_back(ms);
            }
            if (ce != cudaSuccess) break;
            std::sort(t.begin(), t.end());
            out->ms[p][k] = t[t.size() / 2];
            if (best == 0 || out->ms[p][k] < best) {
                best = out->ms[p][k];
                out->consumer_warps[p] = cw;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(ce);
    // counters back to zero for the next step (its reduction would reset them too)
    CUDA_TRY(cudaMemsetAsync(s->counter_err.p, 0, sizeof(int), c->stream));
    CUDA_TRY(cudaMemsetAsync(s->counter_err.p + 2, 0, sizeof(int), c->stream));
    SEAS_TRY(seas_scenario_check(s));
    for (int p = 0; p < 2; ++p) s->cw[p] = out->consumer_warps[p];
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return fail(SEAS_EINVAL, "cannot append to tuning cache %s", cache_path);
        fprintf(f, "%s %d %d %.6f %.6f %.6f %.6f\n", key.c_str(), s->cw[0], s->cw[1], out->ms[0][0], out->ms[0][1],
                out->ms[1][0], out->ms[1][1]);
        fclose(f);
    }
    return SEAS_OK;
}

namespace {
constexpr int64_t kDynRing = 1024;     // pinned host copies of per-step values in flight
}

extern "C" seas_status seas_scenario_graph_create(seas_scn *s, const double *V, double *tau, double *parts) {
    if (!s || !V || !tau) return fail(SEAS_EINVAL, "NULL argument");
    if (s->gexec) return fail(SEAS_ESTATE, "the scenario already has a captured step");
    if (s->timing) return fail(SEAS_ESTATE, "kernel timing is on: a captured step records no timing events");
    seas_op &op = *s->op;
    seas_ctx *c = op.net->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    SEAS_TRY(s->d_dyn.alloc(c, 1));
    SEAS_TRY(s->h_dyn.alloc(sizeof(DynDev) * kDynRing));
    for (cudaEvent_t &e : s->dyn_ev)
        if (!e) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    StepArgs a = step_args(*s, s->n);
    a.dyn = s->d_dyn.p;
    // captured on a stream of its own (the context's stream may be the legacy default stream, which cannot be
    // captured); the graph is launched on the context's stream
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    cudaStream_t st = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{st};
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    cudaError_t e = launch_push(a, V, nullptr, 0, 1, 1, st);
    if (e == cudaSuccess) e = launch_fft_forward(a, st);
    if (e == cudaSuccess) e = launch_step_kernels(*s, a, tau, parts, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(SEAS_ECUDA, "step capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t x = nullptr;
    const cudaError_t e3 = cudaGraphInstantiate(&x, g, 0);
    if (e3 != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(SEAS_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e3));
    }
    s->graph = g;
    s->gexec = x;
    s->dyn_used = 0;
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_graph_step(seas_scn *s) {
    if (!s) return fail(SEAS_EINVAL, "NULL scenario");
    if (!s->gexec) return fail(SEAS_ESTATE, "no captured step (seas_scenario_graph_create)");
    seas_op &op = *s->op;
    seas_ctx *c = op.net->ctx;
    if (!(op.hp.flags & SEAS_FLAG_LAG_CAP))
        for (int b = 0; b < s->B; ++b)
            if (s->active[b] && s->n - s->start[b] >= op.hp.max_steps)
                return fail(SEAS_ESTATE, "push %lld of member %d beyond max_steps %d",
                            (long long)(s->n - s->start[b]), b, op.hp.max_steps);
    CUDA_TRY(cudaSetDevice(c->device));
    // a ring slot is written again only after the uploads issued kDynRing steps earlier have run
    const int64_t i = s->dyn_used;
    if (i % (kDynRing / 4) == 0) {
        cudaEvent_t &ev = s->dyn_ev[(i / (kDynRing / 4)) % 4];
        if (i >= kDynRing) CUDA_TRY(cudaEventSynchronize(ev));
        CUDA_TRY(cudaEventRecord(ev, c->stream));
    }
    s->n++;
    s->last_gamma = 1;
    const StepArgs a = step_args(*s, s->n - 1);
    DynDev *h = static_cast<DynDev *>(s->h_dyn.p) + (i % kDynRing);
    *h = DynDev{a.step, a.lag_max, a.n_tasks_active, a.n_ztasks_active};
    CUDA_TRY(cudaMemcpyAsync(s->d_dyn.p, h, sizeof(DynDev), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaGraphLaunch(s->gexec, c->stream));
    s->dyn_used++;
    return SEAS_OK;
}

extern "C" seas_status seas_scenario_step(const seas_scn *s, int64_t *n) {
    if (!s || !n) return fail(SEAS_EINVAL, "NULL argument");
    *n = s->n;
    return SEAS_OK;
}

extern "C" seas_status seas_destroy_scn(seas_scn *s) {
    if (!s) return SEAS_OK;
    cudaSetDevice(s->op->net->ctx->device);
    cudaStreamSynchronize(s->op->net->ctx->stream);
    s->op->children--;
    delete s;
    return SEAS_OK;
}

// ------------------------------------------------------------------------------------------------------------
// checkpoint / resume
// ------------------------------------------------------------------------------------------------------------

namespace {

struct CkptHeader {
    char magic[8];
    int32_t version, B, N, F;
    int64_t n, ring, dring_len, n_modes_total;
};

seas_status dump(FILE *fp, const void *dev, size_t bytes) {
    std::vector<char> h(bytes);
    if (bytes) CUDA_TRY(cudaMemcpy(h.data(), dev, bytes, cudaMemcpyDeviceToHost));
    if (bytes && fwrite(h.data(), 1, bytes, fp) != bytes) return fail(SEAS_EIO, "short write");
    return SEAS_OK;
}

seas_status slurp(FILE *fp, void *dev, size_t bytes) {
    std::vector<char> h(bytes);
    if (bytes && fread(h.data(), 1, bytes, fp) != bytes) return fail(SEAS_EIO, "short read");
    if (bytes) CUDA_TRY(cudaMemcpy(dev, h.data(), bytes, cudaMemcpyHostToDevice));
    return SEAS_OK;
}

}  // namespace

extern "C" seas_status seas_scenario_save(seas_scn *s, const char *path) {
    if (!s || !path) return fail(SEAS_EINVAL, "NULL argument");
    seas_op &op = *s->op;
    CUDA_TRY(cudaSetDevice(op.net->ctx->device));
    CUDA_TRY(cudaStreamSynchronize(op.net->ctx->stream));
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(SEAS_EIO, "cannot open %s for writing", path);
    CkptHeader h{};
    std::memcpy(h.magic, "SEASCKP1", 8);
    h.version = 3;
    h.B = s->B;
    h.N = op.net->N;
    h.F = op.net->F;
    h.n = s->n;
    h.ring = op.ring;
    h.dring_len = s->dring_len;
    h.n_modes_total = op.n_modes_total;
    seas_status st = SEAS_OK;
    if (fwrite(&h, sizeof h, 1, fp) != 1) st = fail(SEAS_EIO, "short write");
    if (st == SEAS_OK && (fwrite(s->start.data(), sizeof(int64_t), s->B, fp) != (size_t)s->B ||
                          fwrite(s->active.data(), 1, s->B, fp) != (size_t)s->B ||
                          fwrite(&s->horizon, sizeof(int64_t), 1, fp) != 1))
        st = fail(SEAS_EIO, "short write");
    if (st == SEAS_OK) st = dump(fp, s->vring.p, s->vring.bytes());
    if (st == SEAS_OK) st = dump(fp, s->slip.p, s->slip.bytes());
    if (st == SEAS_OK) st = dump(fp, s->slip_prev.p, s->slip_prev.bytes());
    if (st == SEAS_OK) st = dump(fp, s->dring.p, s->dring.bytes());
    if (st == SEAS_OK) st = dump(fp, s->xring.p, s->xring.bytes());
    if (st == SEAS_OK) st = dump(fp, s->sring.p, s->sring.bytes());
    if (fclose(fp) != 0 && st == SEAS_OK) st = fail(SEAS_EIO, "close failed");
    return st;
}

extern "C" seas_status seas_scenario_load(seas_op *op, const char *path, seas_scn **out) {
    if (!op || !path || !out) return fail(SEAS_EINVAL, "NULL argument");
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(op->net->ctx->device));
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(SEAS_EIO, "cannot open %s", path);
    CkptHeader h{};
    if (fread(&h, sizeof h, 1, fp) != 1 || std::memcmp(h.magic, "SEASCKP1", 8) != 0 || h.version != 3) {
        fclose(fp);
        return fail(SEAS_EIO, "%s is not a scenario checkpoint", path);
    }
    if (h.N != op->net->N || h.F != op->net->F || h.ring != op->ring || h.n_modes_total != op->n_modes_total ||
        h.B < 1 || h.n < 0) {
        fclose(fp);
        return fail(SEAS_EIO, "checkpoint does not match this operator");
    }
    if (h.B > kMaxBatch) {
        fclose(fp);
        return fail(SEAS_EIO, "checkpoint batch %d exceeds %d", h.B, kMaxBatch);
    }
    std::vector<int64_t> start(h.B);
    std::vector<char> active(h.B);
    int64_t horizon = -1;
    if (fread(start.data(), sizeof(int64_t), h.B, fp) != (size_t)h.B || fread(active.data(), 1, h.B, fp) != (size_t)h.B ||
        fread(&horizon, sizeof(int64_t), 1, fp) != 1) {
        fclose(fp);
        return fail(SEAS_EIO, "%s: truncated member table", path);
    }
    std::unique_ptr<seas_scn> s;
    seas_status st = scenario_alloc(op, h.B, s);
    if (st == SEAS_OK && h.dring_len != s->dring_len) st = fail(SEAS_EIO, "checkpoint spectral ring size mismatch");
    if (st == SEAS_OK) {
        const cudaError_t e = cudaStreamSynchronize(op->net->ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(SEAS_ECUDA, "cudaStreamSynchronize failed: %s", cudaGetErrorString(e));
        }
    }
    if (st == SEAS_OK) st = slurp(fp, s->vring.p, s->vring.bytes());
    if (st == SEAS_OK) st = slurp(fp, s->slip.p, s->slip.bytes());
    if (st == SEAS_OK) st = slurp(fp, s->slip_prev.p, s->slip_prev.bytes());
    if (st == SEAS_OK) st = slurp(fp, s->dring.p, s->dring.bytes());
    if (st == SEAS_OK) st = slurp(fp, s->xring.p, s->xring.bytes());
    if (st == SEAS_OK) st = slurp(fp, s->sring.p, s->sring.bytes());
    fclose(fp);
    if (st != SEAS_OK) return st;
    s->n = h.n;
    s->start = start;
    s->active = active;
    s->horizon = horizon;
    op->children++;
    *out = s.release();
    return SEAS_OK;
}

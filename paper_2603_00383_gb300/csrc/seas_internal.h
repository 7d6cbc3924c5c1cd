// Internal declarations shared by the host orchestration (seas_api.cu), the operator-build kernels
// (seas_build.cu) and the per-step kernels (seas_step.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "seas.h"

namespace seas {

constexpr int kThreads = 256;       // threads per CTA of every kernel
constexpr int kMaxFFT = 7168;       // largest N_f: two N_f-point complex buffers fit in shared memory
constexpr int kMaxStages = 16;      // radix stages of one FFT plan
constexpr int kFftCluster = 8;      // CTAs of the thread-block cluster that runs one large fault's FFT
constexpr int kFftClusterMin = 2048;  // N_f from which a fault's FFTs run on a cluster (when N_f factors suitably)
constexpr int kMaxBlockSide = 1024; // rows / columns of one H-matrix block (4 accumulator rows per thread)
constexpr int kRowsPerThread = kMaxBlockSide / kThreads;
constexpr int kItemRows = 256;      // rows of one pass-2 item (bounds its staged history / z rows)
constexpr int kMaxBatch = 8;        // scenarios per scenario handle (one pass of the interaction kernel)
constexpr int kItemBytes = 24 * 1024;   // largest pass-2 item (operator bytes)
constexpr int kStageBytes = 68 * 1024;  // one shared-memory stage of the interaction pipeline
constexpr int kStages = 3;              // stages in flight per CTA
constexpr int kStageItems = 31;         // units per stage (one producer lane each)
constexpr int64_t kTaskBytes = 1 << 20; // operator bytes per task (one deterministic partial sum)
constexpr int kCopyTail = 1024;         // bytes past the history ring and z buffer that widened copies may read

__host__ __device__ inline int pad2(int n) { return n + (n & 1); }

// BF16 operators with batches of 5..8 run on the tensor-core consumers, whose B operands (history and z rows) are
// stored pre-split into bfloat16 (high, low) pairs, 8 scenarios wide.
__host__ __device__ inline bool xsplit_of(int prec, int batch) { return prec == 1 && batch > 4; }

// Storage precision of the interaction operator (values of seas_hparams::precision).
constexpr int kPrecFP64 = 0;   // double entries, FP64 arithmetic
constexpr int kPrecBF16 = 1;   // bfloat16 entries, FP32 arithmetic with compensated accumulation
constexpr int kPrecFP16 = 2;   // float16 entries with a per-slice scale, FP32 compensated accumulation
constexpr int kPrecDF64 = 3;   // FP32 (hi, lo) pairs, double-float arithmetic on the FP32 pipes

__host__ __device__ inline int elem_bytes(int prec) { return prec == kPrecBF16 || prec == kPrecFP16 ? 2 : 8; }
// Row length padded so that every row starts on a 16-byte boundary.
__host__ __device__ inline int pad_row(int n, int prec) {
    const int e = 16 / elem_bytes(prec);
    return (n + e - 1) / e * e;
}

// Rows of 2-byte operator units (BF16, FP16) are stored with their 16-byte chunks rotated: logical chunk c of row r
// (counted from the unit's first row) of a unit whose rows have nch chunks sits at chunk (c + rot) mod nch, rot =
// (r / period) mod g with g = gcd(nch, 8) and period = 8 / g.  Then the same logical chunk of 8 consecutive rows falls
// in 8 different 16-byte bank groups of shared memory whatever the row length, so the matrix loads of the tensor-core
// consumers (8 rows, one chunk each) are conflict free.  The operator build applies it once; every consumer of a
// 2-byte arena reads through it.
__host__ __device__ inline int chunk_rot(int r, int nch) {
    int g = nch & -nch;
    if (g > 8) g = 8;
    const int shift = g == 8 ? 0 : g == 4 ? 1 : g == 2 ? 2 : 3;   // log2(8 / g)
    return (r >> shift) & (g - 1);
}
__host__ __device__ inline int chunk_at(int c, int r, int nch) {
    const int q = c + chunk_rot(r, nch);
    return q >= nch ? q - nch : q;
}

// One fault of the spectral self-effect path.
struct FaultDev {
    int32_t off;        // first element (global index)
    int32_t nf;         // N_f (complex FFT size); the padded real transform has M = 2 N_f points
    int32_t mode_off;   // first entry of this fault in the per-mode arrays (N_f + 1 entries, modes 0..N_f)
    int32_t ring;       // R_f: slots of the spectral history ring
    int64_t dring_off;  // first double2 of this fault's ring: [batch][N_f + 1][R_f]
    int64_t tw_off;     // first double2 of the twiddles: N_f entries e^{-2 pi i k/N_f}, then N_f + 1 entries
                        // e^{-2 pi i k/(2 N_f)}
    int32_t nstages;
    int32_t radix[kMaxStages];
    double kfac;        // -(mu / 2) * pi / L_f, so that F_n = kfac * n * sum_T w_n^T D_n^{t-T}
    // four-step plan of a large fault's FFT on a cluster of kFftCluster CTAs: N_f = n1 n2, both multiples of
    // kFftCluster (n1 = 0: the fault's FFTs run on one CTA)
    int32_t n1, n2, nst1, nst2;
    int32_t radix1[kMaxStages], radix2[kMaxStages];
};

// One spectral mode n >= 1 of one fault.
struct ModeDev {
    int64_t w_off;      // first weight of w_n^0..w_n^W
    int32_t W;          // last lag of the window
    int32_t fault;
    int32_t n;
    int32_t pad;
    double tailc;       // static tail: weight mass beyond the window, (2/pi) Si(n pi) - sum_{T<=W} w_n^T (0: none)
};

// One H-matrix block: receiver rows [r0, r0 + p), source columns [c0, c0 + q) (global element indices).
struct BlockDev {
    int32_t r0, p, c0, q;
};

// The interaction runs in two passes per step (two launches of the persistent kernel):
//   pass 1 (source side): for every far slice (b, T), z = V_{b,T}^T x^{step - T}, with x the slip-rate history of the
//     block's source columns.  Work is grouped by source cluster: a run holds the V^T rows (q2 elements each) of all
//     far slices with the same source columns at one lag, so one staged history slice serves all of them; each
//     row's z goes to the z buffer row given by zmap.
//   pass 2 (receiver side): for every block, y += sum over its slices of U_{b,T} z (far) or A_{b,T}^T x (dense),
//     accumulated per task over consecutive lags and written to the task's partial rows.
// The z buffer of a scenario has one row per row of the pass-2 arena ([row][batch]); rows of dense slices are
// unused.  Work that needs no history beyond the scenario's start multiplies zeros, so whole tasks are switched on
// by their first lag only.

// Pass-2 unit: rows of one block stored contiguously at `a` (rows of p2 = pad_row(p) elements of the storage
// precision).  Consecutive items of a task are adjacent in memory.
//   dense (k < 0): rows i0..i1-1 of A^T of one lag T:  y += sum_j A^T[j][:] x_{c0+j}^{step-T}
//   far   (k > 0): k rows of U^T of consecutive lags from T on, whose z rows are zrow .. zrow + k - 1
struct ItemDev {
    int32_t T;
    int32_t k;
    int32_t i0, i1;
    const void *a;
    float scale;        // dense: stored values times scale = operator values (1 except FP16); far: 1 (pass 1 scales z)
    int32_t pad;
    int64_t zrow;
};

// Pass-1 unit: `rows` V^T rows (q2 elements each) at `v`, the far slices of one source cluster at lag T; row r's z
// goes to z row zmap[map + r] (times zscale[map + r] for FP16).  Consecutive runs of a task are adjacent in memory.
struct RunDev {
    int32_t T;
    int32_t rows;
    const void *v;
    int64_t map;
};

// A run of units whose rows share one partial slot (pass 2: items of one block; pass 1: runs of one source
// cluster at consecutive lags, `block` then names the source cluster).  Pass 2 partial sums:
// partial[b * n_partial + part_off + row].
struct TaskDev {
    int32_t block;
    int32_t item_begin;
    int32_t item_end;
    int32_t T_start;
    int64_t part_off;
};

// Source cluster of pass 1: columns [c0, c0 + q).
struct SrcDev {
    int32_t c0, q;
};

// One (block, lag) slice produced during the build.
struct SliceGen {
    int32_t block;
    int32_t T;
    int32_t far;        // 1: admissible (compress), 0: near (store dense)
    int32_t pad;
    int64_t scratch;    // first double of its p*q entries (layout A^T: q rows of p) in the scratch buffers
};

// Result of compressing one slice.
struct SliceOut {
    int32_t k;          // 0: zero slice, -1: dense, > 0: rank
    int32_t pad;
    double norm;        // Frobenius norm of the slice
    double resid;       // Frobenius norm of the residual (low rank) or 0
};

// ---- build kernels (seas_build.cu) ----
struct GeomDev {
    const double2 *x;     // centroids
    const double2 *e1;    // along-fault unit vectors
    const double2 *nrm;   // normals
    const double *ds;     // element lengths
    double cs, dt, scale; // scale = -mu / (2 c_s)
};

cudaError_t launch_gen_slices(const GeomDev &g, const BlockDev *blocks, const SliceGen *slices, int n_slices,
                              const int64_t *entry_prefix, int64_t n_entries, double *scratch, cudaStream_t s);
cudaError_t launch_compress(const BlockDev *blocks, const SliceGen *slices, int n_slices, const double *scratch,
                            double *resid, double *factors, SliceOut *out, double tol, cudaStream_t s);
cudaError_t launch_pack(const BlockDev *blocks, const SliceGen *slices, const SliceOut *out, int n_slices,
                        const double *scratch, const double *factors, const int64_t *dst_off, void *dst,
                        const int64_t *vdst_off, void *vdst, float *scales, int prec, cudaStream_t s);
// dst[i] = src[i] for n runs of bytes[i] bytes (16-byte multiples, 16-byte aligned)
cudaError_t launch_gather(const void *const *src, void *const *dst, const int32_t *bytes, int n, cudaStream_t s);
// One operator unit of a 2-byte arena for the chunk rotation: its first row, rows and 16-byte chunks per row.
struct UnitRows {
    void *p;
    int32_t rows, nch;
};
cudaError_t launch_rotate_rows(const UnitRows *units, int n, cudaStream_t s);
cudaError_t launch_spectral_tables(const ModeDev *modes, int n_modes, const int64_t *g_prefix, int64_t n_g,
                                   const double *mode_L, double cs_dt, const double *gl_x, const double *gl_w,
                                   int gl_n, double *G, double *w, cudaStream_t s);

// ---- step kernels (seas_step.cu) ----
// Per-step values a replayed CUDA graph reads from device memory instead of its baked kernel parameters.
struct DynDev {
    int64_t step, lag_max;
    int32_t n_tasks_active, n_ztasks_active;
};

struct StepArgs {
    int N, F, B, n_modes_total;   // elements, faults, batch, sum over the owned faults of (N_f + 1)
    int n_self;                   // faults with a spectral self effect in this operator (the owned ones)
    int max_nf;                   // largest N_f (shared memory of the FFT kernels)
    // caller's vectors (V, slip in; tau, parts out) with a free surface (method of images): N_io real elements per
    // scenario, io_map[i] = the real element of element i, -1 - j for the image of real element j; NULL otherwise
    // (the caller's layout is the network's, N per scenario)
    const int32_t *io_map;
    int N_io;
    // faults whose FFTs run on a thread-block cluster (indices into faults), and how many run on one CTA
    const int32_t *big;
    int n_big, n_small;
    int64_t step;                 // tick of the step being evaluated (ring slots are tick mod depth)
    int64_t lag_max;              // largest lag with nonzero history: the oldest active member's step (<= step);
                                  // members admitted later have zero history before their first tick
    int ring;                     // slip-rate ring depth R
    int64_t ring_stride;          // doubles per ring slot: layout [slot][element][scenario], padded to even + 2
    double dt, rad;               // rad = -mu / (2 c_s)
    const FaultDev *faults;
    const ModeDev *modes;         // modes n >= 1 of all faults
    int n_modes;
    const double *w;              // spectral weights
    const double2 *tw;            // FFT twiddles
    double *vring;                // [R][ring_stride]
    void *xring;                  // history in the operator's arithmetic: float2 (DF64) or float (BF16/FP16), same
                                  // layout; NULL for FP64.  Split layout (xsplit): 32 bytes per element, the bfloat16
                                  // high parts of scenarios 0..7 then their low parts (scenarios >= B zero)
    int prec;
    int xsplit;                   // 1: BF16 operator with a batch of 5..8 (tensor-core consumers): history and z rows
                                  // held as bfloat16 (high, low) pairs of their FP32 values, 8 scenarios wide
    double *slip, *slip_prev;     // [B][N]
    double2 *dring;               // spectral rings
    double2 *fmodes;              // [B][n_modes_total]
    double *fint;                 // [B][N]
    // interaction
    const BlockDev *blocks;
    const ItemDev *items;
    const TaskDev *tasks;
    int n_tasks_active;           // pass-2 tasks with T_start <= lag_max (a prefix of the T_start-sorted list)
    const RunDev *runs;           // pass 1
    const TaskDev *ztasks;
    const SrcDev *srcs;
    const int32_t *zmap;
    const float *zscale;          // FP16 only
    int n_ztasks_active;
    void *zbuf;                   // [z rows][B] in the arithmetic's dot type (double, float2 or float)
    int pass;                     // 1 or 2: which pass a launch of the interaction kernel runs
    int cw[2];                    // consumer warps of pass 1 and 2 (0: the default of the precision and batch)
    const DynDev *dyn;            // non-null in a captured step: step, lag_max and task counts come from here
    double *partial;              // [B][n_partial]
    int64_t n_partial;
    int *counter;                 // [0]: pass-2 task counter, [2]: pass-1 task counter (reset by the reduction)
    int *err;                     // device error word (bounded waits that ran out)
    uint64_t wait_ns;             // bound of one device wait (wall clock), per scenario
    // reduction: per element the blocks it receives from; per block its tasks' first lags
    const int32_t *cover_ptr, *cover_blk;
    const int32_t *blk_task_ptr, *blk_task_T;
    const int64_t *blk_part;      // first partial of each block
    int n_sms;
    // static tail (SEAS_FLAG_STATIC_TAIL): the elastostatic response of the history the windows drop
    int tail;                     // 1: on (the mode tails live in ModeDev::tailc)
    int sring_depth;              // slots of the slip ring
    double *sring;                // [sring_depth][N][B]: slip after each push
    const double *smat;           // [N][N]: -(mu / 2 c_s) A^static, receiver-major (same-fault entries unused)
    const int32_t *pair_last;     // [F][F]: last lag of each ordered fault pair's window
    const int32_t *block_last;    // with cluster-level windows: last lag of each block (NULL: the pair's)
};

// Allocation-free stepping (seas_stress_step_static): scratch in a static device array of this many doubles.
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 22;
constexpr int kMaxDevices = 64;
cudaError_t static_scratch(double **ptr);   // device address of the array on the current device

// View of a scenario for the earthquake-cycle integrator (seas_integ.cu), and device allocations charged to the
// scenario's context budget.
struct ScnView {
    cudaStream_t stream;
    int device, B, N;
    double dt, rad;          // rad = mu / (2 c_s)
    int64_t n;               // pushes so far
    int32_t first_lag;       // smallest lag of any stored interaction slice (INT32_MAX: none)
};
int scenario_view(const seas_scn *s, ScnView *v);
int scn_alloc(seas_scn *s, size_t bytes, void **p);
void scn_free(seas_scn *s, void *p, size_t bytes);

cudaError_t launch_push(const StepArgs &a, const double *V, const double *slip_in, int replace_last, int j,
                        int gamma, cudaStream_t s);
cudaError_t launch_fft_forward(const StepArgs &a, cudaStream_t s);
cudaError_t launch_modeconv(const StepArgs &a, cudaStream_t s);
cudaError_t launch_interaction(const StepArgs &a, int pass, cudaStream_t s);   // pass 1, then pass 2
// Consumer warp counts compiled for the interaction pass of a precision and batch (the default first); returns how
// many (1 or 2) it wrote to cw.
int interaction_options(int prec, int batch, int pass, int *cw);
cudaError_t launch_reduce(const StepArgs &a, cudaStream_t s);
cudaError_t launch_static_tail(const StepArgs &a, cudaStream_t s);
cudaError_t launch_ifft_assemble(const StepArgs &a, double *tau, double *parts, cudaStream_t s);
cudaError_t launch_wait_probe(const StepArgs &a, cudaStream_t s);
cudaError_t launch_reset_member(const StepArgs &a, int member, cudaStream_t s);

}  // namespace seas

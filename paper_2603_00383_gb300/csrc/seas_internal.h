// Internal declarations shared by the host orchestration (seas_api.cu), the operator-build kernels
// (seas_build.cu) and the per-step kernels (seas_step.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace seas {

constexpr int kThreads = 256;       // threads per CTA of every kernel
constexpr int kMaxFFT = 7168;       // largest N_f: two N_f-point complex buffers fit in shared memory
constexpr int kMaxStages = 16;      // radix stages of one FFT plan
constexpr int kMaxBlockSide = 1024; // rows / columns of one H-matrix block (4 accumulator rows per thread)
constexpr int kRowsPerThread = kMaxBlockSide / kThreads;
constexpr int kMaxItemRank = 128;   // rank-1 terms of one low-rank work item (shared-memory z buffer)
constexpr int kMaxBatch = 8;        // scenarios per scenario handle (one pass of the interaction kernel)
constexpr int kItemBytes = 24 * 1024;   // largest work item (operator bytes)
constexpr int kStageBytes = 64 * 1024;  // one shared-memory stage of the interaction pipeline
constexpr int kStages = 3;              // stages in flight per CTA
constexpr int kStageItems = 31;         // work items per stage
constexpr int64_t kTaskBytes = 1 << 20; // operator bytes per task (one deterministic partial sum)

__host__ __device__ inline int pad2(int n) { return n + (n & 1); }

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

// One unit of interaction work: the inner range [i0, i1) of one (block, lag) slice, stored contiguously at `a`
// (rows padded to 16 bytes: p2 = pad_row(p), q2 = pad_row(q) elements of the storage precision):
//   dense   (k < 0): rows i0..i1-1 of A^T, each p2 elements:  y += sum_j A^T[j][:] x_{c0+j}
//   lowrank (k > 0): k = i1 - i0 rows of V^T (each q2 elements) followed by k rows of U^T (each p2 elements):
//                    y += sum_l U^T[l][:] (V^T[l][:] . x)
// Consecutive items of a task are adjacent in memory.
struct ItemDev {
    int32_t T;
    int32_t k;
    int32_t i0, i1;
    const void *a;
    float scale;        // stored values times scale = operator values (1 except FP16)
    int32_t pad;
};

// A run of items of one block (sorted by lag, adjacent in memory) whose partial sums land in one slot:
// partial[b * n_partial + part_off + row].
struct TaskDev {
    int32_t block;
    int32_t item_begin;
    int32_t item_end;
    int32_t T_start;
    int64_t part_off;
};

// One (block, lag) slice produced during the build.
struct SliceGen {
    int32_t block;
    int32_t T;
    int32_t far;        // 1: admissible (compress), 0: near (store dense)
    int32_t group;      // rank-1 terms per stored low-rank item (packing layout)
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
                        float *scales, int prec, cudaStream_t s);
cudaError_t launch_spectral_tables(const ModeDev *modes, int n_modes, const int64_t *g_prefix, int64_t n_g,
                                   const double *mode_L, double cs_dt, const double *gl_x, const double *gl_w,
                                   int gl_n, double *G, double *w, cudaStream_t s);

// ---- step kernels (seas_step.cu) ----
struct StepArgs {
    int N, F, B, n_modes_total;   // elements, faults, batch, sum over faults of (N_f + 1)
    int max_nf;                   // largest N_f (shared memory of the FFT kernels)
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
                                  // layout; NULL for FP64
    int prec;
    double *slip, *slip_prev;     // [B][N]
    double2 *dring;               // spectral rings
    double2 *fmodes;              // [B][n_modes_total]
    double *fint;                 // [B][N]
    // interaction
    const BlockDev *blocks;
    const ItemDev *items;
    const TaskDev *tasks;
    int n_tasks_active;           // tasks with T_start <= step (a prefix of the T_start-sorted list)
    double *partial;              // [B][n_partial]
    int64_t n_partial;
    int *counter;                 // dynamic task counter (reset by the reduction)
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
};

// Allocation-free stepping (seas_stress_step_static): scratch in a static device array of this many doubles.
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 22;
constexpr int kMaxDevices = 64;
cudaError_t static_scratch(double **ptr);   // device address of the array on the current device

cudaError_t launch_push(const StepArgs &a, const double *V, const double *slip_in, int replace_last,
                        cudaStream_t s);
cudaError_t launch_fft_forward(const StepArgs &a, cudaStream_t s);
cudaError_t launch_modeconv(const StepArgs &a, cudaStream_t s);
cudaError_t launch_interaction(const StepArgs &a, cudaStream_t s);
cudaError_t launch_reduce(const StepArgs &a, cudaStream_t s);
cudaError_t launch_static_tail(const StepArgs &a, cudaStream_t s);
cudaError_t launch_ifft_assemble(const StepArgs &a, double *tau, double *parts, cudaStream_t s);
cudaError_t launch_wait_probe(const StepArgs &a, cudaStream_t s);
cudaError_t launch_reset_member(const StepArgs &a, int member, cudaStream_t s);

}  // namespace seas

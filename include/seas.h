/*
 * seas.h -- C ABI of the GB300 engine for the per-time-step elastodynamic stress-transfer functional of
 * Ciardo & Romanet, "A divide-and-conquer strategy for fast elastodynamic simulation of earthquakes and aseismic
 * slip on fault networks" (arXiv 2603.00383), anti-plane (mode III) setting.
 *
 * At step n (t_n = n dt) the library returns, for every element i of a network of planar faults,
 *
 *     tau_i^n = -(mu / 2 c_s) V_i^n  +  f_self,i^n  +  f_int,i^n                           (Eq. superimposition2)
 *
 *   * f_self: the non-replicating spectral self effect of the element's own fault (Sec. 2.3.1): slip zero-padded
 *     to a 2 L_f domain, D_n = FFT, F_n = -(mu k_n / 2) sum_{T=0}^{W_f(n)} w_n^T D_n^{t-T}
 *     (Eq. funcational_discretized_form, Eq. mode_dependent_truncation), then the inverse FFT;
 *   * f_int: the fault-to-fault space-time convolution f_i = -(mu/2c_s) n_l^i sum_j sum_T K_3l^{ijT} V_j^{t-T}
 *     (Eq. fault-to-fault_interactions_discretized) with kernels from the primitives of Eq. (primitives) and
 *     Eq. (kernel_interactions), evaluated through a selective H-matrix stack (Sec. 2.3.2): one binary cluster
 *     tree per fault, self blocks excluded, dual-tree traversal with the admissibility test of
 *     Eq. (admissibility_condition), low-rank far blocks (adaptive cross approximation), dense near blocks, and
 *     causal windows per block (exact first nonzero lag; end at (1 + eta_Tmax) T_max, Sec. 2.3.2).
 *   * the elastodynamic normal-stress change is identically zero in mode III (Sec. 2.1).
 *
 * Conventions
 *   * Fault f: centre (cx, cy), strike phi, e'_1 = (cos phi, sin phi), normal n = e'_2 = (sin phi, -cos phi)
 *     (e'_1 = e'_3 x e'_2, Sec. 3.1).  Element j (0-based) of fault f has centroid c + (-L/2 + (j + 1/2) ds) e'_1,
 *     ds = L / N_f.  Elements are numbered fault after fault in the order given.
 *   * dt = beta * min_f ds_f / c_s (Sec. 2.3.1, Sec. 3.1; beta = 1/2 in the paper).
 *   * Push n (n = 0, 1, ...) supplies V^n, the slip rate on (t_{n-1}, t_n]; slip delta^n = delta^{n-1} + dt V^n
 *     (delta^{-1} = 0) unless the caller passes delta^n.  seas_stress_step after push n returns tau at t_n,
 *     including lag 0 (the instantaneous part).
 *   * Vectors are [batch][N] row-major float64 (scenario-major), N = total number of elements.
 *
 * Ownership and errors
 *   * The library owns every buffer it allocates; handles are freed child first (destroying a parent with live
 *     children returns SEAS_EBUSY).  The caller owns V / slip / tau buffers.
 *   * Device work is asynchronous on the context's stream; host outputs (mem = SEAS_MEM_HOST) are complete when
 *     the call returns, device outputs after seas_sync() or any later stream-ordered operation.
 *   * Every call returns a status (< 0 on error) and never aborts or exits.  A failed call leaves its handles
 *     usable unless it returned SEAS_ECUDA (a CUDA error; the context should then be destroyed).
 *   * Thread safety: one context per host thread; handles of one context must not be used concurrently.
 */
#ifndef SEAS_H
#define SEAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int seas_status;

#define SEAS_OK 0
#define SEAS_EINVAL (-1)       /* bad argument or geometry (non-finite input, size limits, touching faults) */
#define SEAS_ENOMEM (-2)       /* device allocation failed or the context's HBM budget would be exceeded */
#define SEAS_ECUDA (-3)        /* a CUDA runtime error; the message is in seas_last_error() */
#define SEAS_ESTATE (-4)       /* call out of order: stress_step before a push, push past max_steps, ... */
#define SEAS_EBUSY (-5)        /* destroying a handle that still has live children */
#define SEAS_ETIMEOUT (-6)     /* a bounded device wait ran out */
#define SEAS_EIO (-7)          /* checkpoint file could not be written / read or is malformed */

#define SEAS_MEM_HOST 0
#define SEAS_MEM_DEVICE 1

/* operator flags */
#define SEAS_FLAG_DENSE 1        /* admissibility never satisfied: every block dense (the plain space-time sum) */
#define SEAS_FLAG_NO_TRUNC 2     /* no causal end truncation; full-length spectral windows (exact operator) */
/* SEAS_FLAG_STATIC_TAIL (not in the paper, which truncates): add back, as an elastostatic response, the history each
 * window drops.  Per spectral mode: (S_n - sum_{T<=W} w_n^T) D_n^{n-W-1}, S_n = (2/pi) Si(n pi) the weights' static
 * limit; per ordered fault pair whose window ends at T_last: A^static delta^{n-T_last-1}, A^static the t -> infinity
 * limit of the kernel over dt (Eq. primitives), delta the slip (per block, with the block's T_last, under
 * SEAS_FLAG_CLUSTER_TRUNC).  FP64 in every precision.  Costs a dense N x N FP64
 * static operator and a slip ring per scenario; ignored with SEAS_FLAG_NO_TRUNC (nothing is dropped). */
#define SEAS_FLAG_STATIC_TAIL 4
/* SEAS_FLAG_LAG_CAP: max_steps caps every window (lags 0 .. max_steps - 1 are kept, older history is dropped like a
 * window end) but does not limit the number of pushes, so scenarios may run any number of steps (used by long-running
 * served requests).  Without it, a push past max_steps returns SEAS_ESTATE. */
#define SEAS_FLAG_LAG_CAP 8
/* SEAS_FLAG_CLUSTER_TRUNC: cluster-level end truncation, the extension Sec. 4.3 proposes.  The criterion of
 * Sec. 2.3.2 is applied per block of the H-matrix partition instead of per fault pair: for the block of receiver
 * cluster A and source cluster B, T_max^AB is the largest distance from the two ends of A's segment to the ends of
 * B's elements over c_s, and the block keeps lags up to min(ceil((1 + eta_Tmax) T_max^AB / dt), max_steps - 1)
 * (never longer than the fault pair's window).  Well-separated cluster pairs then store and evaluate fewer lags.
 * With SEAS_FLAG_STATIC_TAIL the tail adds, per block, the static response of the slip at the block's own window
 * end.  Ignored with SEAS_FLAG_NO_TRUNC. */
#define SEAS_FLAG_CLUSTER_TRUNC 16

/* storage precision and arithmetic of the interaction operator */
#define SEAS_PREC_FP64 0   /* FP64 entries, FP64 arithmetic */
#define SEAS_PREC_BF16 1   /* bfloat16 entries, FP32 arithmetic, Kahan-compensated accumulation over the history */
#define SEAS_PREC_FP16S 2  /* float16 entries with a per-slice scale, FP32 compensated arithmetic */
#define SEAS_PREC_DF64 3   /* FP32 (hi, lo) pairs per entry (8 bytes, ~48-bit significand), double-float arithmetic
                            * on the FP32 pipes; the spectral path and assembly stay FP64 in every mode */

typedef struct seas_ctx seas_ctx;
typedef struct seas_net seas_net;
typedef struct seas_op seas_op;
typedef struct seas_scn seas_scn;

/* One planar fault: centre (m), strike phi (rad), length L (m), number of elements N_f (>= 1), flags
 * (SEAS_FAULT_*, 0 for a fault in the full space). */
typedef struct {
    double cx, cy, strike_rad, length;
    int32_t n_elem;
    int32_t flags;
} seas_fault;

/* SEAS_FAULT_SURFACE_START: a traction-free surface passes through the fault's start end c - (L/2) e'_1, normal to
 * the fault, with the medium on the e'_1 side (a fault breaking the surface, as the single-fault verification of
 * App. B).  The library applies the method of images: each fault is continued by its mirror image beyond the start
 * end (a fault of 2 L_f and 2 N_f elements, the doubled domain of App. B) whose slip rate is the real one continued
 * evenly across the surface, delta(-z) = delta(z) (which makes the shear traction on the surface vanish), and the
 * full-space functional of the doubled network is evaluated; the image half's receivers are computed and dropped.
 * Either every fault of a network carries the flag or none does; flagged faults must be parallel with the same
 * orientation and have their start ends on one line normal to them (the common surface), else SEAS_EINVAL.
 * Every vector the caller passes or receives (V, slip, tau, sigma_n, parts, the integrator's state) holds the real
 * elements only, N = sum N_f; the self windows are those of the doubled faults (L -> 2 L_f, N_f -> 2 N_f), and the
 * operator queries (seas_plan_hmatrix, seas_op_blocks, seas_op_mode_windows) report the doubled network: its fault
 * f holds elements 2 off_f .. 2 off_f + 2 N_f - 1, of which 2 off_f + N_f + j is real element off_f + j. */
#define SEAS_FAULT_SURFACE_START 1

/* Homogeneous medium: shear modulus mu (Pa), shear speed c_s (m/s), P speed c_p (recorded; unused in mode III),
 * and beta in dt = beta * min ds / c_s (the paper uses 1/2). */
typedef struct {
    double mu, cs, cp, beta;
} seas_medium;

/* Operator parameters (Table 1 names): leaf = eta_leaf (max elements in a leaf cluster), eta_h = eta_H of
 * Eq. (admissibility_condition), aca_tol = relative Frobenius tolerance per (block, lag) slice (the paper's
 * eps_SVD with ACA in place of SVD), eta_tmin (reported only: windows start at the exact first nonzero lag),
 * eta_tmax, eta_w, q_w (<= 0: q_w = N_f, i.e. no mode-dependent shortening), max_steps = largest number of pushes
 * the operator serves (lags 0 .. max_steps - 1), precision = SEAS_PREC_*, flags = SEAS_FLAG_*. */
typedef struct {
    int32_t leaf;
    int32_t q_w;
    double eta_h, aca_tol, eta_tmin, eta_tmax, eta_w;
    int32_t max_steps;
    int32_t precision;
    int32_t flags;
    int32_t max_block;   /* largest cluster side of an admissible block (0: 64; at most 1024).  Large admissible
                          * blocks are split further: the wavefront cuts a smaller block for fewer lags, which
                          * keeps more of its slices low rank. */
} seas_hparams;

typedef struct {
    double dt;
    int32_t n_faults;
    int32_t n_elem;      /* N */
} seas_net_info;

typedef struct {
    int64_t n_blocks_near, n_blocks_far;
    int64_t n_slices_dense, n_slices_lowrank, n_slices_zero;
    int64_t bytes_interaction;      /* stored interaction operator (all lags) */
    int64_t bytes_dense_causal;     /* the same slices stored dense (rank-0 slices excluded) */
    double compression_ratio;       /* bytes_interaction / bytes_dense_causal, in percent */
    int64_t bytes_self;             /* spectral weight tables */
    int32_t max_rank;
    int32_t ring_depth;             /* slip-rate history slots kept per scenario */
    double mean_rank;
    double build_seconds;
    int64_t n_tasks;                /* interaction work units */
} seas_op_stats;

/* Creates a context on CUDA device `device`.  hbm_budget: bytes the library may allocate (0: no limit).
 * cuda_stream: a cudaStream_t the library issues all work on (NULL: the library creates and owns one; the
 * legacy default stream is passed as cudaStreamLegacy, (void *)1).  Device buffers the caller passes must be
 * ready in this stream's order. */
seas_status seas_create(seas_ctx **ctx, int device, size_t hbm_budget, void *cuda_stream);

/* Device bytes the context's handles hold now (operators, scenarios, networks) and its budget (0: none). */
seas_status seas_ctx_get_memory(const seas_ctx *ctx, size_t *used, size_t *budget);

/* Builds the discretised network (Sec. 2.3.1 "Discretization", Sec. 3.1 frames).  Rejects non-finite or
 * non-positive sizes, N_f with a prime factor above 23 (the FFT's radices), N_f > 7168, and receiver centroids lying
 * on another fault (within 1e-6 ds of one of its elements, where the kernel is singular: faults that cross must do
 * so at an element boundary, as the X-shaped network of Sec. 3.2 does). */
seas_status seas_build_network(seas_ctx *ctx, const seas_fault *faults, int n_faults, const seas_medium *medium,
                               seas_net **net);
seas_status seas_net_get_info(const seas_net *net, seas_net_info *info);
/* Element centroids [N][2] and normals [N][2] (host buffers of the caller). */
seas_status seas_net_get_elements(const seas_net *net, double *centroids, double *normals);

/* Builds the selective H-matrix stack and the spectral tables on the device (Sec. 2.3.1, Sec. 2.3.2).
 * stats may be NULL. */
seas_status seas_build_hmatrix(seas_net *net, const seas_hparams *hp, seas_op **op, seas_op_stats *stats);
/* The part of the operator whose receivers lie on `faults` (n_faults indices): their spectral self effects and the
 * H-matrix blocks of their rows, for sharding one scenario across GPUs by receiver faults (each GPU steps the same
 * full slip-rate history -- gathered from the GPUs that own its parts -- and returns tau on its own faults).
 * seas_stress_step then writes tau, and parts, only on the owned faults' elements; other entries of the output
 * buffers are left as they were.  Not with SEAS_FLAG_STATIC_TAIL (SEAS_EINVAL).  No counterpart in the paper, which
 * names the method inherently parallel. */
seas_status seas_build_hmatrix_part(seas_net *net, const seas_hparams *hp, const int32_t *faults, int n_faults,
                                    seas_op **op, seas_op_stats *stats);
/* Per ordered fault pair (receiver a, source b): last lag of the window, [F][F] int32, -1 on the diagonal. */
seas_status seas_op_pair_windows(const seas_op *op, int32_t *last_lag);
/* Per fault f and mode n = 0..N_f: last lag W_f(n) of the spectral window (flattened fault after fault). */
seas_status seas_op_mode_windows(const seas_op *op, int32_t *w);

/* The operator's H-matrix blocks (the leaf blocks of the dual traversal of Sec. 2.3.2, in build order): row i of
 * `blocks` ([cap][7] int32, host) is (r0, p, c0, q, far, first_lag, last_lag) for receivers r0 .. r0 + p - 1 and
 * sources c0 .. c0 + q - 1; far = 1 for an admissible (low-rank) block; the block's window is
 * first_lag .. last_lag (empty when first_lag > last_lag; first_lag is a lower bound: exactly-zero slices at the
 * start of the window are not stored).  *n_blocks receives the count; at most cap rows are
 * written (blocks may be NULL with cap = 0 to query the count). */
seas_status seas_op_blocks(const seas_op *op, int32_t *blocks, int64_t cap, int64_t *n_blocks);

/* Allocates the history ring buffers of `batch` (1..8) independent scenarios sharing the operator.  BF16 operators
 * with batches of 5..8 run on tensor-core consumers that tile at most 128 receivers per block (SEAS_EINVAL
 * otherwise; the default max_block of 64 always fits). */
seas_status seas_scenario_create(seas_op *op, int batch, seas_scn **scn);

/* Pushes V^n ([batch][N] float64) and optionally delta^n (same layout; NULL: integrate).  mem: where V and slip
 * live.  replace_last != 0 overwrites the previous push instead (the corrector of Sec. 2.4 step 3).
 * SEAS_ESTATE after max_steps pushes.  Host inputs are checked for finiteness (SEAS_EINVAL). */
seas_status seas_push_slip_rate(seas_scn *scn, const double *V, const double *slip, int mem, int replace_last);

/* A slip rate held over gamma >= 1 consecutive lattice steps (t_n, t_{n+gamma}] (the time step gamma dt_min of
 * Sec. 2.4, step 1): V ([batch][N]) goes into gamma ring slots and the slip of lattice step n + j is
 * delta^n + j dt V (j = 1..gamma), or, with slip given, the straight line from delta^n to slip at j = gamma; the
 * spectral history gets every lattice step.  seas_stress_step then returns tau at t_{n+gamma}.  replace_last != 0
 * overwrites the previous push, which must have held the same gamma (SEAS_EINVAL otherwise).  gamma = 1 is
 * seas_push_slip_rate; a push counts gamma steps against max_steps. */
seas_status seas_push_slip_rate_steps(seas_scn *scn, const double *V, const double *slip, int mem, int gamma,
                                      int replace_last);

/* tau at the last pushed step into tau ([batch][N]); sigma_n (nullable) receives zeros; parts (nullable,
 * [3][batch][N]) receives radiation damping, f_self and f_int separately. */
seas_status seas_stress_step(seas_scn *scn, double *tau, double *sigma_n, double *parts, int mem);

/* Allocation-free variant of seas_stress_step, for callers that must not allocate device memory while stepping:
 * a solver embedded in a host code whose own allocator has already reserved the GPU's memory, or a time loop that
 * cannot afford cudaMalloc/cudaFree, which may synchronize the whole device.  seas_stress_step itself allocates
 * nothing per step either (seas_scenario_create allocates the scenario's scratch once, and still does so for
 * scenarios stepped only through this call); the difference is only where the per-call scratch lives.  The paper has
 * no counterpart; this is a property of the library only.  tau ([batch][N]) and parts (nullable, [3][batch][N]) are
 * DEVICE pointers that the caller owns; the call computes what seas_stress_step computes (same kernels, same
 * summation order) on the context's stream, but is not counted by seas_scenario_set_timing.  Its scratch (the
 * interaction's per-task partial sums and the summed interaction term) is a file-scope static device array of
 * 4,194,304 doubles (32 MiB), held by every GPU that loads the library until the process exits; a scenario whose
 * partial-sum rows times batch plus batch * N exceed that gets SEAS_EINVAL and nothing runs.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, which allocates nothing), so make that first
 * call before any stream capture.  All calls share the array, which keeps the last call's contents (every entry a
 * call reads it first writes); calls that overlap on the GPU (other streams, threads or contexts of this process)
 * race on it. */
seas_status seas_stress_step_static(seas_scn *scn, double *tau, double *parts);

/* Watchdog of the scenario's device waits (the interaction kernel's producer/consumer hand-offs).  Every wait is
 * bounded by `seconds` of wall time (default 2 s; accepted range [1e-6, 60]); a wait that runs out sets the
 * scenario's device error word, which is sticky: seas_scenario_check and host-output seas_stress_step then return
 * SEAS_ETIMEOUT, and later interaction launches of the scenario return at once.  The context stays usable (other
 * scenarios are unaffected).  No counterpart in the paper. */
seas_status seas_scenario_set_wait_limit(seas_scn *scn, double seconds);
/* Launches one thread that waits, with the scenario's bound, on a device barrier nothing arrives on, so the wait
 * runs out and takes the same path as a stalled pipeline (error word set, SEAS_ETIMEOUT reported by the next
 * seas_scenario_check).  For testing the watchdog on a live context: no copy is in flight and no other thread is
 * involved.  No counterpart in the paper. */
seas_status seas_scenario_probe_wait(seas_scn *scn);

/* Autotuner of the interaction kernel's launch shape: for each pass (0: source side, 1: receiver side) the number of
 * consumer warps per CTA (8 or 16, where the library compiles both for this precision and batch) that runs the
 * pass fastest on this scenario's operator, measured with CUDA events over `reps` launches of the pass (1..100,
 * median; one untimed launch first) with every task of the operator active, as at full history depth.  The choice
 * holds for the scenario's later steps; it changes no result beyond the summation order of the task reductions.
 * The passes' per-step scratch is overwritten, so call it between steps.  cache_path (NULL: none) names a text file
 * of earlier choices, one line per key (device name, SM count, precision, batch and the operator's work shape): a
 * matching line is applied without timing (from_cache = 1), otherwise the new choice is appended.  SEAS_ESTATE with
 * a captured graph (its kernels are fixed) or while kernel timing is on.  No counterpart in the paper. */
typedef struct {
    int consumer_warps[2];      /* chosen per pass */
    int candidates[2][2];       /* counts compiled per pass (0: none; the first is the default) */
    double ms[2][2];            /* median launch time of each candidate (0: not timed) */
    int from_cache;
} seas_tune;
seas_status seas_scenario_autotune(seas_scn *scn, const char *cache_path, int reps, seas_tune *out);

/* CUDA-graph stepping.  seas_scenario_graph_create captures one step of the scenario -- a push of the slip rate in
 * the caller's device buffer V ([batch][N], slip integrated) and a stress step into the device buffers tau
 * ([batch][N]) and parts (nullable, [3][batch][N]) -- as one graph of all its kernels (interaction passes on every
 * SM).  seas_scenario_graph_step then advances the scenario by one step: it uploads the step's index, lag horizon
 * and task counts (asynchronously, from a pinned ring) and launches the graph, so a step costs two API calls
 * instead of one launch per kernel.  V and tau are read and written at the addresses given at capture; the caller
 * refills V between steps in stream order.  Results equal those of seas_push_slip_rate + seas_stress_step bit for
 * bit; ordinary pushes and steps may be interleaved with graph steps.  Not available while kernel timing is on
 * (SEAS_ESTATE); the graph lives until the scenario is destroyed.  No counterpart in the paper. */
seas_status seas_scenario_graph_create(seas_scn *scn, const double *V, double *tau, double *parts);
seas_status seas_scenario_graph_step(seas_scn *scn);

/* Number of pushes so far (ticks of the batch; equal to every member's step count unless members were admitted
 * later). */
seas_status seas_scenario_step(const seas_scn *scn, int64_t *n);

/* Continuous batching (no counterpart in the paper, which runs one scenario): the members of a batch need not start
 * together.  seas_scenario_admit(scn, m) makes member m a fresh scenario whose first push is the batch's next push:
 * its slip-rate, slip and spectral histories are set to zero on the device (asynchronously on the context stream,
 * no allocation), so its tau from then on equals that of a scenario of its own (to rounding: the summation order
 * depends on the batch width).  Every member shares the batch's ring slots (tick mod depth); a member admitted at
 * tick s reads zeros for lags beyond its own step n - s.  seas_scenario_retire(scn, m) stops counting member m:
 * its outputs are then meaningless and its pushes are ignored by the max_steps check; the interaction kernel skips
 * lags beyond the oldest active member's step.  A member's own step count must stay below max_steps (SEAS_ESTATE
 * from push otherwise); the batch's tick may grow past it.  seas_scenario_member_step returns member m's pushes
 * since admission (-1 when retired).  All members start active at seas_scenario_create. */
seas_status seas_scenario_admit(seas_scn *scn, int member);
seas_status seas_scenario_retire(seas_scn *scn, int member);
seas_status seas_scenario_member_step(const seas_scn *scn, int member, int64_t *n);

seas_status seas_sync(seas_ctx *ctx);
/* Synchronises the scenario's stream and reports SEAS_ETIMEOUT if a bounded device wait of its kernels ran out
 * (host-output stress_step calls check this themselves). */
seas_status seas_scenario_check(seas_scn *scn);
const char *seas_strerror(seas_status s);
/* Thread-local description of the last error of this thread (empty when none). */
const char *seas_last_error(void);

/* Host-only planning (no device work): the block partition, windows and time step the operator build would use.
 * blocks (nullable): [cap][7] int32 rows (r0, p, c0, q, far, first_lag, last_lag) -- receiver rows [r0, r0 + p),
 * source columns [c0, c0 + q), far = 1 for an admissible (low-rank) block, first_lag = conservative first nonzero
 * lag, last_lag = the block's window end (its fault pair's, or its own with SEAS_FLAG_CLUSTER_TRUNC); *n_blocks
 * receives the total count even when it exceeds cap.  pair_last (nullable): [F][F] last lags.
 * mode_windows (nullable): W_f(n), n = 0..N_f, fault after fault.  dt (nullable). */
seas_status seas_plan_hmatrix(const seas_fault *faults, int n_faults, const seas_medium *medium,
                              const seas_hparams *hp, int32_t *blocks, int64_t cap, int64_t *n_blocks,
                              int32_t *pair_last, int32_t *mode_windows, double *dt);

/* Kernel timing on the context stream (tracing).  set_timing(1) resets and starts recording a CUDA event pair
 * around every kernel the scenario launches; get_timing synchronises and returns, per kernel class (0 push,
 * 1 forward FFT, 2 mode convolution, 3 interaction receiver side (pass 2: U z and A x sums), 4 interaction reduction
 * (with the static tail when that flag is set), 5 inverse FFT + assembly, 6 interaction source side (pass 1:
 * z = V^T x)), the launch count and the summed device time, plus the algorithmic bytes the two interaction passes
 * streamed (seas_op_step_bytes summed over the timed steps).  The first set_timing(1) of a
 * scenario creates its events (8192 pairs), so that timed steps pay only for the event records. */
typedef struct {
    int64_t launches[7];
    double ms[7];
    int64_t interaction_bytes;
    int64_t steps;
} seas_timing;
seas_status seas_scenario_set_timing(seas_scn *scn, int enable);
seas_status seas_scenario_get_timing(seas_scn *scn, seas_timing *out);
/* Algorithmic interaction-operator bytes of step `step`: the values of every stored slice with lag <= step
 * (p q near, k (p + q) far) times the storage element size; the 16-byte row padding is not counted. */
seas_status seas_op_step_bytes(const seas_op *op, int64_t step, int64_t *bytes);

/* ---- earthquake-cycle stepping on top of the functional (Sec. 2.2, Sec. 2.4) ----
 * Rate-and-state friction of one element: f = f_* + a ln(V / V_*) + b ln(V theta / D_c) (Eq. R&S_friction) under the
 * background normal stress sigma_n (Pa, compressive positive); the state follows Eq. state_evolution_law with the
 * integrator's eps in (0, 1] (1: the aging law). */
typedef struct {
    double a, b, dc, f0, v0, sigma_n;
} seas_friction;

typedef struct seas_integ seas_integ;

/* Creates an integrator on a scenario that has no pushes yet.  fr: n_fr = 1 (every element) or N entries (element
 * j of every batch member); tau0: background shear stress [batch][N] (Pa); V0, theta0: initial slip rate and state
 * [batch][N]; mem: where tau0, V0 and theta0 live.  The initial rate starts the first predictor but is no slip-rate
 * history (no slip before t = 0).  SEAS_EINVAL if a lag-0 interaction slice exists (faults closer than c_s dt: the
 * per-element Newton solves would couple) or a parameter is out of range; SEAS_ESTATE if the scenario has pushes.
 * The integrator owns its device state (charged to the context's budget); destroy it before the scenario. */
seas_status seas_integrator_create(seas_scn *scn, const seas_friction *fr, int n_fr, double eps, const double *tau0,
                                   const double *V0, const double *theta0, int mem, seas_integ **out);
/* Advances `steps` time steps of dt (the operator's lattice step) on the device, asynchronously on the context
 * stream.  One step (Sec. 2.4): predictor delta* = delta + dt V, theta* = theta + dt thetadot; push of a zero slip
 * rate with slip delta* and a stress step give the elastic stress without its instantaneous part; Newton in ln V per
 * element on tau_known + tau0 - (mu / 2 c_s) V = sigma_n f(V, theta*) to |residual| <= 1e-8 (|tau| + sigma_n);
 * thetadot*; the corrector repeats this with V -> (V + V*)/2, thetadot -> (thetadot + thetadot*)/2 (replacing the
 * pushed slip); the step's slot is then replaced by V**.  Three pushes and two stress steps per step, all FP64. */
seas_status seas_integrator_step(seas_integ *it, int steps);
/* One time step of gamma lattice steps (dt = gamma dt_min, Sec. 2.4 step 1): the predictor and corrector hold their
 * rate over the step's lattice steps (seas_push_slip_rate_steps) and the slip grows linearly along them; the lattice
 * history then receives V** on each of them.  gamma = 1 is one seas_integrator_step. */
seas_status seas_integrator_step_gamma(seas_integ *it, int gamma);
/* `steps` adaptive time steps: gamma = ceil(dt_ev / dt_min) with dt_ev = min over elements of xi D_c / V (Sec. 2.4,
 * step 1), clamped to [1, gamma_max]; xi is the caller's (the paper takes it from a stiffness criterion of the
 * literature).  Synchronises once per step to read dt_ev.  *lattice_steps (nullable) receives the lattice steps
 * advanced. */
seas_status seas_integrator_step_adaptive(seas_integ *it, double xi, int gamma_max, int steps, int64_t *lattice_steps);
/* Synchronises and copies V, theta and slip ([batch][N] each, nullable) into host or device buffers; SEAS_ESTATE if
 * a Newton solve did not converge in 100 iterations since the integrator was created. */
seas_status seas_integrator_state(seas_integ *it, double *V, double *theta, double *slip, int mem);
seas_status seas_destroy_integrator(seas_integ *it);

/* Device probe (no counterpart in the paper; used for roofline reporting): the FP64 fused multiply-add rate of GPU
 * `device` in FMA/s, measured by a kernel of independent FMA chains on every SM (best of three ~30 ms launches).
 * Allocates and frees a few bytes; SEAS_EINVAL for a bad device, SEAS_ECUDA on a CUDA error. */
seas_status seas_measure_fp64_peak(int device, double *fma_per_second);

/* Checkpoint/resume of a scenario: the step counter, the members' start ticks and states, the interaction's lag
 * horizon, slip-rate ring, slip and spectral ring (and the slip ring of the static tail when that flag is set). */
seas_status seas_scenario_save(seas_scn *scn, const char *path);
seas_status seas_scenario_load(seas_op *op, const char *path, seas_scn **scn);

seas_status seas_destroy_scn(seas_scn *scn);
seas_status seas_destroy_op(seas_op *op);
seas_status seas_destroy_net(seas_net *net);
seas_status seas_destroy_ctx(seas_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SEAS_H */

// Per-step kernels of the stress-transfer functional (Eq. superimposition2): slip-rate push, spectral self effect
// (Sec. 2.3.1: FFT of zero-padded slip, per-mode causal convolution, inverse FFT) and the H-matrix space-time
// interaction (Sec. 2.3.2), then assembly with the radiation-damping term.
#include "seas_internal.h"

namespace seas {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// ------------------------------------------------------------------------------------------------------------
// Self-sorting (Stockham) mixed-radix FFT of N points held in shared memory, radices 2, 3, 4, 5.  Stage with
// radix R after sub-transforms of size Ns: butterfly j takes src[j + r N/R] (r < R), twiddles it by
// W_{Ns R}^{r (j mod Ns)}, takes an R-point DFT and writes dst[(j / Ns) Ns R + (j mod Ns) + t Ns].
// tw[k] = e^{-2 pi i k / N}; the inverse (unnormalised) uses conjugate twiddles.  Returns the buffer holding the
// result.  All threads of the CTA must call it.
// ------------------------------------------------------------------------------------------------------------
__device__ double2 *fft_stockham(double2 *src, double2 *dst, int N, const int *radix, int nstages,
                                 const double2 *__restrict__ tw, bool inverse) {
    int Ns = 1;
    for (int st = 0; st < nstages; ++st) {
        const int R = radix[st];
        const int NR = N / R;
        const int tstride = N / (Ns * R);
        for (int j = threadIdx.x; j < NR; j += blockDim.x) {
            const int k = j % Ns;
            double2 v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                if (r < R) {
                    double2 x = src[j + r * NR];
                    if (r > 0) {
                        double2 w = tw[k * r * tstride];
                        if (inverse) w = cconj(w);
                        x = cmul(x, w);
                    }
                    v[r] = x;
                }
            }
            const int d = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                if (t < R) {
                    double2 acc = v[0];
#pragma unroll
                    for (int r = 1; r < 5; ++r) {
                        if (r < R) {
                            double2 w = tw[((r * t) % R) * NR];
                            if (inverse) w = cconj(w);
                            acc = cadd(acc, cmul(v[r], w));
                        }
                    }
                    dst[d + t * Ns] = acc;
                }
            }
        }
        __syncthreads();
        double2 *tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }
    return src;
}

__global__ void k_push(StepArgs a, const double *__restrict__ V, const double *__restrict__ slip_in,
                       int replace_last) {
    const int64_t BN = (int64_t)a.B * a.N;
    const int slot = (int)(a.step % a.ring);
    double *vr = a.vring + (int64_t)slot * BN;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < BN; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = V[e];
        vr[e] = v;
        double s;
        if (slip_in) {
            s = slip_in[e];
        } else {
            const double base = replace_last ? a.slip_prev[e] : a.slip[e];
            s = __dadd_rn(base, __dmul_rn(v, a.dt));   // delta^n = delta^{n-1} + dt V^n
        }
        if (!replace_last) a.slip_prev[e] = a.slip[e];
        a.slip[e] = s;
    }
}

// Spectral coefficients of the zero-padded slip (Eq. functional_no_replication): D_k = (1/M) sum_{j<N_f}
// delta_j e^{-2 pi i k j / M}, M = 2 N_f, k = 0..N_f, from one N_f-point complex FFT of z_j = x_{2j} + i x_{2j+1}
// (x = delta padded with zeros): X_k = E_k + e^{-2 pi i k/M} O_k, E_k = (Z_k + conj Z_{N-k})/2,
// O_k = (Z_k - conj Z_{N-k})/(2i).  One CTA per (fault, scenario); D^n goes to ring slot n mod R_f.
__global__ void __launch_bounds__(kThreads) k_fft_forward(StepArgs a) {
    extern __shared__ double2 smem[];
    const FaultDev fd = a.faults[blockIdx.x];
    const int b = blockIdx.y;
    const int N = fd.nf;
    double2 *b0 = smem, *b1 = smem + N;
    const double *x = a.slip + (int64_t)b * a.N + fd.off;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int e = 2 * j, o = 2 * j + 1;
        b0[j] = make_double2(e < N ? x[e] : 0.0, o < N ? x[o] : 0.0);
    }
    __syncthreads();
    const double2 *tw = a.tw + fd.tw_off;
    const double2 *post = tw + N;
    double2 *Z = fft_stockham(b0, b1, N, fd.radix, fd.nstages, tw, false);
    const double invM = 1.0 / (2.0 * N);
    const int slot = (int)(a.step % fd.ring);
    double2 *ring = a.dring + fd.dring_off + (int64_t)b * (N + 1) * fd.ring + slot;
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        const double2 zk = Z[k == N ? 0 : k];
        const double2 zc = cconj(Z[k == 0 ? 0 : N - k]);
        const double2 E = make_double2(0.5 * (zk.x + zc.x), 0.5 * (zk.y + zc.y));
        const double2 dd = csub(zk, zc);
        const double2 O = make_double2(0.5 * dd.y, -0.5 * dd.x);
        const double2 X = cadd(E, cmul(post[k], O));
        ring[(int64_t)k * fd.ring] = make_double2(X.x * invM, X.y * invM);
    }
}

// Per-mode causal convolution (Eq. funcational_discretized_form):
//   F_n = -(mu k_n / 2) sum_{T=0}^{min(W_f(n), step)} w_n^T D_n^{step - T},  k_n = pi n / L_f.
// One warp per (mode, scenario); lanes stride the lags; the ring is mode-major so the lanes read contiguous slots.
__global__ void __launch_bounds__(kThreads) k_modeconv(StepArgs a) {
    const int md = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.y;
    if (md >= a.n_modes) return;
    const ModeDev mo = a.modes[md];
    const FaultDev fd = a.faults[mo.fault];
    const int R = fd.ring;
    const int64_t Tmax = mo.W < a.step ? mo.W : a.step;
    const double2 *ring = a.dring + fd.dring_off + ((int64_t)b * (fd.nf + 1) + mo.n) * R;
    const double *w = a.w + mo.w_off;
    const int slot0 = (int)(a.step % R);
    double re = 0.0, im = 0.0;
    for (int T = lane; T <= Tmax; T += 32) {
        int s = slot0 - T;
        if (s < 0) s += R;
        const double2 d = ring[s];
        const double wt = w[T];
        re += wt * d.x;
        im += wt * d.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        const double f = fd.kfac * mo.n;
        a.fmodes[(int64_t)b * a.n_modes_total + fd.mode_off + mo.n] = make_double2(f * re, f * im);
    }
}

// Inverse transform and assembly: f_self,j = sum_{n=-N_f+1}^{N_f} F_n e^{2 pi i n j / M} (F_{-n} = conj F_n,
// F_0 = 0), kept for j < N_f, from one N_f-point inverse complex FFT; then
// tau = -(mu / 2 c_s) V + f_self + f_int (Eq. superimposition2).
__global__ void __launch_bounds__(kThreads) k_ifft_assemble(StepArgs a, double *__restrict__ tau,
                                                            double *__restrict__ parts) {
    extern __shared__ double2 smem[];
    const FaultDev fd = a.faults[blockIdx.x];
    const int b = blockIdx.y;
    const int N = fd.nf;
    double2 *b0 = smem, *b1 = smem + N;
    const double2 *Fm = a.fmodes + (int64_t)b * a.n_modes_total + fd.mode_off;
    const double2 *tw = a.tw + fd.tw_off;
    const double2 *post = tw + N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double2 A = k == 0 ? make_double2(0.0, 0.0) : Fm[k];
        const double2 Bc = cconj(Fm[N - k]);
        const double2 E = make_double2(0.5 * (A.x + Bc.x), 0.5 * (A.y + Bc.y));
        const double2 dd = cmul(csub(A, Bc), cconj(post[k]));
        const double2 O = make_double2(0.5 * dd.x, 0.5 * dd.y);
        b0[k] = make_double2(E.x - O.y, E.y + O.x);      // Z_k = E_k + i O_k
    }
    __syncthreads();
    const double2 *z = fft_stockham(b0, b1, N, fd.radix, fd.nstages, tw, true);
    const int64_t BN = (int64_t)a.B * a.N;
    const int slot = (int)(a.step % a.ring);
    const double *V = a.vring + (int64_t)slot * BN + (int64_t)b * a.N + fd.off;
    const double *fi = a.fint + (int64_t)b * a.N + fd.off;
    double *t = tau + (int64_t)b * a.N + fd.off;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        const double2 zz = z[m >> 1];
        const double fs = 2.0 * ((m & 1) ? zz.y : zz.x);
        const double rad = a.rad * V[m];
        const double f = fi[m];
        t[m] = rad + fs + f;
        if (parts) {
            const int64_t o = (int64_t)b * a.N + fd.off + m;
            parts[o] = rad;
            parts[BN + o] = fs;
            parts[2 * BN + o] = f;
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Space-time interaction (Eq. fault-to-fault_interactions_discretized) through the H-matrix stack: one CTA per
// task (a run of work items of one block, sorted by lag); items with lag > step are not yet causal.  Thread t owns
// receiver rows t, t + 256, ... of the block and accumulates over all items of the task; the sum is flushed with
// one atomic add per row and scenario.  BT scenarios per CTA share every operator load.
// ------------------------------------------------------------------------------------------------------------
template <int BT>
__global__ void __launch_bounds__(kThreads) k_interaction(StepArgs a) {
    extern __shared__ double sh[];
    double *xs = sh;                                  // [BT][kMaxBlockSide]
    double *zs = sh + BT * kMaxBlockSide;             // [BT][kMaxItemRank]
    const TaskDev task = a.tasks[blockIdx.x];
    const BlockDev blk = a.blocks[task.block];
    const int b0 = blockIdx.y * BT;
    const int p = blk.p, q = blk.q;
    const int64_t BN = (int64_t)a.B * a.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc[kRowsPerThread][BT];
#pragma unroll
    for (int s = 0; s < kRowsPerThread; ++s)
#pragma unroll
        for (int bb = 0; bb < BT; ++bb) acc[s][bb] = 0.0;

    for (int it = task.item_begin; it < task.item_end; ++it) {
        const ItemDev item = a.items[it];
        if (item.T > a.step) break;
        const int slot = (int)((a.step - item.T) % a.ring);
        const double *vsrc = a.vring + (int64_t)slot * BN + blk.c0;
        const int j0 = item.k < 0 ? item.i0 : 0;
        const int j1 = item.k < 0 ? item.i1 : q;
#pragma unroll
        for (int bb = 0; bb < BT; ++bb) {
            if (b0 + bb < a.B) {
                for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
                    xs[bb * kMaxBlockSide + j] = vsrc[(int64_t)(b0 + bb) * a.N + j];
            } else {
                for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) xs[bb * kMaxBlockSide + j] = 0.0;
            }
        }
        __syncthreads();
        if (item.k < 0) {
            const double *rows = item.a;
#pragma unroll 4
            for (int j = j0; j < j1; ++j) {
                const double *row = rows + (int64_t)(j - j0) * p;
#pragma unroll
                for (int s = 0; s < kRowsPerThread; ++s) {
                    const int i = threadIdx.x + s * kThreads;
                    if (i < p) {
                        const double v = row[i];
#pragma unroll
                        for (int bb = 0; bb < BT; ++bb) acc[s][bb] += v * xs[bb * kMaxBlockSide + j];
                    }
                }
            }
        } else {
            const int nl = item.i1 - item.i0;
            for (int l = warp; l < nl; l += kThreads / 32) {
                const double *row = item.a + (int64_t)l * q;
                double z[BT];
#pragma unroll
                for (int bb = 0; bb < BT; ++bb) z[bb] = 0.0;
                for (int j = lane; j < q; j += 32) {
                    const double v = row[j];
#pragma unroll
                    for (int bb = 0; bb < BT; ++bb) z[bb] += v * xs[bb * kMaxBlockSide + j];
                }
#pragma unroll
                for (int bb = 0; bb < BT; ++bb) {
                    for (int o = 16; o > 0; o >>= 1) z[bb] += __shfl_xor_sync(0xffffffffu, z[bb], o);
                    if (lane == 0) zs[bb * kMaxItemRank + l] = z[bb];
                }
            }
            __syncthreads();
#pragma unroll 4
            for (int l = 0; l < nl; ++l) {
                const double *row = item.b + (int64_t)l * p;
#pragma unroll
                for (int s = 0; s < kRowsPerThread; ++s) {
                    const int i = threadIdx.x + s * kThreads;
                    if (i < p) {
                        const double v = row[i];
#pragma unroll
                        for (int bb = 0; bb < BT; ++bb) acc[s][bb] += v * zs[bb * kMaxItemRank + l];
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < kRowsPerThread; ++s) {
        const int i = threadIdx.x + s * kThreads;
        if (i < p) {
#pragma unroll
            for (int bb = 0; bb < BT; ++bb)
                if (b0 + bb < a.B) atomicAdd(a.fint + (int64_t)(b0 + bb) * a.N + blk.r0 + i, acc[s][bb]);
        }
    }
}

template <int BT>
cudaError_t launch_interaction_bt(const StepArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)BT * (kMaxBlockSide + kMaxItemRank) * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_interaction<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(a.n_tasks_active, (a.B + BT - 1) / BT);
    k_interaction<BT><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_push(const StepArgs &a, const double *V, const double *slip_in, int replace_last,
                        cudaStream_t s) {
    const int64_t BN = (int64_t)a.B * a.N;
    int grid = (int)((BN + kThreads - 1) / kThreads);
    if (grid > 152 * 8) grid = 152 * 8;
    k_push<<<grid, kThreads, 0, s>>>(a, V, slip_in, replace_last);
    return cudaGetLastError();
}

static cudaError_t fft_smem(const void *fn, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_fft_forward(const StepArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)2 * a.max_nf * sizeof(double2);
    cudaError_t e = fft_smem((const void *)k_fft_forward, smem);
    if (e != cudaSuccess) return e;
    k_fft_forward<<<dim3(a.F, a.B), kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_modeconv(const StepArgs &a, cudaStream_t s) {
    if (a.n_modes == 0) return cudaSuccess;
    dim3 grid((a.n_modes + kThreads / 32 - 1) / (kThreads / 32), a.B);
    k_modeconv<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_interaction(const StepArgs &a, cudaStream_t s) {
    if (a.n_tasks_active <= 0) return cudaSuccess;
    if (a.B >= 8) return launch_interaction_bt<8>(a, s);
    if (a.B >= 4) return launch_interaction_bt<4>(a, s);
    if (a.B >= 2) return launch_interaction_bt<2>(a, s);
    return launch_interaction_bt<1>(a, s);
}

cudaError_t launch_ifft_assemble(const StepArgs &a, double *tau, double *parts, cudaStream_t s) {
    const size_t smem = (size_t)2 * a.max_nf * sizeof(double2);
    cudaError_t e = fft_smem((const void *)k_ifft_assemble, smem);
    if (e != cudaSuccess) return e;
    k_ifft_assemble<<<dim3(a.F, a.B), kThreads, smem, s>>>(a, tau, parts);
    return cudaGetLastError();
}

}  // namespace seas

// Per-step kernels of the stress-transfer functional (Eq. superimposition2): slip-rate push, spectral self effect
// (Sec. 2.3.1: FFT of zero-padded slip, per-mode causal convolution, inverse FFT) and the H-matrix space-time
// interaction (Sec. 2.3.2), then assembly with the radiation-damping term.
#include "seas_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cooperative_groups.h>

#include <atomic>
#include <type_traits>

namespace seas {

// Scratch of seas_stress_step_static: the per-task partial sums and the summed interaction term of one call.
// It lives for the life of the process on every GPU that loads the library.  In host code the symbol is only a
// stand-in: the device address comes from cudaGetSymbolAddress (static_scratch below).
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

namespace {

// In a replayed graph the step-dependent fields come from device memory.
__device__ __forceinline__ void apply_dyn(StepArgs &a) {
    if (a.dyn) {
        const DynDev d = *a.dyn;
        a.step = d.step;
        a.lag_max = d.lag_max;
        a.n_tasks_active = d.n_tasks_active;
        a.n_ztasks_active = d.n_ztasks_active;
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// ------------------------------------------------------------------------------------------------------------
// Self-sorting (Stockham) mixed-radix FFTs of N points held in shared memory, radices 2, 3, 4, 5, 7, 11, 13, 17, 19,
// 23 (the odd primes as plain R-point DFTs); nb independent transforms stored one after another.  Stage with radix R
// after sub-transforms of size Ns: butterfly j takes src[j + r N/R] (r < R), twiddles it by
// W_{Ns R}^{r (j mod Ns)}, takes an R-point DFT and writes dst[(j / Ns) Ns R + (j mod Ns) + t Ns].
// tw[k ts] = e^{-2 pi i k / N} (ts = 1 for the fault's own table; a factor of the fault's N_f reads that table with
// stride N_f / N); the inverse (unnormalised) uses conjugate twiddles.  Returns the buffer holding the result.
// All threads of the CTA must call it; wsh is shared scratch of kFftRadixMax entries (the DFT constants of the
// odd-prime radices >= 7, read there as broadcasts instead of held in registers: with them in registers every
// stage of the kernel was compiled at the register limit with spills).
// ------------------------------------------------------------------------------------------------------------
constexpr int kFftRadixMax = 23;

template <int R>
__device__ __forceinline__ void fft_stage(const double2 *__restrict__ src, double2 *__restrict__ dst, int N, int Ns,
                                          const double2 *__restrict__ tw, int ts, int nb, bool inverse,
                                          double2 *wsh) {
    const int NR = N / R;
    const int tstride = N / (Ns * R);
    // R-point DFT constants W_R^m, m < R (conjugated for the inverse)
    constexpr bool kShared = R >= 7;
    double2 wr[kShared ? 1 : R];
    if constexpr (kShared) {
        for (int m = threadIdx.x; m < R; m += blockDim.x) {
            const double2 w = tw[m * NR * ts];
            wsh[m] = inverse ? cconj(w) : w;
        }
        __syncthreads();
    } else {
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const double2 w = tw[m * NR * ts];
            wr[m] = inverse ? cconj(w) : w;
        }
    }
    for (int jt = threadIdx.x; jt < nb * NR; jt += blockDim.x) {
        const int sub = jt / NR, j = jt - sub * NR;       // sub-transform, butterfly within it
        const double2 *__restrict__ sv = src + sub * N;
        double2 *__restrict__ dv = dst + sub * N;
        const int k = j % Ns;
        double2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double2 x = sv[j + r * NR];
            if (r > 0) {
                double2 w = tw[k * r * tstride * ts];
                x = cmul(x, inverse ? cconj(w) : w);
            }
            v[r] = x;
        }
        const int d = (j / Ns) * Ns * R + k;
        if (R == 2) {
            dv[d] = cadd(v[0], v[1]);
            dv[d + Ns] = csub(v[0], v[1]);
        } else if (R == 4) {
            // W_4 = -i (forward), +i (inverse)
            const double2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
            const double2 b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
            const double2 jb1 = inverse ? make_double2(-b1.y, b1.x) : make_double2(b1.y, -b1.x);
            dv[d] = cadd(a0, b0);
            dv[d + Ns] = cadd(a1, jb1);
            dv[d + 2 * Ns] = csub(a0, b0);
            dv[d + 3 * Ns] = csub(a1, jb1);
        } else {
            if constexpr (kShared) {
                // one output at a time (the R inputs stay in registers), constants W_R^{r t mod R} from shared
#pragma unroll 1
                for (int t = 0; t < R; ++t) {
                    double2 acc = v[0];
                    int idx = 0;
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        idx += t;
                        if (idx >= R) idx -= R;
                        acc = cadd(acc, cmul(v[r], wsh[idx]));
                    }
                    dv[d + t * Ns] = acc;
                }
            } else {
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    double2 acc = v[0];
#pragma unroll
                    for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], wr[(r * t) % R]));
                    dv[d + t * Ns] = acc;
                }
            }
        }
    }
}

__device__ double2 *fft_stockham(double2 *src, double2 *dst, int N, const int *radix, int nstages,
                                 const double2 *__restrict__ tw, int ts, int nb, bool inverse, double2 *wsh) {
    int Ns = 1;
    for (int st = 0; st < nstages; ++st) {
        const int R = radix[st];
        switch (R) {
            case 2: fft_stage<2>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 3: fft_stage<3>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 4: fft_stage<4>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 5: fft_stage<5>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 7: fft_stage<7>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 11: fft_stage<11>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 13: fft_stage<13>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 17: fft_stage<17>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            case 19: fft_stage<19>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
            default: fft_stage<23>(src, dst, N, Ns, tw, ts, nb, inverse, wsh); break;
        }
        __syncthreads();
        double2 *tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }
    return src;
}

// Push j (1..gamma) of a slip rate held over gamma lattice steps: V into the ring slot of the tick, and the slip
// delta^{n+j} = delta^n + j dt V (or the caller's slip delta^{n+gamma} on the straight line from delta^n); delta^n is
// kept in slip_prev for the corrector's replacement.  gamma = 1: one ordinary push.
__global__ void k_push(StepArgs a_, const double *__restrict__ V, const double *__restrict__ slip_in,
                       int replace_last, int j, int gamma) {
    StepArgs a = a_;
    apply_dyn(a);
    const int64_t BN = (int64_t)a.B * a.N;
    const int slot = (int)(a.step % a.ring);
    double *vr = a.vring + (int64_t)slot * a.ring_stride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < BN; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / a.N, i = e - b * a.N;
        // the caller's element: itself, or with a free surface the real element whose rate an image carries
        int64_t ue = e;
        if (a.io_map) {
            const int m = a.io_map[i];
            ue = b * a.N_io + (m >= 0 ? m : -1 - m);
        }
        const double v = V[ue];
        vr[i * a.B + b] = v;                           // ring layout [slot][element][scenario]
        if (a.prec == kPrecDF64) {
            const float hi = (float)v;
            reinterpret_cast<float2 *>(a.xring)[(int64_t)slot * a.ring_stride + i * a.B + b] =
                make_float2(hi, (float)(v - (double)hi));
        } else if (a.xsplit) {
            // the FP32 value as bfloat16 high part + bfloat16 of the remainder (the tensor-core B operand)
            __nv_bfloat16 *xr = reinterpret_cast<__nv_bfloat16 *>(a.xring) + ((int64_t)slot * a.ring_stride + i * 8) * 2;
            const float f = (float)v;
            const __nv_bfloat16 h = __float2bfloat16_rn(f);
            xr[b] = h;
            xr[8 + b] = __float2bfloat16_rn(f - __bfloat162float(h));
        } else if (a.prec != kPrecFP64) {
            reinterpret_cast<float *>(a.xring)[(int64_t)slot * a.ring_stride + i * a.B + b] = (float)v;
        }
        const double base = replace_last || j > 1 ? a.slip_prev[e] : a.slip[e];
        double s;
        if (slip_in) {
            s = gamma == 1 ? slip_in[ue] : base + (slip_in[ue] - base) * ((double)j / (double)gamma);
        } else {
            s = __dadd_rn(base, __dmul_rn(v, (double)j * a.dt));   // delta^n = delta^{n-1} + dt V^n
        }
        if (!replace_last && j == 1) a.slip_prev[e] = a.slip[e];
        a.slip[e] = s;
        if (a.tail) a.sring[(a.step % a.sring_depth) * BN + i * a.B + b] = s;
    }
}

// The padded real transform from the half-length complex one: X_k = E_k + e^{-2 pi i k/M} O_k with
// E_k = (Z_k + conj Z_{N-k}) / 2, O_k = (Z_k - conj Z_{N-k}) / (2i); zc = conj Z_{N-k}, pk = e^{-2 pi i k/M}.
__device__ __forceinline__ double2 real_post(double2 zk, double2 zc, double2 pk) {
    const double2 E = make_double2(0.5 * (zk.x + zc.x), 0.5 * (zk.y + zc.y));
    const double2 dd = csub(zk, zc);
    const double2 O = make_double2(0.5 * dd.y, -0.5 * dd.x);
    return cadd(E, cmul(pk, O));
}

// The inverse: Z_k = E_k + i O_k from the modes F_k (F_0 = 0) and conj F_{N-k}, pk = e^{-2 pi i k/M}.
__device__ __forceinline__ double2 real_pre(const double2 *__restrict__ Fm, int k, int N, double2 pk) {
    const double2 A = k == 0 ? make_double2(0.0, 0.0) : Fm[k];
    const double2 Bc = cconj(Fm[N - k]);
    const double2 E = make_double2(0.5 * (A.x + Bc.x), 0.5 * (A.y + Bc.y));
    const double2 dd = cmul(csub(A, Bc), cconj(pk));
    const double2 O = make_double2(0.5 * dd.x, 0.5 * dd.y);
    return make_double2(E.x - O.y, E.y + O.x);
}

// Spectral coefficients of the zero-padded slip (Eq. functional_no_replication): D_k = (1/M) sum_{j<N_f}
// delta_j e^{-2 pi i k j / M}, M = 2 N_f, k = 0..N_f, from one N_f-point complex FFT of z_j = x_{2j} + i x_{2j+1}
// (x = delta padded with zeros): X_k = E_k + e^{-2 pi i k/M} O_k, E_k = (Z_k + conj Z_{N-k})/2,
// O_k = (Z_k - conj Z_{N-k})/(2i).  One CTA per (fault, scenario); D^n goes to ring slot n mod R_f.
__global__ void __launch_bounds__(kThreads) k_fft_forward(StepArgs a_) {
    StepArgs a = a_;
    apply_dyn(a);
    extern __shared__ double2 smem[];
    const FaultDev &fd = a.faults[blockIdx.x];
    if (fd.n1 > 0) return;                             // a large fault: its FFT runs on a cluster
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
    double2 *Z = fft_stockham(b0, b1, N, fd.radix, fd.nstages, tw, 1, 1, false, smem + 2 * a.max_nf);
    const double invM = 1.0 / (2.0 * N);
    const int slot = (int)(a.step % fd.ring);
    double2 *ring = a.dring + fd.dring_off + (int64_t)b * (N + 1) * fd.ring + slot;
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        const double2 X = real_post(Z[k == N ? 0 : k], cconj(Z[k == 0 ? 0 : N - k]), post[k]);
        ring[(int64_t)k * fd.ring] = make_double2(X.x * invM, X.y * invM);
    }
}

// Per-mode causal convolution (Eq. funcational_discretized_form):
//   F_n = -(mu k_n / 2) sum_{T=0}^{min(W_f(n), step)} w_n^T D_n^{step - T},  k_n = pi n / L_f.
// One warp per (mode, scenario); lanes stride the lags, four lags a lane in flight (the loop is latency-bound:
// windows run to ~2000 lags); the ring is mode-major so the lanes read contiguous slots.
__global__ void __launch_bounds__(kThreads) k_modeconv(StepArgs a_) {
    StepArgs a = a_;
    apply_dyn(a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // batches: one block per mode, one warp per scenario, so the warps read the mode's weights together (L1 hits
    // after the first); one scenario: eight modes per block
    const int md = a.B > 1 ? blockIdx.x : blockIdx.x * (kThreads / 32) + warp;
    const int b = a.B > 1 ? warp : 0;
    if (md >= a.n_modes) return;
    const ModeDev mo = a.modes[md];
    const FaultDev fd = a.faults[mo.fault];
    const int R = fd.ring;
    const int64_t Tmax = mo.W < a.lag_max ? mo.W : a.lag_max;
    const double2 *ring = a.dring + fd.dring_off + ((int64_t)b * (fd.nf + 1) + mo.n) * R;
    const double *w = a.w + mo.w_off;
    const int slot0 = (int)(a.step % R);
    double re = 0.0, im = 0.0;
#pragma unroll 4
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
        if (a.tail && a.lag_max > mo.W) {
            // static tail: the spectrum at the window's far edge times the weight mass beyond the window
            int s = slot0 - mo.W - 1;
            if (s < 0) s += R;
            const double2 d = ring[s];
            re += mo.tailc * d.x;
            im += mo.tailc * d.y;
        }
        const double f = fd.kfac * mo.n;
        a.fmodes[(int64_t)b * a.n_modes_total + fd.mode_off + mo.n] = make_double2(f * re, f * im);
    }
}

// Element m of fault fd in scenario b: tau = radiation damping + self (fs) + interaction, and the three parts, in
// the caller's layout: [B][N], or with a free surface [B][N_io] holding the real elements only.
__device__ __forceinline__ void assemble_out(const StepArgs &a, const FaultDev &fd, int b, int m, double fs,
                                            const double *__restrict__ V, double *__restrict__ tau,
                                            double *__restrict__ parts) {
    int64_t o = (int64_t)b * a.N + fd.off + m;
    int64_t BNo = (int64_t)a.B * a.N;
    if (a.io_map) {
        const int u = a.io_map[fd.off + m];
        if (u < 0) return;                             // an image element: computed, not returned
        o = (int64_t)b * a.N_io + u;
        BNo = (int64_t)a.B * a.N_io;
    }
    const double rad = a.rad * V[(int64_t)(fd.off + m) * a.B + b];
    const double f = a.fint[(int64_t)b * a.N + fd.off + m];
    tau[o] = rad + fs + f;
    if (parts) {
        parts[o] = rad;
        parts[BNo + o] = fs;
        parts[2 * BNo + o] = f;
    }
}

// Inverse transform and assembly: f_self,j = sum_{n=-N_f+1}^{N_f} F_n e^{2 pi i n j / M} (F_{-n} = conj F_n,
// F_0 = 0), kept for j < N_f, from one N_f-point inverse complex FFT; then
// tau = -(mu / 2 c_s) V + f_self + f_int (Eq. superimposition2).
__global__ void __launch_bounds__(kThreads) k_ifft_assemble(StepArgs a_, double *__restrict__ tau,
                                                            double *__restrict__ parts) {
    StepArgs a = a_;
    apply_dyn(a);
    extern __shared__ double2 smem[];
    const FaultDev &fd = a.faults[blockIdx.x];
    if (fd.n1 > 0) return;                             // a large fault: its FFT runs on a cluster
    const int b = blockIdx.y;
    const int N = fd.nf;
    double2 *b0 = smem, *b1 = smem + N;
    const double2 *Fm = a.fmodes + (int64_t)b * a.n_modes_total + fd.mode_off;
    const double2 *tw = a.tw + fd.tw_off;
    const double2 *post = tw + N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) b0[k] = real_pre(Fm, k, N, post[k]);
    __syncthreads();
    const double2 *z = fft_stockham(b0, b1, N, fd.radix, fd.nstages, tw, 1, 1, true, smem + 2 * a.max_nf);
    const double *V = a.vring + (int64_t)(a.step % a.ring) * a.ring_stride;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        const double2 zz = z[m >> 1];
        assemble_out(a, fd, b, m, 2.0 * ((m & 1) ? zz.y : zz.x), V, tau, parts);
    }
}

// Large faults (N_f = n1 n2, both multiples of kFftCluster): the FFTs run on a thread-block cluster of
// kFftCluster CTAs, one per SM, because one SM's FP64 pipe (2 FMA per clock) bounds a one-CTA transform of a few
// thousand points at ~0.1 ms.  Four-step factorisation: with j = n2' n1 + n2 (n2' = n2 of the plan) and
// k = k1 + n1 k2,  Z_k = sum_{n2} W_{n2'}^{n2 k2} [W_N^{n2 k1} sum_{n1} W_{n1'}^{n1 k1} z_j]: CTA r transforms the
// columns n2 in [r c2, (r + 1) c2) (c2 = n2' / C) and keeps them, twiddled, in its shared memory; after a cluster
// barrier it gathers the rows k1 in [r c1, (r + 1) c1) from all CTAs' shared memory (distributed shared memory)
// and transforms them.  Each CTA then holds Z_k for its rows; the forward pass reads conj Z_{N-k} from the CTA
// holding row (n1' - k1) mod n1'.
namespace cg = cooperative_groups;

struct FftCl {
    int N, N1, N2, c1, c2, chunk, r;
    double2 *Y, *w0, *w1, *wsh;
};

__device__ __forceinline__ FftCl fft_cl_setup(const FaultDev &fd, double2 *smem, int r) {
    FftCl q;
    q.N = fd.nf;
    q.N1 = fd.n1;
    q.N2 = fd.n2;
    q.c1 = q.N1 / kFftCluster;
    q.c2 = q.N2 / kFftCluster;
    q.chunk = q.N / kFftCluster;
    q.r = r;
    q.Y = smem;
    q.w0 = smem + q.chunk;
    q.w1 = smem + 2 * q.chunk;
    q.wsh = smem + 3 * q.chunk;
    return q;
}

// Columns (already in w0 as [c2][n1']) -> twiddled Y; cluster barrier; rows gathered into w0 ([c1][n2']) and
// transformed.  Returns the buffer holding Z_{k1 + n1' k2} at [p][k2], k1 = r c1 + p.
__device__ const double2 *fft_cl_run(cg::cluster_group &cl, const FaultDev &fd, const FftCl &q,
                                     const double2 *__restrict__ tw, bool inverse) {
    const double2 *A = fft_stockham(q.w0, q.w1, q.N1, fd.radix1, fd.nst1, tw, q.N2, q.c2, inverse, q.wsh);
    for (int t = threadIdx.x; t < q.chunk; t += blockDim.x) {
        const int c = t / q.N1, k1 = t - c * q.N1;
        const double2 w = tw[(q.r * q.c2 + c) * k1];                 // W_N^{n2 k1}
        q.Y[t] = cmul(A[t], inverse ? cconj(w) : w);
    }
    cl.sync();
    for (int t = threadIdx.x; t < q.chunk; t += blockDim.x) {
        const int p = t / q.N2, n2 = t - p * q.N2;
        const double2 *Yr = cl.map_shared_rank(q.Y, n2 / q.c2);
        q.w0[t] = Yr[(n2 % q.c2) * q.N1 + q.r * q.c1 + p];
    }
    __syncthreads();
    return fft_stockham(q.w0, q.w1, q.N2, fd.radix2, fd.nst2, tw, q.N1, q.c1, inverse, q.wsh);
}

__global__ void __cluster_dims__(kFftCluster, 1, 1) __launch_bounds__(kThreads) k_fft_forward_cl(StepArgs a_) {
    StepArgs a = a_;
    apply_dyn(a);
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double2 smem[];
    const FaultDev &fd = a.faults[a.big[blockIdx.x / kFftCluster]];
    const FftCl q = fft_cl_setup(fd, smem, (int)cl.block_rank());
    const int b = blockIdx.y, N = q.N;
    const double2 *tw = a.tw + fd.tw_off;
    const double *x = a.slip + (int64_t)b * a.N + fd.off;
    for (int t = threadIdx.x; t < q.chunk; t += blockDim.x) {      // z_j = x_2j + i x_2j+1, j = n2' n1 + n2
        const int c = t / q.N1, n1 = t - c * q.N1;
        const int j = q.N2 * n1 + q.r * q.c2 + c;
        const int e = 2 * j, o = 2 * j + 1;
        q.w0[t] = make_double2(e < N ? x[e] : 0.0, o < N ? x[o] : 0.0);
    }
    __syncthreads();
    const double2 *Z = fft_cl_run(cl, fd, q, tw, false);
    cl.sync();
    const double2 *post = tw + N;
    const double invM = 1.0 / (2.0 * N);
    const int slot = (int)(a.step % fd.ring);
    double2 *ring = a.dring + fd.dring_off + (int64_t)b * (N + 1) * fd.ring + slot;
    const int count = q.chunk + (q.r == 0 ? 1 : 0);                // rank 0 also writes k = N_f (from Z_0)
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        const int tt = t == q.chunk ? 0 : t;
        const int p = tt / q.N2, k2 = tt - p * q.N2;
        const int k1 = q.r * q.c1 + p;
        const int k = t == q.chunk ? N : k1 + q.N1 * k2;
        // N - k mod N = (n1' - k1) + n1' (n2' - 1 - k2) for k1 > 0, n1' ((n2' - k2) mod n2') for k1 = 0
        const int k1p = k1 == 0 ? 0 : q.N1 - k1;
        const int k2p = k1 == 0 ? (q.N2 - k2) % q.N2 : q.N2 - 1 - k2;
        const double2 *Zr = cl.map_shared_rank(Z, k1p / q.c1);
        const double2 X = real_post(Z[tt], cconj(Zr[(k1p % q.c1) * q.N2 + k2p]), post[k]);
        ring[(int64_t)k * fd.ring] = make_double2(X.x * invM, X.y * invM);
    }
    cl.sync();                                                     // others read this CTA's rows until here
}

__global__ void __cluster_dims__(kFftCluster, 1, 1) __launch_bounds__(kThreads)
    k_ifft_assemble_cl(StepArgs a_, double *__restrict__ tau, double *__restrict__ parts) {
    StepArgs a = a_;
    apply_dyn(a);
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double2 smem[];
    const FaultDev &fd = a.faults[a.big[blockIdx.x / kFftCluster]];
    const FftCl q = fft_cl_setup(fd, smem, (int)cl.block_rank());
    const int b = blockIdx.y, N = q.N;
    const double2 *tw = a.tw + fd.tw_off;
    const double2 *post = tw + N;
    const double2 *Fm = a.fmodes + (int64_t)b * a.n_modes_total + fd.mode_off;
    for (int t = threadIdx.x; t < q.chunk; t += blockDim.x) {
        const int c = t / q.N1, n1 = t - c * q.N1;
        const int j = q.N2 * n1 + q.r * q.c2 + c;
        q.w0[t] = real_pre(Fm, j, N, post[j]);
    }
    __syncthreads();
    const double2 *z = fft_cl_run(cl, fd, q, tw, true);
    cl.sync();                                                     // every CTA has gathered its rows
    const double *V = a.vring + (int64_t)(a.step % a.ring) * a.ring_stride;
    for (int t = threadIdx.x; t < q.chunk; t += blockDim.x) {
        const int p = t / q.N2, k2 = t - p * q.N2;
        const int k = q.r * q.c1 + p + q.N1 * k2;                    // z_k carries elements 2k and 2k + 1
        const double2 zz = z[t];
        if (2 * k < N) assemble_out(a, fd, b, 2 * k, 2.0 * zz.x, V, tau, parts);
        if (2 * k + 1 < N) assemble_out(a, fd, b, 2 * k + 1, 2.0 * zz.y, V, tau, parts);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Space-time interaction (Eq. fault-to-fault_interactions_discretized) through the H-matrix stack.
//
// Persistent kernel, one CTA per SM: the last warp produces, the CW warps before it consume.  The producer takes
// tasks from a dynamic counter (tasks with T_start <= step form a prefix of the task list), packs consecutive
// causal items (lag <= step) of the task into a shared-memory stage and issues one 1-D bulk copy (cp.async.bulk)
// for their operator bytes; each lane copies one item's slip-rate history slice x^{step - T} (cp.async, 16 bytes
// when aligned).  Each stage completes on an mbarrier (transaction bytes plus the lanes' copy arrivals);
// consumers release it on a second mbarrier.  Consumers compute z = V^T x for the rank rows (phase A) and the
// row updates (phase B), pipelined over stages, accumulating each receiver column of the task in registers; at
// the task's end the column sums, reduced over thread groups in a fixed order, go to the task's own slot of the
// partial buffer.  No atomics: a run is bitwise reproducible.
// Every wait is bounded; a wait that runs out sets the error word and the CTA stops.
// ------------------------------------------------------------------------------------------------------------
// Threads of the interaction kernel for a batch width BT: CW consumer warps (16 while the accumulators are small
// enough for 120 registers, which hides more shared-memory and pipe latency) plus one producer warp; RV values per
// flush round keep the reduction buffer at 16 KB.
// The default count per (precision, batch width, pass); ALT: the other count (8 <-> 16) is compiled too, for the
// autotuner (where 16 warps keep every instantiation within 120 registers: batch widths up to 4, and the BF16
// tensor-core consumers).
template <int PREC, int BT, int PASS> struct InterDefault {
    // the tensor-core consumers (BF16, 8 scenarios): 16 warps on the receiver side; on the source side, where a
    // stage holds few pieces, 8
    static constexpr int CW = BT <= 2 || (PREC == kPrecBF16 && BT == 8 && PASS == 2) ? 16 : 8;
    static constexpr bool ALT = BT <= 4 || PREC == kPrecBF16;
};
template <int PREC, int BT, int PASS, int CWv> struct InterShape {
    static constexpr int CW = CWv;
    static constexpr int NC = CW * 32;
    static constexpr int NT = NC + 32;
    static constexpr int RV = CW == 8 ? 8 : 4;
};
// One unit in a stage: pass 2 -- an item (k < 0: dense rows i0..i1-1 of A^T, k > 0: far rows of U^T); pass 1 -- a
// run (k = its V^T rows).  Rows of all units of a stage are numbered consecutively (row_end: running count).
struct StageItem {
    int32_t k, i0, i1;
    int32_t data_off, x_off;     // byte offsets in the stage of the unit's operator rows and of its history / z rows
    int32_t row_end;
    float scale;
    int32_t map_off;             // pass 1: byte offset in the stage of the run's z-row map (int32 per row)
    int64_t map;                 // pass 1: first zmap entry of the run
};

struct StageInfo {
    int32_t task;                // -1: no more work
    int32_t n;                   // units in the stage
    int32_t flush;               // last stage of the task (pass 2)
    int32_t p, q, r0, c0;        // pass 2: the block; pass 1: q and c0 of the source cluster (p = 0, r0 = 0)
    int32_t n_rows;              // rows of the stage's units
    int64_t part_off;
    StageItem it[kStageItems];
};

// Dynamic shared memory of the interaction kernel for batch width BT, in bytes from the start: the stages, their
// descriptors, the flush buffer and the full/empty mbarriers.  The kernel and its launcher both use this, and the
// kernel checks the end against the size it was launched with.
template <int PREC, int BT, int PASS, int CWv> struct InterLayout {
    static constexpr size_t info = (size_t)kStages * kStageBytes;
    static constexpr size_t red = info + kStages * sizeof(StageInfo);
    static constexpr size_t bars =
        red + (size_t)InterShape<PREC, BT, PASS, CWv>::NC * InterShape<PREC, BT, PASS, CWv>::RV * sizeof(double);
    static constexpr size_t total = bars + (2 * kStages + 1) * sizeof(uint64_t);   // full, empty, consumers
    static_assert(sizeof(StageInfo) % 8 == 0 && red % 8 == 0 && bars % 8 == 0, "8-byte alignment");
    static_assert(total <= 227 * 1024, "shared memory per CTA");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n"
        " .reg .b64 st;\n"
        " mbarrier.arrive.shared::cta.b64 st, [%0];\n"
        "}\n" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n"
        " .reg .b64 st;\n"
        " mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n"
        "}\n" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait (limit_ns of wall time, 2 s unless the scenario sets another, and at most 2^30 polls); false, with
// the error word set, if the phase never completes.  The producer's lane 0 waits and shares the outcome with its warp;
// every lane of a consumer warp waits and the warp combines the outcomes, so an abort is uniform per warp.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < (1u << 30); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && global_ns() - t0 > limit_ns) break;
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte asynchronous copy global -> shared (L2 only), tracked by the issuing thread's cp.async group.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// 4- or 8-byte asynchronous copy global -> shared (any element alignment).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}

// Arrive on the mbarrier once all cp.async copies this thread issued so far have landed (count preset).
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Every consumer lane waits on a stage's full barrier itself; the warp goes on only if all its lanes saw it.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int *err, uint64_t limit_ns) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, err, limit_ns));
}

// A warp is done with a stage: its lanes' shared-memory reads are ordered before lane 0's arrive (release) on the
// stage's empty barrier, which counts one arrival per consumer warp.
__device__ __forceinline__ void warp_release(uint64_t *bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// Meeting of all consumer warps (the task-end reduction through shared memory): an mbarrier counting one arrival per
// warp, waited on with the same bound as the stages, so that a warp that left on an error cannot hang the others.
// ph: this thread's phase bit of the barrier.
__device__ __forceinline__ bool consumers_meet(uint64_t *bar, uint32_t &ph, int *err, uint64_t limit_ns) {
    warp_release(bar);
    const bool ok = warp_wait(bar, ph, err, limit_ns);
    ph ^= 1u;
    return ok;
}

// ------------------------------------------------------------------------------------------------------------
// Arithmetic of each storage precision: stored element S, history element X, dot-product value Z, accumulator
// Acc; mac = acc += s * x; dot = z += s * x.
//   FP64: FP64 FMA.
//   DF64: double-float (FP32 pairs): products by FMA-based TwoProd, sums by TwoSum, the low parts carried along;
//         about 2^-48 relative per operation, on the FP32 pipes (GB300 runs FP64 at 1/58 of the FP32 rate).
//   BF16 / FP16: FP32 products, Kahan-compensated accumulation along the history (the task's lags); the FP16
//         per-slice scale is folded into x (dense) or z (low rank).
// ------------------------------------------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_prod(float2 a, float2 x) {
    const float p = a.x * x.x;
    float e = fmaf(a.x, x.x, -p);
    e = fmaf(a.x, x.y, e);
    e = fmaf(a.y, x.x, e);
    return DF{p, e};
}

__device__ __forceinline__ void df_add(DF &s, DF v) {
    const float t = s.hi + v.hi;
    const float bv = t - s.hi;
    const float err = (s.hi - (t - bv)) + (v.hi - bv);
    s.lo += err + v.lo;
    s.hi = t;
}

__device__ __forceinline__ DF df_norm(DF s) {
    const float t = s.hi + s.lo;
    return DF{t, s.lo - (t - s.hi)};
}

template <int PREC> struct PT;

template <> struct PT<kPrecFP64> {
    using S = double;
    using X = double;
    using Z = double;
    using Acc = double;
    __device__ static Acc zero() { return 0.0; }
    __device__ static void mac(Acc &a, S s, X x) { a = fma(s, x, a); }
    __device__ static void macz(Acc &a, S s, Z z) { a = fma(s, z, a); }
    __device__ static Z zz() { return 0.0; }
    __device__ static void dot(Z &z, S s, X x) { z = fma(s, x, z); }
    __device__ static Z shfl_add(Z z, int o, int w) { return z + __shfl_xor_sync(0xffffffffu, z, o, w); }
    __device__ static X xscale(X x, float) { return x; }
    __device__ static Z zscale(Z z, float) { return z; }
    __device__ static double to_d(const Acc &a) { return a; }
};

template <> struct PT<kPrecDF64> {
    using S = float2;
    using X = float2;
    using Z = float2;
    using Acc = DF;
    __device__ static Acc zero() { return DF{0.f, 0.f}; }
    __device__ static void mac(Acc &a, S s, X x) { df_add(a, df_prod(s, x)); }
    __device__ static void macz(Acc &a, S s, Z z) { df_add(a, df_prod(s, z)); }
    __device__ static Z zz() { return make_float2(0.f, 0.f); }
    __device__ static void dot(Z &z, S s, X x) {
        DF d{z.x, z.y};
        df_add(d, df_prod(s, x));
        z = make_float2(d.hi, d.lo);
    }
    __device__ static Z shfl_add(Z z, int o, int w) {
        DF d{z.x, z.y};
        df_add(d, DF{__shfl_xor_sync(0xffffffffu, z.x, o, w), __shfl_xor_sync(0xffffffffu, z.y, o, w)});
        d = df_norm(d);
        return make_float2(d.hi, d.lo);
    }
    __device__ static X xscale(X x, float) { return x; }
    __device__ static Z zscale(Z z, float) {
        const DF d = df_norm(DF{z.x, z.y});
        return make_float2(d.hi, d.lo);
    }
    __device__ static double to_d(const Acc &a) { return (double)a.hi + (double)a.lo; }
};

template <typename H> struct PTHalf {
    using S = H;
    using X = float;
    using Z = float;
    using Acc = float2;     // (sum, compensation)
    __device__ static float f(S s);
    __device__ static Acc zero() { return make_float2(0.f, 0.f); }
    __device__ static void kahan(Acc &a, float v) {
        const float y = v - a.y;
        const float t = a.x + y;
        a.y = (t - a.x) - y;
        a.x = t;
    }
    __device__ static void mac(Acc &a, S s, X x) { kahan(a, f(s) * x); }
    __device__ static void macz(Acc &a, S s, Z z) { kahan(a, f(s) * z); }
    __device__ static Z zz() { return 0.f; }
    __device__ static void dot(Z &z, S s, X x) { z = fmaf(f(s), x, z); }
    __device__ static Z shfl_add(Z z, int o, int w) { return z + __shfl_xor_sync(0xffffffffu, z, o, w); }
    __device__ static X xscale(X x, float sc) { return x * sc; }
    __device__ static Z zscale(Z z, float sc) { return z * sc; }
    __device__ static double to_d(const Acc &a) { return (double)a.x - (double)a.y; }
};
template <> __device__ __forceinline__ float PTHalf<__nv_bfloat16>::f(__nv_bfloat16 s) { return __bfloat162float(s); }
template <> __device__ __forceinline__ float PTHalf<__half>::f(__half s) { return __half2float(s); }
template <> struct PT<kPrecBF16> : PTHalf<__nv_bfloat16> {};
template <> struct PT<kPrecFP16> : PTHalf<__half> {};

// Vector view of the stored operator: VE values of 16 or 8 bytes per load, converted to the arithmetic type E
// (double, DF pair or float).
template <int PREC, int VE> struct VecLoad;
template <int VE> struct VecLoad<kPrecFP64, VE> {
    using E = double;
    __device__ static void ld(const double *p, E *o) {
        if (VE == 2) {
            const double2 v = *reinterpret_cast<const double2 *>(p);
            o[0] = v.x;
            o[VE > 1 ? 1 : 0] = v.y;
        } else {
            o[0] = p[0];
        }
    }
};
template <int VE> struct VecLoad<kPrecDF64, VE> {
    using E = float2;
    __device__ static void ld(const float2 *p, E *o) {
        if (VE == 2) {
            const float4 v = *reinterpret_cast<const float4 *>(p);
            o[0] = make_float2(v.x, v.y);
            o[VE > 1 ? 1 : 0] = make_float2(v.z, v.w);
        } else {
            o[0] = p[0];
        }
    }
};
template <typename H, int VE> struct VecLoadHalf {
    using E = float;
    __device__ static float2 pair(uint32_t w);
    __device__ static void ld(const H *p, E *o) {
        if (VE == 8) {
            const uint4 v = *reinterpret_cast<const uint4 *>(p);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = pair(w[k]);
                o[(2 * k) % VE] = f.x;
                o[(2 * k + 1) % VE] = f.y;
            }
        } else {
            const uint2 v = *reinterpret_cast<const uint2 *>(p);
            const uint32_t w[2] = {v.x, v.y};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float2 f = pair(w[k]);
                o[(2 * k) % VE] = f.x;
                o[(2 * k + 1) % VE] = f.y;
            }
        }
    }
};
template <> __device__ __forceinline__ float2 VecLoadHalf<__nv_bfloat16, 8>::pair(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}
template <> __device__ __forceinline__ float2 VecLoadHalf<__nv_bfloat16, 4>::pair(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}
template <> __device__ __forceinline__ float2 VecLoadHalf<__half, 8>::pair(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <> __device__ __forceinline__ float2 VecLoadHalf<__half, 4>::pair(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <int VE> struct VecLoad<kPrecBF16, VE> : VecLoadHalf<__nv_bfloat16, VE> {};
template <int VE> struct VecLoad<kPrecFP16, VE> : VecLoadHalf<__half, VE> {};

// Elements per vector load: 16 bytes, halved for larger batches to bound the accumulator registers.
template <int PREC, int BT> struct VecWidth {
    static constexpr int SB = PREC == kPrecBF16 || PREC == kPrecFP16 ? 2 : 8;
    static constexpr int value = SB == 2 ? (BT <= 2 ? 8 : 4) : (BT <= 4 ? 2 : 1);
};

// The chunk rotation of 2-byte operator rows (chunk_at) with its row-length terms computed once: rot(r) is row r's
// rotation, at(c, rot) the stored chunk of logical chunk c.  Same mapping as chunk_at.
struct ChunkRot {
    int nch, sh, gm;
    __device__ __forceinline__ explicit ChunkRot(int n) : nch(n) {
        int g = n & -n;
        if (g > 8) g = 8;
        sh = g == 8 ? 0 : g == 4 ? 1 : g == 2 ? 2 : 3;
        gm = g - 1;
    }
    __device__ __forceinline__ int rot(int r) const { return (r >> sh) & gm; }
    __device__ __forceinline__ int at(int c, int rt) const {
        const int q = c + rt;
        return q >= nch ? q - nch : q;
    }
};

// Element offset of vector uu (VE elements) of a row with rotation rt: 2-byte operator rows are stored
// chunk-rotated, 8-byte ones as they are.
template <int PREC, int VE>
__device__ __forceinline__ int vec_off(const ChunkRot &cr, int uu, int rt) {
    if constexpr (PREC == kPrecBF16 || PREC == kPrecFP16) {
        if constexpr (VE == 8) return cr.at(uu, rt) * 8;
        else return cr.at(uu >> 1, rt) * 8 + (uu & 1) * 4;
    } else {
        return uu * VE;
    }
}

// Multiply-accumulate of one converted operator value with one coefficient.
__device__ __forceinline__ void emac(double &acc, double v, double c) { acc = fma(v, c, acc); }
__device__ __forceinline__ void emac(DF &acc, float2 v, float2 c) { df_add(acc, df_prod(v, c)); }
__device__ __forceinline__ void emac(float &acc, float v, float c) { acc = fmaf(v, c, acc); }
// Dot-product step z += v x in the dot type Z (double, (hi, lo) float2, float).
__device__ __forceinline__ void edot(double &z, double v, double x) { z = fma(v, x, z); }
__device__ __forceinline__ void edot(float2 &z, float2 v, float2 x) {
    DF d{z.x, z.y};
    df_add(d, df_prod(v, x));
    z = make_float2(d.hi, d.lo);
}
__device__ __forceinline__ void edot(float &z, float v, float x) { z = fmaf(v, x, z); }

// N values of 4 to 16 bytes each, N * size a multiple of 16, from a 16-byte aligned shared-memory address.
// [tensor-core consumers: begin]
// ------------------------------------------------------------------------------------------------------------
// Tensor-core consumers for BF16 storage with 8 scenarios: with B = 8 the interaction is a multi-right-hand-side
// contraction, and each 16 receivers x 8 scenarios x 16 sources tile is one warp-level MMA (m16n8k16, BF16 inputs,
// FP32 accumulation) instead of 2048 FFMAs and their shared-memory operand loads.  The FP32 history values (x, z)
// are split into BF16 hi + lo parts (two MMAs), so they keep 16 mantissa bits; the BF16 operator is used as stored.
// Per stage the MMA accumulators are FP32 and are added, Kahan-compensated, into the task's accumulator.
// ------------------------------------------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// d += A b: A 16 x 16 row-major BF16 (four registers), b 16 x 8 BF16 (two registers), d 16 x 8 FP32.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Two BF16 values in one register, the first in the low half (the lower index of an MMA fragment pair).
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// B fragments (rows k = 2 tg + {0, 1} and 2 tg + 8 + {0, 1} of a 16 x 8 tile, column g) of four FP32 values,
// split into hi and lo BF16 parts.
// Zero the halves of A-fragment registers whose inner index (k = k0 + 2 tg + {0, 1}, and + 8 for registers 2, 3)
// is not below kvalid: operand bytes past an item are not guaranteed to be finite numbers.
__device__ __forceinline__ void mask_a_k(uint32_t (&a)[4], int tg, int kvalid) {
    const int k0 = 2 * tg;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int k = k0 + (r >= 2 ? 8 : 0);
        const uint32_t keep = (k < kvalid ? 0x0000ffffu : 0u) | (k + 1 < kvalid ? 0xffff0000u : 0u);
        a[r] &= keep;
    }
}

// Splits the FP32 operand rows [rows][8] of one unit, in place, into packed BF16 (hi, lo) pairs laid out as MMA B
// Consumer warps of k_interaction<BF16, 8, PASS>.  B operand rows (history values of source columns, z values)
// arrive split: 16 bytes of bfloat16 high parts of scenarios 0..7, then 16 bytes of low parts; one ldmatrix.trans
// per 16-row K step yields both halves' fragments (rows past the unit's staged rows are clamped to its last row:
// finite values, multiplied by A fragments masked to zero there).
//   Pass 1: each (run, 16 rows) piece is one warp's Z tile over the run's source columns; its rows go to the z rows
//   that the staged z-row map gives, written split as well.
//   Pass 2: the task's receivers form mt 16-row tiles; warp w owns tile w mod mtp in group w / mtp (mtp = mt
//   rounded up to 1, 2, 4 or 8) and the stage's (unit, 16-row chunk) pieces are dealt round-robin to the groups; at
//   the task's end the groups are added in a fixed order.  Blocks are at most 128 receivers wide here (scenario
//   creation checks).
template <int CW, int PASS>
__device__ __forceinline__ void consume_mma(const StepArgs &a, StageInfo *info, unsigned char *stage_mem, double *red,
                                            uint64_t *full, uint64_t *empty) {
    constexpr int NC = CW * 32;
    constexpr int B8 = 8;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int g = lane >> 2, tg = lane & 3, mi = lane >> 3, rr = lane & 7;
    uint32_t *zg = static_cast<uint32_t *>(a.zbuf);       // z rows: 4 words of high pairs, 4 of low pairs
    int cur = -1, mt = 1, mtp = 1, G = CW, grp = 0, tile = 0;
    int ts = 0;                                            // pass 2: the stage's index within its task
    bool act = true;
    float2 acc[4];
    // products with the hi and the lo parts of the operand, in two sets that alternate from piece to piece (four
    // independent MMA chains per warp)
    float dst[4], dsl[4], dst2[4], dsl2[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        acc[v] = make_float2(0.f, 0.f);
        dst[v] = 0.f;
        dsl[v] = 0.f;
        dst2[v] = 0.f;
        dsl2[v] = 0.f;
    }
    bool alt = false;
    // Warps run through the stages on their own: each waits for a stage, takes its share of the pieces (dealt from a
    // start that rotates with the stage, so that no warp always gets the extra ones) and releases the stage; they
    // meet only to add the groups of a finished task.  On the receiver side the rotation follows the stage's index
    // within its task, which the task alone fixes: a group's sums, hence the result, do not depend on which CTA ran
    // the task.
    uint32_t mph = 0;
    for (int gi = 0;; ++gi) {
        const int slot = gi % kStages;
        if (!warp_wait(&full[slot], (gi / kStages) & 1, a.err, a.wait_ns)) return;
        const StageInfo &si = info[slot];
        if (si.task < 0) break;
        unsigned char *base = stage_mem + (size_t)slot * kStageBytes;
        if constexpr (PASS == 1) {
            const int q2 = pad_row(si.q, kPrecBF16);
            const ChunkRot cr(q2 / 8);
            int u = 0;
            for (int m = 0; m < si.n; ++m) {
                const StageItem &it = si.it[m];
                const int rows = it.k;
                const __nv_bfloat16 *V = reinterpret_cast<const __nv_bfloat16 *>(base + it.data_off);
                const unsigned char *xr = base + it.x_off;                  // q2 split history rows
                const int32_t *zm = reinterpret_cast<const int32_t *>(base + it.map_off);
                const int pieces = (rows + 15) >> 4;
                for (int pc = (warp - (u + gi) % CW + CW) % CW; pc < pieces; pc += CW) {
                    const int r0 = pc * 16;
                    // four independent accumulator chains: (hi, lo) parts of x times (even, odd) K steps
                    float d[4][4] = {};
                    const int arow = min(r0 + (mi & 1) * 8 + rr, rows - 1);     // rows past the run: not read
                    const int art = cr.rot(arow);
                    for (int K0 = 0, kk = 0; K0 < q2; K0 += 16, kk ^= 1) {
                        uint32_t af[4];
                        // chunk K0 / 8 (+1) of the row, rotated; past the row (a last piece of 8 columns) its last
                        // chunk, against B rows and A columns masked to zero
                        const int ach = min(K0 / 8 + (mi >> 1), cr.nch - 1);
                        ldsm_x4(af, V + (int64_t)arow * q2 + cr.at(ach, art) * 8);
                        if (q2 - K0 < 16) mask_a_k(af, tg, q2 - K0);
                        // B: matrices (high, K0..K0+7), (high, K0+8..), (low, K0..), (low, K0+8..); columns past
                        // the slice (a last piece of 8) read its last row, against A columns masked to zero
                        uint32_t bf[4];
                        const int brow = min(K0 + (mi & 1) * 8 + rr, q2 - 1);
                        ldsm_x4_t(bf, xr + brow * 32 + (mi >> 1) * 16);
                        if (kk == 0) {
                            mma_bf16(d[0], af, bf[0], bf[1]);
                            mma_bf16(d[1], af, bf[2], bf[3]);
                        } else {
                            mma_bf16(d[2], af, bf[0], bf[1]);
                            mma_bf16(d[3], af, bf[2], bf[3]);
                        }
                    }
                    // D fragment: v = 0, 1 -> row g, scenarios 2 tg, 2 tg + 1; v = 2, 3 -> row g + 8.  Each z value
                    // goes out split (scenarios >= B hold zero history, hence zero z)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = r0 + g + 8 * h;
                        if (row < rows) {
                            const float z0 = (d[0][2 * h] + d[1][2 * h]) + (d[2][2 * h] + d[3][2 * h]);
                            const float z1 = (d[0][2 * h + 1] + d[1][2 * h + 1]) + (d[2][2 * h + 1] + d[3][2 * h + 1]);
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(z0), h1 = __float2bfloat16_rn(z1);
                            const __nv_bfloat16 l0 = __float2bfloat16_rn(z0 - __bfloat162float(h0));
                            const __nv_bfloat16 l1 = __float2bfloat16_rn(z1 - __bfloat162float(h1));
                            uint32_t *zr = zg + (int64_t)zm[row] * 8;
                            zr[tg] = pack_bf16(h0, h1);
                            zr[4 + tg] = pack_bf16(l0, l1);
                        }
                    }
                }
                u += pieces;
            }
            warp_release(&empty[slot]);
        } else {
            const int p = si.p, p2 = pad_row(p, kPrecBF16);
            const int flush = si.flush;
            const int64_t part_off = si.part_off;
            if (si.task != cur) {
                cur = si.task;
                ts = 0;
                mt = (p2 + 15) / 16;
                mtp = mt <= 1 ? 1 : mt <= 2 ? 2 : mt <= 4 ? 4 : 8;
                G = CW / mtp;
                grp = warp / mtp;
                tile = warp % mtp;
                act = tile < mt;
            }
            int u = 0;
            const int i0 = tile * 16;
            // the warp's receiver chunk (+1 for matrices 1 and 3) in every row; past the row (receivers >= p2) its
            // last chunk: those receivers' sums are never written
            const ChunkRot cr2(p2 / 8);
            const int ach2 = min(i0 / 8 + (mi & 1), cr2.nch - 1);
            for (int m = 0; m < si.n; ++m) {
                const StageItem &it = si.it[m];
                const int rows = it.k < 0 ? it.i1 - it.i0 : it.k;
                const __nv_bfloat16 *S = reinterpret_cast<const __nv_bfloat16 *>(base + it.data_off);
                // B operand rows (history values of dense items, z values of far items), split
                const unsigned char *br = base + it.x_off;
                const int pieces = (rows + 15) >> 4;
                // fragments of piece pc: A (receivers x 16 unit rows, rotated chunks; rows past the unit are not
                // read and masked to zero), B ((high, k0..k0+7), (high, k0+8..), (low, k0..), (low, k0+8..); rows
                // past the unit read its last row, against A entries masked to zero)
                auto load = [&](int pc, uint32_t (&af)[4], uint32_t (&bf)[4]) {
                    const int k0 = pc * 16;
                    const int arow = min(k0 + (mi >> 1) * 8 + rr, rows - 1);
                    ldsm_x4_t(af, S + (int64_t)arow * p2 + cr2.at(ach2, cr2.rot(arow)) * 8);
                    if (rows - k0 < 16) mask_a_k(af, tg, rows - k0);
                    const int brow = min(k0 + (mi & 1) * 8 + rr, rows - 1);
                    ldsm_x4_t(bf, br + brow * 32 + (mi >> 1) * 16);
                };
                int pc = (grp - u - ts) & (G - 1);                  // G: a power of two
                if (act && pc < pieces) {
                    // software-pipelined: the next piece's fragments load while this piece's MMAs issue
                    uint32_t af[4], bf[4];
                    load(pc, af, bf);
                    for (;;) {
                        const int pn = pc + G;
                        uint32_t an[4] = {0u, 0u, 0u, 0u}, bn[4] = {0u, 0u, 0u, 0u};
                        if (pn < pieces) load(pn, an, bn);
                        if (alt) {
                            mma_bf16(dst2, af, bf[0], bf[1]);
                            mma_bf16(dsl2, af, bf[2], bf[3]);
                        } else {
                            mma_bf16(dst, af, bf[0], bf[1]);
                            mma_bf16(dsl, af, bf[2], bf[3]);
                        }
                        alt = !alt;
                        if (pn >= pieces) break;
                        pc = pn;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            af[e] = an[e];
                            bf[e] = bn[e];
                        }
                    }
                }
                u += pieces;
            }
            warp_release(&empty[slot]);
            ++ts;
#pragma unroll
            for (int v = 0; v < 4; ++v) {                      // compensated accumulation, once per stage
                PTHalf<__nv_bfloat16>::kahan(acc[v], (dst[v] + dsl[v]) + (dst2[v] + dsl2[v]));
                dst[v] = 0.f;
                dsl[v] = 0.f;
                dst2[v] = 0.f;
                dsl2[v] = 0.f;
            }
            alt = false;
            if (flush) {
                // D fragment: v = 0, 1 -> receiver row g, scenario 2 tg + v; v = 2, 3 -> row g + 8.  Groups added in
                // a fixed order by the thread that owns each (receiver, scenario); a second meeting frees red.
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    red[(warp * 32 + lane) * 4 + v] = act ? (double)acc[v].x - (double)acc[v].y : 0.0;
                if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                for (int o = t; o < p2 * B8; o += NC) {
                    const int i = o >> 3, nn = o & 7, ti = i >> 4, ii = i & 15;
                    const int lo = (ii & 7) * 4 + (nn >> 1), reg = (ii >> 3) * 2 + (nn & 1);
                    if (i < p && nn < a.B) {
                        double sum = 0.0;
                        for (int gg = 0; gg < G; ++gg) sum += red[((gg * mtp + ti) * 32 + lo) * 4 + reg];
                        a.partial[(int64_t)nn * a.n_partial + part_off + i] = sum;
                    }
                }
                if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[v] = make_float2(0.f, 0.f);
                cur = -1;
            }
        }
    }
}

// [tensor-core consumers: end]
template <int PREC, int BT, int PASS, int CWv>
__global__ void __launch_bounds__(InterShape<PREC, BT, PASS, CWv>::NT, 1) k_interaction(StepArgs a_) {
    StepArgs a = a_;
    apply_dyn(a);
    constexpr int CW = InterShape<PREC, BT, PASS, CWv>::CW, NC = InterShape<PREC, BT, PASS, CWv>::NC;
    constexpr int RV = InterShape<PREC, BT, PASS, CWv>::RV;
    using T = PT<PREC>;
    using S = typename T::S;
    using X = typename T::X;
    using Z = typename T::Z;
    using Acc = typename T::Acc;
    static_assert(sizeof(X) == sizeof(Z), "history and z values are staged alike");
    constexpr int SB = (int)sizeof(S);
    constexpr int XB = (int)sizeof(X);
    constexpr bool kSplitB = PREC == kPrecBF16 && BT == 8;   // split B rows (tensor-core consumers)
    // History / z rows and z-row maps: one bulk copy per unit, except for DF64, whose consumers wait longer for bulk
    // copies of these small slices than for warp-wide element copies (measured: 2.85 vs 1.67 ms for the receiver pass
    // of the six-fault network at depth 2000; FP64 is the same either way and BF16 gains 30 %)
    constexpr bool kBulkX = PREC != kPrecDF64;
    constexpr int XA = 16 / XB;                               // history elements per 16 bytes
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using LY = InterLayout<PREC, BT, PASS, CWv>;
    unsigned char *stage_mem = smem_raw;                                            // kStages x kStageBytes
    StageInfo *info = reinterpret_cast<StageInfo *>(smem_raw + LY::info);
    double *red = reinterpret_cast<double *>(smem_raw + LY::red);                  // [NC][RV]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + LY::bars);
    uint64_t *empty = full + kStages;
    __shared__ int sh_flag;
    const X *xring = PREC == kPrecFP64 ? reinterpret_cast<const X *>(a.vring) : reinterpret_cast<const X *>(a.xring);
    const Z *zbuf = reinterpret_cast<const Z *>(a.zbuf);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        uint32_t dyn;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        if (dyn < LY::total) {                     // launched with less shared memory than the layout needs
            atomicExch(a.err, 2);
            sh_flag = 2;
        } else {
            for (int s = 0; s < kStages; ++s) {
                // the producer's arrive (with the transaction bytes), and with element copies each lane's arrive
                // once its copies have landed
                mbar_init(&full[s], kBulkX ? 1 : 1 + 32);
                mbar_init(&empty[s], CW);          // one release per consumer warp
            }
            mbar_init(&empty[kStages], CW);        // the consumers' meeting barrier
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            sh_flag = *(volatile int *)a.err;      // an earlier launch already failed: do nothing
        }
    }
    __syncthreads();
    if (sh_flag) return;

    if (warp == CW) {
        // ------------------------------------------------------------------ producer warp
        // A task's units are adjacent in memory: their operator rows go in one bulk copy per stage (lane 0).  The
        // history (pass 1 runs, pass 2 dense items) or z rows (pass 2 far items) of each unit are copied by the
        // whole warp with 16-byte cp.async when aligned; each lane arrives on the stage barrier when its copies
        // have landed.  Lane l holds the descriptor of unit it + l; after a stage of n units the descriptors shift
        // down by n and the tail is fetched at once.
        const int n_active = PASS == 1 ? a.n_ztasks_active : a.n_tasks_active;
        const TaskDev *tasks = PASS == 1 ? a.ztasks : a.tasks;
        int task = -1, it = 0, ie = 0;
        TaskDev td{};
        int p = 0, q = 0, r0 = 0, c0 = 0;
        struct Unit {
            int32_t T, k, i0, i1;
            const void *a;
            float scale;
            int64_t map;       // pass 1: zmap offset; pass 2: first z row (far)
        } u{};
        auto load = [&](int idx) {
            Unit r{};
            if (PASS == 1) {
                const RunDev rd = a.runs[idx];
                r = Unit{rd.T, rd.rows, 0, rd.rows, rd.v, 1.f, rd.map};
            } else {
                const ItemDev id = a.items[idx];
                r = Unit{id.T, id.k, id.i0, id.i1, id.a, id.scale, id.zrow};
            }
            return r;
        };
        bool have = false;                          // descriptors of `it` are loaded
        for (int g = 0;; ++g) {
            const int slot = g % kStages;
            if (g >= kStages) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&empty[slot], ((g / kStages) - 1) & 1, a.err, a.wait_ns);
                if (!__shfl_sync(0xffffffffu, ok, 0)) return;
            }
            if (it >= ie) {                        // next task
                int t = 0;
                if (lane == 0) t = atomicAdd(PASS == 1 ? a.counter + 2 : a.counter, 1);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t >= n_active) {
                    if (lane == 0) {
                        info[slot].task = -1;
                        mbar_arrive(&full[slot]);
                    }
                    if (!kBulkX) cp_async_arrive(&full[slot]);
                    return;
                }
                task = t;
                td = tasks[t];
                if (PASS == 1) {
                    const SrcDev sd = a.srcs[td.block];
                    p = 0; r0 = 0; q = sd.q; c0 = sd.c0;
                } else {
                    const BlockDev bd = a.blocks[td.block];
                    p = bd.p; r0 = bd.r0; q = bd.q; c0 = bd.c0;
                }
                it = td.item_begin;
                ie = td.item_end;
                have = false;
            }
            if (!have && it + lane < ie) u = load(it + lane);
            const bool valid = it + lane < ie;
            const int w2 = PASS == 1 ? pad_row(q, PREC) : pad_row(p, PREC);     // operator row length
            // Each unit's history / z rows and z-row map arrive in one bulk copy each, issued by the unit's lane and
            // widened to 16-byte bounds (the consumers index past the skew; values past a unit's count are finite
            // neighbours that multiply zero padding or are masked).  A row holds RW values of the history type: the
            // batch, or 8 for the split rows of the tensor-core consumers (8 bfloat16 high parts, 8 low parts).
            const int RW = kSplitB ? 8 : a.B;
            int data_bytes = 0, x_bytes = 0, nrow = 0;
            int map_bytes = 0;
            if (valid) {
                nrow = u.k < 0 ? u.i1 - u.i0 : u.k;
                data_bytes = SB * nrow * w2;
                const int brows = PASS == 1 ? pad_row(q, PREC) : nrow;
                x_bytes = (XB * brows * RW + 15) / 16 * 16 + 16;
                if (PASS == 1) {                   // the run's z-row map follows its history slice
                    map_bytes = (4 * nrow + 15) / 16 * 16 + 16;
                    x_bytes += map_bytes;
                }
            }
            // units in the stage: the longest prefix of valid lanes (at most kStageItems) whose bytes fit
            int incl = data_bytes + x_bytes;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned fit = __ballot_sync(0xffffffffu, valid && lane < kStageItems && incl <= kStageBytes);
            const int n = __ffs(~fit) - 1 < 0 ? 32 : __ffs(~fit) - 1;
            if (n == 0) {                          // a unit larger than a stage (the build rules this out): stop
                if (lane == 0) {
                    atomicExch(a.err, 3);
                    info[slot].task = -1;
                    mbar_arrive(&full[slot]);
                }
                if (!kBulkX) cp_async_arrive(&full[slot]);
                return;
            }
            const bool in = lane < n;
            int dincl = in ? data_bytes : 0, rincl = in ? nrow : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int d = __shfl_up_sync(0xffffffffu, dincl, o);
                const int r = __shfl_up_sync(0xffffffffu, rincl, o);
                if (lane >= o) {
                    dincl += d;
                    rincl += r;
                }
            }
            // the units' history / z areas follow the operator bytes in the same order: their inclusive sums are
            // incl - dincl over the stage's lanes
            const int xincl = incl - dincl;
            const int total_data = __shfl_sync(0xffffffffu, dincl, 31);
            const int total_rows = __shfl_sync(0xffffffffu, rincl, 31);
            StageInfo *si = &info[slot];
            if (lane == 0) {
                si->task = task;
                si->n = n;
                si->flush = it + n >= ie ? 1 : 0;
                si->p = p;
                si->q = q;
                si->r0 = r0;
                si->c0 = c0;
                si->n_rows = total_rows;
                si->part_off = td.part_off;
            }
            const int data_off = dincl - (in ? data_bytes : 0);
            const int x_off = total_data + xincl - (in ? x_bytes : 0);
            const int map_off = x_off + x_bytes - map_bytes;
            unsigned char *dst = stage_mem + (size_t)slot * kStageBytes;
            // source, count and span (count plus the tail that padding columns multiply) of each unit's history /
            // z values
            const X *xsrc = nullptr;
            int xspan = 0;
            if (in) {
                xspan = (PASS == 1 ? pad_row(q, PREC) : nrow) * RW;
                if (PASS == 2 && u.k > 0) {
                    xsrc = reinterpret_cast<const X *>(zbuf + u.map * RW);
                } else {
                    // lags past the step (whole tasks are switched on) read a slot not yet written: zeros
                    const int64_t back = (a.step - u.T) % a.ring;
                    const int slot_v = (int)(back < 0 ? back + a.ring : back);
                    const int e0 = c0 + (PASS == 1 ? 0 : u.i0);
                    xsrc = xring + (int64_t)slot_v * a.ring_stride + (int64_t)e0 * RW;
                }
            }
            // bulk copies: 16-byte aligned source and length; the skew (a multiple of the element size) moves the
            // unit's view in the stage
            const int32_t *msrc = PASS == 1 ? a.zmap + u.map : nullptr;
            int xskew = 0, mskew = 0;
            uint32_t xcopy = 0, mcopy = 0;
            if (in) {
                xskew = (int)(reinterpret_cast<uintptr_t>(xsrc) & 15);
                if (PASS == 1) mskew = (int)(reinterpret_cast<uintptr_t>(msrc) & 15);
                if (kBulkX) {
                    xcopy = (uint32_t)((xskew + XB * xspan + 15) & ~15);
                    if (PASS == 1) mcopy = (uint32_t)((mskew + 4 * nrow + 15) & ~15);
                }
            }
            if (in)
                si->it[lane] = StageItem{u.k, u.i0, u.i1, data_off, x_off + xskew, rincl, u.scale, map_off + mskew,
                                         u.map};
            uint32_t tx = xcopy + mcopy;
            for (int o = 16; o > 0; o >>= 1) tx += __shfl_xor_sync(0xffffffffu, tx, o);
            __syncwarp();
            if (lane == 0) mbar_arrive_tx(&full[slot], (uint32_t)total_data + tx);
            __syncwarp();
            // lane 0 holds unit `it`, the first of the n adjacent units: their operator bytes in one bulk copy
            if (lane == 0 && total_data > 0) bulk_g2s(dst, u.a, (uint32_t)total_data, &full[slot]);
            if (kBulkX) {
                if (xcopy)
                    bulk_g2s(dst + x_off, reinterpret_cast<const unsigned char *>(xsrc) - xskew, xcopy, &full[slot]);
                if (mcopy)
                    bulk_g2s(dst + map_off, reinterpret_cast<const unsigned char *>(msrc) - mskew, mcopy, &full[slot]);
            } else {
                // the warp copies each unit's slice (16 bytes a lane when the skew is zero) at the same skewed place
                for (int m = 0; m < n; ++m) {
                    const int cnt = __shfl_sync(0xffffffffu, xspan, m);
                    const int sk = __shfl_sync(0xffffffffu, xskew, m);
                    const X *src = reinterpret_cast<const X *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(xsrc), m));
                    X *xd = reinterpret_cast<X *>(dst + __shfl_sync(0xffffffffu, x_off, m) + sk);
                    if (sk == 0) {
                        const int n16 = cnt / XA;
                        for (int c = lane; c < n16; c += 32) cp_async16(xd + c * XA, src + c * XA);
                        for (int c = n16 * XA + lane; c < cnt; c += 32) cp_async_elem<XB>(xd + c, src + c);
                    } else {
                        for (int c = lane; c < cnt; c += 32) cp_async_elem<XB>(xd + c, src + c);
                    }
                }
                if (PASS == 1) {
                    for (int m = 0; m < n; ++m) {
                        const int rows = __shfl_sync(0xffffffffu, nrow, m);
                        const int64_t mp = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)u.map, m);
                        int32_t *md = reinterpret_cast<int32_t *>(dst + __shfl_sync(0xffffffffu, map_off, m) +
                                                                  __shfl_sync(0xffffffffu, mskew, m));
                        for (int c = lane; c < rows; c += 32) cp_async_elem<4>(md + c, a.zmap + mp + c);
                    }
                }
                cp_async_arrive(&full[slot]);
            }
            it += n;
            // shift the descriptors of units it .. it + 31 down and fetch the tail now
            if (it < ie) {
                Unit nx;
                nx.T = __shfl_sync(0xffffffffu, u.T, (lane + n) & 31);
                nx.k = __shfl_sync(0xffffffffu, u.k, (lane + n) & 31);
                nx.i0 = __shfl_sync(0xffffffffu, u.i0, (lane + n) & 31);
                nx.i1 = __shfl_sync(0xffffffffu, u.i1, (lane + n) & 31);
                nx.scale = __shfl_sync(0xffffffffu, u.scale, (lane + n) & 31);
                nx.a = reinterpret_cast<const void *>(
                    __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(u.a), (lane + n) & 31));
                nx.map = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)u.map, (lane + n) & 31);
                if (lane + n < 32) u = nx;
                else if (it + lane < ie) u = load(it + lane);
                have = true;
            } else {
                have = false;
            }
        }
    }

    // [tensor-core consumers: begin]
    if constexpr (PREC == kPrecBF16 && BT == 8) {
        consume_mma<CW, PASS>(a, info, stage_mem, red, full, empty);
        return;
    }
    // [tensor-core consumers: end]
    // ---------------------------------------------------------------------- consumer warps
    const int t = threadIdx.x;
    constexpr int VE = VecWidth<PREC, BT>::value;
    using E = typename VecLoad<PREC, VE>::E;
    if constexpr (PASS == 1) {
        // z = V^T x for every row of the stage's runs.  L lanes share a row, each summing at least four vectors
        // before the shuffle tree (the tree's adds run on the same pipe as the products); DF64 takes one lane per
        // row, its shuffle adds costing a dozen FP32 operations each.  The lanes of row slot rw start their sweep
        // rw * L vectors further on, so the rows a warp reads fall in different shared-memory banks.  History values
        // are read one by one (16-byte vector reads of them measured slower).
        Z *zout = reinterpret_cast<Z *>(a.zbuf);
        // Warps run through the stages on their own (each waits for a stage and releases it); the row slots of a
        // stage start at a warp that rotates with the stage, so that the short last sweep moves from warp to warp.
        for (int g = 0;; ++g) {
            const int slot = g % kStages;
            if (!warp_wait(&full[slot], (g / kStages) & 1, a.err, a.wait_ns)) return;
            const StageInfo &sx = info[slot];
            if (sx.task < 0) break;
            const unsigned char *bx = stage_mem + (size_t)slot * kStageBytes;
            const int nz = sx.n_rows;
            const int qv = pad_row(sx.q, PREC) / VE;
            const int q2 = qv * VE;
            // lanes per row: each lane sums at least four vectors (FP64: eight, since every add of the shuffle tree
            // costs an FP64 pipe slot like a product: 0.91 -> 0.83 ms for the six-fault source pass)
            const int q4 = PREC == kPrecDF64 ? 0 : PREC == kPrecFP64 ? qv >> 3 : qv >> 2;
            const int L = q4 >= 32 ? 32 : q4 >= 16 ? 16 : q4 >= 8 ? 8 : q4 >= 4 ? 4 : q4 >= 2 ? 2 : 1;
            const int subs = 32 / L, SA = CW * subs;
            const int wr = (warp + g) % CW;                        // the warp's place in this stage
            const int sl = lane % L, rw = lane / L, slotA = wr * subs + rw;
            const int rot = (rw * L) % qv;
            const ChunkRot cr1(q2 * (int)sizeof(S) / 16);
            // sweeps that reach at least one of the warp's row slots (uniform over the warp)
            const int trips = nz > wr * subs ? (nz - wr * subs + SA - 1) / SA : 0;
            int k = 0, zstart = 0;
            for (int r = 0; r < trips; ++r) {
                const int f = slotA + r * SA;
                const bool act = f < nz;
                Z z[BT];
#pragma unroll
                for (int bb = 0; bb < BT; ++bb) z[bb] = T::zz();
                int64_t zrow = 0;
                float sc = 1.f;
                if (act) {
                    while (f >= sx.it[k].row_end) {
                        zstart = sx.it[k].row_end;
                        ++k;
                    }
                    const StageItem &itm = sx.it[k];
                    const S *vr = reinterpret_cast<const S *>(bx + itm.data_off) + (int64_t)(f - zstart) * q2;
                    const X *x = reinterpret_cast<const X *>(bx + itm.x_off);
                    zrow = reinterpret_cast<const int32_t *>(bx + itm.map_off)[f - zstart];
                    if (PREC == kPrecFP16) sc = a.zscale[itm.map + (f - zstart)];
                    const int rt1 = cr1.rot(f - zstart);
                    for (int i = sl; i < qv; i += L) {
                        int uu = i + rot;
                        if (uu >= qv) uu -= qv;
                        E v[VE];
                        VecLoad<PREC, VE>::ld(vr + vec_off<PREC, VE>(cr1, uu, rt1), v);
#pragma unroll
                        for (int e = 0; e < VE; ++e)
#pragma unroll
                            for (int bb = 0; bb < BT; ++bb)
                                edot(z[bb], v[e], x[(uu * VE + e) * a.B + (bb < a.B ? bb : 0)]);
                    }
                }
#pragma unroll
                for (int bb = 0; bb < BT; ++bb) {
                    for (int o = L / 2; o > 0; o >>= 1) z[bb] = T::shfl_add(z[bb], o, L);
                    if (act && sl == 0 && bb < a.B) zout[zrow * a.B + bb] = T::zscale(z[bb], sc);
                }
            }
            warp_release(&empty[slot]);
        }
        return;
    } else {
        // Thread t works in group t / P and owns the VE-wide column vectors (t mod P) + s P, s < nvt, of the block's
        // rows (P a power of two, G = NC / P groups for NC consumer threads).  The stage's rows (rows of A^T times a
        // history value, rows of U^T times a z value) form one flat list dealt round-robin to the groups; a
        // monotone cursor maps a flat index to its unit.  BF16/FP16: plain FP32 partial sums inside a stage, added
        // into the Kahan-compensated accumulator once per stage.
        // vectors per thread and row: aim at 8 multiply-adds per row (fewer index operations per product); at
        // least enough vectors for the widest block when all NC consumers share a row
        constexpr int NVT_T = 8 / (VE * BT) > 1 ? 8 / (VE * BT) : 1;
        constexpr int NVT_MIN = (kMaxBlockSide + VE * NC - 1) / (VE * NC);
        constexpr int NVT = NVT_T > NVT_MIN ? NVT_T : NVT_MIN;
        constexpr bool MP = PREC == kPrecBF16 || PREC == kPrecFP16;
        using PAcc = typename std::conditional<MP, float, Acc>::type;                 // per-stage partial
        int cur = -1, P = 1, G = 1, vec = 0, grp = 0, nvt = 1;
        Acc acc[NVT][VE][BT];
        PAcc part[NVT][VE][BT];
        // Warps run through the stages on their own; the groups' share of a stage's rows starts at a group that
        // rotates (by whole warps) with the stage's index within its task (fixed by the task, so that the sums do not
        // depend on which CTA ran it); all warps meet only for the task-end reduction.
        uint32_t mph = 0;
        int ts = 0;
        for (int g = 0;; ++g) {
            const int slot = g % kStages;
            if (!warp_wait(&full[slot], (g / kStages) & 1, a.err, a.wait_ns)) return;
            const StageInfo &si = info[slot];
            const int task = si.task;
            if (task < 0) break;
            const int p = si.p, p2 = pad_row(p, PREC);
            const int flush = si.flush;
            const int64_t part_off = si.part_off;
            if (task != cur) {
                cur = task;
                ts = 0;
                // P: threads per row, a power of two, so that groups tile the warps (P <= 32) or whole warps
                // tile a group (P > 32)
                const int pv = p2 / VE;
                const int pn = (pv + NVT_T - 1) / NVT_T;
                P = 1;
                while (P < pn && P < NC) P <<= 1;
                G = NC / P;
                vec = t % P;
                grp = t / P;
                nvt = (pv + P - 1) / P;
#pragma unroll
                for (int s = 0; s < NVT; ++s)
#pragma unroll
                    for (int e = 0; e < VE; ++e)
#pragma unroll
                        for (int bb = 0; bb < BT; ++bb) {
                            acc[s][e][bb] = T::zero();
                            part[s][e][bb] = PAcc{};
                        }
            }
            const unsigned char *base = stage_mem + (size_t)slot * kStageBytes;
            const ChunkRot cr2(p2 * (int)sizeof(S) / 16);
            if (grp < G) {
                const int nr = si.n_rows;
                const int gpw = P >= 32 ? 1 : 32 / P;              // groups per warp
                const int f0 = (grp + ts * gpw) & (G - 1);         // G = NC / P: a power of two
                int k = 0, rstart = 0;
                // one row's coefficients (history or z values) and its operator vectors, then its products (fetching
                // the next row during the current one's products measured slower for BF16: 0.51 -> 0.62 ms; this
                // form is 5-13 % faster than loads and products interleaved for batches up to 4)
                struct RowFetch {
                    E cv[BT];
                    E v[NVT][VE];
                };
                auto fetch = [&](int f, RowFetch &rw) {
                    while (f >= si.it[k].row_end) {
                        rstart = si.it[k].row_end;
                        ++k;
                    }
                    const StageItem &itm = si.it[k];
                    const int r = f - rstart;
                    const S *rowp = reinterpret_cast<const S *>(base + itm.data_off) + (int64_t)r * p2;
                    const int rt2 = cr2.rot(r);
                    if (itm.k < 0) {
                        const X *x = reinterpret_cast<const X *>(base + itm.x_off);
#pragma unroll
                        for (int bb = 0; bb < BT; ++bb) {
                            const X xv = T::xscale(x[r * a.B + (bb < a.B ? bb : 0)], itm.scale);
                            rw.cv[bb] = *reinterpret_cast<const E *>(&xv);
                        }
                    } else {
                        const Z *zr = reinterpret_cast<const Z *>(base + itm.x_off);
#pragma unroll
                        for (int bb = 0; bb < BT; ++bb) {
                            const Z zv = zr[r * a.B + (bb < a.B ? bb : 0)];
                            rw.cv[bb] = *reinterpret_cast<const E *>(&zv);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < NVT; ++s) {
                        const int uu = vec + s * P;
                        if (s < nvt && uu * VE < p2) VecLoad<PREC, VE>::ld(rowp + vec_off<PREC, VE>(cr2, uu, rt2), rw.v[s]);
                    }
                };
                auto compute = [&](const RowFetch &rw) {
#pragma unroll
                    for (int s = 0; s < NVT; ++s) {
                        const int uu = vec + s * P;
                        if (s < nvt && uu * VE < p2) {
#pragma unroll
                            for (int e = 0; e < VE; ++e)
#pragma unroll
                                for (int bb = 0; bb < BT; ++bb) {
                                    if constexpr (MP) emac(part[s][e][bb], rw.v[s][e], rw.cv[bb]);
                                    else emac(acc[s][e][bb], rw.v[s][e], rw.cv[bb]);
                                }
                        }
                    }
                };
                if constexpr (BT < 8) {
                    for (int f = f0; f < nr; f += G) {
                        RowFetch rw;
                        fetch(f, rw);
                        compute(rw);
                    }
                } else {
                    // 8-wide batches: loads and products interleaved row by row (the fetch-then-compute form above
                    // measured 4x slower for FP64 with 8 scenarios; faster for narrower batches)
                    for (int f = f0; f < nr; f += G) {
                        while (f >= si.it[k].row_end) {
                            rstart = si.it[k].row_end;
                            ++k;
                        }
                        const StageItem &itm = si.it[k];
                        const int r = f - rstart;
                        const S *rowp = reinterpret_cast<const S *>(base + itm.data_off) + (int64_t)r * p2;
                        const int rt2 = cr2.rot(r);
                        E cv[BT];
                        if (itm.k < 0) {
                            const X *x = reinterpret_cast<const X *>(base + itm.x_off);
#pragma unroll
                            for (int bb = 0; bb < BT; ++bb) {
                                const X xv = T::xscale(x[r * a.B + (bb < a.B ? bb : 0)], itm.scale);
                                cv[bb] = *reinterpret_cast<const E *>(&xv);
                            }
                        } else {
                            const Z *zr = reinterpret_cast<const Z *>(base + itm.x_off);
#pragma unroll
                            for (int bb = 0; bb < BT; ++bb) {
                                const Z zv = zr[r * a.B + (bb < a.B ? bb : 0)];
                                cv[bb] = *reinterpret_cast<const E *>(&zv);
                            }
                        }
#pragma unroll
                        for (int s = 0; s < NVT; ++s) {
                            if (s < nvt) {
                                const int uu = vec + s * P;
                                if (uu * VE < p2) {
                                    E v[VE];
                                    VecLoad<PREC, VE>::ld(rowp + vec_off<PREC, VE>(cr2, uu, rt2), v);
#pragma unroll
                                    for (int e = 0; e < VE; ++e)
#pragma unroll
                                        for (int bb = 0; bb < BT; ++bb) {
                                            if constexpr (MP) emac(part[s][e][bb], v[e], cv[bb]);
                                            else emac(acc[s][e][bb], v[e], cv[bb]);
                                        }
                                }
                            }
                        }
                    }
                }
                if constexpr (MP) {                                // compensated accumulation, once per stage
#pragma unroll
                    for (int s = 0; s < NVT; ++s)
#pragma unroll
                        for (int e = 0; e < VE; ++e)
#pragma unroll
                            for (int bb = 0; bb < BT; ++bb) {
                                PTHalf<__half>::kahan(acc[s][e][bb], part[s][e][bb]);
                                part[s][e][bb] = PAcc{};
                            }
                }
            }
            warp_release(&empty[slot]);
            ++ts;
            if (flush) {
                // column c = (vec + s P) VE + e; value v of a thread: vector s = v / (VE BT), element e = (v / BT) mod
                // VE, scenario bb = v mod BT.  The G groups are reduced in a fixed order, RV values per round through
                // shared memory; rounds past the task's vectors are skipped (uniform).  Each round's reads are
                // followed by a second meeting, which frees red for the next writes.
                constexpr int NV = NVT * VE * BT;
                const int nv = nvt * VE * BT;
                if (G == 1) {
#pragma unroll
                    for (int s = 0; s < NVT; ++s)
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            const int c = (vec + s * P) * VE + e;
                            if (s < nvt && c < p)
#pragma unroll
                                for (int bb = 0; bb < BT; ++bb)
                                    if (bb < a.B)
                                        a.partial[(int64_t)bb * a.n_partial + part_off + c] = T::to_d(acc[s][e][bb]);
                        }
                } else if (NV <= 8 && P <= 16) {
                    // Reduce-scatter over the 32 / P groups of a warp: at the level with lane distance o a lane keeps
                    // the half of its values selected by lane bit o and adds its partner's copy of that half, so the
                    // values per lane halve at each level (plain adds once a single value is left).  Lane l then holds
                    // values base(l) .. base(l) + cnt - 1 of column vector l mod P, summed over the warp's groups.
                    // The CW warp sums of each (vector, value) are added by one of P NV threads.
                    double vals[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) vals[v] = T::to_d(acc[v / (VE * BT)][(v / BT) % VE][v % BT]);
                    int base = 0, cnt = NV;
                    bool writer = true;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const int o = 16 >> k;
                        if (o < P) break;
                        const bool upper = (lane & o) != 0;
                        if ((NV >> k) >= 2) {
                            const int half = (NV >> k) / 2;
#pragma unroll
                            for (int j = 0; j < NV / 2; ++j) {
                                if (j < half) {
                                    const double send = upper ? vals[j] : vals[j + half];
                                    const double keep = upper ? vals[j + half] : vals[j];
                                    vals[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                                }
                            }
                            if (upper) base += half;
                            cnt = half;
                        } else {
                            vals[0] += __shfl_xor_sync(0xffffffffu, vals[0], o);
                            if (upper) writer = false;             // the partner holds the same sum
                        }
                    }
                    const int vv = lane % P;
                    if (writer) {
#pragma unroll
                        for (int j = 0; j < NV; ++j)
                            if (j < cnt) red[(warp * P + vv) * NV + base + j] = vals[j];
                    }
                    if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                    if (t < P * NV) {
                        const int vt = t % P, v = t / P;
                        const int sv = v / (VE * BT), e = (v / BT) % VE, bb = v % BT;
                        const int c = (vt + sv * P) * VE + e;
                        if (v < nv && c < p && bb < a.B) {
                            double sum = 0.0;
#pragma unroll
                            for (int w = 0; w < CW; ++w) sum += red[(w * P + vt) * NV + v];
                            a.partial[(int64_t)bb * a.n_partial + part_off + c] = sum;
                        }
                    }
                    if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                } else if (P <= 32) {
                    // the 32 / P groups of a warp by a shuffle tree, then the CW warp sums of each (column, value) by
                    // one of RV P threads
#pragma unroll
                    for (int r0 = 0; r0 < NV; r0 += RV) {
                        if (r0 >= nv) break;
#pragma unroll
                        for (int m = 0; m < RV; ++m) {
                            const int v = r0 + m;
                            if (v < NV) {
                                double x = T::to_d(acc[v / (VE * BT)][(v / BT) % VE][v % BT]);
                                for (int o = 16; o >= P; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                                if (lane < P) red[(warp * 32 + lane) * RV + m] = x;
                            }
                        }
                        if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                        if (t < RV * P) {
                            const int m = t / P, vv = t % P, v = r0 + m;
                            const int sv = v / (VE * BT), e = (v / BT) % VE, bb = v % BT;
                            const int c = (vv + sv * P) * VE + e;
                            if (v < nv && c < p && bb < a.B) {
                                double sum = 0.0;
#pragma unroll
                                for (int w = 0; w < CW; ++w) sum += red[(w * 32 + vv) * RV + m];
                                a.partial[(int64_t)bb * a.n_partial + part_off + c] = sum;
                            }
                        }
                        if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                    }
                } else {
                    // 2 to 8 groups of whole warps: group 0 adds the others' values
#pragma unroll
                    for (int r0 = 0; r0 < NV; r0 += RV) {
                        if (r0 >= nv) break;
#pragma unroll
                        for (int m = 0; m < RV; ++m) {
                            const int v = r0 + m;
                            if (v < NV) red[t * RV + m] = T::to_d(acc[v / (VE * BT)][(v / BT) % VE][v % BT]);
                        }
                        if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                        if (grp == 0) {
#pragma unroll
                            for (int m = 0; m < RV; ++m) {
                                const int v = r0 + m;
                                const int sv = v / (VE * BT), e = (v / BT) % VE, bb = v % BT;
                                const int c = (vec + sv * P) * VE + e;
                                if (v < nv && c < p && bb < a.B) {
                                    double sum = 0.0;
                                    for (int gg = 0; gg < G; ++gg) sum += red[(gg * P + vec) * RV + m];
                                    a.partial[(int64_t)bb * a.n_partial + part_off + c] = sum;
                                }
                            }
                        }
                        if (!consumers_meet(&empty[kStages], mph, a.err, a.wait_ns)) return;
                    }
                }
                cur = -1;
            }
        }
    }
}

// Static tail of the interaction (flag SEAS_FLAG_STATIC_TAIL, not in the paper): for receiver e on fault a and each
// source fault b whose window ends at lag T_last(a, b) < step, f_int[e] += sum_{j in b} smat[e][j] delta_j^{step -
// T_last - 1}: the dropped lags T > T_last carry A^T ~ dt A^static, and dt times their slip rates is that slip.  With
// cluster-level windows the same per block covering e, with the block's T_last.  One warp per receiver element,
// lanes over the source columns, a fixed shuffle tree: deterministic.
__global__ void __launch_bounds__(kThreads) k_static_tail(StepArgs a_) {
    StepArgs a = a_;
    apply_dyn(a);
    const int64_t e = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= a.N) return;
    int fa = 0;
    while (fa + 1 < a.F && a.faults[fa + 1].off <= e) ++fa;
    const double *row = a.smat + e * (int64_t)a.N;
    const int64_t BN = (int64_t)a.B * a.N;
    double sum[kMaxBatch];
#pragma unroll
    for (int bb = 0; bb < kMaxBatch; ++bb) sum[bb] = 0.0;
    // source columns j0 .. j1 - 1 whose window ends at lag back - 1
    auto add = [&](int j0, int j1, int64_t back) {
        if (a.lag_max < back) return;                   // no member's window has passed yet
        const double *sl = a.sring + ((a.step - back) % a.sring_depth) * BN;
        for (int j = j0 + lane; j < j1; j += 32) {
            const double m = row[j];
#pragma unroll
            for (int bb = 0; bb < kMaxBatch; ++bb)
                if (bb < a.B) sum[bb] = fma(m, sl[(int64_t)j * a.B + bb], sum[bb]);
        }
    };
    if (a.block_last) {
        // cluster-level windows: every block covering the receiver, with its own window end
        for (int c = a.cover_ptr[e]; c < a.cover_ptr[e + 1]; ++c) {
            const int blk = a.cover_blk[c];
            const BlockDev &bd = a.blocks[blk];
            add(bd.c0, bd.c0 + bd.q, (int64_t)a.block_last[blk] + 1);
        }
    } else {
        for (int fb = 0; fb < a.F; ++fb)
            if (fb != fa)
                add(a.faults[fb].off, a.faults[fb].off + a.faults[fb].nf, (int64_t)a.pair_last[fa * a.F + fb] + 1);
    }
#pragma unroll
    for (int bb = 0; bb < kMaxBatch; ++bb) {
        if (bb < a.B) {
            double v = sum[bb];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) a.fint[(int64_t)bb * a.N + e] += v;
        }
    }
}

// f_int[b][e] = sum over the blocks that element e receives from, and over their causal tasks, of the tasks'
// partial sums; one warp per element, lane c takes covering blocks c, c + 32, ... (its tasks in lag order), then
// a fixed tree: the summation order never depends on timing.  Also resets the task counter for the next step.
__global__ void __launch_bounds__(kThreads) k_reduce(StepArgs a_) {
    StepArgs a = a_;
    apply_dyn(a);
    const int64_t e = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.counter[0] = 0;                                   // pass-2 task counter
        a.counter[2] = 0;                                   // pass-1 task counter
    }
    if (e >= a.N) return;
    double sum[kMaxBatch];
#pragma unroll
    for (int bb = 0; bb < kMaxBatch; ++bb) sum[bb] = 0.0;
    const int c1 = a.cover_ptr[e + 1];
    for (int c = a.cover_ptr[e] + lane; c < c1; c += 32) {
        const int blk = a.cover_blk[c];
        const BlockDev bd = a.blocks[blk];
        const int t0 = a.blk_task_ptr[blk], t1 = a.blk_task_ptr[blk + 1];
        int lo = t0, hi = t1;                               // causal tasks: T_start <= step
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.blk_task_T[mid] <= a.lag_max) lo = mid + 1; else hi = mid;
        }
        const int64_t base = a.blk_part[blk] + (e - bd.r0);
        for (int k = 0; k < lo - t0; ++k) {
            const int64_t o = base + (int64_t)k * bd.p;
#pragma unroll
            for (int bb = 0; bb < kMaxBatch; ++bb)
                if (bb < a.B) sum[bb] += a.partial[(int64_t)bb * a.n_partial + o];
        }
    }
#pragma unroll
    for (int bb = 0; bb < kMaxBatch; ++bb) {
        if (bb < a.B) {
            double v = sum[bb];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) a.fint[(int64_t)bb * a.N + e] = v;
        }
    }
}

// Admission of member `mb` of a batch (continuous batching): its whole history -- every slot of the slip-rate ring
// (and of its reduced-precision mirror and the slip ring of the static tail), its slip, and its spectral rings --
// is set to zero, so that the member starts as a scenario with no slip before the next push.
__global__ void __launch_bounds__(kThreads) k_reset_member(StepArgs a, int mb) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    const int64_t BN = (int64_t)a.B * a.N;
    for (int64_t e = tid; e < (int64_t)a.ring * a.N; e += nt) {
        const int64_t slot = e / a.N, i = e - slot * a.N, o = slot * a.ring_stride + i * a.B + mb;
        a.vring[o] = 0.0;
        if (a.prec == kPrecDF64) {
            reinterpret_cast<float2 *>(a.xring)[o] = make_float2(0.f, 0.f);
        } else if (a.xsplit) {
            __nv_bfloat16 *xr = reinterpret_cast<__nv_bfloat16 *>(a.xring) + (slot * a.ring_stride + i * 8) * 2;
            xr[mb] = __float2bfloat16_rn(0.f);
            xr[8 + mb] = __float2bfloat16_rn(0.f);
        } else if (a.prec != kPrecFP64) {
            reinterpret_cast<float *>(a.xring)[o] = 0.f;
        }
    }
    if (a.tail)
        for (int64_t e = tid; e < (int64_t)a.sring_depth * a.N; e += nt) {
            const int64_t slot = e / a.N, i = e - slot * a.N;
            a.sring[slot * BN + i * a.B + mb] = 0.0;
        }
    for (int64_t i = tid; i < a.N; i += nt) {
        a.slip[(int64_t)mb * a.N + i] = 0.0;
        a.slip_prev[(int64_t)mb * a.N + i] = 0.0;
    }
    for (int f = 0; f < a.F; ++f) {
        const FaultDev fd = a.faults[f];
        const int64_t len = (int64_t)(fd.nf + 1) * fd.ring;
        double2 *d = a.dring + fd.dring_off + (int64_t)mb * len;
        for (int64_t e = tid; e < len; e += nt) d[e] = make_double2(0.0, 0.0);
    }
}

// Watchdog check: one thread waits, with the scenario's bound, on an mbarrier that no thread arrives on.  The wait
// runs out and sets the scenario's error word exactly as a stalled interaction pipeline would, without any copy in
// flight or any other thread involved, so the timeout path can be exercised on a live context.
__global__ void k_wait_probe(StepArgs a) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0, a.err, a.wait_ns);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
}

template <int PREC, int BT, int PASS, int CWv>
cudaError_t launch_interaction_cw(const StepArgs &a, cudaStream_t s) {
    // a captured step does not know its task counts at launch: every SM, CTAs without a task return
    const int n = a.dyn ? a.n_sms : PASS == 1 ? a.n_ztasks_active : a.n_tasks_active;
    if (n <= 0) return cudaSuccess;
    const size_t smem = InterLayout<PREC, BT, PASS, CWv>::total;
    cudaError_t e = cudaFuncSetAttribute(k_interaction<PREC, BT, PASS, CWv>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n < a.n_sms ? n : a.n_sms;
    k_interaction<PREC, BT, PASS, CWv><<<grid, InterShape<PREC, BT, PASS, CWv>::NT, smem, s>>>(a);
    return cudaGetLastError();
}

// The pass with the scenario's consumer warp count (a.cw[pass - 1]; 0 or a count not compiled: the default).
template <int PREC, int BT, int PASS>
cudaError_t launch_interaction_pass(const StepArgs &a, cudaStream_t s) {
    using D = InterDefault<PREC, BT, PASS>;
    constexpr int OTHER = D::CW == 8 ? 16 : 8;
    const int want = a.cw[PASS - 1];
    if constexpr (D::ALT) {
        if (want == OTHER) return launch_interaction_cw<PREC, BT, PASS, OTHER>(a, s);
    }
    return launch_interaction_cw<PREC, BT, PASS, D::CW>(a, s);
}

template <int PREC, int BT, int PASS>
int interaction_options_pass(int *cw) {
    using D = InterDefault<PREC, BT, PASS>;
    cw[0] = D::CW;
    if (!D::ALT) return 1;
    cw[1] = D::CW == 8 ? 16 : 8;
    return 2;
}

// pass 1: z = V^T x of the far slices (source side); pass 2: the receivers' sums.  Pass 2 reads what pass 1 wrote,
// so the launcher issues them in this order on one stream.
template <int PREC, int BT>
cudaError_t launch_interaction_bt(const StepArgs &a, int pass, cudaStream_t s) {
    return pass == 1 ? launch_interaction_pass<PREC, BT, 1>(a, s) : launch_interaction_pass<PREC, BT, 2>(a, s);
}

template <int PREC, int BT>
int interaction_options_bt(int pass, int *cw) {
    return pass == 1 ? interaction_options_pass<PREC, BT, 1>(cw) : interaction_options_pass<PREC, BT, 2>(cw);
}

template <int PREC>
int interaction_options_prec(int batch, int pass, int *cw) {
    if (batch > 4) return interaction_options_bt<PREC, 8>(pass, cw);
    if (batch > 2) return interaction_options_bt<PREC, 4>(pass, cw);
    if (batch > 1) return interaction_options_bt<PREC, 2>(pass, cw);
    return interaction_options_bt<PREC, 1>(pass, cw);
}

template <int PREC>
cudaError_t launch_interaction_prec(const StepArgs &a, int pass, cudaStream_t s) {
    if (a.B > 4) return launch_interaction_bt<PREC, 8>(a, pass, s);
    if (a.B > 2) return launch_interaction_bt<PREC, 4>(a, pass, s);
    if (a.B > 1) return launch_interaction_bt<PREC, 2>(a, pass, s);
    return launch_interaction_bt<PREC, 1>(a, pass, s);
}

}  // namespace

cudaError_t static_scratch(double **ptr) {
    // device address of the scratch array, looked up once per device with that device current
    // (threads that race here look up and store the same address)
    static std::atomic<double *> cache[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    double *p = cache[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        e = cudaGetSymbolAddress(&q, g_static_scratch);
        if (e != cudaSuccess) return e;
        p = static_cast<double *>(q);
        cache[dev].store(p, std::memory_order_release);
    }
    *ptr = p;
    return cudaSuccess;
}

cudaError_t launch_push(const StepArgs &a, const double *V, const double *slip_in, int replace_last, int j,
                        int gamma, cudaStream_t s) {
    const int64_t BN = (int64_t)a.B * a.N;
    int grid = (int)((BN + kThreads - 1) / kThreads);
    if (grid > 152 * 8) grid = 152 * 8;
    k_push<<<grid, kThreads, 0, s>>>(a, V, slip_in, replace_last, j, gamma);
    return cudaGetLastError();
}

static cudaError_t fft_smem(const void *fn, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static size_t fft_cl_smem(const StepArgs &a) {
    return (size_t)(3 * (a.max_nf / kFftCluster) + kFftRadixMax) * sizeof(double2);
}

cudaError_t launch_fft_forward(const StepArgs &a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (a.n_small > 0) {
        const size_t smem = (size_t)(2 * a.max_nf + kFftRadixMax) * sizeof(double2);
        e = fft_smem((const void *)k_fft_forward, smem);
        if (e != cudaSuccess) return e;
        k_fft_forward<<<dim3(a.n_self, a.B), kThreads, smem, s>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && a.n_big > 0) {
        const size_t smem = fft_cl_smem(a);
        e = fft_smem((const void *)k_fft_forward_cl, smem);
        if (e != cudaSuccess) return e;
        k_fft_forward_cl<<<dim3(a.n_big * kFftCluster, a.B), kThreads, smem, s>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_modeconv(const StepArgs &a, cudaStream_t s) {
    if (a.n_modes == 0) return cudaSuccess;
    if (a.B > 1) k_modeconv<<<a.n_modes, 32 * a.B, 0, s>>>(a);
    else k_modeconv<<<(a.n_modes + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int interaction_options(int prec, int batch, int pass, int *cw) {
    switch (prec) {
        case kPrecDF64: return interaction_options_prec<kPrecDF64>(batch, pass, cw);
        case kPrecBF16: return interaction_options_prec<kPrecBF16>(batch, pass, cw);
        case kPrecFP16: return interaction_options_prec<kPrecFP16>(batch, pass, cw);
        default: return interaction_options_prec<kPrecFP64>(batch, pass, cw);
    }
}

cudaError_t launch_interaction(const StepArgs &a, int pass, cudaStream_t s) {
    if (!a.dyn && (pass == 1 ? a.n_ztasks_active : a.n_tasks_active) <= 0) return cudaSuccess;
    switch (a.prec) {
        case kPrecDF64: return launch_interaction_prec<kPrecDF64>(a, pass, s);
        case kPrecBF16: return launch_interaction_prec<kPrecBF16>(a, pass, s);
        case kPrecFP16: return launch_interaction_prec<kPrecFP16>(a, pass, s);
        default: return launch_interaction_prec<kPrecFP64>(a, pass, s);
    }
}

cudaError_t launch_reset_member(const StepArgs &a, int member, cudaStream_t s) {
    k_reset_member<<<152 * 4, kThreads, 0, s>>>(a, member);
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(const StepArgs &a, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const StepArgs &a, cudaStream_t s) {
    const int grid = (a.N + kThreads / 32 - 1) / (kThreads / 32);
    k_reduce<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_static_tail(const StepArgs &a, cudaStream_t s) {
    if (!a.tail) return cudaSuccess;
    const int grid = (a.N + kThreads / 32 - 1) / (kThreads / 32);
    k_static_tail<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ifft_assemble(const StepArgs &a, double *tau, double *parts, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (a.n_small > 0) {
        const size_t smem = (size_t)(2 * a.max_nf + kFftRadixMax) * sizeof(double2);
        e = fft_smem((const void *)k_ifft_assemble, smem);
        if (e != cudaSuccess) return e;
        k_ifft_assemble<<<dim3(a.n_self, a.B), kThreads, smem, s>>>(a, tau, parts);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && a.n_big > 0) {
        const size_t smem = fft_cl_smem(a);
        e = fft_smem((const void *)k_ifft_assemble_cl, smem);
        if (e != cudaSuccess) return e;
        k_ifft_assemble_cl<<<dim3(a.n_big * kFftCluster, a.B), kThreads, smem, s>>>(a, tau, parts);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace seas

// Operator-build kernels: space-time interaction kernel slices (Sec. 2.3.2), their low-rank compression, and the
// pre-integrated spectral self-effect weights (Sec. 2.3.1).  Run once per seas_build_hmatrix call.
#include "seas_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

namespace seas {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ------------------------------------------------------------------------------------------------------------
// Interaction kernel entry.
//
// Eq. (primitives) with S(t) = sqrt((c_s t)^2 - r^2) = r sqrt((c_s t / r)^2 - 1) for c_s t > r (0 otherwise):
//   I_31 = -(1/pi) r2 S / r^2
//   I_32 = H(r1) H(c_s t - |r2|) + (1/pi) sgn(r1) [ |r1| S / r^2 - atan2(S, |r1|) ]
// (arccos(|r1| / sqrt(c_s^2 t^2 - r2^2)) = atan2(S, |r1|) because c_s^2 t^2 - r2^2 = S^2 + r1^2).  The lag-T
// kernel of Eq. (kernel_interactions) is the time difference t1 = (T+1) dt minus t0 = T dt of the space difference
// r1 + ds/2 minus r1 - ds/2.  The time differences are taken in closed form,
//   S1 - S0 = c_s^2 (t1^2 - t0^2) / (S1 + S0),   atan2(S1, a) - atan2(S0, a) = atan2(a (S1 - S0), a^2 + S1 S0),
// so that late lags (primitives growing like c_s t / r, differences like dt ds / r^2) keep their digits.
// ------------------------------------------------------------------------------------------------------------

struct EndTerm {          // one end (r1 +- ds/2) of the source element: its contribution to K_31 and K_32
    double k31, k32;
};

__device__ __forceinline__ EndTerm end_term(double r1, double r2, double ct0, double ct1) {
    EndTerm e{0.0, 0.0};
    const double r = hypot(r1, r2);
    const double ar1 = fabs(r1);
    const double ar2 = fabs(r2);
    // plane-wave part H(r1) H(c_s t - |r2|), time difference t1 - t0
    if (r1 > 0.0) e.k32 += (ct1 > ar2 ? 1.0 : 0.0) - (ct0 > ar2 ? 1.0 : 0.0);
    if (!(ct1 > r) || !(r > 0.0)) return e;
    const double S1 = sqrt((ct1 - r) * (ct1 + r));
    const bool on0 = ct0 > r;
    const double S0 = on0 ? sqrt((ct0 - r) * (ct0 + r)) : 0.0;
    const double dS = on0 ? (ct1 - ct0) * (ct1 + ct0) / (S1 + S0) : S1;
    const double ir2 = 1.0 / (r * r);
    e.k31 = -(1.0 / kPi) * r2 * dS * ir2;
    if (r1 != 0.0) {
        const double dA = atan2(ar1 * dS, ar1 * ar1 + S1 * S0);
        const double br = ar1 * dS * ir2 - dA;
        e.k32 += (r1 > 0.0 ? br : -br) / kPi;
    }
    return e;
}

// Projected, scaled entry -mu/(2 c_s) (n'_1 K_31 + n'_2 K_32) for receiver i and source j at lag T.
__device__ __forceinline__ double interaction_entry(const GeomDev &g, int i, int j, int T) {
    const double2 xi = g.x[i], xj = g.x[j], e1 = g.e1[j], n2 = g.nrm[j], ni = g.nrm[i];
    const double dx = __dadd_rn(xi.x, -xj.x), dy = __dadd_rn(xi.y, -xj.y);
    const double r1 = __dadd_rn(__dmul_rn(dx, e1.x), __dmul_rn(dy, e1.y));
    const double r2 = __dadd_rn(__dmul_rn(dx, n2.x), __dmul_rn(dy, n2.y));
    const double n1p = ni.x * e1.x + ni.y * e1.y;
    const double n2p = ni.x * n2.x + ni.y * n2.y;
    const double h = 0.5 * g.ds[j];
    const double ct0 = __dmul_rn(g.cs, __dmul_rn((double)T, g.dt));
    const double ct1 = __dmul_rn(g.cs, __dmul_rn((double)(T + 1), g.dt));
    const EndTerm a = end_term(r1 + h, r2, ct0, ct1);
    const EndTerm b = end_term(r1 - h, r2, ct0, ct1);
    return g.scale * (n1p * (a.k31 - b.k31) + n2p * (a.k32 - b.k32));
}

__global__ void k_gen_slices(GeomDev g, const BlockDev *__restrict__ blocks, const SliceGen *__restrict__ slices,
                             int n_slices, const int64_t *__restrict__ prefix, int64_t n_entries,
                             double *__restrict__ scratch) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_entries;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_slices - 1;
        while (lo < hi) {           // last slice whose first entry is <= e
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const SliceGen s = slices[lo];
        const BlockDev b = blocks[s.block];
        const int64_t local = e - prefix[lo];
        const int j = (int)(local / b.p);
        const int i = (int)(local - (int64_t)j * b.p);
        scratch[s.scratch + local] = interaction_entry(g, b.r0 + i, b.c0 + j, s.T);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Block reductions
// ------------------------------------------------------------------------------------------------------------

struct MaxLoc {
    double v;
    int64_t idx;
};

__device__ __forceinline__ MaxLoc better(MaxLoc a, MaxLoc b) {
    if (b.v > a.v || (b.v == a.v && b.idx < a.idx)) return b;
    return a;
}

// Sum and arg-max of |.| over the CTA; every thread gets the result.
__device__ void block_reduce(double &sum, MaxLoc &m, double *sh_sum, double *sh_v, int64_t *sh_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        MaxLoc other{__shfl_xor_sync(0xffffffffu, m.v, o), __shfl_xor_sync(0xffffffffu, m.idx, o)};
        m = better(m, other);
    }
    __syncthreads();
    if (lane == 0) {
        sh_sum[warp] = sum;
        sh_v[warp] = m.v;
        sh_i[warp] = m.idx;
    }
    __syncthreads();
    sum = 0.0;
    m = MaxLoc{-1.0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sum += sh_sum[w];
        m = better(m, MaxLoc{sh_v[w], sh_i[w]});
    }
}

// ------------------------------------------------------------------------------------------------------------
// Compression of one (block, lag) slice per CTA.
//
// Admissible blocks: adaptive cross approximation with complete pivoting (the slice is already materialised, so
// the pivot search over the whole residual costs one sweep per rank step and is robust to slices that the
// wavefront cuts into a zero and a nonzero part).  Rank-1 terms u_k v_k^T with u_k = R[:, j*], v_k = R[i*, :] /
// R[i*, j*] are subtracted until ||R||_F <= tol ||S||_F (relative Frobenius tolerance per slice).  If that needs
// k (p + q) >= p q numbers, the slice is stored dense.  Near blocks: dense.  Exactly-zero slices: nothing.
// Layout: slice S (p x q) is stored as A^T, S[i][j] = A[j * p + i].
// ------------------------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) k_compress(const BlockDev *__restrict__ blocks,
                                                       const SliceGen *__restrict__ slices,
                                                       const double *__restrict__ scratch, double *__restrict__ resid,
                                                       double *__restrict__ factors, SliceOut *__restrict__ out,
                                                       double tol) {
    __shared__ double sh_sum[32], sh_v[32];
    __shared__ int64_t sh_i[32];
    __shared__ double us[kMaxBlockSide], vs[kMaxBlockSide];
    const SliceGen s = slices[blockIdx.x];
    const BlockDev b = blocks[s.block];
    const int p = b.p, q = b.q;
    const int64_t pq = (int64_t)p * q;
    const double *S = scratch + s.scratch;
    double *R = resid + s.scratch;

    double sum = 0.0;
    MaxLoc m{-1.0, 0};
    for (int64_t e = threadIdx.x; e < pq; e += blockDim.x) {
        const double v = S[e];
        if (s.far) R[e] = v;
        sum += v * v;
        m = better(m, MaxLoc{fabs(v), e});
    }
    block_reduce(sum, m, sh_sum, sh_v, sh_i);
    const double norm2 = sum;
    if (norm2 == 0.0 || !s.far) {
        if (threadIdx.x == 0) out[blockIdx.x] = SliceOut{norm2 == 0.0 ? 0 : -1, 0, sqrt(norm2), 0.0};
        return;
    }
    const int kmax = (int)((pq - 1) / (p + q));
    double *Ut = factors + s.scratch;                  // rows of p
    double *Vt = factors + s.scratch + (int64_t)kmax * p;  // rows of q
    const double tol2 = tol * tol * norm2;
    double r2 = norm2;
    int k = 0;
    while (r2 > tol2 && k < kmax) {
        const int jm = (int)(m.idx / p), im = (int)(m.idx - (int64_t)jm * p);
        const double piv = R[m.idx];
        if (piv == 0.0) break;
        __syncthreads();
        for (int i = threadIdx.x; i < p; i += blockDim.x) {
            const double u = R[(int64_t)jm * p + i];
            us[i] = u;
            Ut[(int64_t)k * p + i] = u;
        }
        for (int j = threadIdx.x; j < q; j += blockDim.x) {
            const double v = R[(int64_t)j * p + im] / piv;
            vs[j] = v;
            Vt[(int64_t)k * q + j] = v;
        }
        __syncthreads();
        sum = 0.0;
        m = MaxLoc{-1.0, 0};
        for (int64_t e = threadIdx.x; e < pq; e += blockDim.x) {
            const int j = (int)(e / p), i = (int)(e - (int64_t)j * p);
            const double v = R[e] - us[i] * vs[j];
            R[e] = v;
            sum += v * v;
            m = better(m, MaxLoc{fabs(v), e});
        }
        block_reduce(sum, m, sh_sum, sh_v, sh_i);
        r2 = sum;
        ++k;
    }
    if (threadIdx.x == 0) {
        const bool ok = r2 <= tol2 && k > 0;
        out[blockIdx.x] = SliceOut{ok ? k : -1, 0, sqrt(norm2), ok ? sqrt(r2) : 0.0};
    }
}

// Storage conversion of one operator value.
template <int PREC> struct Store;
template <> struct Store<kPrecFP64> {
    using T = double;
    __device__ static T cv(double v) { return v; }
};
template <> struct Store<kPrecDF64> {
    using T = float2;                                  // (hi, lo): hi = fl32(v), lo = fl32(v - hi)
    __device__ static T cv(double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    }
};
template <> struct Store<kPrecBF16> {
    using T = __nv_bfloat16;
    __device__ static T cv(double v) { return __float2bfloat16_rn((float)v); }
};
template <> struct Store<kPrecFP16> {
    using T = __half;
    __device__ static T cv(double v) { return __float2half_rn((float)v); }
};

// Largest |v| over n values (CTA reduction).
__device__ double block_absmax(const double *v, int64_t n, int64_t stride_rows, int row_len, double *sh) {
    double m = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int64_t r = e / row_len, c = e - r * row_len;
        m = fmax(m, fabs(v[r * stride_rows + c]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    return m;
}

// Scale putting the largest value near 2^14, inside float16's range with room to spare.
__device__ __forceinline__ double fp16_scale(double amax) { return amax > 0.0 ? amax / 16384.0 : 1.0; }

// Copies each stored slice into the operator arenas in the storage precision, rows padded to 16 bytes
// (p2 = pad_row(p), q2 = pad_row(q) elements):
//   dense   -> receiver-side arena at dst: A^T, q rows of p2;
//   lowrank -> receiver-side arena at dst: U^T, k rows of p2; source-side arena at vdst: V^T, k rows of q2.
// FP16 stores values divided by a per-slice scale (dense: one; low rank: one for U and one for V); the scale of
// the product (1 for the other precisions) goes to scales[slice].
template <int PREC>
__global__ void k_pack(const BlockDev *__restrict__ blocks, const SliceGen *__restrict__ slices,
                       const SliceOut *__restrict__ out, const double *__restrict__ scratch,
                       const double *__restrict__ factors, const int64_t *__restrict__ dst_off,
                       typename Store<PREC>::T *__restrict__ dst, const int64_t *__restrict__ vdst_off,
                       typename Store<PREC>::T *__restrict__ vdst, float *__restrict__ scales) {
    using T = typename Store<PREC>::T;
    __shared__ double sh[32];
    const SliceGen s = slices[blockIdx.x];
    const SliceOut o = out[blockIdx.x];
    if (o.k == 0) return;
    const BlockDev b = blocks[s.block];
    const int p = b.p, q = b.q, p2 = pad_row(p, PREC), q2 = pad_row(q, PREC);
    const int64_t pq = (int64_t)p * q;
    T *d = dst + dst_off[blockIdx.x];
    if (o.k < 0) {
        const double *S = scratch + s.scratch;
        double inv = 1.0;
        if (PREC == kPrecFP16) {
            const double sc = fp16_scale(block_absmax(S, pq, p, p, sh));
            inv = 1.0 / sc;
            if (threadIdx.x == 0) scales[blockIdx.x] = (float)sc;
        } else if (threadIdx.x == 0) {
            scales[blockIdx.x] = 1.0f;
        }
        const int64_t n = (int64_t)q * p2;
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
            const int j = (int)(e / p2), i = (int)(e - (int64_t)j * p2);
            d[e] = Store<PREC>::cv(i < p ? S[(int64_t)j * p + i] * inv : 0.0);
        }
        return;
    }
    const int kmax = (int)((pq - 1) / (p + q));
    const double *Ut = factors + s.scratch;
    const double *Vt = factors + s.scratch + (int64_t)kmax * p;
    double inv_u = 1.0, inv_v = 1.0;
    if (PREC == kPrecFP16) {
        const double su = fp16_scale(block_absmax(Ut, (int64_t)o.k * p, p, p, sh));
        const double sv = fp16_scale(block_absmax(Vt, (int64_t)o.k * q, q, q, sh));
        inv_u = 1.0 / su;
        inv_v = 1.0 / sv;
        if (threadIdx.x == 0) scales[blockIdx.x] = (float)(su * sv);
    } else if (threadIdx.x == 0) {
        scales[blockIdx.x] = 1.0f;
    }
    T *vd = vdst + vdst_off[blockIdx.x];
    const int64_t nu = (int64_t)o.k * p2, nv = (int64_t)o.k * q2;
    for (int64_t e = threadIdx.x; e < nu; e += blockDim.x) {
        const int l = (int)(e / p2), i = (int)(e - (int64_t)l * p2);
        d[e] = Store<PREC>::cv(i < p ? Ut[(int64_t)l * p + i] * inv_u : 0.0);
    }
    for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) {
        const int l = (int)(e / q2), j = (int)(e - (int64_t)l * q2);
        vd[e] = Store<PREC>::cv(j < q ? Vt[(int64_t)l * q + j] * inv_v : 0.0);
    }
}

// One warp per run: 16-byte copies.
__global__ void __launch_bounds__(kThreads) k_gather(const void *const *__restrict__ src, void *const *__restrict__ dst,
                                                     const int32_t *__restrict__ bytes, int n) {
    const int w = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= n) return;
    const uint4 *s = static_cast<const uint4 *>(src[w]);
    uint4 *d = static_cast<uint4 *>(dst[w]);
    const int n16 = bytes[w] >> 4;
    for (int c = lane; c < n16; c += 32) d[c] = s[c];
}

// Chunk rotation of 2-byte operator units (chunk_at): one warp per unit, one row at a time, in place (a row's
// chunks are all read before any is written).  Rows have at most 128 chunks (1024 columns).
__global__ void __launch_bounds__(kThreads) k_rotate_rows(const UnitRows *__restrict__ units, int n) {
    const int w = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= n) return;
    const UnitRows u = units[w];
    uint4 *base = static_cast<uint4 *>(u.p);
    for (int r = 0; r < u.rows; ++r) {
        uint4 *row = base + (int64_t)r * u.nch;
        uint4 v[4];
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            if (c < u.nch) v[k] = row[c];
        }
        __syncwarp();
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            if (c < u.nch) row[chunk_at(c, r, u.nch)] = v[k];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------------------------
// Spectral weights.  With m = n pi and rho = c_s t / L_f, the time integral of Eq. (non_replicant_kernel),
//   G(rho) = c_s k_n int_0^t K(n, s) ds = (2/pi) int_0^{psi_m} cos^2(psi) sin(m rho sin psi) / sin(psi) dpsi,
//   psi_m = pi/2 for rho <= 1 and arcsin(1/rho) for rho > 1,
// (K written over psi in [0, pi/2] with the indicator c_s s sin psi < L; the s-integral of cos(k_n c_s s sin psi)
// in closed form; the cut-off term carries sin(k_n L) = sin(n pi) = 0).  Then w_n^T = G(rho_{T+1}) - G(rho_T).
// Composite Gauss-Legendre in psi; the phase changes by at most ~pi per panel.
// ------------------------------------------------------------------------------------------------------------

__device__ double spectral_G(int n, double rho, const double *gl_x, const double *gl_w, int gl_n) {
    if (rho <= 0.0) return 0.0;
    const double m = kPi * n;
    const double psim = rho <= 1.0 ? 0.5 * kPi : asin(1.0 / rho);
    const double a = m * rho;
    const int panels = 4 + (int)ceil(0.5 * kPi * n * fmin(rho, 1.0));
    const double hw = 0.5 * psim / panels;
    double total = 0.0;
    for (int P = 0; P < panels; ++P) {
        const double mid = (2 * P + 1) * hw;
        double part = 0.0;
        for (int g = 0; g < gl_n; ++g) {
            const double psi = mid + hw * gl_x[g];
            double sp, cp;
            sincos(psi, &sp, &cp);
            part += gl_w[g] * cp * cp * sin(a * sp) / sp;
        }
        total += part * hw;
    }
    return (2.0 / kPi) * total;
}

__global__ void k_spectral_G(const ModeDev *__restrict__ modes, int n_modes, const int64_t *__restrict__ g_prefix,
                             int64_t n_g, const double *__restrict__ mode_L, double cs_dt,
                             const double *__restrict__ gl_x, const double *__restrict__ gl_w, int gl_n,
                             double *__restrict__ G) {
    __shared__ double sx[32], sw[32];
    for (int i = threadIdx.x; i < gl_n; i += blockDim.x) {
        sx[i] = gl_x[i];
        sw[i] = gl_w[i];
    }
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_g; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_modes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g_prefix[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int T = (int)(e - g_prefix[lo]);
        const double rho = cs_dt * (double)T / mode_L[lo];
        G[e] = spectral_G(modes[lo].n, rho, sx, sw, gl_n);
    }
}

__global__ void k_spectral_w(const ModeDev *__restrict__ modes, int n_modes, const int64_t *__restrict__ g_prefix,
                             const double *__restrict__ G, double *__restrict__ w) {
    const int md = blockIdx.x;
    if (md >= n_modes) return;
    const ModeDev mo = modes[md];
    const double *g = G + g_prefix[md];
    for (int T = threadIdx.x; T <= mo.W; T += blockDim.x) w[mo.w_off + T] = g[T + 1] - g[T];
}

int grid_for(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_gen_slices(const GeomDev &g, const BlockDev *blocks, const SliceGen *slices, int n_slices,
                              const int64_t *entry_prefix, int64_t n_entries, double *scratch, cudaStream_t s) {
    if (n_entries <= 0) return cudaSuccess;
    k_gen_slices<<<grid_for(n_entries), kThreads, 0, s>>>(g, blocks, slices, n_slices, entry_prefix, n_entries,
                                                          scratch);
    return cudaGetLastError();
}

cudaError_t launch_compress(const BlockDev *blocks, const SliceGen *slices, int n_slices, const double *scratch,
                            double *resid, double *factors, SliceOut *out, double tol, cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    k_compress<<<n_slices, kThreads, 0, s>>>(blocks, slices, scratch, resid, factors, out, tol);
    return cudaGetLastError();
}

cudaError_t launch_pack(const BlockDev *blocks, const SliceGen *slices, const SliceOut *out, int n_slices,
                        const double *scratch, const double *factors, const int64_t *dst_off, void *dst,
                        const int64_t *vdst_off, void *vdst, float *scales, int prec, cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    switch (prec) {
        case kPrecFP64:
            k_pack<kPrecFP64><<<n_slices, kThreads, 0, s>>>(blocks, slices, out, scratch, factors, dst_off,
                                                            static_cast<double *>(dst), vdst_off,
                                                            static_cast<double *>(vdst), scales);
            break;
        case kPrecDF64:
            k_pack<kPrecDF64><<<n_slices, kThreads, 0, s>>>(blocks, slices, out, scratch, factors, dst_off,
                                                            static_cast<float2 *>(dst), vdst_off,
                                                            static_cast<float2 *>(vdst), scales);
            break;
        case kPrecBF16:
            k_pack<kPrecBF16><<<n_slices, kThreads, 0, s>>>(blocks, slices, out, scratch, factors, dst_off,
                                                            static_cast<__nv_bfloat16 *>(dst), vdst_off,
                                                            static_cast<__nv_bfloat16 *>(vdst), scales);
            break;
        default:
            k_pack<kPrecFP16><<<n_slices, kThreads, 0, s>>>(blocks, slices, out, scratch, factors, dst_off,
                                                            static_cast<__half *>(dst), vdst_off,
                                                            static_cast<__half *>(vdst), scales);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const void *const *src, void *const *dst, const int32_t *bytes, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int per = kThreads / 32;
    k_gather<<<(n + per - 1) / per, kThreads, 0, s>>>(src, dst, bytes, n);
    return cudaGetLastError();
}

cudaError_t launch_rotate_rows(const UnitRows *units, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int per = kThreads / 32;
    k_rotate_rows<<<(n + per - 1) / per, kThreads, 0, s>>>(units, n);
    return cudaGetLastError();
}

cudaError_t launch_spectral_tables(const ModeDev *modes, int n_modes, const int64_t *g_prefix, int64_t n_g,
                                   const double *mode_L, double cs_dt, const double *gl_x, const double *gl_w,
                                   int gl_n, double *G, double *w, cudaStream_t s) {
    if (n_modes <= 0) return cudaSuccess;
    k_spectral_G<<<grid_for(n_g), kThreads, 0, s>>>(modes, n_modes, g_prefix, n_g, mode_L, cs_dt, gl_x, gl_w, gl_n,
                                                    G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_spectral_w<<<n_modes, kThreads, 0, s>>>(modes, n_modes, g_prefix, G, w);
    return cudaGetLastError();
}

}  // namespace seas

// Earthquake-cycle time stepping on top of the stress-transfer functional (Sec. 2.2 rate-and-state friction,
// Eq. R&S_friction, with the intermediate state law, Eq. state_evolution_law; Sec. 2.4 one-time-step integration):
// a second-order predictor-corrector with a Newton solve of the force balance per element, all in FP64 on the device.
//
// One step of gamma lattice steps (dt = gamma dt_min; gamma = 1 for fixed steps):
//   1. predictor: delta* = delta + dt V, theta* = theta + dt thetadot;
//   2. push V over the gamma lattice steps with slip growing linearly to delta* and evaluate the functional: its
//      self and interaction parts are the elastic stress at the step's end without the instantaneous part (the self
//      term of delta*, the interaction of the history, the interval's own lags 1 .. gamma - 1 carrying V); the
//      only instantaneous term is the radiation damping -(mu / 2 c_s) V (across faults the lag-0 kernel vanishes
//      once faults are farther apart than c_s dt_min, which the integrator checks);
//   3. Newton in u = ln V on  tau_known + tau^o - (mu / 2 c_s) V = sigma_n f(V, theta*), then thetadot*;
//   4. corrector: the same with V -> (V + V*)/2 and thetadot -> (thetadot + thetadot*)/2 (the push replaced),
//      Newton from V*;
//   5. the step's lattice slots are replaced by V** (slip to delta**), which later steps read as history.
// The initial rate V^0 sets the first predictor but is not slip-rate history (no slip before t = 0).
#include "seas.h"
#include "seas_internal.h"

#include <cmath>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

namespace seas {
namespace {

struct FrictionDev {
    const double *a, *b, *dc, *f0, *v0, *sigma;   // per element
    double eps;
};

__device__ __forceinline__ double state_rate(double V, double theta, double dc, double eps) {
    const double om = V * theta / dc;
    return eps == 1.0 ? 1.0 - om : (pow(om, -eps) - 1.0) * om / eps;
}

// V > 0 with tk - rad V = sigma (f0 + a ln(V / v0) + b ln(V theta / dc)), by Newton in u = ln V (the left side
// minus the right side decreases strictly in u, so the root is unique); steps clipped to +-10 in u; stops when
// |g| <= tol (|tk| + sigma).  Returns false if 100 iterations do not get there.
__device__ __forceinline__ bool newton(double tk, double theta, double a, double b, double dc, double f0, double v0,
                                       double sigma, double rad, double v_start, double tol, double &V) {
    double u = log(v_start);
    const double c = f0 - a * log(v0) + b * log(theta / dc);
    const double scale = fabs(tk) + sigma;
    for (int it = 0; it < 100; ++it) {
        const double ev = exp(u);
        const double g = tk - rad * ev - sigma * (c + (a + b) * u);
        if (fabs(g) <= tol * scale) {
            V = ev;
            return true;
        }
        const double dg = -rad * ev - sigma * (a + b);
        u += fmin(10.0, fmax(-10.0, -g / dg));
    }
    V = exp(u);
    return false;
}

// Step 1 (predictor of slip and state).
__global__ void k_predict(int64_t BN, double dt, const double *V, const double *delta, const double *theta,
                          const double *thd, double *d1, double *th1) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < BN; e += (int64_t)gridDim.x * blockDim.x) {
        d1[e] = delta[e] + dt * V[e];
        th1[e] = theta[e] + dt * thd[e];
    }
}

// Steps 3-4: Newton for V*, thetadot*, and the corrector's rate, slip and state.
__global__ void k_newton_predict(int64_t BN, int N, double dt, double rad, FrictionDev fr, const double *parts,
                                 const double *tau0, const double *V, const double *delta, const double *theta,
                                 const double *thd, const double *th1, double *V1, double *thd1, double *d2,
                                 double *th2, double *vavg, int *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < BN; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const double tk = parts[BN + e] + parts[2 * BN + e] + tau0[e];      // self + interaction + background
        double v;
        if (!newton(tk, th1[e], fr.a[i], fr.b[i], fr.dc[i], fr.f0[i], fr.v0[i], fr.sigma[i], rad, V[e], 1e-8, v))
            atomicExch(err, 1);
        V1[e] = v;
        const double td = state_rate(v, th1[e], fr.dc[i], fr.eps);
        thd1[e] = td;
        const double va = 0.5 * (V[e] + v);
        vavg[e] = va;
        d2[e] = delta[e] + dt * va;
        th2[e] = theta[e] + dt * 0.5 * (thd[e] + td);
    }
}

// Step 4-5: Newton for V**, then the new state.
__global__ void k_newton_correct(int64_t BN, int N, double rad, FrictionDev fr, const double *parts,
                                 const double *tau0, const double *V1, const double *d2, const double *th2, double *V,
                                 double *delta, double *theta, double *thd, int *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < BN; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const double tk = parts[BN + e] + parts[2 * BN + e] + tau0[e];
        double v;
        if (!newton(tk, th2[e], fr.a[i], fr.b[i], fr.dc[i], fr.f0[i], fr.v0[i], fr.sigma[i], rad, V1[e], 1e-8, v))
            atomicExch(err, 1);
        V[e] = v;
        delta[e] = d2[e];
        theta[e] = th2[e];
        thd[e] = state_rate(v, th2[e], fr.dc[i], fr.eps);
    }
}

__global__ void k_state_rate(int64_t BN, int N, FrictionDev fr, const double *V, const double *theta, double *thd) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < BN; e += (int64_t)gridDim.x * blockDim.x)
        thd[e] = state_rate(V[e], theta[e], fr.dc[(int)(e % N)], fr.eps);
}

// min over elements of xi D_c / V (the evolution time step of Sec. 2.4, step 1), one CTA.
__global__ void __launch_bounds__(kThreads) k_dt_ev(int64_t BN, int N, double xi, const double *dc, const double *V,
                                                    double *out) {
    __shared__ double sh[kThreads / 32];
    double m = INFINITY;
    for (int64_t e = threadIdx.x; e < BN; e += blockDim.x) m = fmin(m, xi * dc[(int)(e % N)] / V[e]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = fmin(m, sh[w]);
        *out = fmin(m, sh[0]);
    }
}

int grid_of(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    return (int)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

}  // namespace
}  // namespace seas

using namespace seas;

struct seas_integ;
namespace {
FrictionDev friction_of(const seas_integ &it);
}

struct seas_integ {
    seas_scn *scn = nullptr;
    ScnView v{};
    double eps = 1.0;
    // friction per element ([6][N]: a, b, D_c, f_*, V_*, sigma_n), then [B][N] state and work arrays
    double *fr = nullptr, *tau0 = nullptr, *V = nullptr, *delta = nullptr, *theta = nullptr, *thd = nullptr;
    double *d1 = nullptr, *th1 = nullptr, *V1 = nullptr, *thd1 = nullptr, *d2 = nullptr, *th2 = nullptr;
    double *vavg = nullptr, *tau = nullptr, *parts = nullptr, *dtev = nullptr;
    int *err = nullptr;
    void *block = nullptr;              // one allocation holding all of the above
    size_t bytes = 0;
    ~seas_integ() {
        if (block) scn_free(scn, block, bytes);
    }
};

namespace {
FrictionDev friction_of(const seas_integ &it) {
    const int N = it.v.N;
    return FrictionDev{it.fr, it.fr + N, it.fr + 2 * N, it.fr + 3 * N, it.fr + 4 * N, it.fr + 5 * N, it.eps};
}
}  // namespace

extern "C" seas_status seas_integrator_create(seas_scn *scn, const seas_friction *fr, int n_fr, double eps,
                                              const double *tau0, const double *V0, const double *theta0, int mem,
                                              seas_integ **out) {
    if (!scn || !fr || !tau0 || !V0 || !theta0 || !out) return SEAS_EINVAL;
    *out = nullptr;
    if (mem != SEAS_MEM_HOST && mem != SEAS_MEM_DEVICE) return SEAS_EINVAL;
    if (!(eps > 0.0 && eps <= 1.0)) return SEAS_EINVAL;
    auto it = std::make_unique<seas_integ>();
    seas_status st = scenario_view(scn, &it->v);
    if (st != SEAS_OK) return st;
    if (it->v.n != 0) return SEAS_ESTATE;
    // the Newton solves are per element only if no lag-0 slice couples elements of different faults
    if (it->v.first_lag == 0) return SEAS_EINVAL;
    const int N = it->v.N;
    if (n_fr != 1 && n_fr != N) return SEAS_EINVAL;
    for (int k = 0; k < n_fr; ++k) {
        const seas_friction &f = fr[k];
        if (!(f.a > 0 && f.b >= 0 && f.dc > 0 && f.v0 > 0 && f.sigma_n > 0 && std::isfinite(f.f0)))
            return SEAS_EINVAL;
    }
    if (cudaSetDevice(it->v.device) != cudaSuccess) return SEAS_ECUDA;
    it->scn = scn;
    it->eps = eps;
    const int64_t BN = (int64_t)it->v.B * N;
    it->bytes = (size_t)(6 * N + 16 * BN + 1) * sizeof(double) + 256;   // 13 [B][N] arrays, parts, dt_ev, err
    st = scn_alloc(scn, it->bytes, &it->block);
    if (st != SEAS_OK) return st;
    double *p = static_cast<double *>(it->block);
    it->fr = p;
    p += 6 * N;
    for (double **b : {&it->tau0, &it->V, &it->delta, &it->theta, &it->thd, &it->d1, &it->th1, &it->V1, &it->thd1,
                       &it->d2, &it->th2, &it->vavg, &it->tau}) {
        *b = p;
        p += BN;
    }
    it->parts = p;
    p += 3 * BN;
    it->dtev = p;
    p += 1;
    it->err = reinterpret_cast<int *>(p);
    std::vector<double> h((size_t)6 * N);
    for (int i = 0; i < N; ++i) {
        const seas_friction &f = fr[n_fr == 1 ? 0 : i];
        const double v[6] = {f.a, f.b, f.dc, f.f0, f.v0, f.sigma_n};
        for (int c = 0; c < 6; ++c) h[(size_t)c * N + i] = v[c];
    }
    const cudaMemcpyKind kind = mem == SEAS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpy(it->fr, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(it->tau0, tau0, BN * sizeof(double), kind) != cudaSuccess ||
        cudaMemcpy(it->V, V0, BN * sizeof(double), kind) != cudaSuccess ||
        cudaMemcpy(it->theta, theta0, BN * sizeof(double), kind) != cudaSuccess ||
        cudaMemset(it->delta, 0, BN * sizeof(double)) != cudaSuccess || cudaMemset(it->err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SEAS_ECUDA;
    }
    const FrictionDev f = friction_of(*it);
    k_state_rate<<<grid_of(BN), kThreads, 0, it->v.stream>>>(BN, N, f, it->V, it->theta, it->thd);
    if (cudaGetLastError() != cudaSuccess) return SEAS_ECUDA;
    *out = it.release();
    return SEAS_OK;
}

namespace {

seas_status step_gamma(seas_integ *it, int gamma) {
    const int N = it->v.N;
    const int64_t BN = (int64_t)it->v.B * N;
    const int G = grid_of(BN);
    const cudaStream_t sm = it->v.stream;
    const FrictionDev f = friction_of(*it);
    const double dtg = gamma * it->v.dt;
    k_predict<<<G, kThreads, 0, sm>>>(BN, dtg, it->V, it->delta, it->theta, it->thd, it->d1, it->th1);
    if (cudaGetLastError() != cudaSuccess) return SEAS_ECUDA;
    seas_status st = seas_push_slip_rate_steps(it->scn, it->V, it->d1, SEAS_MEM_DEVICE, gamma, 0);
    if (st != SEAS_OK) return st;
    st = seas_stress_step(it->scn, it->tau, nullptr, it->parts, SEAS_MEM_DEVICE);
    if (st != SEAS_OK) return st;
    k_newton_predict<<<G, kThreads, 0, sm>>>(BN, N, dtg, it->v.rad, f, it->parts, it->tau0, it->V, it->delta,
                                              it->theta, it->thd, it->th1, it->V1, it->thd1, it->d2, it->th2, it->vavg,
                                              it->err);
    if (cudaGetLastError() != cudaSuccess) return SEAS_ECUDA;
    st = seas_push_slip_rate_steps(it->scn, it->vavg, it->d2, SEAS_MEM_DEVICE, gamma, 1);
    if (st != SEAS_OK) return st;
    st = seas_stress_step(it->scn, it->tau, nullptr, it->parts, SEAS_MEM_DEVICE);
    if (st != SEAS_OK) return st;
    k_newton_correct<<<G, kThreads, 0, sm>>>(BN, N, it->v.rad, f, it->parts, it->tau0, it->V1, it->d2, it->th2, it->V,
                                              it->delta, it->theta, it->thd, it->err);
    if (cudaGetLastError() != cudaSuccess) return SEAS_ECUDA;
    return seas_push_slip_rate_steps(it->scn, it->V, it->delta, SEAS_MEM_DEVICE, gamma, 1);
}

}  // namespace

extern "C" seas_status seas_integrator_step(seas_integ *it, int steps) {
    if (!it || steps < 0) return SEAS_EINVAL;
    if (cudaSetDevice(it->v.device) != cudaSuccess) return SEAS_ECUDA;
    for (int s = 0; s < steps; ++s) {
        const seas_status st = step_gamma(it, 1);
        if (st != SEAS_OK) return st;
    }
    return SEAS_OK;
}

extern "C" seas_status seas_integrator_step_gamma(seas_integ *it, int gamma) {
    if (!it || gamma < 1) return SEAS_EINVAL;
    if (cudaSetDevice(it->v.device) != cudaSuccess) return SEAS_ECUDA;
    return step_gamma(it, gamma);
}

extern "C" seas_status seas_integrator_step_adaptive(seas_integ *it, double xi, int gamma_max, int steps,
                                                     int64_t *lattice_steps) {
    if (!it || !(xi > 0.0) || gamma_max < 1 || steps < 0) return SEAS_EINVAL;
    if (cudaSetDevice(it->v.device) != cudaSuccess) return SEAS_ECUDA;
    const int64_t BN = (int64_t)it->v.B * it->v.N;
    int64_t done = 0;
    for (int s = 0; s < steps; ++s) {
        k_dt_ev<<<1, kThreads, 0, it->v.stream>>>(BN, it->v.N, xi, it->fr + 2 * it->v.N, it->V, it->dtev);
        double dt_ev = 0.0;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&dt_ev, it->dtev, sizeof(double), cudaMemcpyDeviceToHost, it->v.stream) != cudaSuccess ||
            cudaStreamSynchronize(it->v.stream) != cudaSuccess)
            return SEAS_ECUDA;
        const double g = std::ceil(dt_ev / it->v.dt);
        const int gamma = g >= gamma_max ? gamma_max : (g < 1.0 ? 1 : (int)g);
        const seas_status st = step_gamma(it, gamma);
        if (st != SEAS_OK) return st;
        done += gamma;
    }
    if (lattice_steps) *lattice_steps = done;
    return SEAS_OK;
}

extern "C" seas_status seas_integrator_state(seas_integ *it, double *V, double *theta, double *slip, int mem) {
    if (!it) return SEAS_EINVAL;
    if (mem != SEAS_MEM_HOST && mem != SEAS_MEM_DEVICE) return SEAS_EINVAL;
    if (cudaSetDevice(it->v.device) != cudaSuccess) return SEAS_ECUDA;
    const int64_t BN = (int64_t)it->v.B * it->v.N;
    if (cudaStreamSynchronize(it->v.stream) != cudaSuccess) return SEAS_ECUDA;
    int err = 0;
    if (cudaMemcpy(&err, it->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SEAS_ECUDA;
    const cudaMemcpyKind kind = mem == SEAS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (V && cudaMemcpy(V, it->V, BN * sizeof(double), kind) != cudaSuccess) return SEAS_ECUDA;
    if (theta && cudaMemcpy(theta, it->theta, BN * sizeof(double), kind) != cudaSuccess) return SEAS_ECUDA;
    if (slip && cudaMemcpy(slip, it->delta, BN * sizeof(double), kind) != cudaSuccess) return SEAS_ECUDA;
    return err ? SEAS_ESTATE : SEAS_OK;
}

extern "C" seas_status seas_destroy_integrator(seas_integ *it) {
    if (!it) return SEAS_OK;
    cudaSetDevice(it->v.device);
    cudaStreamSynchronize(it->v.stream);
    delete it;
    return SEAS_OK;
}

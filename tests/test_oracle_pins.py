"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU, no CUDA library).

Each test checks the oracle against something other than itself: a textbook identity, a closed form, a printed
number, a physical limit, an independent discretisation of the same operator, or the same computation in extended
precision.  A dropped term, a wrong sign, index or normalisation, or a transposed operand fails at least one.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import seas_oracle as O
from paper_2603_00383_gb300 import synth

CS = 3464.0
MU = 32e9


# ---------------------------------------------------------------- spectral kernel K(n, t) and its weights ------

@pytest.mark.parametrize("n", [1, 3, 17])
def test_K_before_cs_t_eq_L_is_J1_over_a(n):
    """P1: for c_s t < L, Eq. (non_replicant_kernel_a) equals J_1(a)/a, a = n pi c_s t / L (textbook integral)."""
    L = 1000.0
    t = np.linspace(0.02, 0.98, 25) * L / CS
    a = n * np.pi * CS * t / L
    np.testing.assert_allclose(O.kernel_K(n, t, L, CS), special.j1(a) / a, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n", [1, 4, 9])
def test_K_branches_meet_at_cs_t_eq_L(n):
    """P2: the two branches of Eq. (non_replicant_kernel) join continuously at c_s t = L."""
    L = 700.0
    lo = O.kernel_K(n, L / CS * (1 - 1e-9), L, CS)
    hi = O.kernel_K(n, L / CS * (1 + 1e-9), L, CS)
    assert abs(lo - hi) < 1e-6 * max(1.0, abs(lo))


@pytest.mark.parametrize("n", [1, 2, 5, 10, 40])
def test_K_decays_monotonically_after_L_while_J1_oscillates(n):
    """P4 (App. D): |K(n,t)| decreases monotonically for c_s t > L; the replicating J_1(a)/a keeps oscillating."""
    L = 1000.0
    t = np.linspace(1.0001, 30.0, 1500) * L / CS
    K = O.kernel_K(n, t, L, CS)
    assert np.all(np.diff(np.abs(K)) < 0)
    assert np.all(np.sign(K) == np.sign(K[0]))
    a = n * np.pi * CS * t / L
    assert np.mean(np.diff(np.abs(special.j1(a) / a)) < 0) < 0.6


@pytest.mark.parametrize("n", [1, 6, 25])
def test_weights_equal_time_integral_of_J1_over_a(n):
    """Weights for intervals with c_s t_1 < L against c_s k_n int J_1(a(t))/a(t) dt (independent closed form of K)."""
    L, dt = 1000.0, 0.5 * 1000.0 / 64 / CS
    kn = np.pi * n / L
    T = np.array([0, 1, 7, 30, 100])
    got = O.spectral_weights(n, T, dt, L, CS)
    for Ti, g in zip(T, got):
        f = lambda t: special.j1(kn * CS * t) / (kn * CS * t) if t > 0 else 0.5
        ref = CS * kn * integrate.quad(f, Ti * dt, (Ti + 1) * dt, epsabs=1e-15, epsrel=1e-13)[0]
        assert abs(g - ref) < 1e-13


@pytest.mark.parametrize("n", [1, 3])
def test_weights_equal_time_integral_of_long_time_branch(n):
    """Weights for c_s t_0 > L against nested quadrature of Eq. (non_replicant_kernel_b) over psi and t."""
    L = 500.0
    dt = 0.5 * L / 32 / CS
    kn = np.pi * n / L

    def Kb(t):
        a = n * np.pi * CS * t / L
        return 2 / np.pi * integrate.quad(lambda p: np.cos(p) ** 2 * np.cos(a * np.sin(p)), 0,
                                          np.arcsin(L / (CS * t)), epsabs=1e-15, limit=200)[0]

    for Ti in [70, 90, 200]:
        assert CS * Ti * dt > L
        ref = CS * kn * integrate.quad(Kb, Ti * dt, (Ti + 1) * dt, epsabs=1e-15, epsrel=1e-12)[0]
        got = O.spectral_weights(n, np.array([Ti]), dt, L, CS)[0]
        assert abs(got - ref) < 2e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_weight_sums_telescope_to_static_limit(n):
    """P3: sum_{T<K} w^T = c_s k_n int_0^{K dt} K dt, which for rho = c_s K dt / L > 1 equals
    (2/pi) int_0^1 sqrt(1 - x^2/rho^2) sin(n pi x)/x dx (substitution x = rho sin psi) and tends to (2/pi) Si(n pi),
    the elastostatic limit, within 1/(pi rho^2)."""
    nf = 4
    L = 40.0
    dt = 0.5 * (L / nf) / CS
    K = 2400
    rho = CS * K * dt / L
    s = O.spectral_weights(n, np.arange(K), dt, L, CS).sum()
    ref = 2 / np.pi * integrate.quad(lambda x: np.sqrt(1 - x * x / rho ** 2) * np.sin(n * np.pi * x) / x, 0, 1,
                                     epsabs=1e-15, limit=200)[0]
    assert abs(s - ref) < 1e-12
    assert abs(s - 2 / np.pi * special.sici(n * np.pi)[0]) < 1.0 / (np.pi * rho ** 2)


def test_dft_pair_reconstructs_zero_padded_slip():
    """The mode range n = -N_f+1..N_f with F_{-n} = conj(F_n) and the 1/M normalisation invert exactly: the
    identity mode operator maps slip back to itself on the physical fault."""
    rng = np.random.default_rng(3)
    for nf in (5, 16, 33):
        d = rng.standard_normal((3, nf))
        D = O.slip_modes(d, nf)
        assert np.allclose(D[:, 0], d.sum(-1) / (2 * nf))
        np.testing.assert_allclose(O.modes_to_space(D, nf), d, atol=1e-13)


def test_mode_window_limits():
    """Eq. (mode_dependent_truncation): q_w = n_max gives T_end(1) for all modes; q_w = 1 gives T_end(1)/n."""
    nf, L, dt = 64, 1280.0, 0.5 * 20.0 / CS
    W_all = O.mode_windows(nf, L, dt, CS, 1.5, 0, 10 ** 6)
    W1 = math.ceil(1.5 * L / CS / dt - 1e-9)
    assert np.all(W_all[1:] == W1)
    W_q1 = O.mode_windows(nf, L, dt, CS, 1.5, 1, 10 ** 6)
    for n in (1, 2, 5, 64):
        assert W_q1[n] == math.ceil(1.5 * L / CS / n / dt - 1e-9)


# ---------------------------------------------------------------- space-time interaction kernel -------------------

def test_primitive_cross_derivatives_agree():
    """P5: I_31 and I_32 derive from one potential off the cut: d I_31/d r2 = d I_32/d r1 (catches garbled terms
    of Eq. primitives)."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        r1, r2 = rng.uniform(-400, 400), rng.uniform(-400, 400)
        r = math.hypot(r1, r2)
        t = r / CS * rng.uniform(1.1, 4.0)
        h = 1e-3
        a = (O.I31(r1, r2 + h, t, CS) - O.I31(r1, r2 - h, t, CS)) / (2 * h)
        b = (O.I32(r1 + h, r2, t, CS) - O.I32(r1 - h, r2, t, CS)) / (2 * h)
        assert abs(a - b) < 1e-6 * (abs(a) + 1e-3)


def test_self_element_lag0_is_radiation_damping():
    """P7: on its own element (r1 = r2 = 0) the lag-0 kernel is K_32 = 1, K_31 = 0, which reproduces the
    instantaneous radiation damping -mu/(2 c_s) V of Eq. (superimposition2) (reading H(0) = 0)."""
    for ds in (20.0, 78.125, 9.92757):
        dt = 0.5 * ds / CS
        k31, k32 = O.kernel_K3l(0.0, 0.0, 0, dt, ds, CS)
        assert abs(k31) == 0.0
        assert abs(k32 - 1.0) < 1e-6


def _seg_dist(r1, r2, ds):
    return np.where(np.abs(r1) <= ds / 2, np.abs(r2), np.hypot(np.abs(r1) - ds / 2, r2))


def test_kernel_zero_exactly_before_arrival():
    """P6: A_ij^T = 0 exactly iff the shear front from the nearest point of the source segment has not reached the
    receiver by t = (T+1) dt; nonzero after."""
    w = synth.tiny(2)
    net = O.network(w.faults, MU, CS)
    d = net.x[:, None, :] - net.x[None, :, :]
    r1 = (d * net.e1[None]).sum(-1)
    r2 = (d * net.nrm[None]).sum(-1)
    dist = _seg_dist(r1, r2, net.ds[None, :])
    other = net.fault_of[:, None] != net.fault_of[None, :]
    checked = 0
    for T in range(0, 160, 3):
        A = O.interaction_slice(net, T)
        front = CS * (T + 1) * net.dt
        clear = np.abs(front - dist) > 1e-9 * dist
        before = (front < dist) & other & clear
        after = (front > dist) & other & clear
        assert np.all(A[before] == 0.0)
        assert np.all(A[after] != 0.0)
        checked += after.sum()
    assert checked > 100


def test_late_time_kernel_tends_to_elastostatic_dislocation_stress():
    """P8: K_3l^T / dt tends to the static anti-plane stress of a uniformly slipped segment (a pair of screw
    dislocations): S_31 = -(c_s/pi)(r2/rho+^2 - r2/rho-^2), S_32 = (c_s/pi)(r1+/rho+^2 - r1-/rho-^2),
    r1+- = r1 +- ds/2, with an error decaying like T^-2."""
    ds = 20.0
    dt = 0.5 * ds / CS
    for r1, r2 in [(300.0, 200.0), (-1000.0, 50.0), (5.0, 400.0)]:
        rp, rm = r1 + ds / 2, r1 - ds / 2
        pp, pm = rp ** 2 + r2 ** 2, rm ** 2 + r2 ** 2
        S31 = -(CS / np.pi) * (r2 / pp - r2 / pm)
        S32 = (CS / np.pi) * (rp / pp - rm / pm)
        errs = []
        for T in (3000, 30000):
            k31, k32 = O.kernel_K3l(r1, r2, T, dt, ds, CS)
            errs.append(abs(k32 / dt - S32) / abs(S32))
            assert abs(k31 / dt - S31) < 1e-4 * abs(S31)
        assert errs[1] < errs[0] / 50 and errs[1] < 2e-5


def test_reciprocity_of_far_field_kernel():
    """Source/receiver reciprocity of the anti-plane Green's function: for well-separated elements,
    A_ij^T / ds_j ~ A_ji^T / ds_i (error O((ds/r)^2)).  Faults of different element sizes make a transposed
    operand, a wrong frame or a receiver/source normal swap fail."""
    faults = np.array([[0.0, 0.0, 0.2, 200.0, 10], [100.0, -900.0, 1.1, 400.0, 10]])
    net = O.network(faults, MU, CS)
    nA = 10
    for T in (300, 500, 800):
        A = O.interaction_slice(net, T)
        ab = A[:nA, nA:] / net.ds[None, nA:]
        ba = A[nA:, :nA].T / net.ds[:nA, None]
        r = np.linalg.norm(net.x[:nA, None, :] - net.x[None, nA:, :], axis=-1)
        assert np.all(CS * T * net.dt > 1.5 * r)
        np.testing.assert_allclose(ab, ba, rtol=3e-3)


# ---------------------------------------------------------------- windows and printed numbers --------------------

def test_printed_two_fault_and_x_fault_numbers(golden_printed):
    """P9: the printed geometry of Sec. 3.1 reproduces the printed dt_min, cell sizes and T_end; Table 2's dt."""
    w = synth.paper_two_fault()
    net = O.network(w.faults, 30e9, CS)
    g = golden_printed
    assert abs(net.dt - g["two_fault.dt_min"][0]) <= g["two_fault.dt_min"][1]
    assert abs(net.ds[0] - g["two_fault.dx_1"][0]) <= g["two_fault.dx_1"][1]
    assert abs(net.ds[-1] - g["two_fault.dx_2"][0]) <= g["two_fault.dx_2"][1]
    _, t_end, _ = O.pair_windows(net, 0.01, 0.01, 10 ** 6)
    assert abs(t_end.max() - g["two_fault.T_end"][0]) <= g["two_fault.T_end"][1]
    xf = O.network(np.array([[0, 0, 0.6, 1000.0, 510], [0, 0, -0.6, 1000.0, 510]]), 30e9, CS)
    assert abs(xf.dt - g["x_fault.dt_min"][0]) <= g["x_fault.dt_min"][1]


def test_exact_first_lag_and_centroid_arrival_time():
    """Window start reading: the first nonzero lag of a fault pair is floor(min segment distance / (c_s dt)) (from
    P6), while the centroid-based T_earl of Eq. (early_time) can come after the true first arrival (a source element
    radiates from its nearest point, so for a receiver just beyond an element end the centroid distance overstates it
    by up to ds/2).  The operator therefore starts each block at its exact first nonzero lag and reports T_init only;
    on this network the paper's T_init = (1 - eta_Tmin) T_earl does include that first lag."""
    w = synth.two_fault_128()
    net = O.network(w.faults, MU, CS)
    t_init, _, _ = O.pair_windows(net, 0.01, 0.01, 400)
    d = net.x[:, None, :] - net.x[None, :, :]
    r1 = (d * net.e1[None]).sum(-1)
    r2 = (d * net.nrm[None]).sum(-1)
    dist = _seg_dist(r1, r2, net.ds[None, :])
    for a, b in [(0, 1), (1, 0)]:
        ra, rb = slice(128 * a, 128 * a + 128), slice(128 * b, 128 * b + 128)
        dmin = dist[ra, rb].min()
        first = next(T for T in range(60) if np.any(O.interaction_slice(net, T)[ra, rb] != 0))
        assert first == math.floor(dmin / (CS * net.dt))
        assert t_init[a, b] / net.dt <= first + 1


# ---------------------------------------------------------------- the whole functional ---------------------------

def test_linearity_and_time_shift_invariance():
    """P10: the functional is linear in the history and Toeplitz in time (pushing one zero step first delays the
    output by one step)."""
    w = synth.tiny(1, steps=24)
    net = O.network(w.faults, MU, CS)
    hp = dict(w.hparams, max_steps=25)
    V1 = w.slip_rate(0, 0, 24)
    V2 = w.slip_rate(1, 0, 24)
    t1 = O.stress_history(net, V1, hp)[0]
    t2 = O.stress_history(net, V2, hp)[0]
    t12 = O.stress_history(net, 2.0 * V1 - 0.5 * V2, hp)[0]
    np.testing.assert_allclose(t12, 2.0 * t1 - 0.5 * t2, rtol=1e-11, atol=1e-9 * np.abs(t1).max())
    Vs = np.vstack([np.zeros((1, net.N)), V1[:-1]])
    ts = O.stress_history(net, Vs, hp)[0]
    np.testing.assert_allclose(ts[1:], t1[:-1], rtol=1e-11, atol=1e-9 * np.abs(t1).max())
    assert np.all(ts[0] == 0.0)


def test_spectral_self_converges_to_space_time_self_sum():
    """P12: on one fault, radiation damping + the non-replicating spectral term and the space-time self sum of the
    same primitives (r2 = 0, K_32 only) are two discretisations of one operator; they agree at O(ds)."""
    L = 1000.0
    errs = []
    for N in (16, 32):
        net = O.network(np.array([[0.0, 0.0, 0.3, L, N]]), MU, CS)
        steps = int(round(3 * L / (CS * net.dt)))
        t = np.arange(steps) * net.dt
        xi = (np.arange(N) + 0.5) / N
        V = np.outer(np.sin(np.pi * CS * t / L) ** 2 * (t < L / CS), np.sin(np.pi * xi) ** 2)
        tab = O.SelfTables(N, L, net.dt, CS, np.full(N + 1, steps - 1))
        spectral = O.self_history(net, 0, O.slip_from_rate(V, net.dt), tab) - MU / (2 * CS) * V
        d = net.x[:, None, :] - net.x[None, :, :]
        r1 = (d * net.e1[None]).sum(-1)
        r2 = (d * net.nrm[None]).sum(-1)
        A = np.stack([O.kernel_K3l(r1, r2, T, net.dt, net.ds[None, :], CS)[1] for T in range(steps)])
        st = np.array([-(MU / (2 * CS)) * np.einsum("tij,tj->i", A[: n + 1], V[n::-1]) for n in range(steps)])
        errs.append(np.linalg.norm(spectral - st) / np.linalg.norm(st))
    assert errs[0] < 0.03 and errs[1] < 0.6 * errs[0]


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="no extended precision long double here")
def test_oracle_rounding_is_far_below_parity_tolerance():
    """P13: the FP64 interaction sum agrees with the same sum in extended precision to << 1e-10 (rel-L2)."""
    w = synth.tiny(3, steps=150)
    net = O.network(w.faults, MU, CS)
    V = w.slip_rate(0, 0, 150)
    f64 = O.interaction_history(net, V)
    fld = O.interaction_history(net, V, dtype=np.longdouble).astype(np.float64)
    assert np.linalg.norm(fld) > 0
    assert np.linalg.norm(f64 - fld) / np.linalg.norm(fld) < 1e-13


def test_normal_stress_change_vanishes_and_parts_add_up():
    """Sec. 2.1: in mode III the elastodynamic normal-stress change is identically zero; tau is the sum of the
    three parts of Eq. (superimposition2) and the radiation part is exactly -mu/(2 c_s) V."""
    w = synth.tiny(1, steps=10)
    net = O.network(w.faults, MU, CS)
    V = w.slip_rate(0, 0, 10)
    tau, rad, fs, fi = O.stress_history(net, V, dict(w.hparams, max_steps=10))
    np.testing.assert_array_equal(rad, -(MU / (2 * CS)) * V)
    np.testing.assert_allclose(tau, rad + fs + fi, rtol=0, atol=0)


# ---------------------------------------------------------------- static tail (flag STATIC_TAIL) -------------------

def _two_small_faults():
    return O.network(np.array([[0.0, 0.0, 0.1, 80.0, 8], [60.0, -150.0, 0.7, 80.0, 8]]), MU, CS)


def test_static_slice_is_the_late_time_limit_of_the_dynamic_slice():
    """P14a: A^static equals lim A^T / dt of the dynamic kernel built from Eq. primitives (projection, frames and
    signs included), with an error decaying like T^-2; same-fault entries are zero."""
    net = _two_small_faults()
    As = O.static_slice(net)
    errs = []
    for T in (2000, 20000):
        Ad = O.interaction_slice(net, T) / net.dt
        errs.append(np.abs(Ad - As).max() / np.abs(As).max())
    assert errs[1] < errs[0] / 50 and errs[1] < 1e-5
    assert np.all(As[:8, :8] == 0) and np.abs(As[:8, 8:]).min() > 0


def test_interaction_static_tail_restores_the_dropped_history_at_late_times():
    """P14b: slip rate only at step 0.  With truncated pair windows the plain sum is zero once the window has
    passed; with the static tail it approaches the untruncated sum (A^m V^0 -> dt A^static V^0) as m grows."""
    net = _two_small_faults()
    steps = 700
    V = np.zeros((steps, net.N))
    V[0] = np.linspace(1.0, 2.0, net.N)
    hp = dict(eta_tmin=0.01, eta_tmax=0.01, eta_w=1.5, q_w=0, max_steps=steps)
    full = O.stress_history(net, V, dict(hp, flags=2))[3]
    trunc = O.stress_history(net, V, dict(hp, flags=0))[3]
    tail = O.stress_history(net, V, dict(hp, flags=4))[3]
    last = O.pair_windows(net, 0.01, 0.01, steps)[2]
    m0 = int(last.max()) + 1
    assert m0 < 150 and np.all(trunc[m0:] == 0)
    e = [np.linalg.norm(tail[m] - full[m]) / np.linalg.norm(full[m]) for m in (300, 690)]
    assert e[0] < 0.05 and e[1] < e[0] / 4 and e[1] < 1e-2
    assert np.all(tail[:int(last.min()) + 1] == trunc[:int(last.min()) + 1])


def test_self_static_tail_completes_the_weight_sum():
    """P14c: slip rate only at step 0 (a slip step).  The untruncated spectral term tends to the static response
    sum_T w_n^T D_n = (2/pi) Si(n pi) D_n; the truncated term plus the static tail reaches it (differences decay
    like the weight mass still missing from the untruncated sum), while the plain truncated term stays off."""
    L, N = 500.0, 16
    net = O.network(np.array([[0.0, 0.0, 0.3, L, N]]), MU, CS)
    steps = 900
    V = np.zeros((steps, N))
    V[0] = np.sin(np.pi * (np.arange(N) + 0.5) / N)
    hp = dict(eta_tmin=0.01, eta_tmax=0.01, eta_w=0.5, q_w=0, max_steps=steps)
    full = O.stress_history(net, V, dict(hp, flags=2))[2]
    trunc = O.stress_history(net, V, dict(hp, flags=0))[2]
    tail = O.stress_history(net, V, dict(hp, flags=4))[2]
    W = O.mode_windows(N, L, net.dt, CS, 0.5, 0, steps)
    assert W[1:].max() < 120
    e_tail = [np.linalg.norm(tail[m] - full[m]) / np.linalg.norm(full[m]) for m in (300, 890)]
    e_trunc = np.linalg.norm(trunc[890] - full[890]) / np.linalg.norm(full[890])
    assert e_tail[1] < e_tail[0] / 2 and e_tail[1] < 2e-3 and e_trunc > 20 * e_tail[1]


# ---------------------------------------------------------------- earthquake-cycle step (oracle only) --------------

from oracle import seas_integrator as SI  # noqa: E402

FR = SI.Friction(a=0.01, b=0.015, dc=1e-3, f0=0.6, v0=1e-9, sigma_n=50e6)


def test_state_law_limits_are_the_aging_and_slip_laws():
    """P15a: Eq. state_evolution_law is the aging law 1 - V theta / D_c at eps = 1 and tends to the slip law
    -(V theta / D_c) ln(V theta / D_c) as eps -> 0."""
    rng = np.random.default_rng(3)
    V = 10.0 ** rng.uniform(-12, 0, 50)
    theta = 10.0 ** rng.uniform(-4, 8, 50)
    om = V * theta / FR.dc
    np.testing.assert_allclose(SI.state_rate(V, theta, FR), 1.0 - om, rtol=1e-12, atol=1e-12)
    slip = SI.Friction(**{**FR.__dict__, "eps": 1e-7})
    np.testing.assert_allclose(SI.state_rate(V, theta, slip), -om * np.log(om), rtol=1e-4, atol=1e-12)


def test_newton_root_equals_an_independent_bisection():
    """P15b: the Newton solve of tau - (mu / 2 c_s) V = sigma_n f(V, theta) (in ln V) agrees with a bisection in
    ln V on the same balance to the 1e-8 tolerance, for stresses spanning creep to seismic slip."""
    rad = 32e9 / (2 * 3464.0)
    rng = np.random.default_rng(5)
    theta = 10.0 ** rng.uniform(-3, 7, 40)
    tau = FR.sigma_n * (FR.f0 + rng.uniform(-0.1, 0.1, 40))
    V, it = SI.solve_v(tau, theta, FR, rad, 1e-9)
    lo, hi = np.full(40, -60.0), np.full(40, 5.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        g = tau - rad * np.exp(mid) - FR.sigma_n * SI.friction(np.exp(mid), theta, FR)
        lo = np.where(g > 0, mid, lo)
        hi = np.where(g > 0, hi, mid)
    np.testing.assert_allclose(V, np.exp(0.5 * (lo + hi)), rtol=1e-6)
    assert it < 60 and V.min() < 1e-6 < V.max()


def test_steady_initial_state_of_the_benchmark_stays_put():
    """P15c: the benchmark's initial condition (V = V_*, theta = D_c / V_*, tau^o = f_* sigma_n + mu V_* / (2 c_s),
    no slip before t = 0) is an equilibrium: over 40 steps V stays at V_* to 1e-6 (a sign error in the radiation
    term or the friction law would move it at once)."""
    net = O.network(np.array([[0.0, 0.0, 0.2, 200.0, 8], [30.0, -300.0, 0.9, 160.0, 8]]), MU, CS)
    tau0 = FR.f0 * FR.sigma_n + MU / (2 * CS) * FR.v0
    it = SI.Integrator(net, FR, np.full(net.N, tau0), FR.v0, FR.dc / FR.v0, max_steps=41)
    for _ in range(40):
        V = it.step()
    assert np.abs(V / FR.v0 - 1).max() < 1e-6


def test_predictor_corrector_converges_at_second_order_without_elasticity():
    """P15d: with negligible elasticity (mu -> 0) a step reduces to the slider ODE dtheta/dt = G(V(theta), theta),
    V(theta) from sigma_n f(V, theta) = tau^o; the oracle's predictor-corrector reaches scipy's solution with an
    error that falls about four times when dt halves."""
    fr = SI.Friction(a=0.01, b=0.015, dc=2e-9, f0=0.6, v0=1e-6, sigma_n=50e6)
    tau0 = fr.f0 * fr.sigma_n
    errs = []
    for n_elem in (4, 8):
        net = O.network(np.array([[0.0, 0.0, 0.0, 10.0, n_elem]]), 1e-3, CS)
        steps = int(round(0.01 / net.dt))
        th0 = 5 * fr.dc / fr.v0
        v_init = math.exp((fr.a * math.log(fr.v0) - fr.b * math.log(th0 / fr.dc)) / (fr.a + fr.b))  # balanced
        it = SI.Integrator(net, fr, np.full(net.N, tau0), v_init, th0, max_steps=steps + 1)
        for _ in range(steps):
            it.step()
        def rhs(t, y):
            th = y[0]
            v = math.exp((fr.a * math.log(fr.v0) - fr.b * math.log(th / fr.dc)) / (fr.a + fr.b))
            return [1.0 - v * th / fr.dc]
        ref = integrate.solve_ivp(rhs, (0, steps * net.dt), [th0], rtol=1e-12, atol=1e-20).y[0, -1]
        errs.append(abs(it.theta[0] - ref) / ref)
    assert errs[1] < errs[0] / 3.5 and errs[1] < 1e-4


# ---------------------------------------------------------------- single-row evaluators and the interaction factor --

def test_interaction_rows_equals_the_full_history_across_chunk_and_window_edges():
    """interaction_rows (one step, chosen receivers, lags in chunks) is the row slice of interaction_history (every
    step, every receiver, one lag stack): checked at steps on both sides of chunk boundaries and of the per-pair
    window ends, with and without windows, for chunk sizes 64 and 128, on a three-fault network."""
    w = synth.tiny(4, n_faults=3, steps=270)
    net = O.network(w.faults, MU, CS)
    V = w.slip_rate(0, 0, 270)
    hi = np.array([[-1, 131, 200], [64, -1, 127], [129, 255, -1]])
    full = O.interaction_history(net, V)
    win = O.interaction_history(net, V, pair_hi=hi)
    assert np.abs(full[200]).max() > 0 and np.abs(win[269] - full[269]).max() > 1e-3 * np.abs(full[269]).max()
    rows = np.array([0, 3, net.offset[1], net.N - 1, net.offset[2] + 1])
    for n in (0, 1, 63, 64, 65, 127, 128, 129, 130, 131, 132, 199, 200, 201, 255, 256, 269):
        for chunk in (64, 128):
            np.testing.assert_allclose(O.interaction_rows(net, V, n, rows, chunk=chunk), full[n, rows],
                                       rtol=1e-12, atol=1e-12 * np.abs(full[n]).max())
            np.testing.assert_allclose(O.interaction_rows(net, V, n, rows, pair_hi=hi, chunk=chunk), win[n, rows],
                                       rtol=1e-12, atol=1e-12 * np.abs(full[n]).max())


def test_self_rows_equals_the_full_history_around_the_window_edge():
    """self_rows (one step, chosen receivers, the slip history from the longest window back) is the row slice of
    self_history (every step): mode-dependent windows (q_w = 3) so that modes have different last lags; steps on
    both sides of the longest window."""
    L, nf = 300.0, 12
    net = O.network(np.array([[10.0, -5.0, 0.4, L, nf]]), MU, CS)
    steps = 140
    W = O.mode_windows(nf, L, net.dt, CS, 1.0, 3, steps)
    assert W[1] > W[nf] and W[1] < steps - 20
    V = synth.Workload("one", np.array([[10.0, -5.0, 0.4, L, nf]]), steps=steps).slip_rate(0, 0, steps)
    delta = O.slip_from_rate(V, net.dt)
    tab = O.SelfTables(nf, L, net.dt, CS, W)
    full = O.self_history(net, 0, delta, tab)
    Wm = int(W.max())
    rows = np.array([0, 5, nf - 1])
    for m in (0, 1, Wm - 1, Wm, Wm + 1, Wm + 2, steps - 1):
        np.testing.assert_allclose(O.self_rows(net, 0, delta[: m + 1], m, tab, rows), full[m, rows],
                                   rtol=1e-11, atol=1e-11 * np.abs(full).max())


def _dislocation_traction(x, nrm, P, b):
    """Traction on planes of normal nrm at points x from a screw dislocation of Burgers vector b at P (the textbook
    anti-plane field sigma_31 = -(mu b / 2 pi) y / r^2, sigma_32 = (mu b / 2 pi) x / r^2, relative coordinates)."""
    d = x - P
    r2 = (d * d).sum(-1)
    s31 = -(MU * b / (2 * np.pi)) * d[..., 1] / r2
    s32 = (MU * b / (2 * np.pi)) * d[..., 0] / r2
    return s31 * nrm[..., 0] + s32 * nrm[..., 1]


def test_interaction_tends_to_the_stress_of_a_slipped_segment():
    """Factor, sign and projection of interaction_history / interaction_rows, pinned to elastostatics: a step of
    slip delta_f on each of three differently oriented faults (slip rate delta_f / dt in step 0, nothing after)
    makes f_int tend, as c_s t grows, to the static stress of uniformly slipped segments, i.e. pairs of screw
    dislocations (+delta at the start c - L/2 e'_1 of the fault, -delta at its end), a closed form independent of
    Eq. primitives.  The convention is fixed by the radiation-damping sign of Eq. superimposition2: slip lowers the
    stress on the slipping segment and raises it beyond its tips.  A wrong -mu / (2 c_s) factor, sign, normal frame
    or transposed operand fails; the error decays like (r / c_s t)^2."""
    faults = np.array([[0.0, 0.0, 0.25, 120.0, 6], [150.0, -90.0, 1.2, 100.0, 5], [-40.0, 160.0, -0.7, 90.0, 9]])
    net = O.network(faults, MU, CS)
    delta = np.array([0.7, -0.4, 1.3])
    ref = np.zeros(net.N)
    for f, (cx, cy, phi, L, _) in enumerate(faults):
        e1 = np.array([math.cos(phi), math.sin(phi)])
        c = np.array([cx, cy])
        o = net.fault_of != f
        ref[o] += _dislocation_traction(net.x[o], net.nrm[o], c - 0.5 * L * e1, delta[f])
        ref[o] += _dislocation_traction(net.x[o], net.nrm[o], c + 0.5 * L * e1, -delta[f])
    errs = []
    for n in (5000, 20000):
        V = np.zeros((n + 1, net.N))
        for f in range(3):
            V[0, net.offset[f]:net.offset[f + 1]] = delta[f] / net.dt
        got = O.interaction_rows(net, V, n, np.arange(net.N))
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[1] < 3e-6 and errs[1] < errs[0] / 8
    # the same through the all-steps evaluator on a shorter run
    V = np.zeros((1500, net.N))
    V[0, : net.offset[1]] = delta[0] / net.dt
    hist = O.interaction_history(net, V)[-1]
    one = np.zeros(net.N)
    o = net.fault_of != 0
    e1 = np.array([math.cos(0.25), math.sin(0.25)])
    one[o] = (_dislocation_traction(net.x[o], net.nrm[o], -60.0 * e1, delta[0])
              + _dislocation_traction(net.x[o], net.nrm[o], 60.0 * e1, -delta[0]))
    assert np.linalg.norm(hist - one) / np.linalg.norm(one) < 2e-3


def test_collinear_halves_self_plus_interaction_converge_to_the_whole_fault():
    """Cutting one straight fault into two collinear halves: the spectral self term of the whole fault (Sec. 2.3.1)
    and the spectral self terms of the halves plus their space-time cross interaction (Sec. 2.3.2,
    interaction_history) are two discretisations of one operator and agree at O(ds) as the mesh is refined (slip
    vanishing at the cut and at the ends, so no tip singularity sits between them).  Dropping the cross term,
    flipping its sign or halving its factor leaves an O(1) error that does not shrink."""
    L, phi = 1000.0, 0.3
    e1 = np.array([math.cos(phi), math.sin(phi)])
    errs, wrong = [], []
    for N in (16, 32):
        whole = O.network(np.array([[0.0, 0.0, phi, L, N]]), MU, CS)
        ca, cb = -0.25 * L * e1, 0.25 * L * e1
        split = O.network(np.array([[ca[0], ca[1], phi, L / 2, N // 2], [cb[0], cb[1], phi, L / 2, N // 2]]),
                          MU, CS)
        assert np.allclose(whole.x, split.x) and whole.dt == split.dt
        steps = int(round(3 * L / (CS * whole.dt)))
        t = np.arange(steps) * whole.dt
        xi = (np.arange(N) + 0.5) / N
        V = np.outer(np.sin(np.pi * CS * t / L) ** 2 * (t < L / CS), np.sin(2 * np.pi * xi) ** 2)
        d = O.slip_from_rate(V, whole.dt)
        fw = O.self_history(whole, 0, d, O.SelfTables(N, L, whole.dt, CS, np.full(N + 1, steps - 1)))
        h = N // 2
        th = O.SelfTables(h, L / 2, whole.dt, CS, np.full(h + 1, steps - 1))
        fs = np.concatenate([O.self_history(split, 0, d[:, :h], th), O.self_history(split, 1, d[:, h:], th)], 1)
        fi = O.interaction_history(split, V)
        nw = np.linalg.norm(fw)
        errs.append(np.linalg.norm(fs + fi - fw) / nw)
        wrong.append(min(np.linalg.norm(fs + c * fi - fw) / nw for c in (0.0, -1.0, 0.5, 2.0)))
    assert errs[0] < 0.02 and errs[1] < 0.6 * errs[0]
    assert min(wrong) > 10 * errs[0]


def test_gamma_step_of_one_is_the_fixed_step():
    """P15e: a step of one lattice step is the fixed-dt step, to the last bit."""
    net = O.network(np.array([[0.0, 0.0, 0.2, 200.0, 8], [30.0, -300.0, 0.9, 160.0, 8]]), MU, CS)
    tau0 = np.full(net.N, FR.f0 * FR.sigma_n + MU / (2 * CS) * FR.v0)
    tau0[:8] += 1.5e6 * np.exp(-((np.arange(8) + 0.5) / 8 - 0.4) ** 2 / 0.04)
    a = SI.Integrator(net, FR, tau0, FR.v0, FR.dc / FR.v0, max_steps=12)
    b = SI.Integrator(net, FR, tau0, FR.v0, FR.dc / FR.v0, max_steps=12)
    for _ in range(10):
        np.testing.assert_array_equal(a.step(), b.step_gamma(1))
    np.testing.assert_array_equal(a.theta, b.theta)


def test_gamma_steps_hold_the_rate_on_the_lattice():
    """P15f: the known stress of a step of gamma lattice steps is the stress functional (stress_history) of the
    lattice history in which the interval holds the pushed rate and the slip grows linearly, minus its radiation
    damping: the integrator's lattice bookkeeping against the functional's own definition."""
    net = O.network(np.array([[0.0, 0.0, 0.2, 200.0, 8], [30.0, -300.0, 0.9, 160.0, 8]]), MU, CS)
    tau0 = np.full(net.N, FR.f0 * FR.sigma_n + MU / (2 * CS) * FR.v0)
    it = SI.Integrator(net, FR, tau0, 1.3 * FR.v0, FR.dc / FR.v0, max_steps=40)
    for g in (1, 3, 2):
        it.step_gamma(g)
    v_push = 2.0 * it.V[-1]
    gamma = 4
    slips = [it.delta[-1] + (j * net.dt) * v_push for j in range(1, gamma + 1)]
    known = it._known_stress_lattice(slips, v_push)
    V_lat = np.stack(it.V[1:] + [v_push] * gamma)
    hp = dict(flags=2, max_steps=40)
    tau, rad, fself, fint = O.stress_history(net, V_lat, hp, slip=np.stack(it.delta[1:] + slips))
    np.testing.assert_allclose(known, (tau - rad)[-1], rtol=1e-12, atol=1e-6)


def test_gamma_steps_converge_at_second_order_without_elasticity():
    """P15g: with negligible elasticity the gamma-step scheme is the predictor-corrector of the slider ODE with
    step gamma dt; its error at a fixed time falls about four times when gamma halves."""
    fr = SI.Friction(a=0.01, b=0.015, dc=2e-9, f0=0.6, v0=1e-6, sigma_n=50e6)
    tau0 = fr.f0 * fr.sigma_n
    net = O.network(np.array([[0.0, 0.0, 0.0, 10.0, 4]]), 1e-3, CS)
    th0 = 5 * fr.dc / fr.v0
    v_init = math.exp((fr.a * math.log(fr.v0) - fr.b * math.log(th0 / fr.dc)) / (fr.a + fr.b))
    lattice = 32
    errs = []
    for gamma in (4, 2):
        it = SI.Integrator(net, fr, np.full(net.N, tau0), v_init, th0, max_steps=lattice + 1)
        for _ in range(lattice // gamma):
            it.step_gamma(gamma)

        def rhs(t, y):
            v = math.exp((fr.a * math.log(fr.v0) - fr.b * math.log(y[0] / fr.dc)) / (fr.a + fr.b))
            return [1.0 - v * y[0] / fr.dc]
        ref = integrate.solve_ivp(rhs, (0, lattice * net.dt), [th0], rtol=1e-12, atol=1e-20).y[0, -1]
        errs.append(abs(it.theta[0] - ref) / ref)
    assert errs[1] < errs[0] / 3.5


def test_adaptive_gamma_follows_the_rate():
    net = O.network(np.array([[0.0, 0.0, 0.2, 200.0, 8]]), MU, CS)
    it = SI.Integrator(net, FR, np.full(net.N, FR.f0 * FR.sigma_n), FR.v0, FR.dc / FR.v0, max_steps=4)
    g = it.adaptive_gamma(0.5, 10 ** 9)
    assert g == math.ceil(0.5 * FR.dc / FR.v0 / net.dt)
    assert it.adaptive_gamma(0.5, 100) == 100
    it.V[-1] = np.full(net.N, 1.0)
    assert it.adaptive_gamma(0.5, 100) == 1


# ------------------------------------------------ cluster trees, H-matrix partition, cluster-level windows ------

def _random_net(seed=7):
    rng = np.random.default_rng(seed)
    faults = np.array([[0.0, 0.0, 0.1, 900.0, 37], [150.0, 700.0, -0.3, 700.0, 29],
                       [1100.0, -250.0, 1.2, 500.0, 21]])
    faults[:, :2] += rng.uniform(-20, 20, (3, 2))
    return O.network(faults, MU, CS)


@pytest.mark.parametrize("leaf,eta_h,max_block,dense", [(4, 2.0, 64, False), (8, 0.7, 8, False),
                                                        (3, 1.5, 64, True)])
def test_hmatrix_blocks_tile_each_fault_pair_once(leaf, eta_h, max_block, dense):
    """P16a: the leaf blocks of each ordered fault pair cover every (receiver, source) element pair exactly once;
    every far block satisfies the admissibility test (centre distance > eta_H (r_A + r_B), radii recomputed here
    from the elements) and the side cap; every near block is a pair of leaves; the tree halves keep consecutive
    elements with the extra one on the left."""
    net = _random_net()
    for f in range(net.F):
        stack = [O.cluster_tree(net, f, leaf)]
        while stack:
            c = stack.pop()
            if c.children:
                l, r = c.children
                assert (l.lo, l.hi, r.lo, r.hi) == (c.lo, c.lo + (c.hi - c.lo + 1) // 2, l.hi, c.hi)
                stack += [l, r]
            else:
                assert 1 <= c.hi - c.lo <= leaf

    def circle(lo, hi):
        c = net.x[lo:hi].mean(axis=0)
        return c, max(math.hypot(*(net.x[i] - c)) + net.ds[i] / 2 for i in range(lo, hi))

    for a in range(net.F):
        for b in range(net.F):
            if a == b:
                continue
            cover = np.zeros((net.n_elem[a], net.n_elem[b]), dtype=int)
            blocks = O.hmatrix_blocks(net, a, b, leaf, eta_h, max_block, dense)
            for r0, p, c0, q, far in blocks:
                cover[r0 - net.offset[a]:r0 - net.offset[a] + p, c0 - net.offset[b]:c0 - net.offset[b] + q] += 1
                if far:
                    (ca, ra), (cb, rb) = circle(r0, r0 + p), circle(c0, c0 + q)
                    assert not dense and math.hypot(*(ca - cb)) > eta_h * (ra + rb) and max(p, q) <= max_block
                else:
                    assert p <= leaf and q <= leaf
            assert (cover == 1).all()
            if not dense:
                assert any(b_[4] for b_ in blocks)


def test_cluster_windows_of_two_collinear_faults_in_closed_form():
    """P16b: two collinear faults of 1000 m on x in [0, 1000] and [4000, 5000], 16 elements each, leaf 8: with
    eta_H = 6 neither the root pair (4000 < 6 x 1000) nor a half against a whole fault (4250, 3750 < 6 x 750) is
    admissible, and the four pairs of halves are (3500 .. 4500 > 6 x 500).  Each block's window ends at
    (1 + eta_Tmax) times the largest distance between the ends of its two half-segments over c_s, here the span
    from the outer end of one half to the outer end of the other: 4000, 4500 or 5000 m; the fault-pair window
    (5000 m) is the longest.  Distances along the line of sight make an end taken at a centroid (ds = 62.5 m) move
    the window by two lags."""
    net = O.network(np.array([[500.0, 0.0, 0.0, 1000.0, 16], [4500.0, 0.0, 0.0, 1000.0, 16]]), MU, CS)
    eta_t = 0.3
    W = O.cluster_windows(net, 8, 6.0, 64, eta_t, 10 ** 6)
    lag = lambda d: math.ceil((1 + eta_t) * d / CS / net.dt - 1e-9)
    assert [lag(d) for d in (4000.0, 4500.0, 5000.0)] == [167, 188, 208]
    blocks = sorted(O.hmatrix_blocks(net, 0, 1, 8, 6.0, 64))
    assert blocks == [(0, 8, 16, 8, True), (0, 8, 24, 8, True), (8, 8, 16, 8, True), (8, 8, 24, 8, True)]
    exp = np.full((32, 32), -1)
    L, R = slice(0, 8), slice(8, 16)
    BL, BR = slice(16, 24), slice(24, 32)
    exp[L, BL], exp[L, BR], exp[R, BL], exp[R, BR] = 188, 208, 167, 188
    exp[BL, L], exp[BL, R], exp[BR, L], exp[BR, R] = 188, 167, 208, 188
    np.testing.assert_array_equal(W, exp)
    _, _, P = O.pair_windows(net, 0.01, eta_t, 10 ** 6)
    assert P[0, 1] == P[1, 0] == 208
    assert (O.cluster_windows(net, 8, 6.0, 64, eta_t, 180) == np.where(exp < 0, -1, np.minimum(exp, 179))).all()


def test_cluster_windows_reduce_to_the_fault_pair_windows_for_one_block_per_pair():
    """P16c: with eta_H so small that every root pair is admissible (and no side cap), each fault pair is one block
    and the cluster-level windows are the fault-pair windows of Sec. 2.3.2, element for element."""
    net = _random_net(3)
    W = O.cluster_windows(net, 4, 1e-3, 10 ** 6, 0.01, 10 ** 6)
    _, _, P = O.pair_windows(net, 0.01, 0.01, 10 ** 6)
    np.testing.assert_array_equal(W, P[net.fault_of][:, net.fault_of])


def test_cluster_windows_never_cut_before_the_whole_source_element_has_arrived():
    """P16d: on a three-fault network with many blocks, each element pair's cluster-level window is no longer than
    its fault-pair window and no shorter than the time for the S-wave from the far end of the source element to
    reach the receiver centroid (brute force over element pairs)."""
    net = _random_net(11)
    W = O.cluster_windows(net, 4, 1.0, 16, 0.0, 10 ** 6)
    _, _, P = O.pair_windows(net, 0.01, 0.0, 10 ** 6)
    Pe = P[net.fault_of][:, net.fault_of]
    other = net.fault_of[:, None] != net.fault_of[None, :]
    assert (W[other] <= Pe[other]).all() and (W[other] < Pe[other]).mean() > 0.3
    for i in range(net.N):
        for j in range(net.N):
            if not other[i, j]:
                assert W[i, j] == -1
                continue
            far = max(math.hypot(*(net.x[i] - net.x[j] - s * 0.5 * net.ds[j] * net.e1[j])) for s in (-1, 1))
            assert W[i, j] >= math.ceil(far / CS / net.dt - 1e-9)


def test_interaction_with_element_windows_equals_a_brute_force_loop():
    """P16e: with a window per element pair, f_int^n = -(mu / 2 c_s) sum_j sum_{T <= min(n, hi_ij)} A_ij^T V_j^{n-T}
    written as plain loops, on two faults of five elements over 14 steps."""
    net = O.network(np.array([[0.0, 0.0, 0.0, 50.0, 5], [10.0, 12.0, 0.4, 40.0, 5]]), MU, CS)
    steps = 14
    rng = np.random.default_rng(5)
    V = rng.normal(size=(steps, net.N))
    hi = rng.integers(0, steps, size=(net.N, net.N))
    A = [O.interaction_slice(net, T) for T in range(steps)]
    ref = np.zeros((steps, net.N))
    for n in range(steps):
        for i in range(net.N):
            s = 0.0
            for j in range(net.N):
                for T in range(min(n, hi[i, j]) + 1):
                    s += A[T][i, j] * V[n - T, j]
            ref[n, i] = -(MU / (2 * CS)) * s
    got = O.interaction_history(net, V, pair_hi=hi)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    rows = np.array([1, 6, 9])
    np.testing.assert_allclose(O.interaction_rows(net, V, steps - 1, rows, pair_hi=hi), ref[-1, rows],
                               rtol=1e-12, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------------------------ traction-free surface, method of images ------

def _surface_fault(x0, depth, n, phi=-math.pi / 2):
    e1 = np.array([math.cos(phi), math.sin(phi)])
    return [x0 + 0.5 * depth * e1[0], 0.5 * depth * e1[1], phi, depth, n]


def test_half_space_static_limit_is_the_stress_of_the_segment_and_its_image():
    """P17a: a fault from the free surface y = 0 down to depth D slips uniformly by delta at step 0.  With the
    static tail after the self windows, the half-space self term is its elastostatic limit, which the method of
    images makes the full-space stress of the segment and its mirror image, i.e. screw dislocations +delta at depth
    -D (the image's far end) and -delta at depth D (textbook field, independent of the oracle's kernels).  The
    spectral series of a slip box converges like 1/N (checked at 32 and 64 real elements, receivers between 0.05 D
    and 0.8 D); the fault alone in a full space (dislocations at 0 and D) is off by more than the stress itself, and
    an odd continuation of the slip would be too."""
    D = 1000.0
    errs = []
    for n in (32, 64):
        faults = np.array([_surface_fault(0.0, D, n)])
        doubled, _, _ = O.image_faults(faults)
        net2 = O.network(doubled, MU, CS)
        steps = int(O.mode_windows(2 * n, 2 * D, net2.dt, CS, 0.25, 0, 10 ** 6).max()) + 5
        V = np.zeros((steps, n))
        V[0] = 1.0 / net2.dt
        fs = O.half_space_stress_history(faults, MU, CS, V, dict(eta_w=0.25, q_w=0, flags=4, max_steps=steps))[2]
        net = O.network(faults, MU, CS)
        down = np.array([0.0, -1.0])
        ref = _dislocation_traction(net.x, net.nrm, -D * down, 1.0) + _dislocation_traction(net.x, net.nrm,
                                                                                               D * down, -1.0)
        alone = _dislocation_traction(net.x, net.nrm, np.zeros(2), 1.0) + _dislocation_traction(net.x, net.nrm,
                                                                                                D * down, -1.0)
        z = -net.x[:, 1]
        sel = (z > 0.05 * D) & (z < 0.8 * D)
        scale = np.abs(ref[sel]).max()
        errs.append(np.abs(fs[-1, sel] - ref[sel]).max() / scale)
        assert np.abs(fs[-1, sel] - alone[sel]).max() / scale > 1.0
    assert errs[1] < 0.05 and errs[0] / errs[1] > 1.6, errs


def test_half_space_response_is_even_across_the_surface():
    """P17b: on two parallel faults breaking the surface (different depths and element counts), the full-space
    tau of the doubled network under the evenly continued slip rate is itself even: each image element carries the
    stress of its real partner, self and interaction parts alike."""
    faults = np.array([_surface_fault(0.0, 300.0, 12), _surface_fault(140.0, 200.0, 10)])
    doubled, mirror, real = O.image_faults(faults)
    net2 = O.network(doubled, MU, CS)
    steps = 70
    V = np.random.default_rng(3).lognormal(size=(steps, 22))
    tau, _, fs, fi = O.stress_history(net2, V[:, mirror], dict(max_steps=steps, flags=2))
    partner = np.concatenate([net2.offset[f] + np.arange(2 * n)[::-1] for f, n in enumerate(faults[:, 4].astype(int))])
    for part in (tau, fs, fi):
        np.testing.assert_allclose(part[:, partner], part, rtol=1e-11, atol=1e-11 * np.abs(part).max())
    assert np.abs(fi).max() > 1e-3 * np.abs(fs).max()
    got = O.half_space_stress_history(faults, MU, CS, V, dict(max_steps=steps, flags=2))[0]
    np.testing.assert_array_equal(got, tau[:, real])


def test_image_faults_maps_and_rejects_networks_off_one_surface():
    """P17c: the index maps of a three-element fault, and the geometry checks (parallel faults, start ends on one
    line normal to them)."""
    doubled, mirror, real = O.image_faults(np.array([_surface_fault(0.0, 30.0, 3), _surface_fault(50.0, 20.0, 2)]))
    assert mirror.tolist() == [2, 1, 0, 0, 1, 2, 4, 3, 3, 4] and real.tolist() == [3, 4, 5, 8, 9]
    np.testing.assert_allclose(doubled[0], [0.0, 0.0, -math.pi / 2, 60.0, 6], atol=1e-12)
    with pytest.raises(ValueError):
        O.image_faults(np.array([_surface_fault(0.0, 30.0, 3), _surface_fault(50.0, 20.0, 2, phi=-1.2)]))
    bad = np.array([_surface_fault(0.0, 30.0, 3), _surface_fault(50.0, 20.0, 2)])
    bad[1, 1] -= 5.0
    with pytest.raises(ValueError):
        O.image_faults(bad)


def test_static_tail_with_cluster_windows_restores_the_dropped_history():
    """P16f: the static tail with a window per element pair (cluster-level truncation).  Slip rate only at step 0:
    once every block's window has passed the plain truncated sum is zero and the tail alone is left; it tends to the
    untruncated sum as the pair-level tail does (P14b), and before any window has ended it adds nothing.  Broadcast
    to element pairs, the fault-pair windows give the fault-pair tail (up to summation order)."""
    net = _two_small_faults()
    steps = 700
    V = np.zeros((steps, net.N))
    V[0] = np.linspace(1.0, 2.0, net.N)
    hp = dict(eta_tmin=0.01, eta_tmax=0.01, eta_w=1.5, q_w=0, max_steps=steps, leaf=2, eta_h=0.5, max_block=4)
    full = O.stress_history(net, V, dict(hp, flags=2))[3]
    trunc = O.stress_history(net, V, dict(hp, flags=16))[3]
    tail = O.stress_history(net, V, dict(hp, flags=16 | 4))[3]
    W = O.cluster_windows(net, 2, 0.5, 4, 0.01, steps)
    other = net.fault_of[:, None] != net.fault_of[None, :]
    _, _, P = O.pair_windows(net, 0.01, 0.01, steps)
    assert len(np.unique(W[other])) > 2 and (W[other] < P[net.fault_of][:, net.fault_of][other]).any()
    m0 = int(W.max()) + 1
    assert np.all(trunc[m0:] == 0)
    e = [np.linalg.norm(tail[m] - full[m]) / np.linalg.norm(full[m]) for m in (300, 690)]
    assert e[0] < 0.05 and e[1] < e[0] / 4 and e[1] < 1e-2
    first = int(W[other].min()) + 1
    assert np.all(tail[:first] == trunc[:first])
    delta = O.slip_from_rate(V, net.dt)
    pair_tail = O.static_tail_history(net, delta, P)
    np.testing.assert_allclose(O.static_tail_history(net, delta, P[net.fault_of][:, net.fault_of]), pair_tail,
                               rtol=1e-13, atol=1e-13 * np.abs(pair_tail).max())

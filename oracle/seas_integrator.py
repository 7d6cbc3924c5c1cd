"""CPU oracle of the earthquake-cycle time step on top of the stress-transfer functional (Ciardo & Romanet,
arXiv 2603.00383): rate-and-state friction (Eq. R&S_friction), the intermediate state evolution law
(Eq. state_evolution_law) and the second-order predictor-corrector step with a Newton solve of the force balance
(Sec. 2.4, "One-time-step integration").

TEST INFRASTRUCTURE ONLY, like ``oracle.seas_oracle``: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU legs may use it.  It builds on ``oracle.seas_oracle`` (the stress functional) and shares nothing with the CUDA
library.

What one step n (t_{n-1} -> t_n, fixed dt; the adaptive dt of step 1 of the scheme is not modelled) computes, in
plain FP64 NumPy, per element:

1. predictor: delta* = delta^{n-1} + dt V^{n-1}, theta* = theta^{n-1} + dt thetadot^{n-1};
2. the elastic stress at t_n without its instantaneous part: the spectral self term of delta* (Eq.
   funcational_discretized_form) plus the interaction sum over lags T >= 1 (Eq.
   fault-to-fault_interactions_discretized; lag 0 across faults is exactly zero for faults farther apart than
   c_s dt, which is checked);
3. Newton in u = ln V on  tau_known + tau^o - (mu / 2 c_s) V = sigma_n f(V, theta*)  to a relative residual of
   1e-8 (the radiation-damping term is the only instantaneous one), f = f_* + a ln(V / V_*) + b ln(V theta / D_c);
4. thetadot* = G(V*, theta*) with G of Eq. state_evolution_law;
5. corrector: the same with V^{n-1} -> (V^{n-1} + V*)/2 and thetadot^{n-1} -> (thetadot^{n-1} + thetadot*)/2 in
   steps 1-4; its V**, delta**, theta**, thetadot** are the new state.

Parity status (tests/test_oracle_pins.py, P15): the state law equals the aging law at eps = 1 and tends to the
slip law as eps -> 0; the Newton root equals an independent bisection; the benchmark's steady initial condition
stays at V_*; without elasticity the predictor-corrector converges to scipy's solution of the slider ODE at
second order.  The coupled network integration is pinned only through those parts (no printed values to compare).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from oracle import seas_oracle as O


@dataclass
class Friction:
    """Rate-and-state parameters (Table 1 names): a, b, D_c (m), f_* and V_* (m/s) of the reference steady state,
    background normal stress sigma_n (Pa, compressive positive) and the state-law parameter eps in (0, 1]
    (1: aging law)."""
    a: float
    b: float
    dc: float
    f0: float
    v0: float
    sigma_n: float
    eps: float = 1.0


def friction(V, theta, fr: Friction):
    """f_c = f_* + a ln(V / V_*) + b ln(V theta / D_c)   (Eq. R&S_friction)."""
    return fr.f0 + fr.a * np.log(V / fr.v0) + fr.b * np.log(V * theta / fr.dc)


def state_rate(V, theta, fr: Friction):
    """dtheta/dt = (1 / eps) [ (V theta / D_c)^(-eps) - 1 ] (V theta / D_c)   (Eq. state_evolution_law)."""
    omega = V * theta / fr.dc
    return (np.power(omega, -fr.eps) - 1.0) * omega / fr.eps


def solve_v(tau_known, theta, fr: Friction, rad: float, v_start, tol: float = 1e-8, max_iter: int = 100):
    """V > 0 with tau_known - rad V = sigma_n f(V, theta), rad = mu / (2 c_s), by Newton in u = ln V:
    g(u) = tau_known - rad e^u - sigma_n (f_* + (a + b) u - a ln V_* + b ln(theta / D_c)) decreases strictly, so the
    root is unique; iterations stop when |g| <= tol * (|tau_known| + sigma_n).  Returns (V, iterations)."""
    tau_known = np.asarray(tau_known, dtype=np.float64)
    u = np.log(np.asarray(v_start, dtype=np.float64) * np.ones_like(tau_known))
    c = fr.f0 - fr.a * math.log(fr.v0) + fr.b * np.log(theta / fr.dc)
    scale = np.abs(tau_known) + fr.sigma_n
    for it in range(1, max_iter + 1):
        ev = np.exp(u)
        g = tau_known - rad * ev - fr.sigma_n * (c + (fr.a + fr.b) * u)
        if np.all(np.abs(g) <= tol * scale):
            return ev, it
        dg = -rad * ev - fr.sigma_n * (fr.a + fr.b)
        step = -g / dg
        u = u + np.clip(step, -10.0, 10.0)       # damped in log space: at most a factor e^10 per iteration
    raise RuntimeError("Newton did not converge")


class Integrator:
    """Fixed-dt earthquake-cycle stepping of a network on top of the oracle's stress functional (untruncated
    windows).  tau0: background shear stress [N]; V0, theta0: initial slip rate and state [N]; no slip or slip
    history before t = 0."""

    def __init__(self, net: O.Network, fr: Friction, tau0, V0, theta0, max_steps: int):
        self.net, self.fr, self.max_steps = net, fr, max_steps
        self.tau0 = np.asarray(tau0, dtype=np.float64)
        self.rad = net.mu / (2.0 * net.cs)
        A = np.stack([O.interaction_slice(net, T) for T in range(max_steps)])
        if np.any(A[0] != 0.0):
            raise ValueError("faults within c_s dt of each other: the lag-0 interaction couples the Newton solves")
        self.A = A
        self.tables = []
        for f in range(net.F):
            n_f = int(net.n_elem[f])
            W = np.full(n_f + 1, max_steps - 1)
            self.tables.append(O.SelfTables(n_f, net.length[f], net.dt, net.cs, W))
        self.V = [np.asarray(V0, dtype=np.float64) * np.ones(net.N)]   # V^0 .. V^n (V^0: the initial rate)
        self.delta = [np.zeros(net.N)]
        self.theta = np.asarray(theta0, dtype=np.float64) * np.ones(net.N)
        self.thetadot = state_rate(self.V[0], self.theta, fr)
        self.iterations = []

    def _known_stress(self, delta_new):
        """Elastic stress at the new step without the radiation-damping term: spectral self term of the slip
        history ending in delta_new, interaction over lags T >= 1 of the slip-rate history."""
        net = self.net
        n = len(self.V)                                   # index of the new step
        hist = np.stack(self.delta[1:] + [delta_new])     # slip at steps 1 .. n (step 0 has zero slip)
        tau = np.zeros(net.N)
        for f in range(net.F):
            o0, o1 = net.offset[f], net.offset[f + 1]
            tau[o0:o1] = O.self_history(net, f, hist[:, o0:o1], self.tables[f])[-1]
        # V^1 .. V^{n-1} (V^0 is the initial rate, not a slip-rate history before t = 0)
        for T in range(1, n):
            tau += -self.rad * (self.A[T] @ self.V[n - T])
        return tau

    def step(self):
        """One predictor-corrector step; returns V^n."""
        net, fr, dt = self.net, self.fr, self.net.dt
        if len(self.V) >= self.max_steps:
            raise RuntimeError("max_steps reached")
        v_old, d_old, th_old, thd_old = self.V[-1], self.delta[-1], self.theta, self.thetadot
        # predictor
        d1 = d_old + dt * v_old
        th1 = th_old + dt * thd_old
        v1, it1 = solve_v(self._known_stress(d1) + self.tau0, th1, fr, self.rad, v_old)
        thd1 = state_rate(v1, th1, fr)
        # corrector
        d2 = d_old + dt * 0.5 * (v_old + v1)
        th2 = th_old + dt * 0.5 * (thd_old + thd1)
        v2, it2 = solve_v(self._known_stress(d2) + self.tau0, th2, fr, self.rad, v1)
        self.V.append(v2)
        self.delta.append(d2)
        self.theta = th2
        self.thetadot = state_rate(v2, th2, fr)
        self.iterations.append((it1, it2))
        return v2

    # ------------------------------------------------------------------------------------------------------------
    # Variable time step on the dt_min lattice (Sec. 2.4, step 1): a step of gamma lattice steps holds one slip rate
    # over the whole interval.
    # ------------------------------------------------------------------------------------------------------------

    def _known_stress_lattice(self, slips_new, v_push):
        """Elastic stress at the end of a step of gamma = len(slips_new) lattice steps, without the radiation-damping
        term: spectral self term of the lattice slip history ending in slips_new; interaction over lags T >= 1 of the
        lattice slip-rate history, in which the interval's own lattice steps (lags 1 .. gamma - 1) carry v_push, the
        rate the predictor (or corrector) holds over the interval."""
        net = self.net
        gamma = len(slips_new)
        n = len(self.V) + gamma - 1                       # lattice index of the new step
        hist = np.stack(self.delta[1:] + list(slips_new))
        tau = np.zeros(net.N)
        for f in range(net.F):
            o0, o1 = net.offset[f], net.offset[f + 1]
            tau[o0:o1] = O.self_history(net, f, hist[:, o0:o1], self.tables[f])[-1]
        Vh = self.V + [v_push] * (gamma - 1)              # lattice rates 0 .. n - 1 (0: the initial rate)
        for T in range(1, n):
            tau += -self.rad * (self.A[T] @ Vh[n - T])
        return tau

    def step_gamma(self, gamma: int):
        """One predictor-corrector step of gamma lattice steps (dt = gamma dt_min): the step's slip rate is held over
        its lattice steps (predictor: V^{n-1}; corrector: (V^{n-1} + V*)/2), the slip grows linearly along them, and
        the lattice history receives gamma copies of V** and the slips delta + j dt (V + V*)/2.  gamma = 1 is step().
        Returns V**."""
        net, fr, dt = self.net, self.fr, self.net.dt
        if len(self.V) + gamma > self.max_steps:
            raise RuntimeError("max_steps reached")
        v_old, d_old, th_old, thd_old = self.V[-1], self.delta[-1], self.theta, self.thetadot
        dtg = gamma * dt
        slips1 = [d_old + (j * dt) * v_old for j in range(1, gamma + 1)]
        th1 = th_old + dtg * thd_old
        v1, it1 = solve_v(self._known_stress_lattice(slips1, v_old) + self.tau0, th1, fr, self.rad, v_old)
        thd1 = state_rate(v1, th1, fr)
        vavg = 0.5 * (v_old + v1)
        slips2 = [d_old + (j * dt) * vavg for j in range(1, gamma + 1)]
        th2 = th_old + dtg * 0.5 * (thd_old + thd1)
        v2, it2 = solve_v(self._known_stress_lattice(slips2, vavg) + self.tau0, th2, fr, self.rad, v1)
        self.V += [v2] * gamma
        self.delta += slips2
        self.theta = th2
        self.thetadot = state_rate(v2, th2, fr)
        self.iterations.append((it1, it2))
        return v2

    def adaptive_gamma(self, xi: float, gamma_max: int) -> int:
        """gamma = ceil(dt_ev / dt_min), dt_ev = min_i xi D_c / V_i (Sec. 2.4, step 1), at least 1 and at most
        gamma_max.  xi is taken as a given constant (the paper refers its stiffness-dependent value elsewhere)."""
        dt_ev = float(np.min(xi * self.fr.dc / self.V[-1]))
        return int(min(gamma_max, max(1, math.ceil(dt_ev / self.net.dt))))

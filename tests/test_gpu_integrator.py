"""Earthquake-cycle stepping on the GPU (rate-and-state friction, intermediate state law, Newton, predictor-corrector;
Sec. 2.2, Sec. 2.4) against the CPU oracle's integrator, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import seas_integrator as SI
from oracle import seas_oracle as O
from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu

MU, CS = 32e9, 3464.0
FR = SI.Friction(a=0.01, b=0.015, dc=1e-3, f0=0.6, v0=1e-9, sigma_n=50e6)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(bump):
    faults = np.array([[0.0, 0.0, 0.2, 200.0, 8], [30.0, -300.0, 0.9, 160.0, 8]])
    net = O.network(faults, MU, CS)
    x = (np.arange(8) + 0.5) / 8
    tau0 = np.full(net.N, FR.f0 * FR.sigma_n + MU / (2 * CS) * FR.v0)
    tau0[:8] += bump * np.exp(-((x - 0.4) / 0.2) ** 2)          # a stress bump on fault 0 drives the slip
    return faults, net, tau0


@pytest.mark.parametrize("bump", [0.0, 1.5e6])
def test_integrator_matches_the_oracle_step_by_step(bump):
    steps = 60
    faults, net, tau0 = case(bump)
    ref = SI.Integrator(net, FR, tau0, FR.v0, FR.dc / FR.v0, max_steps=steps + 1)
    ref_V = np.array([ref.step() for _ in range(steps)])
    w = synth.Workload("integ", faults, mu=MU, cs=CS, steps=steps + 1,
                       hparams=dict(max_steps=steps + 1, leaf=4, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC))
    fr = (FR.a, FR.b, FR.dc, FR.f0, FR.v0, FR.sigma_n)
    with seas.Session(w) as s:
        it = seas.seas_integrator_create(s.scn, fr, 1.0, tau0, np.full(net.N, FR.v0), np.full(net.N, FR.dc / FR.v0))
        got_V = []
        for _ in range(steps):
            seas.seas_integrator_step(it, 1)
            got_V.append(seas.seas_integrator_state(it)[0])
        V, th, d = seas.seas_integrator_state(it)
        seas.seas_destroy_integrator(it)
    got_V = np.array(got_V)
    eV, eth, ed = rel(got_V, ref_V), rel(th, ref.theta), rel(d, ref.delta[-1])
    print(f"bump {bump:.1e}: V rises x{ref_V[-1].max() / FR.v0:.1f}; rel-L2 V {eV:.2e}, theta {eth:.2e}, "
          f"slip {ed:.2e}")
    if bump == 0.0:
        assert np.abs(got_V / FR.v0 - 1).max() < 1e-6               # the steady state stays put
    else:
        assert ref_V[-1].max() > 3 * FR.v0                         # the bump does drive the slip
    # both stop Newton at |residual| <= 1e-8 (|tau| + sigma_n); the iterates they stop at may differ by that much
    assert eV < 1e-6 and eth < 1e-6 and ed < 1e-6


def test_integrator_rejects_touching_faults_and_bad_parameters():
    w = synth.Workload("close", np.array([[0.0, 0.0, 0.0, 100.0, 4], [0.0, -6.0, 0.0, 100.0, 4]]), steps=10,
                       hparams=dict(max_steps=10, leaf=2, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC))
    fr = (FR.a, FR.b, FR.dc, FR.f0, FR.v0, FR.sigma_n)
    with seas.Session(w) as s:
        z = np.full(w.N, 1.0)
        with pytest.raises(seas.SeasError) as e:
            seas.seas_integrator_create(s.scn, fr, 1.0, z, z * 1e-9, z)
        assert e.value.status == seas.SEAS_EINVAL               # a lag-0 slice couples the faults
    faults, net, tau0 = case(0.0)
    w2 = synth.Workload("ok", faults, mu=MU, cs=CS, steps=10,
                        hparams=dict(max_steps=10, leaf=4, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC))
    with seas.Session(w2) as s:
        z = np.full(w2.N, 1.0)
        for bad in ((0.0,) + fr[1:], fr[:5] + (-1.0,)):
            with pytest.raises(seas.SeasError):
                seas.seas_integrator_create(s.scn, bad, 1.0, tau0, z * 1e-9, z)
        with pytest.raises(seas.SeasError):
            seas.seas_integrator_create(s.scn, fr, 0.0, tau0, z * 1e-9, z)


def test_multi_step_push_equals_the_lattice_functional():
    """A slip rate held over gamma lattice steps (seas_push_slip_rate_steps) is the functional of the lattice history
    with that rate repeated gamma times (oracle stress_history on the expanded lattice), at every step's end; with
    the caller's end slip, and through replace_last of a whole multi-step push."""
    w = synth.tiny(2, n_faults=3, steps=200)
    net = O.network(w.faults, w.mu, w.cs)
    gammas = [1, 3, 2, 5, 1, 4, 7, 2, 6, 3, 1, 5]
    rates = w.slip_rate(0, 0, len(gammas))
    lattice = np.concatenate([np.repeat(rates[k][None], g, 0) for k, g in enumerate(gammas)])
    ref = O.stress_history(net, lattice, dict(w.hparams, flags=seas.SEAS_FLAG_NO_TRUNC, max_steps=w.steps))
    ends = np.cumsum(gammas) - 1
    slip_lat = O.slip_from_rate(lattice, net.dt)
    for mode in ("integrated", "caller_slip", "replaced"):
        with seas.Session(w, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC) as s:
            t = np.zeros(w.N)
            P = np.zeros(3 * w.N)
            out = []
            for k, g in enumerate(gammas):
                V = np.ascontiguousarray(rates[k])
                if mode == "caller_slip":
                    seas.seas_push_slip_rate_steps(s.scn, V, g, slip=np.ascontiguousarray(slip_lat[ends[k]]))
                elif mode == "replaced":
                    seas.seas_push_slip_rate_steps(s.scn, 3.0 * V + 1.0, g)
                    seas.seas_push_slip_rate_steps(s.scn, V, g, replace_last=True)
                else:
                    seas.seas_push_slip_rate_steps(s.scn, V, g)
                seas.seas_stress_step(s.scn, t, parts=P)
                out.append(np.concatenate([t, P]))
            if mode == "replaced":
                with pytest.raises(seas.SeasError) as e:
                    seas.seas_push_slip_rate_steps(s.scn, V, gammas[-1] + 1, replace_last=True)
                assert e.value.status == seas.SEAS_EINVAL
        out = np.array(out)
        errs = [rel(out[:, :w.N], ref[0][ends])] + [rel(out[:, (k + 1) * w.N:(k + 2) * w.N], ref[k + 1][ends])
                                                   for k in range(3)]
        print(f"multi-step push ({mode}): rel-L2 tau/rad/self/int {errs}")
        assert max(errs) <= 1e-10


def test_gamma_and_adaptive_steps_match_the_oracle():
    """Time steps of several lattice steps (Sec. 2.4 step 1) on the GPU against the oracle's gamma steps: a fixed
    gamma sequence, then adaptive steps whose gamma the GPU picks from min xi D_c / V and the oracle recomputes."""
    steps = 160
    faults, net, tau0 = case(1.5e6)
    fr = (FR.a, FR.b, FR.dc, FR.f0, FR.v0, FR.sigma_n)
    w = synth.Workload("integ", faults, mu=MU, cs=CS, steps=steps,
                       hparams=dict(max_steps=steps, leaf=4, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC))
    gammas = [1, 2, 4, 3, 8, 5, 2, 6]
    ref = SI.Integrator(net, FR, tau0, FR.v0, FR.dc / FR.v0, max_steps=steps)
    ref_V = [ref.step_gamma(g) for g in gammas]
    with seas.Session(w) as s:
        it = seas.seas_integrator_create(s.scn, fr, 1.0, tau0, np.full(net.N, FR.v0), np.full(net.N, FR.dc / FR.v0))
        got_V = []
        for g in gammas:
            seas.seas_integrator_step_gamma(it, g)
            got_V.append(seas.seas_integrator_state(it)[0])
        # adaptive: xi chosen so that gamma stays between 1 and 12 on this run
        xi = 12 * net.dt * FR.v0 / FR.dc
        adaptive_ref, adaptive_got = [], []
        for _ in range(6):
            g = ref.adaptive_gamma(xi, 12)
            if len(ref.V) + g > steps:
                break
            adaptive_ref.append(g)
            ref.step_gamma(g)
            adaptive_got.append(seas.seas_integrator_step_adaptive(it, xi, 12, 1))
        V, th, d = seas.seas_integrator_state(it)
        seas.seas_destroy_integrator(it)
    eV = rel(np.array(got_V), np.array(ref_V))
    print(f"gamma steps {gammas}: rel-L2 V {eV:.2e}; adaptive gammas GPU {adaptive_got} oracle {adaptive_ref}; "
          f"final rel-L2 V {rel(V, ref.V[-1]):.2e} theta {rel(th, ref.theta):.2e} slip {rel(d, ref.delta[-1]):.2e}")
    assert eV < 1e-6
    assert adaptive_got == adaptive_ref and max(adaptive_ref) > 1
    assert rel(V, ref.V[-1]) < 1e-6 and rel(th, ref.theta) < 1e-6 and rel(d, ref.delta[-1]) < 1e-6

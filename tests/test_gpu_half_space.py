"""A traction-free surface by the method of images (App. B) through the C ABI: faults whose start end breaks the
surface (SEAS_FAULT_SURFACE_START) against the oracle's doubled network with the slip continued evenly, for the
stress step (one fault; two parallel faults through the H-matrix) and for the earthquake-cycle integrator."""
import math

import numpy as np
import pytest

from oracle import seas_integrator as SI
from oracle import seas_oracle as O
from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu

MU, CS = 32e9, 3464.0
S = seas.SEAS_FAULT_SURFACE_START


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def surface_fault(x0, depth, n, phi=-math.pi / 2):
    e1 = (math.cos(phi), math.sin(phi))
    return [x0 + 0.5 * depth * e1[0], 0.5 * depth * e1[1], phi, depth, n, S]


def run(w, steps, **hp):
    V = w.slip_rate(0, 0, steps)
    tau = np.zeros((steps, w.N))
    P = np.zeros((steps, 3, w.N))
    t, p = np.zeros(w.N), np.zeros(3 * w.N)
    with seas.Session(w, **hp) as s:
        info = seas.seas_net_get_info(s.net)
        cen, _ = seas.seas_net_get_elements(s.net)
        stats = s.stats
        for n in range(steps):
            seas.seas_push_slip_rate(s.scn, np.ascontiguousarray(V[n]))
            seas.seas_stress_step(s.scn, t, parts=p)
            tau[n], P[n] = t, p.reshape(3, w.N)
    return V, tau, P, info, cen, stats


def test_surface_fault_matches_the_doubled_network_of_the_oracle():
    """One 640 m fault of 64 elements from the surface down (the single-fault problem of App. B at small size),
    300 steps with the self windows of the doubled fault: tau and its parts equal the oracle's full-space functional
    of the doubled fault under the evenly continued slip rate, on the real elements; the library reports the real
    elements only.  The surface changes tau against the fault alone in a full space."""
    steps = 300
    faults = np.array([surface_fault(0.0, 640.0, 64)])
    w = synth.Workload("surface1", faults, mu=MU, cs=CS, steps=steps, hparams=dict(max_steps=steps, leaf=16))
    V, tau, P, info, cen, _ = run(w, steps)
    assert info["n_elem"] == 64
    np.testing.assert_allclose(cen, O.network(faults[:, :5], MU, CS).x, atol=1e-9)
    ref = O.half_space_stress_history(faults[:, :5], MU, CS, V, w.hparams)
    alone = O.stress_history(O.network(faults[:, :5], MU, CS), V, w.hparams)
    errs = [rel(tau, ref[0]), rel(P[:, 0], ref[1]), rel(P[:, 1], ref[2])]
    print(f"surface fault: rel-L2 tau/rad/self {errs}; surface vs full space {rel(ref[0], alone[0]):.2e}")
    assert max(errs) <= 1e-10
    assert np.abs(P[:, 2]).max() == 0.0
    assert rel(ref[0], alone[0]) > 1e-3


@pytest.mark.parametrize("mode", ["dense", "hmatrix"])
def test_parallel_surface_faults_match_the_oracle(mode):
    """Two parallel faults breaking the surface (400 m / 48 elements and 300 m / 32 elements, 150 m apart): each
    doubled fault carries its image, so the interaction includes the images of the other fault; windows truncate
    inside the 260 steps.  Exact with dense blocks, at the ACA tolerance with low-rank far blocks."""
    steps = 260
    faults = np.array([surface_fault(0.0, 400.0, 48), surface_fault(150.0, 300.0, 32)])
    hp = dict(max_steps=steps, leaf=8, eta_h=1.0, eta_tmax=0.01)
    w = synth.Workload("surface2", faults, mu=MU, cs=CS, steps=steps, hparams=hp)
    extra = dict(flags=seas.SEAS_FLAG_DENSE) if mode == "dense" else dict(aca_tol=1e-10)
    V, tau, P, info, _, stats = run(w, steps, **extra)
    assert info["n_elem"] == 80
    ref = O.half_space_stress_history(faults[:, :5], MU, CS, V, dict(hp, **extra))
    errs = [rel(tau, ref[0]), rel(P[:, 0], ref[1]), rel(P[:, 1], ref[2]), rel(P[:, 2], ref[3])]
    print(f"two surface faults ({mode}): rel-L2 tau/rad/self/int {errs}; far blocks {stats['n_blocks_far']}")
    assert max(errs) <= (1e-10 if mode == "dense" else 1e-8)
    assert np.abs(ref[3]).max() > 1e-3 * np.abs(ref[2]).max()
    if mode == "hmatrix":
        assert stats["n_blocks_far"] > 0


def test_integrator_on_a_surface_fault_matches_the_oracle_on_the_doubled_fault():
    """The earthquake-cycle integrator on a fault breaking the surface (state on the real elements only) against
    the oracle's integrator on the doubled fault with mirrored initial conditions, whose real half it must follow
    (the Newton solve stops at |residual| <= 1e-8, so iterates may differ by that much)."""
    steps = 50
    fr = SI.Friction(a=0.01, b=0.015, dc=1e-3, f0=0.6, v0=1e-9, sigma_n=50e6)
    faults = np.array([surface_fault(0.0, 200.0, 16)])
    z = (np.arange(16) + 0.5) / 16
    tau0 = fr.f0 * fr.sigma_n + MU / (2 * CS) * fr.v0 + 1.5e6 * np.exp(-((z - 0.3) / 0.2) ** 2)
    doubled, mirror, real = O.image_faults(faults[:, :5])
    ref = SI.Integrator(O.network(doubled, MU, CS), fr, tau0[mirror], fr.v0, fr.dc / fr.v0, max_steps=steps + 1)
    ref_V = np.array([ref.step()[real] for _ in range(steps)])
    w = synth.Workload("surface_integ", faults, mu=MU, cs=CS, steps=steps + 1,
                       hparams=dict(max_steps=steps + 1, leaf=4, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC))
    with seas.Session(w) as s:
        it = seas.seas_integrator_create(s.scn, (fr.a, fr.b, fr.dc, fr.f0, fr.v0, fr.sigma_n), 1.0, tau0,
                                         np.full(16, fr.v0), np.full(16, fr.dc / fr.v0))
        got_V = []
        for _ in range(steps):
            seas.seas_integrator_step(it, 1)
            got_V.append(seas.seas_integrator_state(it)[0])
        V, th, d = seas.seas_integrator_state(it)
        seas.seas_destroy_integrator(it)
    got_V = np.array(got_V)
    eV, eth, ed = rel(got_V, ref_V), rel(th, ref.theta[real]), rel(d, ref.delta[-1][real])
    print(f"surface integrator: V rises x{ref_V[-1].max() / fr.v0:.1f}; rel-L2 V {eV:.2e}, theta {eth:.2e}, "
          f"slip {ed:.2e}")
    assert ref_V[-1].max() > 3 * fr.v0
    assert eV < 1e-6 and eth < 1e-6 and ed < 1e-6


def test_surface_networks_off_one_surface_are_rejected():
    ok = surface_fault(0.0, 100.0, 8)
    tilted = surface_fault(60.0, 100.0, 8, phi=-1.3)
    lower = surface_fault(60.0, 100.0, 8)
    lower[1] -= 10.0
    free = list(ok[:5]) + [0]
    with seas.Session(synth.Workload("s", np.array([ok]), steps=4, hparams=dict(max_steps=4))):
        pass
    for bad in ([ok, tilted], [ok, lower], [ok, free]):
        w = synth.Workload("bad", np.array(bad), steps=4, hparams=dict(max_steps=4))
        with pytest.raises(seas.SeasError) as e:
            seas.Session(w)
        assert e.value.status == seas.SEAS_EINVAL


def test_surface_faults_in_an_eight_scenario_bf16_batch():
    """The tensor-core BF16 path with 8 scenarios on two parallel surface faults: member b pushed (1 + b / 8) times
    the rates gets that multiple of the oracle's half-space stress (the functional is linear): self and radiation
    parts in FP64 within 1e-10, the BF16 interaction within the BF16 bound of the parity tests (5e-3)."""
    steps = 200
    faults = np.array([surface_fault(0.0, 400.0, 48), surface_fault(150.0, 300.0, 32)])
    hp = dict(max_steps=steps, leaf=8, eta_h=1.0, eta_tmax=0.01)
    w = synth.Workload("surface2_b8", faults, mu=MU, cs=CS, steps=steps, hparams=hp)
    V = w.slip_rate(0, 0, steps)
    scale = 1.0 + np.arange(8) / 8.0
    P = np.zeros((steps, 3, 8, w.N))
    p = np.zeros(3 * 8 * w.N)
    t = np.zeros(8 * w.N)
    with seas.Session(w, batch=8, precision=seas.SEAS_PREC_BF16) as s:
        for n in range(steps):
            seas.seas_push_slip_rate(s.scn, np.concatenate([c * V[n] for c in scale]))
            seas.seas_stress_step(s.scn, t, parts=p)
            P[n] = p.reshape(3, 8, w.N)
    ref = O.half_space_stress_history(faults[:, :5], MU, CS, V, hp)
    worst = [0.0, 0.0, 0.0]
    for b, c in enumerate(scale):
        for k in range(3):
            worst[k] = max(worst[k], rel(P[:, k, b], c * ref[k + 1]))
    print(f"surface faults, BF16 x 8: worst member rel-L2 rad/self/int {worst}")
    assert worst[0] <= 1e-10 and worst[1] <= 1e-10 and worst[2] <= 5e-3

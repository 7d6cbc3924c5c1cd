"""Intersecting faults (the X-shaped network of Sec. 3.2) and fault sizes with the odd prime radices up to 23 (the
paper's 510-element faults are 2 * 3 * 5 * 17), through the C ABI against the oracle; and the compression trend of
Table 3 as the interaction window grows."""
import numpy as np
import pytest

from oracle import seas_oracle as O
from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu

EXACT = 1e-10
DENSE_EXACT = dict(flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(w, **hp):
    V = w.slip_rate(0, 0, w.steps)
    tau = np.zeros((w.steps, w.N))
    P = np.zeros((w.steps, 3, w.N))
    t, p = np.zeros(w.N), np.zeros(3 * w.N)
    with seas.Session(w, **hp) as s:
        for n in range(w.steps):
            seas.seas_push_slip_rate(s.scn, np.ascontiguousarray(V[n]))
            seas.seas_stress_step(s.scn, t, parts=p)
            tau[n], P[n] = t, p.reshape(3, w.N)
        stats = s.stats
    return V, tau, P, stats


@pytest.mark.parametrize("mode", ["dense", "hmatrix"])
def test_x_shaped_faults_crossing_at_an_element_boundary(mode):
    """Two faults crossing at their midpoints (an element boundary, Sec. 3.2): receivers next to the crossing sit
    within half an element of the other fault, and the lag-0 interaction across the crossing is nonzero.  There the
    oracle's plain four-term difference of the primitives loses digits in FP64 (5.6e-10 against its own
    extended-precision evaluation on this network), so the interaction part is compared with the oracle evaluated
    in extended precision; tau, radiation and self parts with the FP64 oracle."""
    L, n, steps = 100.0, 40, 90
    w = synth.Workload("x40", np.array([[0.0, 0.0, 0.6, L, n], [0.0, 0.0, -0.6, L, n]]), mu=30e9, steps=steps,
                       hparams=dict(max_steps=steps, leaf=4, flags=seas.SEAS_FLAG_NO_TRUNC))
    hp = DENSE_EXACT if mode == "dense" else dict(leaf=4, eta_h=1.0, aca_tol=1e-13, flags=seas.SEAS_FLAG_NO_TRUNC)
    V, tau, P, stats = run(w, **hp)
    net = O.network(w.faults, w.mu, w.cs)
    ref = O.stress_history(net, V, dict(w.hparams, flags=seas.SEAS_FLAG_NO_TRUNC))
    ref_int = O.interaction_history(net, V, dtype=np.longdouble).astype(np.float64)
    assert np.any(O.interaction_slice(net, 0) != 0)            # the crossing couples the faults at lag 0
    if mode == "hmatrix":
        assert stats["n_blocks_far"] > 0
    errs = [rel(tau, ref[0]), rel(P[:, 0], ref[1]), rel(P[:, 1], ref[2]), rel(P[:, 2], ref_int)]
    print(f"X faults ({mode}): rel-L2 tau/rad/self/int(extended) {errs}; FP64 oracle's own interaction error "
          f"{rel(ref[3], ref_int):.2e}")
    assert max(errs) <= EXACT


def test_fault_sizes_with_the_odd_prime_radices():
    """Self terms of faults of 14, 22, 26, 34, 38 and 46 elements (radices 7, 11, 13, 17, 19, 23) against the
    oracle's direct DFT."""
    sizes = [14, 22, 26, 34, 38, 46]
    faults = np.array([[0.0, 300.0 * k, 0.1 * k, 2.0 * n, n] for k, n in enumerate(sizes)])
    w = synth.Workload("radix", faults, steps=60, hparams=dict(max_steps=60, leaf=8, flags=seas.SEAS_FLAG_NO_TRUNC))
    V, tau, P, _ = run(w, **DENSE_EXACT)
    net = O.network(w.faults, w.mu, w.cs)
    ref = O.stress_history(net, V, dict(w.hparams, flags=seas.SEAS_FLAG_NO_TRUNC))
    for f, n in enumerate(sizes):
        cols = slice(net.offset[f], net.offset[f + 1])
        e = rel(P[:, 1, cols], ref[2][:, cols])
        assert e <= EXACT, (n, e)
    assert rel(tau, ref[0]) <= EXACT


def test_x_fault_compression_falls_as_the_interaction_window_grows():
    """Table 3's trend on the X-shaped network of Table 2 (2 x 510 elements, leaf 50, eta_H 1.5, tolerance 1e-4):
    as eta_Tmax grows from 0.01 to 2 the windows lengthen and the stored fraction of the causal dense operator
    falls (the late lags compress better); the printed ratios (51.5, 44.8, 28.2, 25.0 %) come from the paper's SVD
    and its windows, so only the trend and the rough level are compared."""
    faults = np.array([[0.0, 0.0, 0.6, 1000.0, 510], [0.0, 0.0, -0.6, 1000.0, 510]])
    ratios, lasts = [], []
    for eta in (0.01, 0.1, 1.0, 2.0):
        w = synth.Workload("x510", faults, mu=30e9, steps=2600,
                           hparams=dict(leaf=50, eta_h=1.5, aca_tol=1e-4, eta_tmin=0.01, eta_tmax=eta, eta_w=1.5,
                                        q_w=102, max_steps=2600))
        with seas.Session(w) as s:
            ratios.append(s.stats["compression_ratio"])
            lasts.append(int(seas.seas_op_pair_windows(s.op).max()))
    print("X faults: eta_Tmax 0.01, 0.1, 1, 2 -> last lags", lasts, "compression %", [round(r, 2) for r in ratios])
    assert lasts == sorted(lasts) and lasts[0] < lasts[-1]
    assert all(a > b for a, b in zip(ratios, ratios[1:]))
    assert 10.0 < ratios[-1] < ratios[0] < 90.0

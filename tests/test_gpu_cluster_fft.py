"""Faults of N_f >= 2048 elements run their FFTs on a thread-block cluster (four-step transform over distributed
shared memory): the self term of such faults against the oracle's direct DFTs, in a full space and doubled across
a free surface, and for a two-scenario batch."""
import math

import numpy as np
import pytest

from oracle import seas_oracle as O
from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu

STEPS = 4


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(w, batch=1, scale=(1.0,)):
    V = w.slip_rate(0, 0, STEPS)
    out = np.zeros((STEPS, batch, 3, w.N))
    t, p = np.zeros(batch * w.N), np.zeros(3 * batch * w.N)
    with seas.Session(w, batch=batch) as s:
        for n in range(STEPS):
            seas.seas_push_slip_rate(s.scn, np.concatenate([c * V[n] for c in scale]))
            seas.seas_stress_step(s.scn, t, parts=p)
            out[n] = p.reshape(3, batch, w.N).transpose(1, 0, 2)
    return V, out


@pytest.mark.parametrize("case", ["full_space_2560", "surface_1024"])
def test_large_fault_self_term_matches_the_oracle(case):
    """N_f = 2560 (four-step 40 x 64, radices 4, 2, 5 and 4, 4, 4) in a full space; a 1024-element fault breaking
    the surface, doubled to 2048 (32 x 64): radiation and self parts within 1e-10 of the oracle over 4 steps."""
    if case == "full_space_2560":
        faults = np.array([[0.0, 0.0, 0.3, 25600.0, 2560]])
    else:
        faults = np.array([[0.0, -5120.0, -0.5 * math.pi, 10240.0, 1024, seas.SEAS_FAULT_SURFACE_START]])
    w = synth.Workload(case, faults, steps=STEPS, hparams=dict(max_steps=STEPS))
    V, P = run(w)
    if case == "full_space_2560":
        ref = O.stress_history(O.network(faults, w.mu, w.cs), V, w.hparams)
    else:
        ref = O.half_space_stress_history(faults[:, :5], w.mu, w.cs, V, w.hparams)
    errs = [rel(P[:, 0, 0], ref[1]), rel(P[:, 0, 1], ref[2])]
    print(f"{case}: rel-L2 rad/self {errs}")
    assert max(errs) <= 1e-10


def test_large_fault_batch_members_are_independent():
    """A two-scenario batch on a 2048-element fault: the second member, pushed twice the first one's rates, gets
    twice its stress (the functional is linear), so the cluster kernels index the scenarios apart."""
    w = synth.Workload("batch2048", np.array([[0.0, 0.0, -0.2, 20480.0, 2048]]), steps=STEPS,
                       hparams=dict(max_steps=STEPS))
    _, P = run(w, batch=2, scale=(1.0, 2.0))
    np.testing.assert_allclose(P[:, 1], 2.0 * P[:, 0], rtol=1e-12, atol=1e-12 * np.abs(P).max())
    assert np.abs(P[:, 0, 1]).max() > 0

"""The allocation-free stress step (seas_stress_step_static) against the ordinary one, through the C ABI.

Both entry points run the same kernels; the static one takes its per-call scratch from a static device array shared
by every call in the process.  Two consecutive steps are checked on each of two workloads taken in turn, so the
second workload starts from the scratch contents the first one left behind.
"""
import numpy as np
import pytest

from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu

EXACT = 1e-10


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


@pytest.mark.parametrize("case", ["two_fault_hmatrix_batch2", "tiny_dense", "two_fault_truncated_first_steps"])
def test_static_step_matches_stress_step(case):
    """The third case runs after the others have filled the array: its first steps, with truncated windows and
    before the waves reach the other fault, leave most interaction tasks inactive, so stale scratch would show."""
    torch = pytest.importorskip("torch")
    if case == "two_fault_hmatrix_batch2":
        w, batch, hp = synth.two_fault_128(), 2, dict(flags=seas.SEAS_FLAG_NO_TRUNC, eta_h=2.0, leaf=32, aca_tol=1e-6)
        first, count = w.steps // 2, 2
    elif case == "tiny_dense":
        w, batch = synth.tiny(3, n_faults=3, steps=60), 1
        hp = dict(flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC)
        first, count = w.steps // 2, 2
    else:
        w, batch, hp = synth.two_fault_128(), 1, dict(flags=0, eta_h=2.0, leaf=32, aca_tol=1e-6)
        first, count = 0, 3
    V = np.stack([w.slip_rate(b, 0, first + count) for b in range(batch)], axis=1).reshape(first + count, -1)
    with seas.Session(w, batch=batch, **hp) as s:
        BN = batch * s.op.N
        assert V.shape[1] == BN
        Vd = torch.from_numpy(V).cuda()
        tau = torch.zeros(BN, dtype=torch.float64, device="cuda")
        parts = torch.zeros(3 * BN, dtype=torch.float64, device="cuda")
        tau_s = torch.full_like(tau, float("nan"))
        parts_s = torch.full_like(parts, float("nan"))
        for n in range(first):
            seas.seas_push_slip_rate(s.scn, Vd[n])
            seas.seas_stress_step(s.scn, tau, parts=parts)
        for n in range(first, first + count):          # calls in a row
            seas.seas_push_slip_rate(s.scn, Vd[n])
            seas.seas_stress_step(s.scn, tau, parts=parts)
            seas.seas_stress_step_static(s.scn, tau_s, parts=parts_s)
            seas.seas_scenario_check(s.scn)
            torch.cuda.synchronize()
            a, b = tau_s.cpu().numpy(), tau.cpu().numpy()
            pa, pb = parts_s.cpu().numpy().reshape(3, BN), parts.cpu().numpy().reshape(3, BN)
            assert np.all(np.isfinite(a)) and np.abs(b).max() > 0
            assert rel(a, b) <= EXACT, (case, n)
            for k in range(3):
                assert rel(pa[k], pb[k]) <= EXACT, (case, n, k)
            tau_s.fill_(float("nan"))
            parts_s.fill_(float("nan"))

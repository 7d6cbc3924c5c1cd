"""Bitwise reproducibility of the interaction at full history depth, where every CTA of the persistent kernel takes
many tasks from the dynamic counter in an order that varies from run to run: two scenarios stepped with the same
slip rates on the same operator give the same tau, bit for bit (no atomics; each task's sums follow an order that
the task alone fixes)."""
import numpy as np
import pytest

from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,batch", [(seas.SEAS_PREC_FP64, 1), (seas.SEAS_PREC_BF16, 8), (seas.SEAS_PREC_BF16, 1),
                                        (seas.SEAS_PREC_DF64, 1)])
def test_two_runs_at_depth_are_bitwise_equal(prec, batch):
    torch = pytest.importorskip("torch")
    steps, K = 2000, 6
    w = synth.six_fault_3072(steps=steps)
    V = np.stack([w.slip_rate(b, 0, steps) for b in range(batch)], axis=1).reshape(steps, -1)
    Vd = torch.from_numpy(V).cuda()
    with seas.Session(w, batch=batch, precision=prec) as s:
        runs = []
        for _ in range(2):
            scn = seas.seas_scenario_create(s.op, batch)
            tau = torch.zeros(batch * w.N, dtype=torch.float64, device="cuda")
            out = []
            for n in range(steps):
                seas.seas_push_slip_rate(scn, Vd[n])
                seas.seas_stress_step(scn, tau)
                if n >= steps - K:
                    out.append(tau.clone())
            seas.seas_scenario_check(scn)
            seas.seas_destroy_scn(scn)
            runs.append(torch.stack(out).cpu().numpy())
    assert np.abs(runs[0]).max() > 0
    np.testing.assert_array_equal(runs[0], runs[1])

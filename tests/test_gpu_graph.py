"""A step captured as a CUDA graph and replayed (seas_scenario_graph_create / _step) gives the same tau, bit for bit,
as seas_push_slip_rate + seas_stress_step, also when the two are interleaved, when the windows are still opening,
and for an 8-member BF16 batch on the tensor-core consumers."""
import numpy as np
import pytest

from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["tiny_hmatrix_fp64", "two_fault_bf16_batch8", "six_fault_truncated_fp64"])
def test_graph_steps_equal_ordinary_steps(case):
    torch = pytest.importorskip("torch")
    if case == "tiny_hmatrix_fp64":
        w, B, hp, steps = synth.tiny(2, n_faults=3, steps=120), 1, dict(leaf=8, eta_h=3.0, aca_tol=1e-13), 120
    elif case == "two_fault_bf16_batch8":
        w, B, hp, steps = synth.two_fault_128(), 8, dict(precision=seas.SEAS_PREC_BF16), 120
    else:
        w, B, hp, steps = synth.six_fault_3072(steps=300), 1, {}, 300
    V = np.stack([w.slip_rate(b, 0, steps) for b in range(B)], axis=1).reshape(steps, -1)
    Vd = torch.from_numpy(V).cuda()
    BN = B * w.N
    out = {}
    for mode in ("plain", "graph", "mixed"):
        with seas.Session(w, batch=B, **hp) as s:
            tau = torch.zeros(BN, dtype=torch.float64, device="cuda")
            vbuf = torch.zeros(BN, dtype=torch.float64, device="cuda")
            res = []
            if mode != "plain":
                seas.seas_scenario_graph_create(s.scn, vbuf, tau)
            for n in range(steps):
                if mode == "graph" or (mode == "mixed" and (n // 7) % 2 == 1):
                    vbuf.copy_(Vd[n])
                    seas.seas_scenario_graph_step(s.scn)
                else:
                    seas.seas_push_slip_rate(s.scn, Vd[n])
                    seas.seas_stress_step(s.scn, tau)
                res.append(tau.clone())
            seas.seas_scenario_check(s.scn)
            out[mode] = torch.stack(res).cpu().numpy()
            assert seas.seas_scenario_step(s.scn) == steps
    assert np.abs(out["plain"]).max() > 0
    np.testing.assert_array_equal(out["graph"], out["plain"])
    np.testing.assert_array_equal(out["mixed"], out["plain"])


def test_graph_capture_rules():
    torch = pytest.importorskip("torch")
    w = synth.tiny(1, steps=20)
    with seas.Session(w, flags=seas.SEAS_FLAG_DENSE | seas.SEAS_FLAG_NO_TRUNC) as s:
        v = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        t = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        with pytest.raises(seas.SeasError) as e:
            seas.seas_scenario_graph_step(s.scn)
        assert e.value.status == seas.SEAS_ESTATE
        seas.seas_scenario_set_timing(s.scn, True)
        with pytest.raises(seas.SeasError) as e:
            seas.seas_scenario_graph_create(s.scn, v, t)
        assert e.value.status == seas.SEAS_ESTATE
        seas.seas_scenario_set_timing(s.scn, False)
        seas.seas_scenario_graph_create(s.scn, v, t)
        for _ in range(20):
            seas.seas_scenario_graph_step(s.scn)
        with pytest.raises(seas.SeasError) as e:
            seas.seas_scenario_graph_step(s.scn)                # past max_steps
        assert e.value.status == seas.SEAS_ESTATE

"""The interaction autotuner (seas_scenario_autotune): it picks, per pass, one of the consumer-warp counts compiled
for the precision and batch by timing them; the choice is cached by key and reapplied without timing; the tuned
scenario gives the untuned one's tau up to the summation order of the reductions; a captured graph fixes the
kernels (SEAS_ESTATE)."""
import numpy as np
import pytest

from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,batch,tol", [(seas.SEAS_PREC_FP64, 1, 1e-13), (seas.SEAS_PREC_BF16, 8, 1e-6),
                                            (seas.SEAS_PREC_DF64, 1, 1e-13)])
def test_autotune_choice_cache_and_result(tmp_path, prec, batch, tol):
    torch = pytest.importorskip("torch")
    steps = 400
    w = synth.six_fault_3072(steps=steps)
    V = np.stack([w.slip_rate(b, 0, steps) for b in range(batch)], axis=1).reshape(steps, -1)
    Vd = torch.from_numpy(V).cuda()
    cache = tmp_path / "tune.txt"
    with seas.Session(w, batch=batch, precision=prec) as s:
        plain = seas.seas_scenario_create(s.op, batch)
        tuned = seas.seas_scenario_create(s.op, batch)
        t = seas.seas_scenario_autotune(tuned, cache, reps=3)
        for p in ("source", "receiver"):
            assert t["consumer_warps"][p] in t["ms"][p]
            assert all(v > 0 for v in t["ms"][p].values())
            assert set(t["ms"][p]) <= {8, 16}
        assert not t["from_cache"]
        again = seas.seas_scenario_create(s.op, batch)
        t2 = seas.seas_scenario_autotune(again, cache, reps=3)
        assert t2["from_cache"] and t2["consumer_warps"] == t["consumer_warps"]
        assert cache.read_text().count("\n") == 1
        out = {}
        for name, scn in (("plain", plain), ("tuned", tuned)):
            tau = torch.zeros(batch * w.N, dtype=torch.float64, device="cuda")
            res = []
            for n in range(steps):
                seas.seas_push_slip_rate(scn, Vd[n])
                seas.seas_stress_step(scn, tau)
                if n % 40 == 39:
                    res.append(tau.clone())
            seas.seas_scenario_check(scn)
            out[name] = torch.stack(res).cpu().numpy()
        scale = np.abs(out["plain"]).max()
        assert scale > 0
        assert np.abs(out["tuned"] - out["plain"]).max() <= tol * scale
        # a captured step fixes its kernels
        v = torch.zeros(batch * w.N, dtype=torch.float64, device="cuda")
        tt = torch.zeros(batch * w.N, dtype=torch.float64, device="cuda")
        seas.seas_scenario_graph_create(again, v, tt)
        with pytest.raises(seas.SeasError) as e:
            seas.seas_scenario_autotune(again, None, reps=1)
        assert e.value.status == seas.SEAS_ESTATE
        for h in (plain, tuned, again):
            seas.seas_destroy_scn(h)

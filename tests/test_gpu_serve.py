"""Serving on the GPU: requests admitted into shared slot groups at different ticks (continuous batching), on two
geometries at once, give each request the result it gets when run alone, and the member API of the C ABI behaves."""
import numpy as np
import pytest

from paper_2603_00383_gb300 import seas, serve, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def geometries(precision=0):
    out = []
    for seed in (2, 3):
        w = synth.tiny(seed, n_faults=3, steps=80)
        w.hparams = dict(w.hparams, leaf=8, eta_h=3.0, aca_tol=1e-13, precision=precision)
        out.append(w)
    return out


def alone(torch, w, req, precision=0):
    src = synth.SlipRateStream(w, req.seed, torch.device("cuda", 0))
    out = []
    with seas.Session(w, precision=precision) as s:
        t = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        for n in range(req.steps):
            seas.seas_push_slip_rate(s.scn, src.row(n).contiguous())
            seas.seas_stress_step(s.scn, t)
            out.append(t.cpu().numpy().copy())
    return np.array(out)


@pytest.mark.parametrize("precision", [seas.SEAS_PREC_FP64, seas.SEAS_PREC_BF16])
def test_each_request_equals_its_solo_run_in_the_mix(precision):
    torch = pytest.importorskip("torch")
    geoms = geometries(precision)
    steps = [30, 55, 12, 70, 41, 25, 64, 18, 50]
    trace = [serve.Request(rid=k, geom=k % 2, steps=steps[k], seed=1000 + k, arrival=0.001 * k)
             for k in range(len(steps))]
    srv = serve.Server(geoms, budget=8 << 30, batch=2, precision=precision, record=True)
    srv.run(trace, time_scale=1e3)
    torch.cuda.synchronize()
    st = srv.sched.requests
    assert all(r.state == "done" and r.done == r.steps for r in st.values())
    admitted_late = [r for r in st.values() if r.admitted > 0]
    assert admitted_late, "every request started at once: no continuous batching exercised"
    # in the BF16 batch of 2 the CUDA-core consumers differ from the solo run only in the summation order
    tol = 1e-12 if precision == seas.SEAS_PREC_FP64 else 1e-6
    worst = 0.0
    for r in trace:
        mix = torch.stack(srv.backend.history[r.rid]).cpu().numpy()
        solo = alone(torch, geoms[r.geom], r, precision)
        assert mix.shape == solo.shape
        worst = max(worst, rel(mix, solo))
    print(f"precision {precision}: worst rel-L2 mix vs alone over {len(trace)} requests: {worst:.2e}; "
          f"{srv.ticks} group ticks, p50 step latency {np.percentile(srv.latency_ms, 50):.3f} ms")
    assert worst <= tol


def test_member_api_admit_retire_and_step_counts():
    torch = pytest.importorskip("torch")
    w = geometries()[0]
    V = torch.from_numpy(np.stack([w.slip_rate(b, 0, w.steps) for b in range(2)], axis=1).reshape(w.steps, -1))
    V = V.cuda()
    with seas.Session(w, batch=2) as s:
        t = torch.zeros(2 * w.N, dtype=torch.float64, device="cuda")
        for n in range(5):
            seas.seas_push_slip_rate(s.scn, V[n])
            seas.seas_stress_step(s.scn, t)
        seas.seas_scenario_admit(s.scn, 1)
        assert seas.seas_scenario_member_step(s.scn, 1) == 0 and seas.seas_scenario_member_step(s.scn, 0) == 5
        seas.seas_scenario_retire(s.scn, 0)
        assert seas.seas_scenario_member_step(s.scn, 0) == -1
        for bad in (-1, 2):
            with pytest.raises(seas.SeasError) as e:
                seas.seas_scenario_admit(s.scn, bad)
            assert e.value.status == seas.SEAS_EINVAL
        # member 1 restarted at tick 5: it now runs like a fresh scenario pushed with V[5:], column 1
        out = []
        for n in range(5, 25):
            seas.seas_push_slip_rate(s.scn, V[n])
            seas.seas_stress_step(s.scn, t)
            out.append(t[w.N:].cpu().numpy().copy())
    Vb = V.reshape(w.steps, 2, w.N)[5:25, 1].contiguous()
    with seas.Session(w) as s1:
        t1 = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        ref = []
        for n in range(20):
            seas.seas_push_slip_rate(s1.scn, Vb[n])
            seas.seas_stress_step(s1.scn, t1)
            ref.append(t1.cpu().numpy().copy())
    assert rel(np.array(out), np.array(ref)) <= 1e-12

"""Partial operators (seas_build_hmatrix_part) for sharding one scenario by receiver faults: stepped with the same
global slip-rate history, each part returns on its own faults the rows of the full operator and leaves every other
entry of the output as it was; the parts of a partition together give the full tau."""
import numpy as np
import pytest

from paper_2603_00383_gb300 import seas, shard, synth

pytestmark = pytest.mark.gpu

SENTINEL = 12345.0


def _run(w, B, hp, steps, owned):
    import torch
    V = np.stack([w.slip_rate(b, 0, steps) for b in range(B)], axis=1).reshape(steps, -1)
    Vd = torch.from_numpy(V).cuda()
    out = []
    with seas.Session(w, batch=B, owned=owned, **hp) as s:
        tau = torch.full((B * w.N,), SENTINEL, dtype=torch.float64, device="cuda")
        for n in range(steps):
            seas.seas_push_slip_rate(s.scn, Vd[n])
            seas.seas_stress_step(s.scn, tau)
            out.append(tau.clone())
        seas.seas_scenario_check(s.scn)
    return torch.stack(out).cpu().numpy().reshape(steps, B, w.N)


@pytest.mark.parametrize("case", ["six_fault_fp64", "six_fault_bf16_batch8"])
def test_parts_return_the_full_operators_rows(case):
    pytest.importorskip("torch")
    if case == "six_fault_fp64":
        w, B, hp, steps = synth.six_fault_3072(steps=300), 1, {}, 300
    else:
        w, B, hp, steps = synth.six_fault_3072(steps=200), 8, dict(precision=seas.SEAS_PREC_BF16), 200
    full = _run(w, B, hp, steps, None)
    scale = np.abs(full).max()
    assert scale > 0
    assembled = np.full_like(full, np.nan)
    for part in shard.partition_faults(w.n_elem, 2) + [[4]]:
        got = _run(w, B, hp, steps, part)
        mine = shard.owned_elements(w.n_elem, part)
        rest = np.setdiff1d(np.arange(w.N), mine)
        assert np.all(got[:, :, rest] == SENTINEL)           # other faults' entries untouched
        err = np.abs(got[:, :, mine] - full[:, :, mine]).max() / scale
        assert err <= 1e-13, (part, err)
        if len(part) > 1:
            assembled[:, :, mine] = got[:, :, mine]
    assert not np.isnan(assembled).any()                      # the two parts cover every element


def test_part_rejects_bad_fault_lists():
    w = synth.tiny(1, n_faults=3, steps=10)
    with pytest.raises(seas.SeasError):
        seas.Session(w, owned=[])
    with pytest.raises(seas.SeasError):
        seas.Session(w, owned=[3])

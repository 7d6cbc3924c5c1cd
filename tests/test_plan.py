"""Host logic of the operator plan (no GPU): block partition of the selective H-matrix (Sec. 2.3.2), causal windows
and spectral windows, checked against the definitions and against the oracle's own window arithmetic."""
import math

import numpy as np
import pytest

from oracle import seas_oracle as O
from paper_2603_00383_gb300 import seas, synth


def plan(w, **hp):
    p = dict(w.hparams)
    p.update(hp)
    return seas.seas_plan_hmatrix(w.faults, w.mu, w.cs, w.cp, w.beta, p), p


def circle(net, a, b):
    xs = net.x[a:b]
    c = xs.mean(0)
    return c, np.max(np.hypot(*(xs - c).T)) + net.ds[a] / 2


@pytest.mark.parametrize("make,hp", [(synth.six_fault_3072, {}), (synth.two_fault_128, {"flags": 0}),
                                     (synth.two_fault_128, {}), (lambda: synth.tiny(2), {"leaf": 2, "eta_h": 1.0})])
def test_partition_covers_every_cross_fault_pair_once(make, hp):
    w = make()
    pl, p = plan(w, **hp)
    net = O.network(w.faults, w.mu, w.cs)
    cover = np.zeros((net.N, net.N), dtype=np.int32)
    for r0, pp, c0, q, far, _, _ in pl["blocks"]:
        cover[r0:r0 + pp, c0:c0 + q] += 1
        assert net.fault_of[r0] == net.fault_of[r0 + pp - 1] != net.fault_of[c0] == net.fault_of[c0 + q - 1]
        ca, ra = circle(net, r0, r0 + pp)
        cb, rb = circle(net, c0, c0 + q)
        adm = np.hypot(*(ca - cb)) > p["eta_h"] * (ra + rb)
        if far:
            assert adm and not (p["flags"] & seas.SEAS_FLAG_DENSE)
        else:
            assert pp <= p["leaf"] and q <= p["leaf"]
            assert not adm or (p["flags"] & seas.SEAS_FLAG_DENSE)
    other = net.fault_of[:, None] != net.fault_of[None, :]
    assert np.all(cover[other] == 1) and np.all(cover[~other] == 0)


def test_dense_flag_gives_only_near_leaf_blocks():
    w = synth.two_fault_128()
    pl, _ = plan(w)
    assert pl["blocks"][:, 4].sum() == 0
    assert pl["blocks"][:, 1].max() <= 32 and pl["blocks"][:, 3].max() <= 32


@pytest.mark.parametrize("make", [synth.two_fault_128, synth.six_fault_3072, synth.paper_two_fault])
def test_windows_and_dt_equal_the_oracle(make):
    w = make()
    pl, p = plan(w, flags=0)
    net = O.network(w.faults, w.mu, w.cs)
    assert abs(pl["dt"] - net.dt) <= 2e-16 * net.dt
    _, _, last = O.pair_windows(net, p["eta_tmin"], p["eta_tmax"], p["max_steps"])
    np.testing.assert_array_equal(pl["pair_last"], last)
    for f in range(net.F):
        W = O.mode_windows(int(net.n_elem[f]), net.length[f], net.dt, net.cs, p["eta_w"], p["q_w"], p["max_steps"])
        np.testing.assert_array_equal(pl["mode_windows"][f][1:], W[1:])


def test_no_trunc_windows_are_the_whole_history():
    w = synth.six_fault_3072(steps=700)
    pl, p = plan(w, flags=seas.SEAS_FLAG_NO_TRUNC)
    off = ~np.eye(w.n_faults, dtype=bool)
    assert np.all(pl["pair_last"][off] == 699)
    assert all(np.all(m[1:] == 699) for m in pl["mode_windows"])


def test_block_first_lag_never_after_the_first_nonzero_lag():
    w = synth.tiny(3, steps=200)
    pl, _ = plan(w, leaf=2, eta_h=1.0, flags=0)
    net = O.network(w.faults, w.mu, w.cs)
    A = np.stack([O.interaction_slice(net, T) for T in range(200)])
    for r0, pp, c0, q, far, first, _ in pl["blocks"]:
        nz = np.nonzero(np.any(A[:, r0:r0 + pp, c0:c0 + q] != 0, axis=(1, 2)))[0]
        if len(nz):
            assert first <= nz[0] <= first + 2


@pytest.mark.parametrize("bad", [
    dict(n=29), dict(n=0), dict(length=-1.0), dict(cx=float("nan")), dict(n=7168 * 2)])
def test_invalid_geometry_is_rejected(bad):
    f = dict(cx=0.0, cy=0.0, strike=0.0, length=100.0, n=8)
    f.update(bad)
    faults = np.array([[f["cx"], f["cy"], f["strike"], f["length"], f["n"]],
                       [0.0, 500.0, 0.0, 100.0, 8]])
    with pytest.raises(seas.SeasError) as e:
        seas.seas_plan_hmatrix(faults, 32e9, 3464.0, 6000.0, 0.5, dict(max_steps=10, leaf=4))
    assert e.value.status == seas.SEAS_EINVAL


def test_receiver_on_another_fault_is_rejected():
    faults = np.array([[0.0, 0.0, 0.0, 100.0, 10], [5.0, 0.0, 0.0, 100.0, 10]])   # collinear, overlapping
    with pytest.raises(seas.SeasError) as e:
        seas.seas_plan_hmatrix(faults, 32e9, 3464.0, 6000.0, 0.5, dict(max_steps=10, leaf=4))
    assert e.value.status == seas.SEAS_EINVAL


def _surface_fault(x0, depth, n, phi=-0.5 * math.pi):
    e1 = (math.cos(phi), math.sin(phi))
    return [x0 + 0.5 * depth * e1[0], 0.5 * depth * e1[1], phi, depth, n, seas.SEAS_FAULT_SURFACE_START]


def test_plan_of_a_surface_network_is_the_oracles_doubled_network():
    """Faults breaking a free surface (method of images): the host plan is that of the doubled network the oracle
    builds (image_faults): the same dt, mode windows of 2 N_f + 1 modes per fault, and the same block partition as
    the oracle's dual traversal of the doubled faults."""
    faults = np.array([_surface_fault(0.0, 400.0, 48), _surface_fault(150.0, 300.0, 32)])
    hp = dict(max_steps=300, leaf=8, eta_h=1.0)
    pl = seas.seas_plan_hmatrix(faults, 32e9, 3464.0, 6000.0, 0.5, hp)
    doubled, mirror, real = O.image_faults(faults[:, :5])
    net2 = O.network(doubled, 32e9, 3464.0)
    assert pl["dt"] == pytest.approx(net2.dt, rel=1e-15)
    assert [len(m) for m in pl["mode_windows"]] == [97, 65]
    for f, n in enumerate((96, 64)):
        W = O.mode_windows(n, doubled[f, 3], net2.dt, 3464.0, 1.5, 0, 300)
        np.testing.assert_array_equal(pl["mode_windows"][f], W)
    ref = set()
    for a in range(2):
        for b in range(2):
            if a != b:
                ref |= {tuple(int(v) for v in blk[:4]) for blk in O.hmatrix_blocks(net2, a, b, 8, 1.0, 64)}
    assert {tuple(int(v) for v in r[:4]) for r in pl["blocks"]} == ref


@pytest.mark.parametrize("bad", ["tilted", "off_surface", "mixed", "unknown_flag"])
def test_surface_networks_off_one_surface_are_rejected_on_the_host(bad):
    ok = _surface_fault(0.0, 100.0, 8)
    other = _surface_fault(60.0, 100.0, 8)
    if bad == "tilted":
        other = _surface_fault(60.0, 100.0, 8, phi=-1.3)
    elif bad == "off_surface":
        other[1] -= 10.0
    elif bad == "mixed":
        other[5] = 0
    else:
        other[5] = 2
    seas.seas_plan_hmatrix(np.array([ok]), 32e9, 3464.0, 6000.0, 0.5, dict(max_steps=4))
    with pytest.raises(seas.SeasError) as e:
        seas.seas_plan_hmatrix(np.array([ok, other]), 32e9, 3464.0, 6000.0, 0.5, dict(max_steps=4))
    assert e.value.status == seas.SEAS_EINVAL


@pytest.mark.parametrize("leaf,eta_h,max_block,dense", [(8, 2.0, 0, False), (4, 1.0, 16, False), (6, 2.0, 0, True)])
def test_plan_block_windows_equal_the_oracle(leaf, eta_h, max_block, dense):
    """The plan's last lag of every block: the fault pair's window without the flag, the oracle's cluster-level
    window (Sec. 4.3 reading) with SEAS_FLAG_CLUSTER_TRUNC, as integers; the partition equals the oracle's."""
    faults = np.array([[0.0, 0.0, 0.1, 400.0, 40], [60.0, 300.0, -0.3, 320.0, 32], [450.0, -150.0, 1.2, 240.0, 24]])
    hp = dict(max_steps=260, leaf=leaf, eta_h=eta_h, max_block=max_block, eta_tmax=0.05,
              flags=seas.SEAS_FLAG_DENSE if dense else 0)
    net = O.network(faults, 32e9, 3464.0)
    _, _, P = O.pair_windows(net, 0.01, 0.05, 260)
    W = O.cluster_windows(net, leaf, eta_h, max_block or 64, 0.05, 260, dense=dense)
    ref = set()
    for a in range(net.F):
        for b in range(net.F):
            if a != b:
                ref |= {tuple(int(v) for v in blk)
                        for blk in O.hmatrix_blocks(net, a, b, leaf, eta_h, max_block or 64, dense)}
    for cluster in (False, True):
        p = dict(hp, flags=hp["flags"] | (seas.SEAS_FLAG_CLUSTER_TRUNC if cluster else 0))
        pl = seas.seas_plan_hmatrix(faults, 32e9, 3464.0, 6000.0, 0.5, p)
        assert {tuple(int(v) for v in r[:5]) for r in pl["blocks"]} == ref
        expect = W if cluster else P[net.fault_of][:, net.fault_of]
        for r0, pp, c0, q, far, first, last in pl["blocks"]:
            assert (expect[r0:r0 + pp, c0:c0 + q] == last).all()
    assert (W[net.fault_of[:, None] != net.fault_of[None, :]] < P[net.fault_of][:, net.fault_of][
        net.fault_of[:, None] != net.fault_of[None, :]]).any()

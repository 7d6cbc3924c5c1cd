"""Cluster-level end truncation (the per-block window of Sec. 4.3) through the C ABI: the library's H-matrix
partition and block windows against the oracle's restatement of the cluster trees, the dual traversal and the
window criterion (integers, exact), and the truncated interaction against the oracle's element-pair windowed sum."""
import numpy as np
import pytest

from oracle import seas_oracle as O
from paper_2603_00383_gb300 import seas, synth

pytestmark = pytest.mark.gpu

FAULTS = np.array([[0.0, 0.0, 0.1, 400.0, 40], [60.0, 300.0, -0.3, 320.0, 32], [450.0, -150.0, 1.2, 240.0, 24]])
STEPS = 260


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def workload(**hp):
    return synth.Workload("cluster3", FAULTS, steps=STEPS, hparams=dict(dict(max_steps=STEPS), **hp))


@pytest.mark.parametrize("leaf,eta_h,max_block,dense", [(8, 2.0, 0, False), (4, 1.0, 16, False),
                                                        (6, 2.0, 0, True)])
def test_blocks_and_block_windows_equal_the_oracle(leaf, eta_h, max_block, dense):
    """Every (r0, p, c0, q, far) block of the library is one of the oracle's leaf blocks and vice versa; each
    block's last lag is the oracle's cluster-level window, and without the flag the fault pair's."""
    flags = seas.SEAS_FLAG_CLUSTER_TRUNC | (seas.SEAS_FLAG_DENSE if dense else 0)
    w = workload(leaf=leaf, eta_h=eta_h, max_block=max_block, eta_tmax=0.05)
    net = O.network(w.faults, w.mu, w.cs)
    mb = max_block or 64
    ref = set()
    for a in range(net.F):
        for b in range(net.F):
            if a != b:
                ref |= {tuple(int(v) for v in blk) for blk in O.hmatrix_blocks(net, a, b, leaf, eta_h, mb, dense)}
    W = O.cluster_windows(net, leaf, eta_h, mb, 0.05, STEPS, dense=dense)
    _, _, P = O.pair_windows(net, 0.01, 0.05, STEPS)
    for fl, expect in ((flags, W), (flags & ~seas.SEAS_FLAG_CLUSTER_TRUNC, P[net.fault_of][:, net.fault_of])):
        with seas.Session(w, flags=fl) as s:
            blk = seas.seas_op_blocks(s.op)
        assert {tuple(int(v) for v in r[:5]) for r in blk} == ref and len(blk) == len(ref)
        for r0, p, c0, q, far, lo, hi in blk:
            assert (expect[r0:r0 + p, c0:c0 + q] == hi).all(), (r0, p, c0, q, hi)
    assert (W < P[net.fault_of][:, net.fault_of]).sum() > 0


@pytest.mark.parametrize("mode", ["dense", "hmatrix"])
def test_cluster_truncated_interaction_matches_the_oracle(mode):
    """tau, radiation, self and interaction parts over 260 steps with block windows that end inside the run,
    against the oracle with the same element-pair windows: exact with every block dense, the ACA tolerance
    (1e-10 per slice) with low-rank far blocks.  The truncation changes the interaction against the fault-pair
    windows by far more than the tolerance, so a library that ignored the flag fails."""
    extra = dict(flags=seas.SEAS_FLAG_CLUSTER_TRUNC | seas.SEAS_FLAG_DENSE) if mode == "dense" else \
        dict(flags=seas.SEAS_FLAG_CLUSTER_TRUNC, aca_tol=1e-10)
    w = workload(leaf=8, eta_h=2.0, eta_tmax=0.01, **extra)
    V = w.slip_rate(0, 0, STEPS)
    tau = np.zeros((STEPS, w.N))
    P = np.zeros((STEPS, 3, w.N))
    t, p = np.zeros(w.N), np.zeros(3 * w.N)
    with seas.Session(w) as s:
        stats = s.stats
        for n in range(STEPS):
            seas.seas_push_slip_rate(s.scn, np.ascontiguousarray(V[n]))
            seas.seas_stress_step(s.scn, t, parts=p)
            tau[n], P[n] = t, p.reshape(3, w.N)
    net = O.network(w.faults, w.mu, w.cs)
    ref = O.stress_history(net, V, w.hparams)
    pair = O.stress_history(net, V, dict(w.hparams, flags=w.hparams["flags"] & ~seas.SEAS_FLAG_CLUSTER_TRUNC))
    errs = [rel(tau, ref[0]), rel(P[:, 0], ref[1]), rel(P[:, 1], ref[2]), rel(P[:, 2], ref[3])]
    moved = rel(ref[3], pair[3])
    print(f"cluster truncation ({mode}): rel-L2 tau/rad/self/int {errs}; change vs pair windows {moved:.2e}; "
          f"far blocks {stats['n_blocks_far']}")
    assert moved > 1e-3
    assert max(errs) <= (1e-10 if mode == "dense" else 1e-8)
    if mode == "hmatrix":
        assert stats["n_blocks_far"] > 0


def test_cluster_truncation_stores_less():
    w = workload(leaf=8, eta_h=2.0, eta_tmax=0.01)
    with seas.Session(w) as a, seas.Session(w, flags=seas.SEAS_FLAG_CLUSTER_TRUNC) as b:
        assert b.stats["bytes_interaction"] < a.stats["bytes_interaction"]


@pytest.mark.parametrize("mode", ["dense", "hmatrix"])
def test_cluster_truncation_with_the_static_tail_matches_the_oracle(mode):
    """The static tail per block (each block's own window end) with cluster-level windows, 260 steps: tau and its
    parts against the oracle; the tail moves the interaction by far more than the tolerance."""
    flags = seas.SEAS_FLAG_CLUSTER_TRUNC | seas.SEAS_FLAG_STATIC_TAIL
    extra = dict(flags=flags | seas.SEAS_FLAG_DENSE) if mode == "dense" else dict(flags=flags, aca_tol=1e-10)
    w = workload(leaf=8, eta_h=2.0, eta_tmax=0.01, **extra)
    V = w.slip_rate(0, 0, STEPS)
    tau = np.zeros((STEPS, w.N))
    P = np.zeros((STEPS, 3, w.N))
    t, p = np.zeros(w.N), np.zeros(3 * w.N)
    with seas.Session(w) as s:
        for n in range(STEPS):
            seas.seas_push_slip_rate(s.scn, np.ascontiguousarray(V[n]))
            seas.seas_stress_step(s.scn, t, parts=p)
            tau[n], P[n] = t, p.reshape(3, w.N)
    net = O.network(w.faults, w.mu, w.cs)
    ref = O.stress_history(net, V, w.hparams)
    plain = O.stress_history(net, V, dict(w.hparams, flags=w.hparams["flags"] & ~seas.SEAS_FLAG_STATIC_TAIL))
    errs = [rel(tau, ref[0]), rel(P[:, 1], ref[2]), rel(P[:, 2], ref[3])]
    moved = rel(ref[3], plain[3])
    print(f"cluster truncation + static tail ({mode}): rel-L2 tau/self/int {errs}; tail moves int by {moved:.2e}")
    assert moved > 1e-3
    assert max(errs) <= (1e-10 if mode == "dense" else 1e-8)

"""Seeded workload generator: determinism, counter-based access, placement constraints."""
import numpy as np

from paper_2603_00383_gb300 import synth


def test_counter_based_slices_agree():
    w = synth.two_fault_128()
    a = w.slip_rate(2, 0, 12)
    b = w.slip_rate(2, 5, 12)
    np.testing.assert_array_equal(a[5:], b)
    assert not np.array_equal(w.slip_rate(3, 0, 2), w.slip_rate(2, 0, 2))


def test_slip_rate_statistics_and_pulse():
    w = synth.six_fault_3072()
    V = w.slip_rate(0, 0, 50)
    bg = V[:, w.faults[0, 4].astype(int):]
    assert 1e-9 <= bg.min() and bg.max() < 1e-6
    assert np.all(np.abs(np.log10(bg).mean() + 7.5) < 0.05)
    n0 = int(w.faults[0, 4])
    assert abs(V[0, :n0].max() - 1.0) < 0.05
    peak = np.argmax(V[40, :n0])
    ds0 = w.faults[0, 3] / n0
    expect = 0.8 * w.cs * w.input_dt() * 40 / ds0
    assert abs(abs(peak + 0.5 - n0 / 2) - expect) < 1.0


def test_six_fault_placement_constraints():
    w = synth.six_fault_3072()
    assert list(w.n_elem) == [256, 384, 512, 512, 640, 768] and w.N == 3072
    ends = []
    for cx, cy, phi, L, n in w.faults:
        e = np.array([np.cos(phi), np.sin(phi)])
        p0, p1 = np.array([cx, cy]) - L / 2 * e, np.array([cx, cy]) + L / 2 * e
        assert np.all(np.abs(p0) <= 20000) and np.all(np.abs(p1) <= 20000)
        assert 0 <= phi <= np.pi / 2
        ends.append((p0, p1))
    for i in range(6):
        for j in range(i):
            assert synth._seg_dist(*ends[i], *ends[j]) >= 500.0


def test_ensemble_networks_are_fft_friendly():
    for g in range(4):
        w = synth.ensemble_network(g)
        assert 2 <= w.n_faults <= 12 and 1000 <= w.steps <= 5000
        for n in w.n_elem:
            m = int(n)
            for p in (2, 3, 5):
                while m % p == 0:
                    m //= p
            assert m == 1

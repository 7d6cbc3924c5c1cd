"""Seeded synthetic workloads for the elastodynamic stress-transfer functional.

This module is shared by the CUDA path (tests, bench) and by the CPU oracle.  It holds none of the method's
arithmetic: it only produces inputs -- fault placements (centre, strike, length, element count), medium constants,
operator parameters, and slip-rate histories -- from a counter-based SplitMix64 stream, so that any (scenario, step,
element) value can be regenerated independently of every other one.

Workloads (shapes follow the paper's benchmarks; the paper's own data are not used):

* ``two_fault_128``   -- two 10 km faults, 128 elements each; fault B rotated 30 deg and offset 3 km along strike and
  2 km along the normal of fault A (the paper's two-fault benchmark shape, Sec. 3.1, at 1/8 of its resolution).
* ``six_fault_3072``  -- six non-intersecting faults of 256..768 elements (3072 in total, 20 m elements) placed at
  random in a 40 x 40 km box (the paper's ~3e3-DOF scale, abstract and Sec. 3.1).
* ``paper_two_fault`` -- the exact two-fault geometry printed in Sec. 3.1 (centroids, lengths, normals; Table 1).
* ``surface_fault_1600`` -- one fault breaking a traction-free surface, 40 km deep, 1600 elements (doubled to
  3200 by the method of images), the shape of the paper's single-fault verification (App. B).
* ``tiny``            -- 2..3 faults of 4..16 elements for brute-force checks.
* ``ensemble``        -- random networks for batched / served runs (2..12 faults, 500..6000 elements).

Slip-rate history: log10 V ~ U[-9, -6] m/s i.i.d. per (element, step), plus on fault 0 a bilateral Gaussian
rupture pulse of peak 1 m/s, width 5 elements, moving outwards from the fault centre at 0.8 c_s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 260300383
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# operator flags (mirrors of the C header's SEAS_FLAG_* values; inputs, not arithmetic)
FLAG_DENSE = 1          # every block stored dense (admissibility never satisfied)
FLAG_NO_TRUNC = 2       # no causal end truncation of pair windows, full spectral windows
FLAG_STATIC_TAIL = 4    # add the elastostatic response of truncated history (default off)
FLAG_LAG_CAP = 8        # max_steps caps the windows but not the number of steps
FLAG_CLUSTER_TRUNC = 16 # interaction windows end per H-matrix block (cluster-level end truncation)

PREC_FP64 = 0
PREC_BF16 = 1
PREC_FP16S = 2


def splitmix64(key: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each counter: mix(key + (counter + 1) * golden).  Counter-based, so vectorisable."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(key: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(key, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Workload:
    """One synthetic stress-transfer workload: network, medium, operator parameters and slip-rate statistics."""

    name: str
    faults: np.ndarray                 # [F, 5]: cx, cy, strike_rad, length, n_elem (+ fault flags, optional)
    mu: float = 32e9
    cs: float = 3464.0
    cp: float = 6000.0
    beta: float = 0.5
    steps: int = 400
    batch: int = 1
    seed: int = SEED
    pulse: bool = True
    hparams: dict = field(default_factory=dict)

    @property
    def n_faults(self) -> int:
        return int(self.faults.shape[0])

    @property
    def n_elem(self) -> np.ndarray:
        return self.faults[:, 4].astype(np.int64)

    @property
    def N(self) -> int:
        return int(self.n_elem.sum())

    def input_dt(self) -> float:
        """The pulse clock: beta * min(L_f / N_f) / c_s, the lattice the workload is specified on."""
        return self.beta * float(np.min(self.faults[:, 3] / self.faults[:, 4])) / self.cs

    def slip_rate(self, scenario: int, step0: int, step1: int) -> np.ndarray:
        """Slip rate V[m][j] for steps m in [step0, step1) of one scenario, in m/s (float64, [steps][N])."""
        N = self.N
        m = np.arange(step0, step1, dtype=np.int64)
        idx = (m[:, None] * N + np.arange(N, dtype=np.int64)[None, :]).astype(np.uint64)
        u = uniform01(self.seed + scenario, idx)
        V = np.power(10.0, -9.0 + 3.0 * u)
        if self.pulse and step1 > step0:
            n0 = int(self.faults[0, 4])
            ds0 = float(self.faults[0, 3]) / n0
            xi = (np.arange(n0) + 0.5 - 0.5 * n0) * ds0
            front = 0.8 * self.cs * self.input_dt() * m.astype(np.float64)
            arg = (np.abs(xi)[None, :] - front[:, None]) / (5.0 * ds0)
            V[:, :n0] += np.exp(-0.5 * arg * arg)
        return V

    def slip_rate_batch(self, step0: int, step1: int) -> np.ndarray:
        """[steps][batch][N] slip rates for scenarios 0..batch-1."""
        return np.stack([self.slip_rate(s, step0, step1) for s in range(self.batch)], axis=1)


def _hp(leaf=32, eta_h=2.0, aca_tol=1e-6, eta_tmin=0.01, eta_tmax=0.01, eta_w=1.5, q_w=0, max_steps=400,
        precision=PREC_FP64, flags=0) -> dict:
    return dict(leaf=leaf, eta_h=eta_h, aca_tol=aca_tol, eta_tmin=eta_tmin, eta_tmax=eta_tmax, eta_w=eta_w,
                q_w=q_w, max_steps=max_steps, precision=precision, flags=flags)


def two_fault_128(steps: int = 400, n_elem: int = 128) -> Workload:
    """Two 10 km faults: A at the origin with strike 0; B at c_A + 3 km e1_A + 2 km n_A with strike +30 deg."""
    fa = (0.0, 0.0, 0.0, 10000.0, n_elem)
    # n_A = (sin 0, -cos 0) = (0, -1); e1_A = (1, 0)
    fb = (3000.0, -2000.0, math.radians(30.0), 10000.0, n_elem)
    return Workload("two_fault_128", np.array([fa, fb], dtype=np.float64), steps=steps,
                    hparams=_hp(max_steps=steps, flags=FLAG_DENSE | FLAG_NO_TRUNC))


def paper_two_fault(n_elem: int = 1000, steps: int = 1447) -> Workload:
    """The two-fault benchmark geometry as printed (Sec. 3.1, Table 1): centroids, lengths and unit normals.

    Strike phi is recovered from the printed normal n = (sin phi, -cos phi)."""
    n1 = (-0.524322, -0.85152)
    n2 = (0.159658, -0.987172)
    s1 = math.atan2(n1[0], -n1[1])
    s2 = math.atan2(n2[0], -n2[1])
    f1 = (-3591.98, -4635.56, s1, 9927.57, n_elem)
    f2 = (214.108, -1037.84, s2, 9578.55, n_elem)
    return Workload("paper_two_fault", np.array([f1, f2], dtype=np.float64), mu=30e9, steps=steps,
                    hparams=_hp(leaf=50, eta_h=1.5, aca_tol=1e-6, eta_tmin=0.01, eta_tmax=0.01, eta_w=1.5,
                                q_w=200, max_steps=steps))


def _seg_dist(p0, p1, q0, q1) -> float:
    """Distance between two segments in the plane (0 when they cross)."""
    def cross(a, b):
        return a[0] * b[1] - a[1] * b[0]

    def pt_seg(p, a, b):
        ab = b - a
        t = np.clip(np.dot(p - a, ab) / np.dot(ab, ab), 0.0, 1.0)
        return float(np.hypot(*(a + t * ab - p)))

    d1, d2 = p1 - p0, q1 - q0
    den = cross(d1, d2)
    if den != 0.0:
        t = cross(q0 - p0, d2) / den
        u = cross(q0 - p0, d1) / den
        if 0.0 <= t <= 1.0 and 0.0 <= u <= 1.0:
            return 0.0
    return min(pt_seg(p0, q0, q1), pt_seg(p1, q0, q1), pt_seg(q0, p0, p1), pt_seg(q1, p0, p1))


def place_faults(n_elem, ds: float, box: float, gap: float, seed: int, max_tries: int = 100000) -> np.ndarray:
    """Rejection-sample fault centres U[-box/2, box/2]^2 and strikes U[0, 90 deg] so that every endpoint stays in
    the box and every pair of faults is at least ``gap`` apart.  Faults are placed in the given order."""
    out = []
    ctr = 0
    half = 0.5 * box
    for nf in n_elem:
        L = nf * ds
        for _ in range(max_tries):
            u = uniform01(seed ^ 0x5EA5, np.arange(ctr, ctr + 3, dtype=np.uint64))
            ctr += 3
            cx, cy = -half + box * u[0], -half + box * u[1]
            phi = 0.5 * math.pi * u[2]
            e1 = np.array([math.cos(phi), math.sin(phi)])
            p0 = np.array([cx, cy]) - 0.5 * L * e1
            p1 = np.array([cx, cy]) + 0.5 * L * e1
            if np.any(np.abs(p0) > half) or np.any(np.abs(p1) > half):
                continue
            ok = True
            for f in out:
                fe1 = np.array([math.cos(f[2]), math.sin(f[2])])
                q0 = np.array(f[:2]) - 0.5 * f[3] * fe1
                q1 = np.array(f[:2]) + 0.5 * f[3] * fe1
                if _seg_dist(p0, p1, q0, q1) < gap:
                    ok = False
                    break
            if ok:
                out.append((cx, cy, phi, L, float(nf)))
                break
        else:
            raise RuntimeError("fault placement failed")
    return np.array(out, dtype=np.float64)


def six_fault_3072(steps: int = 2000) -> Workload:
    """Six faults of 256, 384, 512, 512, 640, 768 elements (20 m), 40 x 40 km box, edge gaps >= 500 m."""
    faults = place_faults([256, 384, 512, 512, 640, 768], 20.0, 40000.0, 500.0, SEED)
    return Workload("six_fault_3072", faults, steps=steps,
                    hparams=_hp(leaf=32, eta_h=2.0, aca_tol=1e-6, eta_tmin=0.01, eta_tmax=0.01, eta_w=1.5,
                                q_w=0, max_steps=steps))


def tiny(seed: int = 1, n_faults: int = 2, steps: int = 30) -> Workload:
    """2..3 faults of 4..16 elements (2,3,5-smooth counts) in a 600 m box, 40 m gaps."""
    u = uniform01(seed ^ 0x71E1, np.arange(n_faults, dtype=np.uint64))
    sizes = [4, 5, 6, 8, 9, 10, 12, 15, 16]
    n_elem = [sizes[int(math.floor(len(sizes) * x))] for x in u]
    faults = place_faults(n_elem, 10.0, 600.0, 40.0, seed)
    return Workload(f"tiny{seed}", faults, steps=steps, seed=SEED + 1000 * seed,
                    hparams=_hp(leaf=4, eta_h=1.0, aca_tol=1e-8, max_steps=steps, flags=FLAG_NO_TRUNC))


def _is_235_smooth(n: int) -> bool:
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def _smooth_sizes(total: int, parts: int, seed: int) -> list:
    """Split ``total`` elements into ``parts`` fault sizes, each a 2,3,5-smooth even number >= 64."""
    smooth = [n for n in range(64, 20001, 2) if _is_235_smooth(n)]
    u = uniform01(seed ^ 0x51CE, np.arange(parts, dtype=np.uint64)) + 0.5
    raw = u / u.sum() * total
    return [min(smooth, key=lambda s: abs(s - r)) for r in raw]


def ensemble_network(geom_id: int, seed: int = SEED) -> Workload:
    """Random network: F in [2, 12], N log-uniform in [500, 6000], 20 m elements, box 40 km * sqrt(N / 3000),
    steps in [1000, 5000] (the batched-ensemble shape)."""
    u = uniform01(seed ^ 0xE45E, np.arange(4 * geom_id, 4 * geom_id + 4, dtype=np.uint64))
    F = 2 + int(11 * u[0])
    N = int(round(math.exp(math.log(500.0) + u[1] * (math.log(6000.0) - math.log(500.0)))))
    steps = 1000 + int(4001 * u[2])
    sizes = _smooth_sizes(N, F, seed + geom_id)
    box = 40000.0 * math.sqrt(sum(sizes) / 3000.0)
    faults = place_faults(sizes, 20.0, box, 500.0, seed + 7919 * geom_id)
    return Workload(f"ensemble{geom_id}", faults, steps=steps, seed=seed + 100000 * geom_id,
                    hparams=_hp(leaf=32, eta_h=2.0, aca_tol=1e-6, max_steps=steps))


FAULT_SURFACE_START = 1   # mirror of the C header's SEAS_FAULT_SURFACE_START (a fault flag; an input)


def surface_fault_1600(steps: int = 2000, n_real: int = 1600, depth: float = 40000.0) -> Workload:
    """The shape of the single-fault verification of App. B: one vertical fault from the free surface (y = 0) down
    to 40 km, 1600 elements of 25 m, which the library doubles across the surface to an 80 km fault of 3200
    elements (method of images); self windows with eta_w = 2 and q_w = N_elts / 2 = 1600 on the doubled fault."""
    fault = (0.0, -0.5 * depth, -0.5 * math.pi, depth, n_real, FAULT_SURFACE_START)
    return Workload("surface_fault_1600", np.array([fault]), steps=steps,
                    hparams=dict(leaf=32, eta_h=2.0, aca_tol=1e-6, eta_tmin=0.01, eta_tmax=0.01, eta_w=2.0,
                                 q_w=n_real, max_steps=steps))


WORKLOADS = {"two_fault_128": two_fault_128, "six_fault_3072": six_fault_3072, "paper_two_fault": paper_two_fault,
             "surface_fault_1600": surface_fault_1600}


def served_network(geom_id: int, seed: int = SEED, n_lo: int = 256, n_hi: int = 8000, max_steps: int = 1000,
                   precision: int = PREC_FP64) -> Workload:
    """Network of the served workload: N log-uniform in [n_lo, n_hi], F in [2, 12] (at most N / 64 faults), 20 m
    elements, box 40 km * sqrt(N / 3000), operator lags capped at ``max_steps`` (the served requests run longer:
    windows end at the cap)."""
    u = uniform01(seed ^ 0x5E4E, np.arange(4 * geom_id, 4 * geom_id + 4, dtype=np.uint64))
    N = int(round(math.exp(math.log(n_lo) + u[1] * (math.log(n_hi) - math.log(n_lo)))))
    F = max(2, min(2 + int(11 * u[0]), N // 64))
    sizes = _smooth_sizes(N, F, seed + 31 * geom_id)
    box = 40000.0 * math.sqrt(sum(sizes) / 3000.0)
    faults = place_faults(sizes, 20.0, box, 500.0, seed + 7907 * geom_id)
    return Workload(f"served{geom_id}", faults, steps=max_steps, seed=seed + 200000 * geom_id,
                    hparams=_hp(leaf=32, eta_h=2.0, aca_tol=1e-6, max_steps=max_steps, precision=precision,
                                flags=FLAG_LAG_CAP))


class SlipRateStream:
    """Slip rates of one served request, generated on the GPU in chunks of ``chunk`` steps with the statistics of
    Workload.slip_rate (log10 V ~ U[-9, -6] per element and step, plus the rupture pulse on fault 0).  The uniform
    numbers come from torch's counter-based Philox generator, seeded per (request seed, chunk), so the values of a
    step depend only on the request's seed and the step, not on what else runs.  Holds no method arithmetic."""

    def __init__(self, workload: Workload, seed: int, device, chunk: int = 256):
        import torch
        self.torch = torch
        self.w = workload
        self.seed = int(seed)
        self.device = device
        self.chunk = int(chunk)
        n0 = int(workload.faults[0, 4])
        ds0 = float(workload.faults[0, 3]) / n0
        self.n0 = n0
        self.xi = torch.from_numpy(np.abs((np.arange(n0) + 0.5 - 0.5 * n0) * ds0)).to(device)
        self.ds0 = ds0
        self.front = 0.8 * workload.cs * workload.input_dt()
        self._k = -1
        self._buf = None

    def _fill(self, k: int):
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed((self.seed * 1000003 + k) & 0x7FFFFFFFFFFFFFFF)
        u = torch.rand((self.chunk, self.w.N), generator=g, device=self.device, dtype=torch.float64)
        V = torch.pow(10.0, -9.0 + 3.0 * u)
        if self.w.pulse:
            m = torch.arange(k * self.chunk, (k + 1) * self.chunk, device=self.device, dtype=torch.float64)
            arg = (self.xi[None, :] - self.front * m[:, None]) / (5.0 * self.ds0)
            V[:, : self.n0] += torch.exp(-0.5 * arg * arg)
        self._k, self._buf = k, V

    def row(self, m: int):
        """V^m, a [N] float64 tensor on the device (a view valid until the next chunk is generated)."""
        k = m // self.chunk
        if k != self._k:
            self._fill(k)
        return self._buf[m - k * self.chunk]

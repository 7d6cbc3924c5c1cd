"""CPU oracle of the per-time-step elastodynamic stress-transfer functional (Ciardo & Romanet, arXiv 2603.00383).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It shares no code, table, constant generator or helper with the CUDA library; it reads only the
seeded inputs of ``paper_2603_00383_gb300.synth`` (which hold none of the method's arithmetic).

What it computes, step by step, in plain FP64 NumPy (no blocking, no compression, no FFT):

1. Network geometry (Sec. 3.1): e'_2 = n = (sin phi, -cos phi), e'_1 = e'_3 x e'_2 = (cos phi, sin phi);
   element j of fault f has centroid c_f + (-L_f/2 + (j + 1/2) ds_f) e'_1 with ds_f = L_f / N_f (Sec. 2.3.1,
   "Discretization"); the lattice step is dt = beta * min_f ds_f / c_s with beta = 1/2 (Sec. 2.3.1; Sec. 3.1).
2. Anti-plane primitives I_31, I_32 exactly as Eq. (primitives) (Sec. 2.3.2), with H(0) = 0 and sgn(0) = 0.
3. The discrete kernel as the four-term space/time difference of the primitives, Eq. (kernel_interactions),
   in the source element's frame; projected on the receiver normal rotated into that frame,
   A_ij^T = n'_1 K_31 + n'_2 K_32 (Eq. fault-to-fault_interactions_discretized).
4. f_int,i^n = -(mu / 2 c_s) sum_{j on other faults} sum_T A_ij^T V_j^{n-T}
   (Eq. fault-to-fault_interactions_discretized), every lag 0..n unless a window restricts T to a plain range.
5. Spectral weights w_{f,n}^T = c_s k_n * int_{T dt}^{(T+1) dt} K(n, t) dt with K of Eq. (non_replicant_kernel),
   k_n = pi n / L_f, evaluated through the equivalent single psi-integral (integrating cos(k c_s t sin psi) over
   t in closed form), by composite Gauss-Legendre quadrature.
6. D_{f,n}^m by direct DFT of the zero-padded slip on the 2 L_f domain (Eq. functional_no_replication),
   F_{f,n}^m = -(mu k_n / 2) sum_{T=0}^{W_f(n)} w_{f,n}^T D_{f,n}^{m-T} (Eq. funcational_discretized_form),
   f_self by direct inverse DFT over the modes n = -N_f + 1 .. N_f with F_{-n} = conj(F_n).
7. tau^n = -(mu / 2 c_s) V^n + f_self^n + f_int^n (Eq. superimposition2); sigma_n^el = 0 (Sec. 2.1).

Windows (optional, off by default): mode-dependent self windows W_f(n) = ceil(T_end(n)/dt) with
T_end(n) = eta_w L_f / c_s * Lcal(n) (Eq. mode_dependent_truncation) and per fault-pair interaction windows ending at
ceil((1 + eta_Tmax) T_max / dt) (Sec. 2.3.2, "Truncation of elastodynamic time-window"), or, with the
cluster-level end truncation of Sec. 4.3 (flag 16), the same criterion per block of the H-matrix partition (the
fault-wise cluster trees and the dual traversal restated in cluster_tree / hmatrix_blocks).  Static tail (flag 4,
not in the paper, off by default): the history a window drops is added back as an elastostatic response, per mode
c_n D_n^{m - W - 1} with c_n = (2/pi) Si(n pi) - sum_{T <= W} w_n^T, per fault pair A^static delta^{m - T_last - 1}.

Half-space (App. B): image_faults doubles each surface-breaking fault across the traction-free surface and
continues the slip evenly; half_space_stress_history is the functional of that doubled network on the real rows.

Parity status: every function here is pinned by tests/test_oracle_pins.py (closed forms, special cases, printed
numbers, brute force in extended precision).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------------------------------------------
# 1. geometry
# ----------------------------------------------------------------------------------------------------------------


@dataclass
class Network:
    mu: float
    cs: float
    dt: float
    fault_of: np.ndarray      # [N] fault index of each element
    x: np.ndarray             # [N, 2] element centroids
    e1: np.ndarray            # [N, 2] along-fault unit vector e'_1 of the element's fault
    nrm: np.ndarray           # [N, 2] unit normal e'_2 = n of the element's fault
    ds: np.ndarray            # [N] element length
    offset: np.ndarray        # [F + 1] first element of each fault
    length: np.ndarray        # [F] fault lengths
    center: np.ndarray        # [F, 2]
    n_elem: np.ndarray        # [F]

    @property
    def N(self) -> int:
        return int(self.offset[-1])

    @property
    def F(self) -> int:
        return int(self.length.shape[0])


def network(faults: np.ndarray, mu: float, cs: float, beta: float = 0.5) -> Network:
    """Element centroids, frames and the time step (Sec. 3.1 frames; Sec. 2.3.1 discretization; dt per Sec. 3.1)."""
    faults = np.asarray(faults, dtype=np.float64)
    xs, e1s, ns, dss, fo = [], [], [], [], []
    offset = [0]
    for f, (cx, cy, phi, L, nf) in enumerate(faults):
        nf = int(nf)
        e1 = np.array([math.cos(phi), math.sin(phi)])
        n = np.array([math.sin(phi), -math.cos(phi)])
        ds = L / nf
        s = -0.5 * L + (np.arange(nf) + 0.5) * ds
        xs.append(np.array([cx, cy])[None, :] + s[:, None] * e1[None, :])
        e1s.append(np.repeat(e1[None, :], nf, 0))
        ns.append(np.repeat(n[None, :], nf, 0))
        dss.append(np.full(nf, ds))
        fo.append(np.full(nf, f))
        offset.append(offset[-1] + nf)
    dt = beta * float(np.min(faults[:, 3] / faults[:, 4])) / cs
    return Network(mu=mu, cs=cs, dt=dt, fault_of=np.concatenate(fo), x=np.concatenate(xs),
                   e1=np.concatenate(e1s), nrm=np.concatenate(ns), ds=np.concatenate(dss),
                   offset=np.array(offset), length=faults[:, 3].copy(), center=faults[:, :2].copy(),
                   n_elem=faults[:, 4].astype(np.int64))


# ----------------------------------------------------------------------------------------------------------------
# 2-4. space-time interaction
# ----------------------------------------------------------------------------------------------------------------


def I31(r1, r2, t, cs):
    """I_31(r1, r2, t) = -(r2 / (pi r)) H(t - r/c_s) sqrt((c_s t / r)^2 - 1)   (Eq. primitives, first line)."""
    r = np.hypot(r1, r2)
    on = (cs * t > r) & (r > 0)
    rs = np.where(on, r, 1.0)
    a = np.where(on, cs * t / rs, 1.0)
    return np.where(on, -(r2 / (np.pi * rs)) * np.sqrt(a * a - 1.0), 0.0)


def I32(r1, r2, t, cs):
    """I_32(r1, r2, t) = H(r1) H(t - |r2|/c_s)
    + (1/pi) sgn(r1) H(t - r/c_s) [ (|r1|/r) sqrt((c_s t / r)^2 - 1) - arccos(|r1| / sqrt((c_s t)^2 - r2^2)) ]
    (Eq. primitives, second line)."""
    r = np.hypot(r1, r2)
    plane = np.where((r1 > 0) & (cs * t > np.abs(r2)), 1.0, 0.0)
    on = (cs * t > r) & (r > 0)
    rs = np.where(on, r, 1.0)
    a = np.where(on, cs * t / rs, 1.0)
    den = np.where(on, np.sqrt(np.maximum((cs * t) ** 2 - r2 * r2, 0.0)), 1.0)
    br = (np.abs(r1) / rs) * np.sqrt(a * a - 1.0) - np.arccos(np.minimum(np.abs(r1) / den, 1.0))
    return plane + np.where(on, np.sign(r1) * br / np.pi, 0.0)


def kernel_K3l(r1, r2, T, dt, ds, cs):
    """(K_31, K_32) at lag T: the four-term difference of Eq. (kernel_interactions),
    K(r1, r2, t) = I(r1 + ds/2, r2, t + dt) - I(r1 - ds/2, r2, t + dt) - I(r1 + ds/2, r2, t) + I(r1 - ds/2, r2, t),
    with t = T dt, so that lag T is the response at t_n to unit slip rate on (t_{n-T-1}, t_{n-T}]."""
    t0 = T * dt
    t1 = (T + 1) * dt
    h = 0.5 * ds
    out = []
    for I in (I31, I32):
        out.append(I(r1 + h, r2, t1, cs) - I(r1 - h, r2, t1, cs) - I(r1 + h, r2, t0, cs) + I(r1 - h, r2, t0, cs))
    return out[0], out[1]


def interaction_slice(net: Network, T, rows=None, cols=None, dtype=np.float64) -> np.ndarray:
    """A_ij^T = n'_1 K_31 + n'_2 K_32 for receivers ``rows`` and sources ``cols`` (default: all).  (r1, r2) are the
    receiver's coordinates in the source element's frame, n' the receiver normal in that frame (Eq.
    fault-to-fault_interactions_discretized).  Same-fault entries are zero: self effects are spectral (Sec. 2.3.2).
    T may be a 1-D array of lags; the result then has a leading lag axis."""
    rows = np.arange(net.N) if rows is None else np.asarray(rows)
    cols = np.arange(net.N) if cols is None else np.asarray(cols)
    x = net.x.astype(dtype)
    d = x[rows][:, None, :] - x[cols][None, :, :]
    e1 = net.e1[cols].astype(dtype)[None, :, :]
    e2 = net.nrm[cols].astype(dtype)[None, :, :]
    r1 = (d * e1).sum(-1)
    r2 = (d * e2).sum(-1)
    nr = net.nrm[rows].astype(dtype)[:, None, :]
    n1 = (nr * e1).sum(-1)
    n2 = (nr * e2).sum(-1)
    cs = dtype(net.cs)
    Ta = np.asarray(T)
    Tb = Ta.astype(dtype)[:, None, None] if Ta.ndim == 1 else dtype(Ta)
    k31, k32 = kernel_K3l(r1, r2, Tb, dtype(net.dt), net.ds[cols].astype(dtype)[None, :], cs)
    A = n1 * k31 + n2 * k32
    same = net.fault_of[rows][:, None] == net.fault_of[cols][None, :]
    return np.where(same, dtype(0), A)


def static_slice(net: Network, rows=None, cols=None) -> np.ndarray:
    """A_ij^static = lim_{T -> inf} A_ij^T / dt: the elastostatic stress at receiver i of unit slip on source element
    j.  As t -> inf, dI_31/dt -> -(c_s / pi) r2 / r^2 and dI_32/dt -> (c_s / pi) r1 / r^2 (Eq. primitives), so the
    element difference of Eq. kernel_interactions gives S_31 = -(c_s/pi)(r2/rho_+^2 - r2/rho_-^2),
    S_32 = (c_s/pi)(r1_+/rho_+^2 - r1_-/rho_-^2), r1_+- = r1 +- ds/2, rho_+-^2 = r1_+-^2 + r2^2; projected like
    interaction_slice.  Same-fault entries are zero."""
    rows = np.arange(net.N) if rows is None else np.asarray(rows)
    cols = np.arange(net.N) if cols is None else np.asarray(cols)
    d = net.x[rows][:, None, :] - net.x[cols][None, :, :]
    e1 = net.e1[cols][None, :, :]
    e2 = net.nrm[cols][None, :, :]
    r1 = (d * e1).sum(-1)
    r2 = (d * e2).sum(-1)
    nr = net.nrm[rows][:, None, :]
    n1 = (nr * e1).sum(-1)
    n2 = (nr * e2).sum(-1)
    h = 0.5 * net.ds[cols][None, :]
    rp, rm = r1 + h, r1 - h
    pp, pm = rp * rp + r2 * r2, rm * rm + r2 * r2
    s31 = -(net.cs / np.pi) * (r2 / pp - r2 / pm)
    s32 = (net.cs / np.pi) * (rp / pp - rm / pm)
    A = n1 * s31 + n2 * s32
    same = net.fault_of[rows][:, None] == net.fault_of[cols][None, :]
    return np.where(same, 0.0, A)


def _element_hi(net: Network, pair_hi, rows=None) -> np.ndarray:
    """Window ends per element pair [rows][N]: ``pair_hi`` given per fault pair [F][F] is broadcast to the elements
    of each pair; given per element pair [N][N] (cluster-level windows) its rows are taken as they are."""
    hi = np.asarray(pair_hi)
    rows = np.arange(net.N) if rows is None else np.asarray(rows)
    if hi.shape == (net.N, net.N):
        return hi[rows]
    fo = net.fault_of
    return hi[fo[rows]][:, fo]


def interaction_history(net: Network, V: np.ndarray, pair_hi=None, dtype=np.float64) -> np.ndarray:
    """f_int^n for every step n of V[steps][N] (Eq. fault-to-fault_interactions_discretized), all rows.

    ``pair_hi`` (optional, [F][F] or [N][N] ints) limits the lags of receiver-fault a / source-fault b (or of
    receiver element i / source element j) to T <= pair_hi[a][b] (pair_hi[i][j])."""
    steps = V.shape[0]
    A = np.stack([interaction_slice(net, T, dtype=dtype) for T in range(steps)])
    if pair_hi is not None:
        hi = _element_hi(net, pair_hi)
        A = np.where(np.arange(steps)[:, None, None] <= hi[None, :, :], A, 0)
    Vd = V.astype(dtype)
    out = np.zeros((steps, net.N), dtype=dtype)
    for n in range(steps):
        out[n] = np.einsum("tij,tj->i", A[: n + 1], Vd[n::-1])
    return -(dtype(net.mu) / (2 * dtype(net.cs))) * out


def interaction_rows(net: Network, V: np.ndarray, n: int, rows, pair_hi=None, chunk: int = 128) -> np.ndarray:
    """f_int^n at receiver ``rows`` only, for one step n, from the slip-rate history V[0..n][N]."""
    rows = np.asarray(rows)
    acc = np.zeros(rows.shape[0])
    hi = None if pair_hi is None else _element_hi(net, pair_hi, rows)
    for T0 in range(0, n + 1, chunk):
        Ts = np.arange(T0, min(n + 1, T0 + chunk))
        A = interaction_slice(net, Ts, rows=rows)               # [lags, rows, N]
        if hi is not None:
            A = np.where(Ts[:, None, None] <= hi[None], A, 0.0)
        acc += np.einsum("tij,tj->i", A, V[n - Ts])
    return -(net.mu / (2 * net.cs)) * acc


def pair_windows(net: Network, eta_tmin: float, eta_tmax: float, max_steps: int, no_trunc: bool = False):
    """Per ordered fault pair (receiver a, source b), Sec. 2.3.2 "Truncation of elastodynamic time-window":

    * T_arr(i, j) = min(r_ij, |r'_2,ij|)/c_s if r'_1,ij > 0 else r_ij / c_s (centroid offsets, source frame);
      T_earl = min T_arr (Eq. early_time); T_init = (1 - eta_Tmin) T_earl.
    * T_max = max over the source elements and the two receiver-fault endpoints of distance / c_s, the distance
      taken to the far end of each source element (so the source fault's endpoints); this reading reproduces the
      printed T_end ~ 3.76 s of Sec. 3.1 (centroid distances give 3.7547 s); T_end = (1 + eta_Tmax) T_max.

    Returns (t_init [F][F] seconds, t_end [F][F] seconds, last_lag [F][F]) where
    last_lag = min(ceil(T_end / dt - 1e-9), max_steps - 1) (the whole history when ``no_trunc``); -1 on the
    diagonal."""
    F = net.F
    t_init = np.zeros((F, F))
    t_end = np.zeros((F, F))
    last = np.full((F, F), -1, dtype=np.int64)
    for a in range(F):
        ra = slice(net.offset[a], net.offset[a + 1])
        ca, e1a = net.center[a], net.e1[net.offset[a]]
        ends = np.stack([ca - 0.5 * net.length[a] * e1a, ca + 0.5 * net.length[a] * e1a])
        for b in range(F):
            if a == b:
                continue
            rb = slice(net.offset[b], net.offset[b + 1])
            d = net.x[ra][:, None, :] - net.x[rb][None, :, :]
            r = np.hypot(d[..., 0], d[..., 1])
            r1 = (d * net.e1[rb][None]).sum(-1)
            r2 = (d * net.nrm[rb][None]).sum(-1)
            tarr = np.where(r1 > 0, np.minimum(r, np.abs(r2)), r) / net.cs
            t_init[a, b] = (1.0 - eta_tmin) * tarr.min()
            hb = 0.5 * net.ds[rb][:, None] * net.e1[rb]
            src_ends = np.concatenate([net.x[rb] - hb, net.x[rb] + hb])
            de = ends[:, None, :] - src_ends[None, :, :]
            tmax = np.hypot(de[..., 0], de[..., 1]).max() / net.cs
            t_end[a, b] = (1.0 + eta_tmax) * tmax
            lag = math.ceil(t_end[a, b] / net.dt - 1e-9)
            last[a, b] = max_steps - 1 if no_trunc else min(lag, max_steps - 1)
    return t_init, t_end, last


@dataclass
class Cluster:
    lo: int                   # first element (global index)
    hi: int                   # one past the last element
    centre: np.ndarray        # mean of the element centroids
    radius: float             # largest centroid distance from the centre plus half an element
    children: tuple = ()


def cluster_tree(net: Network, f: int, leaf: int) -> Cluster:
    """The binary cluster tree of fault f (Sec. 2.3.2, "Fault-wise hierarchical decomposition"): the root holds the
    fault's elements in order; a cluster of more than ``leaf`` elements is cut into two halves of consecutive
    elements, the left half taking the extra element of an odd count."""
    def make(lo, hi):
        pts = net.x[lo:hi]
        c = pts.mean(axis=0)
        r = float(np.max(np.hypot(*(pts - c).T) + 0.5 * net.ds[lo:hi]))
        node = Cluster(lo, hi, c, r)
        if hi - lo > leaf:
            mid = lo + (hi - lo + 1) // 2
            node.children = (make(lo, mid), make(mid, hi))
        return node
    return make(int(net.offset[f]), int(net.offset[f + 1]))


def hmatrix_blocks(net: Network, a: int, b: int, leaf: int, eta_h: float, max_block: int, dense: bool = False):
    """Leaf blocks of the dual-tree traversal of receiver fault a against source fault b (Sec. 2.3.2,
    Eq. admissibility_condition): a cluster pair whose centre distance exceeds eta_H (r_A + r_B), and whose sides
    are at most ``max_block``, is an admissible (far) block; a pair of two leaves that is not admissible is a near
    block; any other pair is refined by cutting the cluster of larger radius (the receiver on a tie within 1e-12,
    the non-leaf one when the other is a leaf).  ``dense``: nothing is admissible.  Returns
    [(r0, p, c0, q, far)] with rows r0 .. r0 + p - 1 and columns c0 .. c0 + q - 1."""
    out = []

    def visit(A: Cluster, B: Cluster):
        p, q = A.hi - A.lo, B.hi - B.lo
        d = float(np.hypot(*(A.centre - B.centre)))
        adm = (not dense) and d > eta_h * (A.radius + B.radius) and p <= max_block and q <= max_block
        if adm or (not A.children and not B.children):
            out.append((A.lo, p, B.lo, q, bool(adm)))
            return
        if not A.children:
            cut_receiver = False
        elif not B.children:
            cut_receiver = True
        else:
            tie = abs(A.radius - B.radius) <= 1e-12 * max(A.radius, B.radius)
            cut_receiver = tie or A.radius > B.radius
        if cut_receiver:
            for C in A.children:
                visit(C, B)
        else:
            for C in B.children:
                visit(A, C)

    visit(cluster_tree(net, a, leaf), cluster_tree(net, b, leaf))
    return out


def cluster_windows(net: Network, leaf: int, eta_h: float, max_block: int, eta_tmax: float, max_steps: int,
                    dense: bool = False, no_trunc: bool = False) -> np.ndarray:
    """Cluster-level end truncation (Sec. 4.3, "Improvement of the algorithm"): the fault-pair criterion of
    Sec. 2.3.2 applied to each block of the H-matrix partition instead of to the whole fault pair.  For a block of
    receiver cluster A and source cluster B, T_max^AB is the largest distance from the two ends of A's segment to
    the ends of B's elements over c_s, and every element pair of the block keeps lags
    T <= min(ceil((1 + eta_Tmax) T_max^AB / dt - 1e-9), max_steps - 1) (every lag with ``no_trunc``).

    Returns last_lag [N][N] (-1 between elements of one fault)."""
    last = np.full((net.N, net.N), -1, dtype=np.int64)
    for a in range(net.F):
        for b in range(net.F):
            if a == b:
                continue
            for r0, p, c0, q, _ in hmatrix_blocks(net, a, b, leaf, eta_h, max_block, dense):
                e1r = net.e1[r0]
                ends = np.stack([net.x[r0] - 0.5 * net.ds[r0] * e1r,
                                 net.x[r0 + p - 1] + 0.5 * net.ds[r0 + p - 1] * e1r])
                cols = slice(c0, c0 + q)
                hb = 0.5 * net.ds[cols][:, None] * net.e1[cols]
                src_ends = np.concatenate([net.x[cols] - hb, net.x[cols] + hb])
                de = ends[:, None, :] - src_ends[None, :, :]
                tmax = np.hypot(de[..., 0], de[..., 1]).max() / net.cs
                lag = math.ceil((1.0 + eta_tmax) * tmax / net.dt - 1e-9)
                last[r0:r0 + p, c0:c0 + q] = max_steps - 1 if no_trunc else min(lag, max_steps - 1)
    return last


# ----------------------------------------------------------------------------------------------------------------
# 5-6. spectral self effect
# ----------------------------------------------------------------------------------------------------------------

_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)


def _gl_panels(a, b, panels):
    """Nodes and weights of a composite 16-point Gauss-Legendre rule with ``panels`` equal panels on [a, b]
    (a, b arrays of the same shape S; result shape S + [panels * 16])."""
    a = np.asarray(a, dtype=np.float64)[..., None]
    b = np.asarray(b, dtype=np.float64)[..., None]
    k = np.arange(panels, dtype=np.float64)
    lo = a + (b - a) * (k / panels)
    h = (b - a) / panels
    x = lo[..., :, None] + 0.5 * h[..., :, None] * (_GL_X + 1.0)
    w = 0.5 * h[..., :, None] * _GL_W * np.ones_like(x)
    return x.reshape(x.shape[:-2] + (-1,)), w.reshape(w.shape[:-2] + (-1,))


def kernel_K(n: int, t, L: float, cs: float) -> np.ndarray:
    """K(n, t) of Eq. (non_replicant_kernel): (1/2pi) int_0^{2pi} cos^2 psi cos(a sin psi) dpsi for c_s t < L and
    (2/pi) int_0^{arcsin(L/(c_s t))} cos^2 psi cos(a sin psi) dpsi for c_s t > L, a = n pi c_s t / L.
    Composite Gauss-Legendre with panels of at most ~one oscillation; used to check the weights (tests)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    a = n * np.pi * cs * t / L
    out = np.empty_like(t)
    short = cs * t < L
    if short.any():
        P = 8 + int(math.ceil(4.0 * float(a[short].max()) / (2 * np.pi)))
        x, w = _gl_panels(np.zeros(short.sum()), np.full(short.sum(), 2 * np.pi), P)
        out[short] = (w * np.cos(x) ** 2 * np.cos(a[short][:, None] * np.sin(x))).sum(-1) / (2 * np.pi)
    if (~short).any():
        pm = np.arcsin(L / (cs * t[~short]))
        P = 8 + int(math.ceil(n * np.pi / (2 * np.pi)))
        x, w = _gl_panels(np.zeros(pm.shape), pm, P)
        out[~short] = (2 / np.pi) * (w * np.cos(x) ** 2 * np.cos(a[~short][:, None] * np.sin(x))).sum(-1)
    return out


def spectral_weights(n: int, T: np.ndarray, dt: float, L: float, cs: float) -> np.ndarray:
    """w_n^T = c_s k_n int_{T dt}^{(T+1) dt} K(n, t) dt, k_n = pi n / L  (Eq. funcational_discretized_form, with the
    pre-integrated kernel of Sec. 2.3.1; reading: the table absorbs c_s k_n so that F_n = -(mu k_n / 2) sum w D).

    Writing K over psi in [0, pi/2] with the indicator c_s t sin(psi) < L (both branches of Eq. non_replicant_kernel)
    and integrating cos(k_n c_s t sin psi) over t in closed form gives, with m = n pi and rho = c_s t / L,
        w = (2/pi) int_0^{psi_0} cos^2(psi) [sin(m min(rho_1 sin psi, 1)) - sin(m min(rho_0 sin psi, 1))] / sin(psi)
    with psi_0 = arcsin(min(1, 1/rho_0)).  The integrand has a kink at arcsin(1/rho_1); the two sides of it are
    integrated separately with panels of at most ~2 oscillations each."""
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    m = n * np.pi
    rho0 = cs * T * dt / L
    rho1 = cs * (T + 1.0) * dt / L
    psi0 = np.where(rho0 > 1.0, np.arcsin(np.minimum(1.0, 1.0 / np.maximum(rho0, 1e-300))), 0.5 * np.pi)
    psia = np.where(rho1 > 1.0, np.arcsin(np.minimum(1.0, 1.0 / rho1)), 0.5 * np.pi)
    psia = np.minimum(psia, psi0)
    phase = m * np.maximum(rho1, 1e-300) * 0.5 * np.pi
    panels = int(2 + math.ceil(float(np.max(np.minimum(phase, m * 2.0))) / (4 * np.pi)))

    def f(x):
        s = np.sin(x)
        return np.cos(x) ** 2 * (np.sin(m * np.minimum(rho1[:, None] * s, 1.0))
                                 - np.sin(m * np.minimum(rho0[:, None] * s, 1.0))) / s

    x, w = _gl_panels(np.zeros_like(psia), psia, panels)
    total = (w * f(x)).sum(-1)
    x, w = _gl_panels(psia, psi0, panels)
    total += (w * f(x)).sum(-1)
    return (2.0 / np.pi) * total


def mode_windows(n_f: int, L: float, dt: float, cs: float, eta_w: float, q_w: int, max_steps: int,
                 no_trunc: bool = False) -> np.ndarray:
    """W_f(n) for n = 0..N_f (index 0 unused): the last lag of mode n's window.
    T_end(n) = T_end(1) Lcal(n), T_end(1) = eta_w L / c_s,
    Lcal(n) = 1/|n| + (q_w - 1)/(n_max - 1) (1 - 1/|n|)   (Eq. mode_dependent_truncation),
    reading n_max = N_f (the padded 2 L_f period carries |n| <= N_f); q_w <= 0 means q_w = n_max;
    W = min(ceil(T_end(n)/dt - 1e-9), max_steps - 1); the whole history when ``no_trunc``."""
    W = np.zeros(n_f + 1, dtype=np.int64)
    qw = n_f if q_w <= 0 else q_w
    for n in range(1, n_f + 1):
        if no_trunc:
            W[n] = max_steps - 1
            continue
        lcal = 1.0 if n_f == 1 else 1.0 / n + (qw - 1.0) / (n_f - 1.0) * (1.0 - 1.0 / n)
        tend = eta_w * L / cs * lcal
        W[n] = min(math.ceil(tend / dt - 1e-9), max_steps - 1)
    return W


def slip_modes(delta: np.ndarray, n_f: int) -> np.ndarray:
    """D_n = (1/M) sum_{j < N_f} delta_j exp(-2 pi i n j / M), n = 0..N_f, M = 2 N_f: the spectral coefficients of
    slip zero-padded to the 2 L_f domain (Eq. functional_no_replication), by direct DFT."""
    M = 2 * n_f
    nn = np.arange(n_f + 1)[:, None]
    jj = np.arange(n_f)[None, :]
    E = np.exp(-2j * np.pi * nn * jj / M) / M
    return delta @ E.T


def modes_to_space(F: np.ndarray, n_f: int, rows=None) -> np.ndarray:
    """f_j = sum_{n=-N_f+1}^{N_f} F_n exp(2 pi i n j / M) with F_{-n} = conj(F_n), kept for j < N_f (the physical
    fault); direct inverse DFT.  F: [..., N_f + 1] for n = 0..N_f."""
    M = 2 * n_f
    j = np.arange(n_f) if rows is None else np.asarray(rows)
    n = np.arange(-n_f + 1, n_f + 1)
    Ffull = np.concatenate([np.conj(F[..., n_f - 1:0:-1]), F[..., : n_f + 1]], axis=-1)
    E = np.exp(2j * np.pi * n[:, None] * j[None, :] / M)
    return (Ffull @ E).real


class SelfTables:
    """Weights w_{f,n}^T for one fault, n = 1..N_f, T = 0..W_f(n); with ``tail``, also the weight mass beyond the
    window, c_n = S_n - sum_{T <= W_f(n)} w_n^T with the static limit S_n = sum_{T >= 0} w_n^T = (2/pi) Si(n pi)
    (the t -> inf limit of Eq. non_replicant_kernel's time integral)."""

    def __init__(self, n_f: int, L: float, dt: float, cs: float, W: np.ndarray, tail: bool = False):
        self.n_f, self.L, self.W = n_f, L, W
        self.w = [np.zeros(0)] + [spectral_weights(n, np.arange(W[n] + 1), dt, L, cs) for n in range(1, n_f + 1)]
        self.c = None
        if tail:
            from scipy.special import sici
            self.c = np.zeros(n_f + 1)
            for n in range(1, n_f + 1):
                self.c[n] = (2.0 / np.pi) * sici(n * np.pi)[0] - self.w[n].sum()


def self_history(net: Network, f: int, delta: np.ndarray, tables: SelfTables) -> np.ndarray:
    """f_self^m on fault f for every step m of its slip history delta[steps][N_f]
    (Eq. funcational_discretized_form then the inverse DFT)."""
    n_f, L = tables.n_f, tables.L
    D = slip_modes(delta, n_f)                     # [steps][N_f + 1]
    steps = delta.shape[0]
    F = np.zeros_like(D)
    for n in range(1, n_f + 1):
        kn = np.pi * n / L
        conv = np.convolve(tables.w[n], D[:, n])[:steps]
        if tables.c is not None:
            # static tail: the slip at the window's far edge, held since t = -inf, times the weight mass beyond
            # the window
            lag = int(tables.W[n]) + 1
            conv[lag:] += tables.c[n] * D[: steps - lag, n]
        F[:, n] = -(net.mu * kn / 2.0) * conv
    return modes_to_space(F, n_f)


def self_rows(net: Network, f: int, delta: np.ndarray, m: int, tables: SelfTables, rows) -> np.ndarray:
    """f_self^m at local ``rows`` of fault f, from delta[0..m][N_f] (windows as in ``tables``; no static tail)."""
    if tables.c is not None:
        raise NotImplementedError("self_rows evaluates the windowed sum only; use self_history with a static tail")
    n_f, L = tables.n_f, tables.L
    Wmax = int(tables.W.max())
    lo = max(0, m - Wmax)
    D = slip_modes(delta[lo: m + 1], n_f)           # D^{lo..m}
    F = np.zeros(n_f + 1, dtype=complex)
    for n in range(1, n_f + 1):
        kn = np.pi * n / L
        T = np.arange(0, min(tables.W[n], m) + 1)
        F[n] = -(net.mu * kn / 2.0) * np.sum(tables.w[n][T] * D[m - T - lo, n])
    return modes_to_space(F, n_f, rows)


# ----------------------------------------------------------------------------------------------------------------
# 7. the whole functional
# ----------------------------------------------------------------------------------------------------------------


def slip_from_rate(V: np.ndarray, dt: float) -> np.ndarray:
    """delta^n = delta^{n-1} + dt V^n, delta^{-1} = 0 (the predictor's slip update, Sec. 2.4, step 2)."""
    return np.cumsum(V * dt, axis=0)


def stress_history(net: Network, V: np.ndarray, hp: dict, slip=None):
    """tau^n for every step of V[steps][N]; returns (tau, rad, self, int), each [steps][N]  (Eq. superimposition2).

    hp: operator parameters (eta_tmin, eta_tmax, eta_w, q_w, max_steps, flags; leaf, eta_h, max_block for
    CLUSTER_TRUNC); windows are applied unless flags has NO_TRUNC (2); with CLUSTER_TRUNC (16) the interaction
    windows end per H-matrix block (cluster_windows; DENSE (1) makes every block a leaf pair).  With STATIC_TAIL
    (4) and windows, the history each window drops is added as a static response: per mode,
    c_n D_n^{m - W_f(n) - 1} (SelfTables); per fault pair, A^static delta^{m - T_last - 1}, the elastostatic stress
    of the slip reached when the pair's window starts (static_slice)."""
    steps = V.shape[0]
    no_trunc = bool(hp.get("flags", 0) & 2)
    tail = bool(hp.get("flags", 0) & 4) and not no_trunc
    max_steps = int(hp.get("max_steps", steps))
    delta = slip_from_rate(V, net.dt) if slip is None else slip
    rad = -(net.mu / (2 * net.cs)) * V
    fself = np.zeros_like(V)
    for f in range(net.F):
        o0, o1 = net.offset[f], net.offset[f + 1]
        n_f = int(net.n_elem[f])
        W = mode_windows(n_f, net.length[f], net.dt, net.cs, hp.get("eta_w", 1.5), hp.get("q_w", 0), max_steps,
                         no_trunc)
        fself[:, o0:o1] = self_history(net, f, delta[:, o0:o1],
                                       SelfTables(n_f, net.length[f], net.dt, net.cs, W, tail=tail))
    _, _, last = pair_windows(net, hp.get("eta_tmin", 0.01), hp.get("eta_tmax", 0.01), max_steps, no_trunc)
    if hp.get("flags", 0) & 16:
        last = cluster_windows(net, int(hp.get("leaf", 32)), float(hp.get("eta_h", 2.0)),
                               int(hp.get("max_block", 0)) or 64, hp.get("eta_tmax", 0.01), max_steps,
                               dense=bool(hp.get("flags", 0) & 1), no_trunc=no_trunc)
    fint = interaction_history(net, V, pair_hi=last)
    if tail:
        fint += static_tail_history(net, delta, last)
    return rad + fself + fint, rad, fself, fint


def static_tail_history(net: Network, delta: np.ndarray, last) -> np.ndarray:
    """Interaction part of the static tail at every step m: -(mu / 2 c_s) sum over source faults b != fault(i) of
    sum_{j in b} A_ij^static delta_j^{m - T_last(a, b) - 1}, where the pair's window still reaches back to step 0
    nothing is added (the dropped lags T > T_last carry A^T ~ dt A^static, and dt sum_{T > T_last} V^{m-T} is that
    slip).  ``last`` per fault pair [F][F], or per element pair [N][N] (cluster-level windows: each element pair's
    own window end T_last(i, j) in place of the pair's)."""
    steps = delta.shape[0]
    As = static_slice(net)
    out = np.zeros((steps, net.N))
    if np.asarray(last).shape == (net.N, net.N) and net.N != net.F:
        L = np.asarray(last)
        other = net.fault_of[:, None] != net.fault_of[None, :]
        for i in range(net.N):
            for lag in np.unique(L[i][other[i]]):
                cols = np.nonzero(other[i] & (L[i] == lag))[0]
                lag = int(lag) + 1
                if lag < steps:
                    out[lag:, i] += delta[: steps - lag, cols] @ As[i, cols]
        return -(net.mu / (2 * net.cs)) * out
    for a in range(net.F):
        ra = slice(net.offset[a], net.offset[a + 1])
        for b in range(net.F):
            if a == b:
                continue
            rb = slice(net.offset[b], net.offset[b + 1])
            lag = int(last[a][b]) + 1
            if lag >= steps:
                continue
            out[lag:, ra] += delta[: steps - lag, rb] @ As[ra, rb].T
    return -(net.mu / (2 * net.cs)) * out


# ----------------------------------------------------------------------------------------------------------------
# traction-free surface by the method of images
# ----------------------------------------------------------------------------------------------------------------


def image_faults(faults: np.ndarray):
    """Method of images for a traction-free surface (App. B; Sec. 4.2 names image methods for simple geometries).

    Every fault's start end c - (L/2) e'_1 lies on the surface; the faults are parallel with e'_1 pointing into the
    medium, and the surface is the line through their start ends normal to e'_1.  Reflection across that line maps
    each fault onto its own continuation beyond the start end.  Continuing the slip evenly, delta(-z) = delta(z)
    with z the distance from the surface, makes the anti-plane displacement even in z, so its z-derivative, and with
    it the shear traction on the surface, vanishes; the full-space functional of the doubled network then gives the
    half-space stress on the real elements.

    Returns (doubled, mirror, real): doubled[f] = (start end x, y, phi, 2 L_f, 2 N_f); mirror[k] = the real element
    whose slip rate element k of the doubled network carries (on fault f: N_f + j and N_f - 1 - j both carry real
    element j); real[i] = the element of the doubled network at real element i (N_f + j)."""
    faults = np.asarray(faults, dtype=np.float64)
    e1 = np.stack([np.cos(faults[:, 2]), np.sin(faults[:, 2])], axis=1)
    start = faults[:, :2] - 0.5 * faults[:, 3:4] * e1
    scale = float(faults[:, 3].max())
    if np.any(e1 @ e1[0] < 1.0 - 1e-12):
        raise ValueError("the faults of a half-space network are parallel, with the same orientation")
    if np.any(np.abs((start - start[0]) @ e1[0]) > 1e-9 * scale):
        raise ValueError("every fault's start end lies on the one free surface")
    doubled = np.column_stack([start, faults[:, 2], 2.0 * faults[:, 3], 2 * faults[:, 4]])
    mirror, real = [], []
    o_real = 0
    o_doubled = 0
    for f in range(faults.shape[0]):
        n = int(faults[f, 4])
        j = np.arange(n)
        mirror.append(np.concatenate([o_real + j[::-1], o_real + j]))
        real.append(o_doubled + n + j)
        o_real += n
        o_doubled += 2 * n
    return doubled, np.concatenate(mirror), np.concatenate(real)


def half_space_stress_history(faults: np.ndarray, mu: float, cs: float, V: np.ndarray, hp: dict,
                              beta: float = 0.5):
    """(tau, rad, self, int) on the real elements of a half-space network, each [steps][N]: stress_history of the
    doubled network of image_faults with the slip rate V[steps][N] continued evenly across the surface.  The
    windows are those of the doubled faults (a self window on the 2 L_f fault, as in App. B)."""
    doubled, mirror, real = image_faults(faults)
    net2 = network(doubled, mu, cs, beta)
    parts = stress_history(net2, V[:, mirror], hp)
    return tuple(p[:, real] for p in parts)

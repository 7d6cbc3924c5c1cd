"""Serving of stress-transfer scenario requests with continuous batching on one GPU.

Requests arrive over time (a seeded Poisson trace); each names a network geometry from a pool, a number of steps
and a seed for its slip-rate history.  The server keeps, per geometry, the H-matrix operator resident in HBM
(built on first use, evicted when idle and the memory is needed) and groups of ``batch`` scenario slots sharing that
operator.  Every tick, each group with an active member advances all its members by one step in one push and one
stress step (one persistent interaction launch serves all members); groups of different geometries run on their
own CUDA streams, so their work overlaps on the device.  A request is admitted into a free slot as soon as one
exists and the HBM budget allows its operator and slot group; a member that finishes is retired at once and its
slot is free for the next request (members of a group start at different ticks: seas_scenario_admit).

The scheduling policy (``Scheduler``) is plain host logic with no device work, so it is tested on the CPU; the
device side (``GpuBackend``) only calls the C ABI.  Per-step latency is measured with CUDA events on each group's
stream.
"""
from __future__ import annotations

import collections
import math
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass
class Request:
    rid: int
    geom: int                    # index into the geometry pool
    steps: int                   # stress steps the request asks for
    seed: int                    # seed of its slip-rate history
    arrival: float               # seconds after the start of the trace
    state: str = "queued"        # queued | active | done | cancelled | rejected
    admitted: float = None       # server clock at admission
    finished: float = None
    done: int = 0                # steps completed
    slot: tuple = None           # (group id, member) while active


def poisson_trace(n_geom: int, rate: float, duration: float, steps_lo: int, steps_hi: int, seed: int = synth.SEED):
    """Requests of a Poisson process of ``rate`` per second over ``duration`` seconds: exponential inter-arrival
    times, geometry uniform over the pool, steps log-uniform in [steps_lo, steps_hi] (SplitMix64 uniforms)."""
    out, t, k = [], 0.0, 0
    while True:
        u = synth.uniform01(seed ^ 0xA44, np.arange(4 * k, 4 * k + 4, dtype=np.uint64))
        t += -math.log(1.0 - u[0]) / rate
        if t >= duration:
            return out
        steps = int(round(math.exp(math.log(steps_lo) + u[2] * (math.log(steps_hi) - math.log(steps_lo)))))
        out.append(Request(rid=k, geom=min(n_geom - 1, int(n_geom * u[1])), steps=steps,
                           seed=int(seed + 7 * k + 1), arrival=t))
        k += 1


@dataclass
class _Group:
    gid: int
    geom: int
    slots: list                  # rid or None per member
    last_used: float = 0.0


class Scheduler:
    """Admission and slot bookkeeping (no device work).

    geom_bytes[g]: device bytes of geometry g's operator; group_bytes[g]: bytes of one slot group (scenario
    handle of ``batch`` members) on it; budget: HBM bytes the server may hold.  ``plan(now)`` returns the actions
    to carry out, in order, and updates the bookkeeping as if they had succeeded:

      ("retire", gid, member, rid)  ("evict", g)  ("drop", gid)  ("build", g)  ("group", g, gid)
      ("admit", gid, member, rid)   ("reject", rid)

    Requests are served first come first served among those that can start; a request whose geometry does not fit
    the whole budget is rejected; one that fits but not now waits while others (on resident geometries) go ahead.
    Idle groups are dropped and idle operators evicted (least recently used first) only when memory is needed."""

    def __init__(self, geom_bytes, group_bytes, budget: int, batch: int):
        self.geom_bytes = list(geom_bytes)
        self.group_bytes = list(group_bytes)
        self.budget = int(budget)
        self.batch = int(batch)
        self.resident = [False] * len(self.geom_bytes)
        self.groups = {}                                     # gid -> _Group
        self.next_gid = 0
        self.used = 0
        self.queue = collections.deque()                     # rids in arrival order
        self.requests = {}
        self.last_use = [0.0] * len(self.geom_bytes)

    # -- requests ------------------------------------------------------------------------------------------------
    def submit(self, req: Request):
        self.requests[req.rid] = req
        self.queue.append(req.rid)

    def cancel(self, rid: int):
        """A queued request leaves the queue; an active one is retired at the next plan()."""
        r = self.requests[rid]
        if r.state == "queued":
            self.queue.remove(rid)
            r.state = "cancelled"
        elif r.state == "active":
            r.state = "cancelled"

    def step_done(self, rid: int):
        """One more completed step of an active request."""
        r = self.requests[rid]
        r.done += 1
        if r.done >= r.steps and r.state == "active":
            r.state = "done"

    # -- planning ------------------------------------------------------------------------------------------------
    def _free_slot(self, g):
        for gr in self.groups.values():
            if gr.geom == g:
                for m, rid in enumerate(gr.slots):
                    if rid is None:
                        return gr, m
        return None, None

    def _idle_group(self, gr):
        return all(rid is None for rid in gr.slots)

    def _make_room(self, need, keep_geom, now, actions):
        """Drop idle groups, then evict idle operators (LRU), until `need` more bytes fit; False if impossible."""
        if self.used + need <= self.budget:
            return True
        for gr in sorted(self.groups.values(), key=lambda x: x.last_used):
            if self._idle_group(gr):
                actions.append(("drop", gr.gid))
                self.used -= self.group_bytes[gr.geom]
                del self.groups[gr.gid]
                if self.used + need <= self.budget:
                    return True
        waiting = {self.requests[rid].geom for rid in self.queue if self.requests[rid].arrival <= now}
        for g in sorted(range(len(self.resident)), key=lambda x: self.last_use[x]):
            if not self.resident[g] or g == keep_geom or g in waiting:
                continue
            if any(gr.geom == g for gr in self.groups.values()):
                continue
            actions.append(("evict", g))
            self.resident[g] = False
            self.used -= self.geom_bytes[g]
            if self.used + need <= self.budget:
                return True
        return self.used + need <= self.budget

    def plan(self, now: float):
        actions = []
        for gr in self.groups.values():
            for m, rid in enumerate(gr.slots):
                if rid is not None and self.requests[rid].state in ("done", "cancelled"):
                    actions.append(("retire", gr.gid, m, rid))
                    gr.slots[m] = None
                    r = self.requests[rid]
                    r.slot = None
                    r.finished = now
        keep = collections.deque()
        while self.queue:
            rid = self.queue.popleft()
            r = self.requests[rid]
            if r.arrival > now:
                keep.append(rid)
                continue
            g = r.geom
            if self.geom_bytes[g] + self.group_bytes[g] > self.budget:
                actions.append(("reject", rid))
                r.state = "rejected"
                continue
            gr, m = self._free_slot(g)
            if gr is None:
                need = self.group_bytes[g] + (0 if self.resident[g] else self.geom_bytes[g])
                if not self._make_room(need, g, now, actions):
                    keep.append(rid)
                    continue
                if not self.resident[g]:
                    actions.append(("build", g))
                    self.resident[g] = True
                    self.used += self.geom_bytes[g]
                gr = _Group(self.next_gid, g, [None] * self.batch, now)
                self.next_gid += 1
                self.groups[gr.gid] = gr
                self.used += self.group_bytes[g]
                actions.append(("group", g, gr.gid))
                m = 0
            gr.slots[m] = rid
            gr.last_used = now
            self.last_use[g] = now
            r.state = "active"
            r.admitted = now
            r.slot = (gr.gid, m)
            actions.append(("admit", gr.gid, m, rid))
        self.queue = keep
        return actions

    def active_groups(self):
        return [gr for gr in self.groups.values() if any(rid is not None for rid in gr.slots)]


# ---------------------------------------------------------------------------------------------------- device side --

class GpuBackend:
    """Carries out a Scheduler's actions through the C ABI: one context (with its own torch stream) and operator per
    resident geometry, one scenario handle of ``batch`` members per group."""

    def __init__(self, geometries, batch: int, device: int = 0, precision: int = 0, record: bool = False,
                 tune: bool = True):
        import tempfile
        import torch
        from . import seas
        self.torch, self.seas = torch, seas
        # the interaction's consumer warps per pass, tuned once per operator when it is built (off the serving clock)
        # and applied to each of its groups from this cache file
        self.tune_cache = os.path.join(tempfile.mkdtemp(prefix="seas_serve_tune_"), "choices.txt") if tune else None
        self.geoms = geometries
        self.batch = batch
        self.device = device
        self.precision = precision
        self.record = record                                  # keep every request's tau history (tests)
        self.ctx, self.net, self.op = {}, {}, {}
        self.stream = {}
        self.groups = {}                                      # gid -> dict(scn, geom, V, tau, members)
        self.streams_of = {}
        self.history = {}                                     # rid -> list of tau rows (record mode)
        self.build_seconds = {}

    def build(self, g):
        torch, seas = self.torch, self.seas
        w = self.geoms[g]
        st = torch.cuda.Stream(device=self.device)
        t0 = time.perf_counter()
        ctx = seas.seas_create(self.device, 0, st)
        net = seas.seas_build_network(ctx, w.faults, w.mu, w.cs, w.cp, w.beta)
        op, stats = seas.seas_build_hmatrix(net, dict(w.hparams, precision=self.precision))
        if self.tune_cache:
            probe = seas.seas_scenario_create(op, self.batch)
            seas.seas_scenario_autotune(probe, self.tune_cache, reps=3)
            seas.seas_destroy_scn(probe)
        self.build_seconds[g] = time.perf_counter() - t0
        self.ctx[g], self.net[g], self.op[g], self.stream[g] = ctx, net, op, st

    def held(self, g):
        """Device bytes the library holds for geometry g (network, operator and its slot groups)."""
        return self.seas.seas_ctx_get_memory(self.ctx[g])[0] if g in self.ctx else 0

    def evict(self, g):
        seas = self.seas
        seas.seas_sync(self.ctx[g])
        seas.seas_destroy_op(self.op.pop(g))
        seas.seas_destroy_net(self.net.pop(g))
        seas.seas_destroy_ctx(self.ctx.pop(g))
        self.stream.pop(g)

    def group(self, g, gid):
        torch, seas = self.torch, self.seas
        w = self.geoms[g]
        scn = seas.seas_scenario_create(self.op[g], self.batch)
        if self.tune_cache:
            seas.seas_scenario_autotune(scn, self.tune_cache, reps=1)          # the operator's choice, cached
        for m in range(self.batch):
            seas.seas_scenario_retire(scn, m)
        with torch.cuda.stream(self.stream[g]):
            V = torch.zeros((self.batch, w.N), dtype=torch.float64, device=self.device)
            tau = torch.zeros((self.batch, w.N), dtype=torch.float64, device=self.device)
        self.groups[gid] = dict(scn=scn, geom=g, V=V, tau=tau, members=[None] * self.batch,
                                ev=None, pending=None)

    def drop(self, gid):
        G = self.groups.pop(gid)
        self.seas.seas_sync(self.ctx[G["geom"]])
        self.seas.seas_destroy_scn(G["scn"])

    def admit(self, gid, m, req):
        G = self.groups[gid]
        w = self.geoms[G["geom"]]
        self.seas.seas_scenario_admit(G["scn"], m)
        with self.torch.cuda.stream(self.stream[G["geom"]]):
            G["members"][m] = (req, synth.SlipRateStream(w, req.seed, self.torch.device("cuda", self.device)))
        if self.record:
            self.history[req.rid] = []

    def retire(self, gid, m):
        G = self.groups[gid]
        self.seas.seas_scenario_retire(G["scn"], m)
        G["members"][m] = None
        with self.torch.cuda.stream(self.stream[G["geom"]]):
            G["V"][m].zero_()

    def tick(self, gid):
        """Issues one step of every active member of the group on its geometry's stream; returns the event pair
        that brackets it.  The previous tick of this group must have completed (the caller waits on its event)."""
        torch, seas = self.torch, self.seas
        G = self.groups[gid]
        st = self.stream[G["geom"]]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            for m, mem in enumerate(G["members"]):
                if mem is not None:
                    req, src = mem
                    G["V"][m].copy_(src.row(req.done), non_blocking=True)
            seas.seas_push_slip_rate(G["scn"], G["V"].view(-1))
            seas.seas_stress_step(G["scn"], G["tau"].view(-1))
            e1.record(st)
            if self.record:
                for m, mem in enumerate(G["members"]):
                    if mem is not None:
                        self.history[mem[0].rid].append(G["tau"][m].clone())
        return e0, e1


class Server:
    """Runs a request trace against the GPU backend in wall-clock time: arrivals are released when the server's
    clock passes them, each loop iteration plans admissions and issues one tick per active group, and the loop waits
    on each group's previous tick before issuing its next one (at most one tick in flight per group)."""

    def __init__(self, geometries, budget: int, batch: int = 8, device: int = 0, precision: int = 0,
                 record: bool = False, geom_bytes=None, group_bytes=None):
        self.backend = GpuBackend(geometries, batch, device, precision, record)
        if geom_bytes is None or group_bytes is None:
            geom_bytes, group_bytes = estimate_bytes(geometries, batch, precision)
        self.sched = Scheduler(geom_bytes, group_bytes, budget, batch)
        self.latency_ms = []                                 # per request-step
        self.element_steps = 0
        self.ticks = 0

    def prebuild(self, geoms):
        """Warm start: builds the operators of ``geoms`` (in order, while they fit the budget) before serving."""
        sch = self.sched
        for g in geoms:
            if sch.resident[g] or sch.used + sch.geom_bytes[g] > sch.budget:
                continue
            self.backend.build(g)
            sch.resident[g] = True
            sch.used += sch.geom_bytes[g]
            self._reconcile_geom(g, self.backend.held(g))

    def run(self, trace, until: float = None, time_scale: float = 1.0):
        """Serves ``trace`` until every request is finished (or the server clock reaches ``until`` seconds);
        returns the wall time.  time_scale > 1 releases arrivals faster than real time."""
        sched, be = self.sched, self.backend
        for r in trace:
            sched.submit(r)
        inflight = {}                                        # gid -> (e0, e1, [rids stepped])
        t_start = time.perf_counter()
        while True:
            now = (time.perf_counter() - t_start) * time_scale
            for gid, (e0, e1, rids) in list(inflight.items()):
                if e1.query():
                    self._complete(gid, e0, e1, rids)
                    del inflight[gid]
            for act in sched.plan(now):
                kind = act[0]
                if kind == "build":
                    g = act[1]
                    be.build(g)
                    self._reconcile_geom(g, be.held(g))
                elif kind == "evict":
                    be.evict(act[1])
                elif kind == "group":
                    g = act[1]
                    before = be.held(g)
                    be.group(g, act[2])
                    self._reconcile_group(g, be.held(g) - before)
                elif kind == "drop":
                    be.drop(act[1])
                elif kind == "admit":
                    be.admit(act[1], act[2], sched.requests[act[3]])
                elif kind == "retire":
                    be.retire(act[1], act[2])
            active = sched.active_groups()
            issued = False
            for gr in active:
                if gr.gid in inflight:
                    continue
                rids = [rid for rid in gr.slots if rid is not None and sched.requests[rid].state == "active"]
                if not rids:
                    continue
                e0, e1 = be.tick(gr.gid)
                inflight[gr.gid] = (e0, e1, rids)
                issued = True
                self.ticks += 1
            pending = [r for r in sched.requests.values() if r.state in ("queued", "active")]
            if not pending and not inflight:
                break
            if until is not None and now >= until:
                for gid, (e0, e1, rids) in inflight.items():
                    e1.synchronize()
                    self._complete(gid, e0, e1, rids)
                break
            if not issued and inflight:
                next(iter(inflight.values()))[1].synchronize()
            elif not issued and not inflight:
                waiting = [r.arrival for r in pending if r.state == "queued"]
                if waiting and min(waiting) > now:
                    time.sleep(min(0.01, (min(waiting) - now) / time_scale))
        return time.perf_counter() - t_start

    def _reconcile_geom(self, g, actual):
        """Replaces the planned bytes of geometry g's operator with what the library holds after the build."""
        sch = self.sched
        sch.used += actual - sch.geom_bytes[g]
        sch.geom_bytes[g] = actual

    def _reconcile_group(self, g, actual):
        sch = self.sched
        sch.used += actual - sch.group_bytes[g]
        sch.group_bytes[g] = actual

    def _complete(self, gid, e0, e1, rids):
        ms = e0.elapsed_time(e1)
        G = self.backend.groups.get(gid)
        N = self.backend.geoms[G["geom"]].N if G is not None else 0
        for rid in rids:
            self.latency_ms.append(ms)
            self.element_steps += N
            self.sched.step_done(rid)


def estimate_bytes(geometries, batch: int, precision: int):
    """Device bytes of each geometry's operator and of one slot group, from the host-only plan: the causal block
    slices at the element size of the precision (dense upper bound, i.e. before compression) plus the spectral
    tables, and per group the slip-rate, spectral and partial-sum buffers."""
    from . import seas
    eb = 2 if precision in (1, 2) else 8
    gb, sb = [], []
    for w in geometries:
        p = seas.seas_plan_hmatrix(w.faults, w.mu, w.cs, w.cp, w.beta, dict(w.hparams, precision=precision))
        blocks, last = p["blocks"], p["pair_last"]
        lags = np.maximum(0, blocks[:, 6].astype(np.int64) - blocks[:, 5] + 1)
        entries = int(np.sum(blocks[:, 1].astype(np.int64) * blocks[:, 3] * lags))
        W = max(int(max(x.max() for x in p["mode_windows"])), 1)
        ring = max(int(last.max()) + 1, 1)
        gb.append(entries * eb + 8 * W * (w.N + w.n_faults))
        sb.append(batch * (ring * w.N * (8 + (0 if eb == 8 else 4)) + (W + 1) * (w.N + w.n_faults) * 16
                           + 16 * w.N * 8) + len(blocks) * 64 * 8 * batch)
    return gb, sb

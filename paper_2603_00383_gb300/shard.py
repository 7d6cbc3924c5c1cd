"""Sharding one scenario across GPUs by receiver faults.

Each rank owns a set of faults: it builds the part of the operator whose receivers lie on them
(seas_build_hmatrix_part: their spectral self effects and their H-matrix block rows) and returns tau on them.  Every
step needs the whole slip-rate history as sources, so the ranks exchange their faults' slip rates with one
all-gather per step (a SEAS solver computes V per fault, Sec. 2.4, so each rank has only its own) and push the
gathered vector.  The operator rows are the expensive part (O(N^2 W)); the exchange moves N * 8 bytes per step.

The exchange and the bookkeeping here are host logic; the stress evaluation is a callable, so the multi-rank path is
tested on the CPU with gloo ranks and any evaluator.
"""
from __future__ import annotations

import numpy as np


def partition_faults(n_elem, world: int):
    """Faults to ranks, largest first to the least loaded rank, the load of a fault being its element count (its
    rows of the operator span every source column, so the work of a rank grows with the elements it owns)."""
    n_elem = [int(n) for n in n_elem]
    order = sorted(range(len(n_elem)), key=lambda f: (-n_elem[f], f))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for f in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(f)
        load[r] += n_elem[f]
    return [sorted(p) for p in parts]


def owned_elements(n_elem, faults):
    """Global element indices of `faults`, in element order."""
    off = np.concatenate([[0], np.cumsum([int(n) for n in n_elem])])
    return np.concatenate([np.arange(off[f], off[f + 1]) for f in sorted(faults)]).astype(np.int64)


class ShardedStepper:
    """One rank's view of a scenario sharded by receiver faults.

    dist: torch.distributed (initialised); n_elem: elements per fault; evaluate(V_full) -> tau over all elements
    (only the owned entries are used; on a GPU a partial operator's seas_push_slip_rate + seas_stress_step)."""

    def __init__(self, dist, n_elem, evaluate, device="cpu"):
        import torch
        self.torch, self.dist = torch, dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.parts = partition_faults(n_elem, self.world)
        self.index = [owned_elements(n_elem, p) for p in self.parts]
        self.mine = self.index[self.rank]
        self.N = int(sum(int(n) for n in n_elem))
        self.width = max(len(ix) for ix in self.index)
        self.evaluate = evaluate
        self.device = device
        self.gather_idx = torch.from_numpy(np.concatenate(self.index)).to(device)

    def gather(self, V_local):
        """The slip rates of every fault from each rank's own (all-gather of equal-width buffers)."""
        torch = self.torch
        buf = torch.zeros(self.width, dtype=torch.float64, device=self.device)
        buf[: len(self.mine)] = V_local
        bufs = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(bufs, buf)
        flat = torch.cat([b[: len(ix)] for b, ix in zip(bufs, self.index)])
        V = torch.empty(self.N, dtype=torch.float64, device=self.device)
        V[self.gather_idx] = flat
        return V

    def step(self, V_local):
        """Exchanges this step's slip rates and returns tau on the owned elements."""
        V = self.gather(V_local)
        tau = self.evaluate(V)
        return tau[self.torch.from_numpy(self.mine).to(tau.device)] if not isinstance(tau, np.ndarray) else \
            tau[self.mine]

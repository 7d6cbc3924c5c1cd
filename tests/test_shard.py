"""Sharding one scenario by receiver faults (no GPU): the partition, and the per-step exchange of slip rates between
two gloo ranks, launched like torchrun would, with the CPU oracle as the evaluator of each rank's rows."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_balances_elements_and_covers_every_fault_once():
    from paper_2603_00383_gb300 import shard
    n_elem = [256, 384, 512, 512, 640, 768]
    for world in (1, 2, 3, 4, 6):
        parts = shard.partition_faults(n_elem, world)
        assert sorted(f for p in parts for f in p) == list(range(6))
        loads = [sum(n_elem[f] for f in p) for p in parts]
        assert max(loads) - min(loads) <= max(n_elem)
    assert shard.partition_faults(n_elem, 2) == [[0, 3, 5], [1, 2, 4]]    # 768+512+256 = 640+512+384
    ix = shard.owned_elements([3, 2, 4], [2, 0])
    assert ix.tolist() == [0, 1, 2, 5, 6, 7, 8]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist
        from oracle import seas_oracle as O
        from paper_2603_00383_gb300 import shard, synth
        dist.init_process_group("gloo", rank=rank, world_size=world)
        w = synth.tiny(3, n_faults=3, steps=30)
        net = O.network(w.faults, w.mu, w.cs)
        hp = dict(w.hparams, flags=2)
        V = w.slip_rate(0, 0, w.steps)
        ref = O.stress_history(net, V, hp)[0]
        hist = []

        def evaluate(Vfull):
            hist.append(Vfull.numpy().copy())
            return torch.from_numpy(O.stress_history(net, np.stack(hist), hp)[0][-1])

        st = shard.ShardedStepper(dist, w.n_elem, evaluate)
        worst_v, worst_t = 0.0, 0.0
        for n in range(w.steps):
            tau = st.step(torch.from_numpy(V[n][st.mine]))
            worst_v = max(worst_v, float(np.abs(hist[-1] - V[n]).max()))
            worst_t = max(worst_t, float(np.abs(tau.numpy() - ref[n][st.mine]).max() / np.abs(ref).max()))
        q.put((rank, st.parts, len(st.mine), worst_v, worst_t))
        dist.destroy_process_group()
    except Exception as e:                                   # report instead of hanging the parent
        q.put(("error", rank, repr(e)))


def test_two_gloo_ranks_exchange_slip_rates_and_own_their_rows():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(o[0] != "error" for o in out), out
    out.sort()
    assert out[0][1] == out[1][1]                            # both ranks derive the same partition
    from paper_2603_00383_gb300 import synth
    assert out[0][2] + out[1][2] == synth.tiny(3, n_faults=3).N
    assert all(o[3] == 0.0 for o in out)                     # the gathered slip rates are the global ones
    # each rank's rows are the unsharded rows (the oracle's self term over histories of different lengths rounds
    # differently, hence a relative 1e-13 rather than 0)
    assert all(o[4] < 1e-13 for o in out), out

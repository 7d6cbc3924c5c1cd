"""The bench's N > 1 path on CPU: two gloo ranks, launched like torchrun would (RANK / WORLD_SIZE / MASTER_*).

Checks the barrier, the max-over-ranks time, independent scenario seeds per rank, the whole-job rate, and that
the oracle arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    try:
        import bench
        from paper_2603_00383_gb300 import synth
        dist, r, w, local = bench.dist_setup(None)
        bench.barrier(dist)
        slowest = bench.max_over_ranks(dist, 1.5 + r, "cpu")        # rank r "took" 1.5 + r seconds
        ref = bench.run_reference(None, synth.two_fault_128(), 396, 4, 3) if r != 0 else "skipped"
        q.put((r, w, local, slowest, bench.rank_seed(r), ref))
        dist.destroy_process_group()
    except Exception as e:                                        # report instead of hanging the parent
        q.put(("error", rank, repr(e)))


def test_two_gloo_ranks_share_only_the_barrier_and_the_max_time():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(o[0] != "error" for o in out), out
    out.sort()
    import bench
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 2.5 for o in out)                         # both see the slowest rank's time
    assert out[0][4] != out[1][4]                                # independent scenarios
    assert out[1][5] is None                                     # the oracle arm does no work off rank 0
    assert bench.job_rate(3072 * 2000, 2, 2.5) == pytest.approx(2 * 3072 * 2000 / 2.5)


def test_timed_window_is_the_deepest_steps_whatever_k_is():
    """The bench always runs the workload for its full length and times its K deepest steps."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_00383_gb300 import synth
    w = synth.six_fault_3072()
    assert bench.window(w, 20) == (1980, 20)
    assert bench.window(w, 5000) == (0, 2000)
    elems, steps = bench.oracle_sample(w, 1980, 20, 48)
    assert steps.min() >= 1980 and steps.max() < 2000 and elems.max() < 256
    rows = bench.oracle_rows(w)
    off = [0, 256, 640, 1152, 1664, 2304, 3072]
    assert all(any(off[f] <= r < off[f + 1] for r in rows) for f in range(6))

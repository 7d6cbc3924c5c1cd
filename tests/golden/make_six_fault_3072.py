"""Writes six_fault_3072_oracle.txt: CPU-oracle values of the six-fault, 3072-element workload at full size (2000
steps, the workload's causal and spectral windows), for the sampled-row parity test.

    python tests/golden/make_six_fault_3072.py [--procs 8]

Calls only ``oracle.seas_oracle`` and the seeded inputs of ``paper_2603_00383_gb300.synth``; nothing here comes
from the CUDA library.  Rows and steps:

* interaction part f_int (Eq. fault-to-fault_interactions_discretized, pair windows of Sec. 2.3.2): 64 receivers
  spread over all six faults, at steps 401, 1597, 1598 and 1999 (1598 is the first step past the shortest pair
  window, which ends at lag 1597);
* spectral self part f_self (Eq. funcational_discretized_form, windows of Eq. mode_dependent_truncation): 8
  receivers of every fault (sizes 256, 384, 512, 512, 640, 768: radix 2, 3 and 5 transforms) at the same steps.

Each line: ``part step global_row value``.  The oracle's spectral tables of the large faults take minutes to
build, which is why the values are stored rather than recomputed inside a GPU test.
"""
import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

STEPS = (401, 1597, 1598, 1999)
OUT = os.path.join(HERE, "six_fault_3072_oracle.txt")


def rows_int(N):
    return np.unique(np.round(np.linspace(0, N - 1, 64)).astype(int))


def rows_self(nf):
    return np.unique(np.round(np.linspace(0, nf - 1, 8)).astype(int))


def _setup():
    from oracle import seas_oracle as O
    from paper_2603_00383_gb300 import synth
    w = synth.six_fault_3072()
    net = O.network(w.faults, w.mu, w.cs)
    V = w.slip_rate(0, 0, w.steps)
    return O, w, net, V


def job_int(args):
    n, rows = args
    O, w, net, V = _setup()
    hp = w.hparams
    _, _, last = O.pair_windows(net, hp["eta_tmin"], hp["eta_tmax"], hp["max_steps"])
    return [("int", n, int(r), float(v)) for r, v in zip(rows, O.interaction_rows(net, V, n, rows, pair_hi=last))]


def job_self(f):
    O, w, net, V = _setup()
    hp = w.hparams
    nf = int(net.n_elem[f])
    W = O.mode_windows(nf, net.length[f], net.dt, net.cs, hp["eta_w"], hp["q_w"], hp["max_steps"])
    tab = O.SelfTables(nf, net.length[f], net.dt, net.cs, W)
    o0 = int(net.offset[f])
    delta = O.slip_from_rate(V, net.dt)[:, o0:o0 + nf]
    rows = rows_self(nf)
    out = []
    for n in STEPS:
        vals = O.self_rows(net, f, delta[: n + 1], n, tab, rows)
        out += [("self", n, o0 + int(r), float(v)) for r, v in zip(rows, vals)]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    N = 3072
    ri = rows_int(N)
    jobs_i = [(n, ri[k:k + 8]) for n in STEPS for k in range(0, len(ri), 8)]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res_s = pool.map_async(job_self, list(range(5, -1, -1)), chunksize=1)
        res_i = pool.map_async(job_int, jobs_i, chunksize=1)
        lines = [x for r in res_s.get() + res_i.get() for x in r]
    lines.sort(key=lambda t: (t[0], t[1], t[2]))
    with open(OUT, "w") as fh:
        fh.write("# CPU-oracle values of six_fault_3072 (2000 steps, workload windows); written by "
                 "make_six_fault_3072.py\n# part step global_row value\n")
        for p, n, r, v in lines:
            fh.write(f"{p} {n} {r} {v!r}\n")
    print(f"wrote {len(lines)} values to {OUT}")


if __name__ == "__main__":
    main()

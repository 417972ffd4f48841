"""Multi-rank host logic on CPU ranks (gloo, world size 2).

Sequences do not shard (problem l+1 needs problem l's vectors), but independent sequences
(k-points of one SCF cycle) do: each rank solves its own seeded sequence with no data-path
collective, and the benchmark combines the ranks' timings (max) and converged pairs (sum).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle.chfsi_oracle as O
        from paper_1206_3768_gb300 import inputs

        seq = inputs.planted_sequence("c1", n=96, N=2, nev=6, blk=10, seed_offset=rank)
        As = [np.tril(p.A.numpy()) for p in seq.problems]
        Bs = [np.tril(p.B.numpy()) for p in seq.problems]
        res = O.chfsi_solve_sequence(As, Bs, 6, 10, 1e-10, deg=10)
        conv = sum(int(np.isfinite(lam).sum()) for lam, _, _ in res)
        err = max(float(np.max(np.abs(lam - p.lam[:6]))) for (lam, _, _), p in zip(res, seq.problems))
        ms = 100.0 + 50.0 * rank
        ms_max, units = bench.combine_ranks(ms, conv)
        out[rank] = (ms_max, units, conv, err, float(seq.problems[0].lam[0]))
    finally:
        dist.destroy_process_group()


def test_weak_scaling_combination_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    # both ranks see the slowest time and the sum of the units
    assert r0[0] == r1[0] == 150.0
    assert r0[1] == r1[1] == r0[2] + r1[2] == 24.0
    # every rank solved its own (different) sequence to the planted spectrum
    assert r0[3] < 1e-10 and r1[3] < 1e-10
    assert r0[4] != r1[4]

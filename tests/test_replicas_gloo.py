"""The N>1 benchmark path on CPU: one process per rank (world size 2, gloo
on 127.0.0.1), each solving its own seeded replica with no collective on
the data path; the only exchange is the max-over-ranks timing reduction.
Each rank's replica equals the same replica solved in a single process."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank):
    from oracle import OracleProblem, pitsbicg
    from paper_2203_10148_gb300 import inputs
    from paper_2203_10148_gb300.replicas import replica_seed
    w = inputs.heat1d(N=8, seed=replica_seed(inputs.SEED_HEAT1D, rank, 0))
    X, info = pitsbicg(OracleProblem.from_workload(w), tol=1e-10)
    return w, X, info


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2203_10148_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, wsize, local = replicas.dist_env()
        assert (r, wsize, local) == (rank, world, rank)
        w, X, info = _replica(rank)
        replicas.barrier()
        # ranks take different times; the job takes the slowest one's
        t = replicas.max_over_ranks([1.0 + rank, 10.0 - rank])
        rate = replicas.whole_job_rate(3, world, t[0])
        out[rank] = {"X": X, "y0": w.y0.copy(), "iters": info.iterations, "t": t, "rate": rate}
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        assert res[rank]["t"] == [2.0, 10.0]
        assert res[rank]["rate"] == pytest.approx(3 * world / 2.0)
    # distinct inputs per rank, each solved exactly as in one process
    assert not np.allclose(res[0]["y0"], res[1]["y0"])
    for rank in range(world):
        _, X, info = _replica(rank)
        assert np.array_equal(res[rank]["X"], X)
        assert res[rank]["iters"] == info.iterations


def test_single_process_helpers():
    from paper_2203_10148_gb300 import replicas
    assert replicas.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert replicas.replica_seed(10, 0, 0) == 10
    seeds = {replicas.replica_seed(0, r, s) for r in range(8) for s in range(13)}
    assert len(seeds) == 8 * 13
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1, 1, 0.0)

"""Multi-rank host logic of bench.py (replicas, weak scaling) on CPU ranks.

The path shards over independent right-hand sides, so the only cross-rank
step of the benchmark is the maximum of the per-rank timings.  Two gloo ranks
on 127.0.0.1 check it, and the whole-job value built from it."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    got_ws, got_rank, got_local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://")
    # rank r took (r + 1) ms for the window and 10 - r ms for the whole job
    ms, whole = bench.max_over_ranks([rank + 1.0, 10.0 - rank], "cpu", ws)
    value = bench.whole_job_value(64, 256, ws, whole)
    out[rank] = (got_ws, got_rank, got_local, ms, whole, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_value():
    ws = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of this multi-threaded process
    out = mgr.dict()
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    for r in range(ws):
        got_ws, got_rank, got_local, ms, whole, value = out[r]
        assert (got_ws, got_rank, got_local) == (ws, r, r)
        assert ms == 2.0          # slowest window over the ranks
        assert whole == 10.0      # slowest whole job over the ranks
        assert value == pytest.approx(64 * 256 * ws / 10e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3.5, 7.0], "cpu", 1) == [3.5, 7.0]
    assert bench.whole_job_value(8, 10, 1, 20.0) == pytest.approx(8 * 10 / 0.02)

"""The multi-GPU path of bench.py is N independent replicas (one lattice per
rank, no collective on the data path): ranks meet only at barriers and in
the max-over-ranks timing.  That host logic runs here as two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    ms = 10.0 + 5.0 * r  # rank 1 is the slow one
    m = bench.max_over_ranks(w, ms)
    out.put((r, w, m, bench.weak_scaling_value(w, 1000, 20, m)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; value = 2 replicas x nodes x steps / that time
    assert [x[2] for x in res] == [15.0, 15.0]
    assert all(x[1] == 2 for x in res)
    assert abs(res[0][3] - 2 * 1000 * 20 / 15e-3 / 1e6) < 1e-9


def test_reference_arm_other_ranks_exit_quietly(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(A(), 2, 1) == 0
    assert capsys.readouterr().out == ""

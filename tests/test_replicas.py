"""The N > 1 path of bench.py, on CPU: two ranks over gloo (one process per rank, rendezvous on
127.0.0.1).  Atmospheres are independent, so the ranks own disjoint shards of the workload and
the process group carries only barriers and the max-over-ranks time; rank 0 alone reports, and
under --impl reference the other ranks exit without work."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch
    r, w, local = bench.dist_env()
    bench.init_replicas(w, local, backend="gloo")
    cpu = torch.device("cpu")
    got = {"rank": r}
    got["max"] = bench.max_over_ranks(10.0 * (r + 1), w, cpu)
    got["sum"] = bench.sum_over_ranks(r + 1, w, cpu)
    got["ids"] = bench.replica_ids(r, 5)
    bench.barrier(w)
    # the reference arm under torchrun: rank 0 alone runs; the others return without output
    if r != 0:
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(None)
        got["reference_output"] = buf.getvalue()
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put(got)


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {d["rank"]: d for d in res}
    assert res[0]["max"] == res[1]["max"] == 20.0
    assert res[0]["sum"] == res[1]["sum"] == 3.0
    assert not set(res[0]["ids"]) & set(res[1]["ids"])
    assert sorted(res[0]["ids"] + res[1]["ids"]) == list(range(10))
    assert res[1]["reference_output"] == ""

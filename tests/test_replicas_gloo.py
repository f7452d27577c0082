"""The multi-process path of bench.py on CPU (gloo, world size 2, 127.0.0.1): the operator does
not shard on one GPU's data, so N ranks run N independent replicas and the only exchange is the
timing reduction -- max of the step times, sum of the applies -- and only rank 0 reports."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.reduce_max_sum(10.0 + 5.0 * rank, 2.0 * (rank + 1))
    bench.barrier()
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "grav16"])
    dist.destroy_process_group()
    q.put((rank, t, u, rc, buf.getvalue()))


def test_two_replicas_reduce_and_report_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, t, u, rc, out = q.get(timeout=240)
        res[rank] = (t, u, rc, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        t, u, rc, _ = res[rank]
        assert (t, u, rc) == (15.0, 6.0, 0)  # max(10, 15), 2 + 4, both ranks exit 0
    line = json.loads(res[0][3].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert res[1][3].strip() == ""  # rank 1 prints nothing

"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

Under torchrun every rank runs its own replica of the workload; the only
cross-rank steps are the barrier and the max over ranks of the timed region.
The reference arm runs on rank 0 alone.
"""
import contextlib
import io
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (ws, rank)
    # the timed region's duration is the max over ranks
    got = bench.dist_max(1.5 + rank, w)
    bench.barrier(w)
    # reference arm: rank 0 prints one JSON line, the others print nothing
    out = io.StringIO()
    args = argparse.Namespace(gpus=ws, steps=1, warmup=0, ref_n=300)
    with contextlib.redirect_stdout(out):
        bench.run_reference(args, w, r)
    dist.destroy_process_group()
    q.put((rank, got, out.getvalue()))


def test_world_size_2_max_and_reference_arm():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(ws):
        rank, got, text = q.get(timeout=120)
        res[rank] = (got, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 2.5
    assert res[1][1] == ""
    line = json.loads(res[0][1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


if __name__ == "__main__":
    pytest.main([__file__, "-q"])

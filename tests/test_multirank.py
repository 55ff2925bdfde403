"""The multi-rank path of bench.py on CPU (gloo, world size 2): rendezvous, barrier, the
max-over-ranks timing reduction, and the weak-scaling split into independent light cones."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, outdir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2111_08744_gb300 import inputs as I
    wsz, r, _ = bench.dist_init()
    assert (wsz, r) == (ws, rank)
    bench.barrier(wsz)
    m = bench.max_over_ranks(10.0 * (rank + 1), wsz)
    base = I.config_plain_small()
    w = bench.rank_workload(base, rank, wsz)
    res = {"max": m, "observer": w.observer.tolist(), "n_rays": w.n_rays,
           "same_field": bool(w.levels is base.levels), "same_dirs": bool(np.array_equal(w.dirs, base.dirs))}
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    assert r[0]["max"] == r[1]["max"] == 20.0
    assert r[0]["observer"] != r[1]["observer"]
    assert all(x["same_field"] and x["same_dirs"] for x in r)
    assert r[0]["n_rays"] == r[1]["n_rays"] == 3072

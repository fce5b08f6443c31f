"""The multi-replica path of bench.py on the host: two gloo ranks (CPU), the timing
barrier, the max / sum reductions and the whole-job throughput they give, and the
reference arm's rank > 0 exit without work.  The ranks are replicas (no data-path
collective), so this is all the multi-GPU logic there is."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out_dir):
    os.environ.update(WORLD_SIZE=str(ws), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init("gloo")
    res = {"ws": w, "rank": r, "local": local}
    bench.barrier(w)
    res["max"] = bench.max_over_ranks(float(rank + 1), w)
    res["sum"] = bench.sum_over_ranks(float(rank + 1), w)
    # rank r processed 10 (r + 1) units in 1 + r seconds
    res["thr"] = bench.job_throughput(10.0 * (rank + 1), 1.0 + rank, w)
    if rank > 0:
        class A:   # the reference arm's arguments
            steps, warmup, cycle = 1, 0, "V"
        res["ref"] = bench.run_reference(A())   # returns at once on ranks > 0
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_replicas(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    for r, g in enumerate(got):
        assert (g["ws"], g["rank"], g["local"]) == (2, r, r)
        assert g["max"] == 2.0 and g["sum"] == 3.0
        assert g["thr"] == pytest.approx((10.0 + 20.0) / 2.0)
    assert got[1]["ref"] is None

"""Host logic of the multi-process (one rank per GPU, replicas only) benchmark path, run as two gloo
ranks on the CPU: the job's time is the maximum over ranks, throughput counts every rank's units,
each replica draws its own catalogue, and the reference arm runs on rank 0 only."""

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_1512_07295_gb300 import catalogs

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_job = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
        cat = catalogs.zeldovich(8, 100.0, rms=4.0, seed=bench.replica_seed(rank))
        args = type("A", (), {"nside": 8, "ng": 16, "box": 100.0, "steps": 1, "warmup": 0, "gpus": world})()
        buf = io.StringIO()
        if rank != 0:  # the reference arm: ranks other than 0 leave without work or output
            with redirect_stdout(buf):
                bench.run_reference(args)
        dist.barrier()
        res = {"ms_job": ms_job, "rate": bench.job_rate(world, 1000, 4, ms_job), "cat0": cat[0].tolist(),
               "ref_out": buf.getvalue()}
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(world)]
    # the job's time is the slowest rank's, on every rank
    assert r[0]["ms_job"] == r[1]["ms_job"] == 15.0
    # whole-job throughput: 2 ranks x 1000 units x 4 steps in 15 ms
    assert r[0]["rate"] == pytest.approx(2 * 1000 * 4 / 15e-3)
    # independent realisations per replica
    assert not np.allclose(r[0]["cat0"], r[1]["cat0"])
    # the reference arm printed nothing on rank 1
    assert r[1]["ref_out"] == ""

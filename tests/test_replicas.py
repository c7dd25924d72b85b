"""Multi-GPU form of the bench: independent replicas, one projection problem per
rank, no collective on the data path; the job's time is the slowest rank's and
its throughput counts every rank's projections.  The host-side logic runs here
as two gloo ranks on the CPU (127.0.0.1)."""
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


def _rank_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_2103_01874_gb300 import fields
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 3.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, dist)
    rate = bench.whole_job_rate(world, 5, ms)
    seed = bench.replica_seed(rank)
    fl = fields.make_fields(8, 8, 8, seed=seed)
    # the reference arm: only rank 0 works under torchrun
    ref = bench.run_reference(None) if rank != 0 else "rank0"
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as fh:
        json.dump({"ms": ms, "rate": rate, "seed": seed, "u0": float(fl.u.ravel()[0]),
                   "ref_is_none": ref is None}, fh)


def test_two_gloo_replicas(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(world)]
    # max over ranks on every rank
    assert r[0]["ms"] == r[1]["ms"] == 13.0
    # whole-job throughput: all ranks' projections over the slowest rank's time
    assert r[0]["rate"] == pytest.approx(world * 5 / 13.0e-3)
    # replicas are independent problems
    assert r[0]["seed"] != r[1]["seed"] and r[0]["u0"] != r[1]["u0"]
    assert r[1]["ref_is_none"]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(1, 20, 1000.0) == pytest.approx(20.0)
    assert np.isfinite(bench.whole_job_rate(8, 20, 1000.0))

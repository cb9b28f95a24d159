"""The N > 1 path of bench.py on CPU: two gloo ranks as independent replicas.

Each rank advances its own copy of the same workload (weak scaling, no SPH
data exchanged); the only collectives are the barrier around the timed
region and the all-reduce of the slowest rank's time, from which rank 0
reports the whole job's particle updates per second."""
import hashlib
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _state_digest(s):
    h = hashlib.sha1()
    for k in sorted(s):
        h.update(k.encode())
        h.update(np.ascontiguousarray(s[k]).tobytes())
    return h.hexdigest()


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(WORLD), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=WORLD)
    try:
        r, world, local = bench.dist_env()
        assert (r, world, local) == (rank, WORLD, rank)
        # every rank builds the same replica from the same seed
        args = bench.parse(["--side", "12", "--gpus", str(WORLD)])
        s, prm = bench.make_workload(args)
        digests = [None] * WORLD
        dist.all_gather_object(digests, (_state_digest(s), len(s["x"]), prm.n_target))
        # rank-dependent stand-in times: the job takes as long as the slowest rank
        dist.barrier()
        ms = 100.0 + 37.5 * rank
        ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
        value = bench.whole_job_rate(world, len(s["x"]), args.steps, ms_max)
        # the reference arm runs on rank 0 only: other ranks return at once
        if rank != 0:
            bench.run_reference(args)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr((digests, ms_max, value)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path, capfd):
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(WORLD)]
    digests, ms_max, value = res[0]
    assert res[1] == res[0]  # both ranks agree on every reported number
    assert len(set(digests)) == 1  # identical replicas
    n = 12 ** 3
    assert digests[0][1] == n
    assert ms_max == 100.0 + 37.5 * (WORLD - 1)
    assert value == pytest.approx(WORLD * n * 20 / (ms_max * 1e-3), rel=1e-15)
    # the non-zero rank's reference arm printed nothing
    assert capfd.readouterr().out.strip() == ""


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.whole_job_rate(1, 1000, 10, 2.0) == pytest.approx(5e6)


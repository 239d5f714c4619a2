"""The N > 1 path of bench.py on CPU: two gloo ranks exchange only the timing (the job's time is
the slowest rank's, its work the sum over the ranks), and every rank draws its own worlds."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = [0.25, 0.75][rank]                 # seconds this rank took
        t_job = bench.max_over_ranks(t_local, world, torch.device("cpu"))
        units = bench.job_units(1024, 10, world)
        out[rank] = (t_job, units / t_job, bench.rank_seed(7, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0][0] == res[1][0] == 0.75             # both ranks see the slowest rank's time
    assert res[0][1] == pytest.approx(2 * 1024 * 10 / 0.75)
    assert res[0][2] != res[1][2]                     # distinct world seeds per rank


def test_ranks_draw_distinct_worlds():
    import bench
    import worldgen as wg
    a = wg.make_biped(num_worlds=2, seed=bench.rank_seed(0, 0))
    b = wg.make_biped(num_worlds=2, seed=bench.rank_seed(0, 1))
    assert not np.allclose(a.body_mass, b.body_mass)


def test_reference_arm_rank_above_zero_does_no_work(capsys):
    import sys
    import bench
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--impl", "reference"]
        args = bench.parse()
    finally:
        sys.argv = argv
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""

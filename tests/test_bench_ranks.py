"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own input pair.

Products are independent, so ranks share no data; the only collectives are the max over
ranks of the timed region and of the end-to-end time. Rank 0 builds the line from the max.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from test_bench_line import args, fake_report

        # each rank its own pair: same shapes, different values
        A, B = bench.workload(6, 4, bench.rank_seed(rank))
        sums = torch.tensor([float(sum(np.abs(c).sum() for c in A))], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, sums)
        assert len({round(float(g.item()), 12) for g in gathered}) == world
        assert [c.shape for c in A] == [c.shape for c in bench.workload(6, 4, bench.rank_seed(0))[0]]

        # the timed region: the slowest rank sets the time
        t_local = 100.0 + 20.0 * rank
        t = bench.max_over_ranks(dist, t_local, "cpu")
        assert t == 100.0 + 20.0 * (world - 1)
        e2e = bench.max_over_ranks(dist, 3.0 - rank, "cpu")
        assert e2e == 3.0
        if rank == 0:
            line = bench.make_line(args(steps=2), [fake_report(), fake_report()], t_local, t, world,
                                   {"value": world * 1 / e2e, "unit": "products/s",
                                    "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
                                   {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0})
            assert line["n_gpus"] == world and line["scaling"] == "weak"
            assert line["value"] == world * 2 / t          # all ranks' products over the max time
            assert line["ms_per_step"] == 1e3 * t / 2
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = os.pathsep.join([root, here] + ([old] if old else []))
    try:
        mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
    finally:
        os.environ["PYTHONPATH"] = old


def test_single_rank_max_is_identity():
    import bench
    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.rank_seed(0) != bench.rank_seed(1)

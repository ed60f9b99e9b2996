"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
independent instance (weak scaling, no data-path collective), combine their
timings into the whole-job figures: the slowest rank's time and the sum of
the ranks' marker-steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    from paper_2103_12194_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank's workload is its own seeded instance
    spec, _ = inputs.microbench_config(n_markers=1000, seed=rank)
    elapsed_ms = 100.0 + 50.0 * rank
    work = 1_000_000 * (rank + 1)
    t, total = bench.combine_ranks(elapsed_ms, work, world, "cpu")
    out.put((rank, t, total, spec["seed"]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_weak_scaling_figures():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, total, seed in res:
        assert t == pytest.approx(0.150)        # the slowest rank's 150 ms
        assert total == 3_000_000               # 1e6 + 2e6 marker-steps
        assert seed == rank                     # independent instances


def test_single_rank_needs_no_collective():
    import bench
    assert bench.combine_ranks(250.0, 12345, 1, "cpu") == (0.25, 12345.0)

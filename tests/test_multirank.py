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


def test_partition_balances_uneven_instances():
    """Longest processing time first: every instance on exactly one rank,
    the heaviest rank within 4/3 of the ideal share (Graham's bound), and the
    assignment deterministic."""
    from paper_2103_12194_gb300 import ranks
    import bench
    from paper_2103_12194_gb300 import inputs
    work = [n for _, n in bench.batch_specs(inputs)]  # the 32-instance sweep
    for world in (1, 2, 3, 8):
        parts = ranks.partition(work, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(work)))
        loads = [sum(work[i] for i in p) for p in parts]
        ideal = max(sum(work) / world, max(work))
        assert max(loads) <= 4.0 / 3.0 * ideal
        assert parts == ranks.partition(work, world)
    assert ranks.partition([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]


class _FakeSim:
    """Stands in for a Simulation of the breakdown search: the bracket of pd
    point p is [p, p + 1] and its gains [p] * n_v."""

    def __init__(self, points, n_v):
        self.points, self.n_v = points, n_v

    def paschen_bisect(self, lo, hi, n_v, rounds, n_seed, **kw):
        import numpy as np
        assert list(lo) == [100.0 + p for p in self.points]
        return (np.array([float(p) for p in self.points]),
                np.array([float(p) + 1 for p in self.points]),
                np.array([[float(p)] * n_v for p in self.points]))

    def close(self):
        pass


def _rank_sweep(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from paper_2103_12194_gb300 import ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    points = list(range(7))
    work = [3, 1, 4, 1, 5, 9, 2]
    mine = ranks.partition(work, world)[rank]
    res = ranks.paschen_bisect_ranks(lambda pts: _FakeSim(pts, 4), points,
                                     [100.0 + p for p in points], [900.0] * 7, n_v=4,
                                     rounds=2, n_seed=10, world=world, rank=rank, work=work)
    got = ranks.gather({("inst", i): rank for i in mine}, world, rank)
    out.put((rank, mine, res, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_a_breakdown_search_and_gather_it():
    """The pd points of a breakdown search are split between two gloo ranks by
    their work; each rank searches its own points, and rank 0 receives every
    point's bracket in pd order (the other rank gets None)."""
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_sweep, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, mine0, res0, got0), (r1, mine1, res1, got1) = res
    assert sorted(mine0 + mine1) == list(range(7)) and mine0 and mine1
    lo, hi = res0
    assert lo == [float(p) for p in range(7)] and hi == [float(p) + 1 for p in range(7)]
    assert res1 is None and got1 is None
    assert got0 == {**{("inst", i): 0 for i in mine0}, **{("inst", i): 1 for i in mine1}}

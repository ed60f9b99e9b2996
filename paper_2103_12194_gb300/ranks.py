"""Instances of a sweep shared among ranks (one process per GPU).

Every (pd, V) instance of a breakdown sweep or of the batched sweep workload
is independent of the others (Sec. V: a Paschen curve is a set of separate
breakdown runs), so the ranks exchange no data while they step.  The only
collective is at the end: each rank's per-instance results are gathered to
rank 0.

- partition(): longest-processing-time-first assignment of instances to
  ranks by their estimated work (markers x steps): instances in decreasing
  work, each to the rank with the least work so far; ties go to the lower
  rank and, within a rank, instances keep increasing order.
- gather(): the ranks' {instance: result} maps merged on rank 0 through
  torch.distributed (gloo on CPU, NCCL on GPUs); other ranks get None.
- paschen_bisect_ranks(): the batched breakdown search over the pd points
  this rank owns, its brackets gathered to rank 0 in pd order.
"""


def partition(work, n_ranks):
    """Indices of the instances each rank takes ([n_ranks] lists, each
    sorted), from the instances' estimated work (any non-negative numbers)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * n_ranks
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(work[i])
    return [sorted(p) for p in parts]


def gather(local, world, rank):
    """Merge the ranks' {instance: result} dicts on rank 0 (None elsewhere);
    results must be picklable.  An instance reported by two ranks is an
    error."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object(dict(local), parts, dst=0)
    if rank != 0:
        return None
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError("instance %r reported by two ranks" % (k,))
            merged[k] = v
    return merged


def paschen_bisect_ranks(make_sim, points, V_lo, V_hi, n_v, rounds, n_seed, world, rank,
                         work=None, **kw):
    """The batched breakdown search (slpic_paschen_bisect) with the pd points
    shared among the ranks.  make_sim(point_indices) returns a Simulation
    with len(point_indices) * n_v instances configured for those points (in
    that order, n_v instances each); work[p] is point p's estimated cost
    (default: equal).  Returns, on rank 0, (V_lo, V_hi) lists over all points
    in their order; None on the other ranks."""
    work = [1.0] * len(points) if work is None else work
    mine = partition(work, world)[rank]
    local = {}
    if mine:
        sim = make_sim(mine)
        lo, hi, gain = sim.paschen_bisect([V_lo[p] for p in mine], [V_hi[p] for p in mine],
                                          n_v=n_v, rounds=rounds, n_seed=n_seed, **kw)
        sim.close()
        for j, p in enumerate(mine):
            local[p] = (float(lo[j]), float(hi[j]), [float(g) for g in gain[j]])
    allres = gather(local, world, rank)
    if allres is None:
        return None
    if sorted(allres) != list(range(len(points))):
        raise RuntimeError("the ranks did not cover every pd point")
    return [allres[p][0] for p in range(len(points))], [allres[p][1] for p in range(len(points))]

"""Case sharding of one GSGP problem over several contexts (gsgp_shard_*).

Every step of a generation is independent per fitness case except the
squared-error sums behind the RMSE (Sec. 2.2, "Fitness computation"), so the
cases can be partitioned: each shard holds a contiguous, 1024-case-aligned
slice, all shards draw the same selections from the shared seed, and per
step they exchange the per-chunk partial sums (an element-wise sum of the
shards' arrays, each array zero outside its own chunks).  The library then
finishes the step on the complete sums in its fixed order, so the sharded
run equals one unsharded run bit for bit.

This module only plans the slices and drives the steps; the exchange is the
caller's (an all-reduce over ranks, or a sum of the arrays when several
shards share one process).
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np

CHUNK = 1024


def plan(n_train: int, n_test: int, shards: int) -> List[Tuple[int, int, int]]:
    """(case0, local training cases, local test cases) of each shard: the
    problem's cases (training first) cut into `shards` contiguous slices on
    1024-case boundaries, as even as the boundaries allow.  Later shards may
    be empty of training cases; a shard is never empty (shards <= chunks)."""
    n = n_train + n_test
    chunks = -(-n // CHUNK)
    if shards < 1 or shards > chunks:
        raise ValueError(f"1 <= shards <= {chunks} (1024-case chunks)")
    bounds = [min(n, (chunks * k // shards) * CHUNK) for k in range(shards + 1)]
    out = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        tr = max(0, min(b, n_train) - a)
        out.append((a, tr, (b - a) - tr))
    return out


def slice_cases(data: Sequence[np.ndarray], case0: int, n_tr: int, n_te: int):
    """The shard's (X_train, y_train, X_test, y_test) from the problem's
    arrays (row-major cases, training then test)."""
    X_tr, y_tr, X_te, y_te = data
    ntr_all = len(y_tr)
    a_tr = min(case0, ntr_all)
    a_te = max(0, case0 - ntr_all)
    return (X_tr[a_tr:a_tr + n_tr], y_tr[a_tr:a_tr + n_tr],
            X_te[a_te:a_te + n_te], y_te[a_te:a_te + n_te])


def _foreign_streams(runs) -> bool:
    """True when a run's work is not queued on torch's current stream (the
    exchange, a torch operation, then needs a device synchronisation on each
    side)."""
    import torch
    cur = torch.cuda.current_stream().cuda_stream
    return any((r.cfg.stream or 0) != cur for r in runs)


def local_sum(runs) -> None:
    """Exchange for shards that share one process: every shard's array
    becomes the element-wise sum of all of them (on torch's current stream;
    runs on other streams are synchronised around it)."""
    import torch
    sync = _foreign_streams(runs)
    if sync:
        torch.cuda.synchronize()
    arrays = [r.shard_partials() for r in runs]
    total = arrays[0].clone()
    for a in arrays[1:]:
        total += a
    for a in arrays:
        a.copy_(total)
    if sync:
        torch.cuda.synchronize()


def init(runs, exchange: Callable[[list], None] = local_sum) -> None:
    """gsgp_init on every shard, the exchange, gsgp_shard_finish."""
    for r in runs:
        r.init()
    exchange(runs)
    for r in runs:
        r.shard_finish()


def evolve(runs, generations: int, exchange: Callable[[list], None] = local_sum) -> None:
    """`generations` generations of every shard, one exchange each."""
    for _ in range(generations):
        for r in runs:
            r.shard_generation()
        exchange(runs)
        for r in runs:
            r.shard_finish()


def allreduce_exchange(group=None) -> Callable[[list], None]:
    """Exchange for one shard per rank: an all-reduce (sum) of the shard's
    array over the process group (torch.distributed, ordered with torch's
    current stream; a shard on another stream is synchronised around it)."""
    import torch
    import torch.distributed as dist

    def ex(runs):
        sync = _foreign_streams(runs)
        if sync:
            torch.cuda.synchronize()
        for r in runs:
            dist.all_reduce(r.shard_partials(), op=dist.ReduceOp.SUM, group=group)
        if sync:
            torch.cuda.synchronize()
    return ex

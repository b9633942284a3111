"""Worker of the two-rank gloo tests (imported by spawned processes)."""

import os

import numpy as np


def gradient_shards(rank, world, port, out_dir):
    """Each rank takes its rows of one batch, computes the oracle gradient of
    the symmetric form on them, and the ranks add their sums (gloo)."""
    import torch
    import torch.distributed as dist

    import oracle
    import synthetic_inputs as si
    from paper_1811_07624_gb300.sharding import allreduce_sum, reduce_max, shard_rows

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, h, batch = 48, 6, 37
        U = si.reflectors(n, h, seed=3, unit=False)
        d = si.spectrum(n, seed=3)
        X = si.vectors(batch, n, seed=4)
        G = si.vectors(batch, n, seed=5)
        r0, r1 = shard_rows(batch, world, rank)
        _, gU, gd = oracle.backward("SYM", U, X[r0:r1], G[r0:r1], d=d)
        tU, td = torch.from_numpy(np.ascontiguousarray(gU)), torch.from_numpy(gd.copy())
        allreduce_sum([tU, td, None], dist)
        slowest = reduce_max(10.0 + rank, dist)
        np.save(os.path.join(out_dir, f"gU_{rank}.npy"), tU.numpy())
        np.save(os.path.join(out_dir, f"gd_{rank}.npy"), td.numpy())
        np.save(os.path.join(out_dir, f"max_{rank}.npy"), np.array([slowest, r0, r1]))
    finally:
        dist.destroy_process_group()

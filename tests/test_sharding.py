"""Multi-GPU partitioning and collectives, checked on the host (gloo, two ranks).

The hot path shards by rows or by whole transforms with no data exchange; the
gradients of the fit are sums over the batch, so the ranks' sums must add up
to the full-batch gradient.  The oracle supplies the per-shard gradients.
"""

import socket

import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from paper_1811_07624_gb300.sharding import shard_rows, shard_transforms, transform_cost


@pytest.mark.parametrize("batch,world", [(0, 1), (1, 2), (7, 3), (262144, 8), (37, 2), (5, 8)])
def test_shard_rows_cover_once_and_balance(batch, world):
    ranges = [shard_rows(batch, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == batch
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [r1 - r0 for r0, r1 in ranges]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == batch
    with pytest.raises(ValueError):
        shard_rows(batch, world, world)


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_shard_transforms_lpt(world):
    specs = [(t["n"], t["h"], t["batch"]) for t in si.ragged_transforms(512)]
    parts = shard_transforms(specs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(specs)))
    loads = [sum(transform_cost(*specs[i]) for i in p) for p in parts]
    lower = max(sum(loads) / world, max(transform_cost(*s) for s in specs))
    assert max(loads) <= 4.0 / 3.0 * lower + 1e-9  # the LPT bound


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_gradient_sum_equals_full_batch(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import dist_worker

    oracle.build_oracle()  # build once, before the ranks load it
    world = 2
    mp.start_processes(dist_worker.gradient_shards, args=(world, _free_port(), str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    n, h, batch = 48, 6, 37
    U = si.reflectors(n, h, seed=3, unit=False)
    d = si.spectrum(n, seed=3)
    X, G = si.vectors(batch, n, seed=4), si.vectors(batch, n, seed=5)
    _, gU, gd = oracle.backward("SYM", U, X, G, d=d)
    covered = 0
    for r in range(world):
        np.testing.assert_allclose(np.load(tmp_path / f"gU_{r}.npy"), gU, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(np.load(tmp_path / f"gd_{r}.npy"), gd, rtol=1e-12, atol=1e-12)
        slowest, r0, r1 = np.load(tmp_path / f"max_{r}.npy")
        assert slowest == 10.0 + world - 1
        covered += int(r1 - r0)
    assert covered == batch

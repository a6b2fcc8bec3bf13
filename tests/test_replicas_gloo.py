"""The multi-process path on CPU: world_size 2 with the gloo backend.

Each rank computes, with the FP64 oracle, its contiguous share of the RIRs
of a small batch; the gathered result must equal the single-process
computation exactly, and the step-time reduction must return the slowest
rank's time.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402

from paper_1810_11359_gb300 import replicas  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _batch():
    L = np.array([3.7, 2.9, 2.3])
    beta = np.array([0.9, 0.8, 0.85, 0.7, 0.95, 0.6])
    rng = np.random.default_rng(21)
    ps = rng.uniform(0.3, 1.0, (5, 3)) * (L - 0.6) + 0.3
    pr = rng.uniform(0.3, 1.0, (5, 3)) * (L - 0.6) + 0.3
    return L, beta, ps, pr


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        L, beta, ps, pr = _batch()
        lo, hi = replicas.shard_range(ps.shape[0], rank, world)
        h = oracle.rir_list(L, beta, 343.0, 16000.0, 32 / 16000, ps[lo:hi], pr[lo:hi], [5, 5, 5], 600)
        full = replicas.gather_shards(torch.from_numpy(np.ascontiguousarray(h)), ps.shape[0])
        t_max = replicas.max_over_ranks(1.0 + rank)
        rate = replicas.whole_job_rate(10.0, world, t_max)
        if rank == 0:
            np.save(os.path.join(out_dir, "full.npy"), full.numpy())
            np.save(os.path.join(out_dir, "tmax.npy"), np.array([t_max, rate]))
    finally:
        dist.destroy_process_group()


def test_shard_range_covers_every_item_once():
    for n in [0, 1, 5, 7, 128]:
        for world in [1, 2, 3, 8]:
            parts = [replicas.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and b - a >= d - c
    with pytest.raises(ValueError):
        replicas.shard_range(4, 2, 2)


def test_two_gloo_ranks_reassemble_the_single_process_result(tmp_path):
    import oracle
    oracle.build()
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    L, beta, ps, pr = _batch()
    ref = oracle.rir_list(L, beta, 343.0, 16000.0, 32 / 16000, ps, pr, [5, 5, 5], 600)
    full = np.load(tmp_path / "full.npy")
    assert full.shape == ref.shape
    assert np.array_equal(full, ref)
    t_max, rate = np.load(tmp_path / "tmax.npy")
    assert t_max == 2.0 and rate == pytest.approx(10.0 * 2 / 2.0)

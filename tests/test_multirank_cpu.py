"""The multi-rank sharding of the transport, on CPU with gloo and world size 2:
each rank follows its own package range with the oracle (frozen mode), the counts
and spectra are summed over ranks, and the result equals one process following all
packages -- bit for bit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _model():
    from paper_1201_3588_gb300 import workloads as w
    m = w.sphere_model(n_base=8, n_bins=12, tau_v=2.0)
    T = np.full((m.n_species, m.tree.n_leaves), 35.0)
    return m, T


def _worker(rank, world, port, n_per_rank, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1201_3588_gb300 import shard
    m, T = _model()
    first, n = shard.package_range(rank, world, n_per_rank)
    t = oracle.transport(m, n, seed=5, first_id=first, mode=oracle.MODE_FROZEN, T_frozen=T,
                         n_total=shard.total_packages(world, n_per_rank))
    cnt = torch.from_numpy(t.count.astype(np.int64))
    sed = torch.from_numpy(t.sed.astype(np.int64))
    shard.sum_over_ranks(cnt)
    shard.sum_over_ranks(sed)
    tot = torch.tensor([t.emitted, t.escaped, t.absorptions], dtype=torch.int64)
    shard.sum_over_ranks(tot)
    if rank == 0:
        np.savez(os.path.join(out_dir, "sum.npz"), cnt=cnt.numpy(), sed=sed.numpy(),
                 tot=tot.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_sum_to_the_single_run(tmp_path):
    import oracle
    world, n = 2, 600
    mp.start_processes(_worker, args=(world, _free_port(), n, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    got = np.load(tmp_path / "sum.npz")
    m, T = _model()
    ref = oracle.transport(m, world * n, seed=5, mode=oracle.MODE_FROZEN, T_frozen=T,
                           n_total=world * n)
    assert (got["cnt"] == ref.count.astype(np.int64)).all()
    assert (got["sed"] == ref.sed.astype(np.int64)).all()
    assert got["tot"].tolist() == [ref.emitted, ref.escaped, ref.absorptions]


def test_package_ranges_partition_the_ids():
    from paper_1201_3588_gb300 import shard
    ids = []
    for r in range(4):
        f, n = shard.package_range(r, 4, 7)
        ids.extend(range(f, f + n))
    assert ids == list(range(28))
    with pytest.raises(ValueError):
        shard.package_range(4, 4, 7)

"""Host logic of the multi-GPU path on the CPU: the shard of each rank, and
two gloo ranks that each count their own chunks (with the oracle, standing in
for a GPU), merge their totals with the one collective of the path and agree
on the slowest time."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth
from paper_1011_0235_gb300 import shard


@pytest.mark.parametrize("count,world", [(0, 1), (1, 2), (64, 2), (64, 3), (7, 8), (4096, 5)])
def test_shards_partition_the_units(count, world):
    seen = []
    sizes = []
    for r in range(world):
        rg = shard.shard(count, world, r)
        seen.extend(rg)
        sizes.append(len(rg))
    assert seen == list(range(count))
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_arguments():
    for args in ((4, 0, 0), (4, 2, 2), (4, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            shard.shard(*args)


def _chunks():
    out = []
    for c in range(10):
        law = synth.degenerate(90, 0.95) if c % 4 < 2 else synth.uniform()
        out.append(synth.host(3000 + 17 * c, law, synth.SEED_BASE + 14, c << 13))
    return out


def _rank(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = shard.env()
    assert (w, r, lr) == (world, rank, rank)
    chunks = _chunks()
    st = oracle.StreamOracle(8192)
    for i in shard.shard(len(chunks), world, rank):
        st.push(chunks[i])
    totals = torch.from_numpy(st.totals.astype(np.int64))
    shard.merge_totals(totals)
    t = shard.slowest(0.25 * (rank + 1))
    np.save(os.path.join(outdir, "r%d.npy" % rank), np.concatenate([totals.numpy(), [int(t * 1000)]]))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_merge_totals_and_time():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank, args=(world, _free_port(), d), nprocs=world, join=True)
        res = [np.load(os.path.join(d, "r%d.npy" % r)) for r in range(world)]
    whole = oracle.hist(np.concatenate(_chunks())).astype(np.int64)
    for r in res:
        assert np.array_equal(r[:256], whole)
        assert r[256] == 500  # max(0.25, 0.5) s

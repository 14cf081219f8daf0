"""Genome sharding across ranks, tested on the CPU: world_size-2 gloo ranks each map the reads
against their own fragment range (the CPU oracle stands in for a GPU), exchange one record per
read with an all-gather, and merge; the merged result must equal the oracle on the whole genome
bit for bit.  Also a single-process check of the merge over 1..5 shards."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import gen
import oracle
from paper_1403_2136_gb300 import shard
from tests.parity_util import assert_hits_equal


def _workload():
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=60_000, reads=24)
    genome, reads = gen.materialize(wl)
    # a planted repeat across a shard border makes ties and duplicate fragments likely
    genome = genome.copy()
    genome[29_000:29_600] = genome[50_000:50_600]
    return wl, genome, reads


def _oracle_shard(genome, F, reads, match, mismatch, world, rank, max_len):
    f0, f1, g0, g1 = shard.shard_bounds(genome.shape[0], F, world, rank, max_len)
    if f1 <= f0:
        return shard.empty_records(reads.count)
    hits, _, _ = oracle.map_batch(genome[g0:g1], F, reads.seq, reads.offsets, match, mismatch)
    return shard.to_records(hits, f0, F)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_merge_equals_whole_genome(world):
    wl, genome, reads = _workload()
    F, ml = 1000, int(np.diff(reads.offsets).max())
    recs = [_oracle_shard(genome, F, reads, 5, -4, world, r, ml) for r in range(world)]
    got = shard.records_to_hits(shard.merge(recs))
    want, _, _ = oracle.map_batch(genome, F, reads.seq, reads.offsets, 5, -4)
    assert_hits_equal(got, want, f"{world} shards")


@pytest.mark.parametrize("genome_len,world", [(4_500, 4), (4_500, 7), (900, 3)])
def test_merge_with_ranks_that_own_no_fragment(genome_len, world):
    """More ranks than fragments (or a rank left over by the rounding of the split): the
    empty ranks contribute empty records and the merge still equals the whole genome; with a
    single fragment the merged second is -1 with score 0."""
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=genome_len, reads=16)
    genome, reads = gen.materialize(wl)
    F, ml = 1000, int(np.diff(reads.offsets).max())
    bounds = [shard.shard_bounds(genome.shape[0], F, world, r, ml) for r in range(world)]
    assert any(f1 <= f0 for f0, f1, _, _ in bounds)           # some rank owns nothing
    recs = [_oracle_shard(genome, F, reads, 5, -4, world, r, ml) for r in range(world)]
    got = shard.records_to_hits(shard.merge(recs))
    want, _, _ = oracle.map_batch(genome, F, reads.seq, reads.offsets, 5, -4)
    assert_hits_equal(got, want, f"{world} shards of {genome_len} bp")
    if genome_len <= F:
        assert np.all(got["second_frag"] == -1) and np.all(got["second_score"] == 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, genome, reads = _workload()
    F, ml = 1000, int(np.diff(reads.offsets).max())
    mine = _oracle_shard(genome, F, reads, 5, -4, world, rank, ml)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine.tobytes())
    recs = [np.frombuffer(b, dtype=shard.REC) for b in gathered]
    merged = shard.records_to_hits(shard.merge(recs))
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks(tmp_path):
    world = 2
    out = str(tmp_path / "merged.npy")
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    got = np.load(out)
    wl, genome, reads = _workload()
    want, _, _ = oracle.map_batch(genome, 1000, reads.seq, reads.offsets, 5, -4)
    assert_hits_equal(got, want, "gloo 2 ranks")

"""Genome sharding across ranks, tested on the CPU: world_size-2 gloo ranks each map the reads
against their own fragment range (the CPU oracle stands in for a GPU) through the library's
``shard.map_sharded``, which exchanges one record per read with an all-gather and merges; the
merged result must equal the oracle on the whole genome bit for bit.  Also a single-process
check of the merge over 1..5 shards, and a tie between a fragment's owner and the partial copy
of it on the rank before (the case that decides which (strand, offset) the merge keeps)."""
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


def _oracle_slice(genome_slice, F, reads_seq, reads_off, match, mismatch, max_len):
    hits, _, _ = oracle.map_batch(genome_slice, F, reads_seq, reads_off, match, mismatch)
    return hits


_COMP = bytes.maketrans(b"ACGT", b"TGCA")


def _tie_case():
    """G = 400, F = 100, two ranks, max_len 40: rank 0 owns fragments 0-1 and sees fragment 2
    on diagonals [200, 239) only.  A 20-base read has its reverse complement planted at 202
    (inside that partial view) and its forward copy at 250 (outside it): both score 20 * 5 in
    fragment 2, and the first argmax of the whole genome is the forward copy (+ strand first)."""
    rng = np.random.default_rng(1403)
    genome = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 400)].copy()
    read = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 20)].copy()
    genome[250:270] = read
    genome[202:222] = np.frombuffer(read.tobytes()[::-1].translate(_COMP), np.uint8)
    seq = read.copy()
    off = np.array([0, 20], dtype=np.int64)
    return genome, seq, off


def test_partial_copy_tie_keeps_the_owners_argmax():
    genome, seq, off = _tie_case()
    F, ml = 100, 40
    want, _, _ = oracle.map_batch(genome, F, seq, off, 5, -4)
    # the whole genome, worked out: fragment 2, 100 = 20 * 5, the + strand copy at 250
    assert (int(want["best_frag"][0]), int(want["best_score"][0]), int(want["offset"][0]),
            int(want["strand"][0])) == (2, 100, 250, 0)
    b0 = shard.shard_bounds(400, F, 2, 0, ml)
    assert b0 == (0, 2, 0, 239)
    rec0 = shard.to_records(_oracle_slice(genome[0:239], F, seq, off, 5, -4, ml), 0, F)
    rec1 = shard.to_records(_oracle_slice(genome[200:400], F, seq, off, 5, -4, ml), 2, F)
    # rank 0's partial view of fragment 2 ties the owner with the reverse copy
    assert (int(rec0["f1"][0]), int(rec0["s1"][0]), int(rec0["offset"][0]), int(rec0["strand"][0])) == \
        (2, 100, 202, 1)
    assert (int(rec1["f1"][0]), int(rec1["s1"][0]), int(rec1["offset"][0]), int(rec1["strand"][0])) == \
        (2, 100, 250, 0)
    for order in ([rec0, rec1], [rec1, rec0]):
        got = shard.records_to_hits(shard.merge(order))
        assert_hits_equal(got, want, "planted partial-copy tie")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_path, case):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if case == "tie":
        genome, seq, off = _tie_case()
        F, ml = 100, 40
    else:
        wl, genome, reads = _workload()
        seq, off = reads.seq, reads.offsets
        F, ml = 1000, int(np.diff(reads.offsets).max())
    merged = shard.map_sharded(genome, F, seq, off, 5, -4, ml, map_slice=_oracle_slice)
    gathered = [None] * world
    dist.all_gather_object(gathered, merged.tobytes())
    if rank == 0:
        assert all(g == gathered[0] for g in gathered), "ranks disagree on the merged hits"
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", ["workload", "tie"])
def test_gloo_two_ranks(tmp_path, case):
    world = 2
    out = str(tmp_path / "merged.npy")
    mp.spawn(_rank_main, args=(world, _free_port(), out, case), nprocs=world, join=True)
    got = np.load(out)
    if case == "tie":
        genome, seq, off = _tie_case()
        F = 100
    else:
        wl, genome, reads = _workload()
        seq, off, F = reads.seq, reads.offsets, 1000
    want, _, _ = oracle.map_batch(genome, F, seq, off, 5, -4)
    assert_hits_equal(got, want, f"gloo 2 ranks ({case})")


def test_neighbour_rule_is_rejected():
    with pytest.raises(ValueError):
        shard.map_sharded(np.zeros(10, np.uint8), 4, np.zeros(0, np.uint8), np.zeros(1, np.int64), 5, -4, 8,
                          exclude_neighbors=True)

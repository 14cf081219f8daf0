"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Integer and index results must be bit-exact (best/second fragment, scores, offset, strand,
flags; NW score, span and CIGAR).
"""
import numpy as np
import pytest

import gen
import oracle
from tests.parity_util import (assert_alns_equal, assert_hits_equal, concat_reads, cpu_count, oracle_map)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mss():
    import torch
    assert torch.cuda.is_available()
    import paper_1403_2136_gb300 as m
    from paper_1403_2136_gb300 import build
    build.build()
    m.load_library()
    return m


def run_both(mss, genome, seq, off, F, match, mismatch, nw=None, max_len=None, tune=None, procs=None, step=1):
    g = mss.mss_load_genome(genome, frag_len=F, max_read_len=max_len or max(1, int(np.diff(off).max())))
    if tune:
        mss.mss_set_tune(g, **tune)
    if step != 1:
        mss.mss_set_read_step(g, step)
    hits = mss.mss_map_reads(g, seq, off, match, mismatch)
    alns = cig = None
    if nw is not None:
        alns, cig = mss.nw_align(g, seq, off, hits, *nw)
    ohits, oalns, ocig = oracle_map(genome, F, seq, off, match, mismatch, nw=nw, procs=procs, step=step)
    g.close()
    return hits, alns, cig, ohits, oalns, ocig


def test_pack_matches_oracle_encoding(mss):
    rng = np.random.default_rng(1)
    G = 100_003
    genome = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), size=G)
    g = mss.mss_load_genome(genome, frag_len=1000, max_read_len=100)
    codes = mss.mss_genome_codes(g, 0, G + 500)
    assert np.array_equal(codes[:G], oracle.encode(genome))
    assert np.all(codes[G:] == 4)      # padding reads as N
    g.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_tiny_50k_all_reads(mss, variant):
    """50 kbp uniform genome, F=1000, 100 x 100 bp reads (10% subs + one indel), +1/-1."""
    wl = gen.workloads()["tiny-50k"]
    genome, reads = gen.materialize(wl)
    hits, alns, cig, oh, oa, oc = run_both(mss, genome, reads.seq, reads.offsets, wl.frag_len, wl.match,
                                           wl.mismatch, nw=wl.nw, tune={"variant": variant}, procs=cpu_count())
    assert_hits_equal(hits, oh, f"tiny-50k variant {variant}")
    assert_alns_equal(alns, cig, oa, oc, f"tiny-50k variant {variant}")
    # the generator's truth: most reads map to the fragment of their true start
    assert np.mean(hits["best_frag"] == reads.true_start // wl.frag_len) > 0.8


@pytest.mark.parametrize("pairs,queries", [(4, 8), (8, 4), (4, 4)])
@pytest.mark.parametrize("variant", [0, 1])
def test_scan_configurations(mss, pairs, queries, variant):
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=60_000, reads=37)
    genome, reads = gen.materialize(wl)
    hits, _, _, oh, _, _ = run_both(mss, genome, reads.seq, reads.offsets, 1000, 5, -4,
                                    tune={"variant": variant, "pairs": pairs, "queries": queries},
                                    procs=cpu_count())
    assert_hits_equal(hits, oh, f"config v{variant} D{pairs} Q{queries}")


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("max_len", [250, 2432])
def test_scan_with_128_threads_per_cta(mss, variant, max_len):
    """The 128-thread CTA shape (tiles of 2,048 diagonals, four CTAs per SM) on a ragged mix of
    read lengths, bit-exact against the oracle; the shapes it is not built for are rejected."""
    wl = gen.scaled(gen.workloads()["chrom-230M"], genome_len=70_000, reads=30)
    genome, reads = gen.materialize(wl)
    hits, _, _, oh, _, _ = run_both(mss, genome, reads.seq, reads.offsets, 1000, 5, -4, max_len=max_len,
                                    tune={"variant": variant, "pairs": 8, "queries": 4, "threads": 128},
                                    procs=cpu_count())
    assert_hits_equal(hits, oh, f"128 threads v{variant} max_len {max_len}")
    g = mss.mss_load_genome(genome, frag_len=1000, max_read_len=250)
    with pytest.raises(mss.MssError):
        mss.mss_set_tune(g, threads=64)
    mss.mss_set_tune(g, pairs=4, queries=8, threads=128)
    with pytest.raises(mss.MssError):
        mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4)
    g.close()


@pytest.mark.parametrize("items", [1, 4, 64])
def test_chunking_is_result_neutral(mss, items):
    """One chunk per group, a few, or many chunks per group must give the same top-2 (the
    cross-chunk merge of fragments split between chunks is exact)."""
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=90_000, reads=20)
    genome, reads = gen.materialize(wl)
    hits, _, _, oh, _, _ = run_both(mss, genome, reads.seq, reads.offsets, 777, 5, -4,
                                    tune={"min_items_per_cta": items}, procs=cpu_count())
    assert_hits_equal(hits, oh, f"items {items}")


def test_adversarial_cases(mss):
    rng = np.random.default_rng(7)
    G = 20_000
    genome = bytearray(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=G).tobytes())
    genome[3000:3400] = genome[12000:12400]           # exact repeat (ties -> lowest fragment)
    genome[7000:7700] = b"N" * 700                    # an all-N stretch covering whole fragments
    genome[15000:15300] = genome[15000:15300].lower()  # lowercase bases are bases
    genome = bytes(genome)
    reads = [
        genome[12050:12150],                           # repeat copy: best == second, repeat flag
        genome[0:60],                                  # genome start
        genome[G - 45:G],                              # genome end (window runs into padding)
        genome[G - 20:G] + b"ACGTACGTAC",              # overhangs the genome end
        genome[7100:7200],                             # all N
        b"N" * 33,                                     # read of N only: best == 0
        genome[4990:5020],                             # junction of fragments (F = 250 below)
        genome[15010:15110],                           # lowercase source
        b"A",                                          # m = 1
        b"GT",                                         # m = 2
        genome[100:131], genome[200:232], genome[300:333],  # m = 31, 32, 33
        genome[400:650],                               # m = 250
        bytes(rng.choice(np.frombuffer(b"ACGTN", np.uint8), size=97).tobytes()),
    ]
    seq, off = concat_reads(reads)
    for F in (250, 16, 1000, 20_000, 30_000):         # F = G and F > G: a single fragment
        for (ma, mm) in ((5, -4), (1, -1), (13, -7), (3, 0)):
            hits, _, _, oh, _, _ = run_both(mss, genome, seq, off, F, ma, mm, max_len=300, procs=1)
            assert_hits_equal(hits, oh, f"adversarial F={F} scores {ma}/{mm}")
            if F == 250:   # the exact repeat copy ties with its source
                assert oh["best_score"][0] == oh["second_score"][0] and oh["flags"][0] == 1
                assert oh["best_score"][5] == 0 and oh["flags"][5] == 1
            if F > 20_000:  # a single fragment: no second
                assert np.all(oh["second_frag"] == -1) and np.all(oh["second_score"] == 0)


def test_longest_reads(mss):
    """m up to the ABI maximum 2432 (int16 path: 2432 * 13 <= 32767)."""
    rng = np.random.default_rng(8)
    genome = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=9000).tobytes()
    reads = [genome[100:100 + 2432], genome[5000:5000 + 2000], genome[3000:3000 + 1024]]
    reads = [bytes(r[:i] + (b"T" if r[i:i + 1] != b"T" else b"A") + r[i + 1:]) for r, i in zip(reads, (7, 99, 512))]
    seq, off = concat_reads(reads)
    for ma, mm in ((13, -2), (1, -1)):
        hits, _, _, oh, _, _ = run_both(mss, genome, seq, off, 512, ma, mm, max_len=2432, procs=3)
        assert_hits_equal(hits, oh, f"long reads {ma}/{mm}")


def test_nw_parameters(mss):
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=40_000, reads=30)
    genome, reads = gen.materialize(wl)
    for nw in ((5, -4, -26, -26, 32), (5, -4, -10, -1, 32), (2, -3, -5, -2, 8), (5, -4, -10, -1, 63),
               (1, -1, -1, -1, 0)):
        hits, alns, cig, oh, oa, oc = run_both(mss, genome, reads.seq, reads.offsets, 2048, 5, -4, nw=nw,
                                               procs=cpu_count())
        assert_hits_equal(hits, oh, f"nw {nw}")
        assert_alns_equal(alns, cig, oa, oc, f"nw {nw}")


def test_device_path_and_graph_replay(mss):
    import torch
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=50_000, reads=64)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=2048, max_read_len=150)
    d_seq = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets).cuda()
    R = reads.count
    d_hits = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):   # capture once, replay
            d_hits.zero_()
            mss.mss_map_reads_device(g, d_seq, d_off, R, 150, 5, -4, d_hits, stream=s)
            mss.mss_sync(g, stream=s)
            got = mss.hits_from_bytes(d_hits.cpu())
            want = mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4)
            assert_hits_equal(got, want, "device path")
    n1 = mss.mss_launch_count(g)
    assert n1 >= 15
    g.close()


def test_errors_are_reported(mss):
    genome = b"ACGT" * 100
    g = mss.mss_load_genome(genome, frag_len=64, max_read_len=100)
    seq, off = concat_reads([b"ACGTX"])
    with pytest.raises(mss.MssError) as e:
        mss.mss_map_reads(g, seq, off, 5, -4)
    assert e.value.status == mss.MSS_EINVAL
    seq, off = concat_reads([b"A" * 101])
    with pytest.raises(mss.MssError) as e:
        mss.mss_map_reads(g, seq, off, 5, -4)
    assert e.value.status == mss.MSS_EREADLEN
    seq, off = concat_reads([b"ACGT"])
    with pytest.raises(mss.MssError) as e:
        mss.mss_map_reads(g, seq, off, 0, -4)
    assert e.value.status == mss.MSS_EINVAL
    g.close()
    g = mss.mss_load_genome(genome, frag_len=64, max_read_len=2432)
    seq, off = concat_reads([b"A" * 2432])
    with pytest.raises(mss.MssError) as e:
        mss.mss_map_reads(g, seq, off, 14, -4)
    assert e.value.status == mss.MSS_EOVERFLOW
    with pytest.raises(mss.MssError):
        mss.mss_load_genome(b"ACGTQ", frag_len=64)
    # the context stays usable after an error
    seq, off = concat_reads([b"ACGTACGT"])
    h = mss.mss_map_reads(g, seq, off, 5, -4)
    assert h["best_score"][0] == 40
    g.close()


def test_empty_batches_and_empty_reads(mss):
    """R = 0 is a no-op on every entry point; a read of length 0 is rejected with
    MSS_EREADLEN (host calls: before any launch; device calls: by the length check of the
    ordering kernel, reported at the next synchronisation) and the context stays usable."""
    import torch
    rng = np.random.default_rng(9)
    genome = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=5000).tobytes()
    g = mss.mss_load_genome(genome, frag_len=500, max_read_len=200)
    seq, off = concat_reads([])
    assert mss.mss_map_reads(g, seq, off, 5, -4).shape == (0,)
    alns, cigs = mss.nw_align(g, seq, off, np.zeros(0, dtype=mss.HIT_DTYPE), 5, -4, -10, -1, 32)
    assert alns.shape == (0,) and cigs == []
    hits, alns, _ = mss.mss_map_align(g, seq, off, 5, -4, (5, -4, -10, -1, 32))
    assert hits.shape == (0,) and alns.shape == (0,)
    d_seq = torch.zeros(16, dtype=torch.uint8, device="cuda")
    d_off = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_hits = torch.zeros(32, dtype=torch.uint8, device="cuda")
    mss.mss_map_reads_device(g, d_seq, d_off, 0, 1, 5, -4, d_hits)
    mss.mss_sync(g)

    reads = [genome[100:200], b"", genome[300:350]]
    seq, off = concat_reads(reads)
    with pytest.raises(mss.MssError) as e:
        mss.mss_map_reads(g, seq, off, 5, -4)
    assert e.value.status == mss.MSS_EREADLEN
    d_seq, d_off = torch.from_numpy(seq).cuda(), torch.from_numpy(off).cuda()
    d_hits = torch.zeros(3 * 32, dtype=torch.uint8, device="cuda")
    mss.mss_map_reads_device(g, d_seq, d_off, 3, 100, 5, -4, d_hits)
    with pytest.raises(mss.MssError) as e:
        mss.mss_sync(g)
    assert e.value.status == mss.MSS_EREADLEN
    # the context stays usable and the next call is exact
    seq, off = concat_reads([genome[100:200], genome[300:350]])
    hits, _, _, oh, _, _ = run_both(mss, genome, seq, off, 500, 5, -4, max_len=200, procs=1)
    assert_hits_equal(hits, oh, "after an empty-read error")
    h = mss.mss_map_reads(g, seq, off, 5, -4)
    assert list(h["best_score"]) == [500, 250]
    g.close()


def test_autotune_keeps_results(mss):
    import torch
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=80_000, reads=48)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=2048, max_read_len=150)
    before = mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4)
    d_seq = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets).cuda()
    t = mss.mss_autotune(g, d_seq, d_off, reads.count, 150, 5, -4, allow_frag_len=False)
    assert t["frag_len"] == 2048
    after = mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4)
    assert_hits_equal(after, before, "autotune")
    # with scan timing on (as in the benchmark) and the fragment length free: the candidates run
    # outside graph capture, the chosen F is one of the candidates, results follow the new F
    mss.mss_scan_timing(g, True)
    t = mss.mss_autotune(g, d_seq, d_off, reads.count, 150, 5, -4, allow_frag_len=True)
    assert t["frag_len"] in (1024, 2048, 4096, 8192) and t["variant"] in (0, 1) and t["pairs"] in (4, 8)
    want, _, _ = oracle_map(genome, t["frag_len"], reads.seq, reads.offsets, 5, -4, procs=cpu_count())
    assert_hits_equal(mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4), want, "autotuned F")
    g.close()


@pytest.mark.parametrize("world", [2, 3])
def test_genome_sharding_on_gpu_equals_unsharded(mss, world):
    """Genome shards mapped one after another on this GPU and merged (the exchange emulated in
    memory) give the oracle's whole-genome result bit for bit, including a planted tie between
    a fragment's owner and the partial copy of it on the rank before."""
    from paper_1403_2136_gb300 import shard
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=300_000, reads=60)
    genome, reads = gen.materialize(wl)
    ml = int(np.diff(reads.offsets).max())
    # plant a tie across rank 0's border: a read whose reverse complement lies in the partial
    # view rank 0 has of the first fragment of rank 1, and whose forward copy lies further
    # into that fragment (outside the view): the owner's + strand copy must win
    genome = genome.copy()
    F = 2048
    f1 = shard.shard_bounds(genome.shape[0], F, world, 0, ml)[1]
    rng = np.random.default_rng(world)
    read = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 100)].copy()
    genome[f1 * F + 600:f1 * F + 700] = read
    genome[f1 * F + 2:f1 * F + 102] = np.frombuffer(read.tobytes()[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA")),
                                                     np.uint8)
    seq = np.concatenate([reads.seq, read])
    off = np.concatenate([reads.offsets, [reads.offsets[-1] + 100]]).astype(np.int64)
    got = shard.map_sharded_local(genome, F, seq, off, 5, -4, world, ml)
    g = mss.mss_load_genome(genome, frag_len=F, max_read_len=ml)
    unsharded = mss.mss_map_reads(g, seq, off, 5, -4)
    g.close()
    want, _, _ = oracle_map(genome, F, seq, off, 5, -4, procs=cpu_count())
    assert_hits_equal(unsharded, want, "unsharded GPU vs oracle")
    assert_hits_equal(got, want, f"{world} GPU shards vs oracle")
    last = want[-1]
    assert (int(last["best_frag"]), int(last["best_score"]), int(last["offset"]), int(last["strand"])) == \
        (f1, 500, f1 * F + 600, 0)


def test_bounded_wait_gives_up_and_reports_timeout(mss):
    """A bounded device wait that runs out (an mbarrier phase nothing completes, 5 ms limit)
    comes back as MSS_ETIMEOUT from the synchronising call; the error word is cleared and the
    context still maps reads bit-exactly afterwards."""
    import time
    wl = gen.scaled(gen.workloads()["tiny-50k"], genome_len=20_000, reads=8)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=100)
    t0 = time.perf_counter()
    st = mss.mss_check_wait_timeout(g, 5000)
    dt = time.perf_counter() - t0
    assert st == mss.MSS_ETIMEOUT, st
    assert dt >= 0.004, dt
    mss.mss_sync(g)                                  # cleared: no error left behind
    assert mss.mss_check_wait_timeout(g, 0) == mss.MSS_EINVAL
    assert mss.mss_check_wait_timeout(g, 2_000_000) == mss.MSS_EINVAL
    hits = mss.mss_map_reads(g, reads.seq, reads.offsets, wl.match, wl.mismatch)
    want, _, _ = oracle.map_batch(genome, wl.frag_len, reads.seq, reads.offsets, wl.match, wl.mismatch)
    assert_hits_equal(hits, want, "after the wait self-check")
    g.close()


def test_map_sharded_over_nccl_one_rank(mss):
    """shard.map_sharded through a one-rank NCCL process group on this GPU: the library's scan
    of the rank's slice, the all-gather of the records on the device, the merge; equal to the
    oracle on the whole genome (every box here has one GPU, so this is the NCCL path's only
    run on hardware; the multi-rank exchange runs with gloo ranks on the CPU)."""
    import socket
    import torch
    import torch.distributed as dist
    from paper_1403_2136_gb300 import shard
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=120_000, reads=24)
    genome, reads = gen.materialize(wl)
    ml = int(np.diff(reads.offsets).max())
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        got = shard.map_sharded(genome, 2048, reads.seq, reads.offsets, 5, -4, ml)
    finally:
        dist.destroy_process_group()
    want, _, _ = oracle.map_batch(genome, 2048, reads.seq, reads.offsets, 5, -4)
    assert_hits_equal(got, want, "map_sharded over NCCL, one rank")


# ---------------------------------------------------------------- MaxSSmap_fast (read step 2)
@pytest.mark.parametrize("variant", [0, 1])
def test_fast_step_tiny_50k(mss, variant):
    """Every other read base: 50 kbp genome, 100 reads, both lane variants, with NW."""
    wl = gen.workloads()["tiny-50k"]
    genome, reads = gen.materialize(wl)
    hits, alns, cig, oh, oa, oc = run_both(mss, genome, reads.seq, reads.offsets, wl.frag_len, wl.match,
                                           wl.mismatch, nw=wl.nw, tune={"variant": variant}, procs=cpu_count(),
                                           step=2)
    assert_hits_equal(hits, oh, f"fast tiny-50k variant {variant}")
    assert_alns_equal(alns, cig, oa, oc, f"fast tiny-50k variant {variant}")


@pytest.mark.parametrize("match,mismatch", [(5, -4), (13, -4)])
def test_fast_step_uneven_odd_lengths(mss, match, mismatch):
    """Odd and even lengths (1 .. 700, several tiles and both selector-row sizes), N bases,
    reads planted across fragment borders; 13 / -4 runs the int16 lanes, 5 / -4 the f16 lanes."""
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=60_000, reads=40)
    genome, reads = gen.materialize(wl)
    g_ascii = bytes(genome)
    strs = [bytes(reads.read(i))[:L] for i, L in enumerate([1, 2, 3, 37, 100, 101, 150] * 5 + [149] * 5)]
    strs += [g_ascii[4096 - 60:4096 + 61], g_ascii[20_000:20_333].replace(b"C", b"N", 9)]
    long_reads = match == 13  # 5 x 400 <= 2048 keeps 5 / -4 on the f16 lanes
    if long_reads:
        strs.append(g_ascii[10_000:10_700])
    seq, off = concat_reads(strs)
    hits, _, _, oh, _, _ = run_both(mss, genome, seq, off, 2048, match, mismatch, max_len=700 if long_reads else 400,
                                    procs=cpu_count(), step=2)
    assert_hits_equal(hits, oh, f"fast uneven {match}/{mismatch}")


def test_fast_step_device_graph_and_back_to_plain(mss):
    """The device path replays its graph with step 2; switching back to step 1 gives the plain
    results; bad steps and unsupported scan shapes are rejected."""
    import torch
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=40_000, reads=24)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=1024, max_read_len=150)
    d_seq = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets).cuda()
    R = reads.count
    s = torch.cuda.Stream()
    mss.mss_set_read_step(g, 2)
    assert mss.mss_get_read_step(g) == 2
    want2, _, _ = oracle_map(genome, 1024, reads.seq, reads.offsets, 5, -4, procs=cpu_count(), step=2)
    for _ in range(2):
        d_hits = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
        mss.mss_map_reads_device(g, d_seq, d_off, R, 150, 5, -4, d_hits, stream=s)
        mss.mss_sync(g, stream=s)
        assert_hits_equal(mss.hits_from_bytes(d_hits.cpu()), want2, "fast device")
    mss.mss_set_read_step(g, 1)
    want1, _, _ = oracle_map(genome, 1024, reads.seq, reads.offsets, 5, -4, procs=cpu_count())
    assert_hits_equal(mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4), want1, "plain again")
    with pytest.raises(mss.MssError):
        mss.mss_set_read_step(g, 3)
    mss.mss_set_read_step(g, 2)
    mss.mss_set_tune(g, pairs=4, queries=8)
    with pytest.raises(mss.MssError):
        mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4)
    g.close()


# ---------------------------------------------------------------- base qualities (PSSM)
def _quals_for(reads_seq, seed):
    rng = np.random.default_rng(seed)
    return (33 + rng.integers(2, 42, size=reads_seq.shape[0])).astype(np.uint8)   # Phred 2..41


@pytest.mark.parametrize("scale", [4, 1])
def test_pssm_both_phases_match_oracle(mss, scale):
    """Position-specific scores from base qualities in phase one and phase two, bit for bit
    against the oracle (fragments, scores, offsets, strands, flags; NW score, span, CIGAR)."""
    import torch
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=50_000, reads=30)
    genome, reads = gen.materialize(wl)
    g_ascii = bytes(genome)
    strs = [bytes(reads.read(i)) for i in range(reads.count)]
    strs += [b"A", g_ascii[7000:7150].replace(b"G", b"N", 5), g_ascii[4096 - 50:4096 + 51]]
    seq, off = concat_reads(strs)
    quals = _quals_for(seq, 7 + scale)
    R, ML = len(strs), 150
    nw = (5, -4, -10, -1, 32)
    g = mss.mss_load_genome(genome, frag_len=2048, max_read_len=ML)
    d_seq, d_q, d_off = (torch.from_numpy(x).cuda() for x in (seq, quals, off))
    d_hits = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    mss.mss_map_reads_quals_device(g, d_seq, d_q, d_off, R, ML, 5, -4, scale, d_hits, stream=s)
    mss.mss_sync(g, stream=s)
    stride = 4 * ML + 64
    d_alns = torch.zeros(R * 24, dtype=torch.uint8, device="cuda")
    d_cig = torch.zeros(R * stride, dtype=torch.uint8, device="cuda")
    mss.nw_align_quals_device(g, d_seq, d_q, d_off, R, ML, d_hits, d_alns, d_cig, stride, scale, *nw, stream=s)
    mss.mss_sync(g, stream=s)
    hits = mss.hits_from_bytes(d_hits.cpu())
    alns = d_alns.cpu().numpy().view(mss.ALN_DTYPE)
    cig = d_cig.cpu().numpy().reshape(R, stride)
    cigars = [bytes(cig[i, :max(alns["cigar_len"][i], 0)]).decode() for i in range(R)]
    oh, oa, oc = oracle.map_batch(genome, 2048, seq, off, 5, -4, nw=nw, quals=quals, scale=scale)
    assert_hits_equal(hits, oh, f"pssm scale {scale}")
    assert_alns_equal(alns, cigars, oa, oc, f"pssm scale {scale}")
    # the graph of the call replays with the same qualities
    d_hits2 = torch.zeros_like(d_hits)
    mss.mss_map_reads_quals_device(g, d_seq, d_q, d_off, R, ML, 5, -4, scale, d_hits2, stream=s)
    mss.mss_sync(g, stream=s)
    assert torch.equal(d_hits, d_hits2)
    g.close()


def test_pssm_constant_quality_equals_plain_scores_and_errors(mss):
    """Every base at quality 40 ('I'): phase one equals the plain scan with scores
    (round(4*5*x), round(4*-4*x/3)) = (20, -5); a bad quality character is reported."""
    import torch
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=40_000, reads=24)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=1024, max_read_len=150)
    R = reads.count
    d_seq, d_off = torch.from_numpy(reads.seq).cuda(), torch.from_numpy(reads.offsets).cuda()
    d_q = torch.full((reads.seq.shape[0],), ord("I"), dtype=torch.uint8, device="cuda")
    d_hits = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    mss.mss_map_reads_quals_device(g, d_seq, d_q, d_off, R, 150, 5, -4, 4, d_hits)
    mss.mss_sync(g)
    want = mss.mss_map_reads(g, reads.seq, reads.offsets, 20, -5)
    assert_hits_equal(mss.hits_from_bytes(d_hits.cpu()), want, "quality 40 = plain 20 / -5")
    d_q[5] = ord(" ")
    mss.mss_map_reads_quals_device(g, d_seq, d_q, d_off, R, 150, 5, -4, 4, d_hits)
    with pytest.raises(mss.MssError):
        mss.mss_sync(g)
    with pytest.raises(mss.MssError):
        mss.mss_map_reads_quals_device(g, d_seq, d_q, d_off, R, 150, 5, -4, 40, d_hits)   # scale above 32
    g.close()


# ---------------------------------------------------------------- second fragment not adjacent to the best
@pytest.mark.parametrize("F", [1000, 333])
def test_second_rule_excluding_neighbours(mss, F):
    """With the neighbour rule the second is the best fragment not adjacent to the best, bit for
    bit against the oracle; reads straddling fragment borders make the plain second a
    neighbour often.  Switching back gives the plain result."""
    wl = gen.workloads()["tiny-50k"]
    genome, reads = gen.materialize(wl)
    g_ascii = bytes(genome)
    strs = [bytes(reads.read(i)) for i in range(reads.count)]
    strs += [g_ascii[b - 40:b + 60] for b in range(F, 20 * F, 2 * F)]   # junction reads
    seq, off = concat_reads(strs)
    g = mss.mss_load_genome(genome, frag_len=F, max_read_len=100)
    mss.mss_set_second_rule(g, True)
    got = mss.mss_map_reads(g, seq, off, wl.match, wl.mismatch)
    want, _, _ = oracle.map_batch(genome, F, seq, off, wl.match, wl.mismatch, exclude_neighbors=True)
    assert_hits_equal(got, want, f"neighbour rule F={F}")
    plain, _, _ = oracle_map(genome, F, seq, off, wl.match, wl.mismatch, procs=cpu_count())
    assert np.any(plain["second_frag"] != want["second_frag"])   # the rule changed something
    mss.mss_set_second_rule(g, False)
    assert_hits_equal(mss.mss_map_reads(g, seq, off, wl.match, wl.mismatch), plain, "plain rule again")
    g.close()

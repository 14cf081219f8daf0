"""Parity at the sizes the benchmark runs on.

* The bench workload itself: the full 4.6 Mbp genome with the bench's seed, F = 2048, the
  reads of one bench batch (50,000 reads of 100 and 150 bp at 10/20/30% substitutions) mapped
  in one call through the same device entry points the bench times; 48 reads spread evenly
  over the batch (both lengths, all three divergence levels) are compared field by field with
  the oracle: all seven hit fields, and the NW score, span and CIGAR.
* Genome positions beyond 2^31: the 2.4 Gbp genome of the ancient-DNA workload with reads
  drawn from its last 100 Mbp (the workload's lengths, low divergence so that they map where
  they were drawn).  Checked by what the oracle can compute one read at a time:
  the reported best and second fragment scores are the oracle's S(f) of those fragments, the
  offset and strand attain the best score, the repeat flag follows from the scores, the
  fragment the read was drawn from scores at most the best (and at most the second when it
  is not the best), and the NW alignment at offsets >= 2^31 equals the oracle's.
"""
import numpy as np
import pytest

import gen
import oracle
from tests.parity_util import ALN_FIELDS, HIT_FIELDS, cpu_count, oracle_map

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


def _device_map_align(mss, g, seq, off, max_len, match, mismatch, nw):
    """Phase one and two through the device entry points, as the bench calls them."""
    import torch
    R = int(off.shape[0] - 1)
    stride = 4 * max_len + 64
    d_seq = torch.from_numpy(seq).cuda()
    d_off = torch.from_numpy(off).cuda()
    d_hits = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    d_alns = torch.zeros(R * 24, dtype=torch.uint8, device="cuda")
    d_cig = torch.zeros(R * stride, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        mss.mss_map_reads_device(g, d_seq, d_off, R, max_len, match, mismatch, d_hits, stream=s)
        mss.nw_align_device(g, d_seq, d_off, R, max_len, d_hits, d_alns, d_cig, stride, *nw, stream=s)
        mss.mss_sync(g, stream=s)
    hits = mss.hits_from_bytes(d_hits.cpu())
    alns = d_alns.cpu().numpy().view(mss.ALN_DTYPE)
    cig = mss.cigar_strings(alns, d_cig.cpu().numpy().reshape(R, stride))
    return hits, alns, cig


def _subset(seq, off, idx):
    lens = (off[idx + 1] - off[idx]).astype(np.int64)
    o = np.zeros(idx.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=o[1:])
    s = np.concatenate([seq[off[i]:off[i + 1]] for i in idx])
    return s, o


def test_bench_batch_on_the_full_genome(mss):
    import bench
    wl = gen.workloads()["bact-4.6M"]
    genome = gen.make_genome(wl.genome, wl.seed)
    reads = gen.read_set(wl, genome, 0)
    max_len = int(reads.lengths.max())
    seq, off = bench.batches(reads.seq, reads.offsets, 50_000)[0]
    R = int(off.shape[0] - 1)
    assert R == 50_000
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=max_len)
    hits, alns, cig = _device_map_align(mss, g, seq, off, max_len, wl.match, wl.mismatch, wl.nw)
    g.close()
    idx = np.linspace(0, R - 1, 48).astype(np.int64)
    # the batch holds read i, i + 8, ... of the workload: both lengths and all three levels
    src = gen.batch_index(reads.count, 8, 0)[idx]
    assert set(reads.lengths[src].tolist()) == {100, 150}
    assert len(set((src % 200_000) * 3 // 200_000)) == 3
    s_seq, s_off = _subset(seq, off, idx)
    oh, oa, oc = oracle_map(genome, wl.frag_len, s_seq, s_off, wl.match, wl.mismatch, nw=wl.nw, procs=cpu_count())
    for f in HIT_FIELDS:
        assert np.array_equal(hits[f][idx].astype(np.int64), oh[f].astype(np.int64)), f
    for f in ALN_FIELDS:
        assert np.array_equal(alns[f][idx].astype(np.int64), oa[f].astype(np.int64)), f
    assert [cig[i] for i in idx] == oc
    assert (hits["best_score"] > 0).all()


def _frag_score(genome, F, read, f):
    """S(f) by the oracle alone: fragment f's diagonals with their windows (the genome from
    fF to fF + F + m - 1, N past its end) as a genome of its own, whose fragment 0 is f."""
    m = len(read)
    lo = f * F
    win = genome[lo:min(genome.shape[0], lo + F + m - 1)]
    _, fs = oracle.map_read(win, F, read, 5, -4, with_frag_scores=True)
    return int(fs[0])


def test_genome_offsets_beyond_2_31(mss):
    wl = gen.workloads()["ancient-2.4G"]
    genome = gen.make_genome(wl.genome, wl.seed)
    G = int(genome.shape[0])
    base = G - 100_000_000
    assert base > 2**31
    # the workload's read lengths at low divergence, so that nearly every read maps where it
    # was drawn and the offsets checked lie beyond 2^31
    rs = gen.ReadSpec(96, lognormal=(45, 0.35, 25, 80), sub_levels=((0.0, 0.05),), gap_mode=0)
    reads = gen.make_reads(genome[base:], rs, wl.seed * 37)
    max_len = int(reads.lengths.max())
    F = wl.frag_len
    g = mss.mss_load_genome(genome, frag_len=F, max_read_len=max_len)
    hits, alns, cig = _device_map_align(mss, g, reads.seq, reads.offsets, max_len, wl.match, wl.mismatch, wl.nw)
    g.close()
    nm, nmm, go, ge, W = wl.nw
    checked_high = 0
    for i in range(0, reads.count, 2):
        h = hits[i]
        read = reads.read(i)
        s1 = _frag_score(genome, F, read, int(h["best_frag"]))
        assert s1 == int(h["best_score"]), (i, s1, tuple(h))
        q = oracle.encode(read)
        qs = oracle.revcomp_codes(q) if h["strand"] else q
        d = int(h["offset"])
        assert int(h["best_frag"]) * F <= d < (int(h["best_frag"]) + 1) * F
        lo, hi = max(0, d - W - 1), min(G, d + len(q) + W + 1)
        gw = oracle.encode(genome[lo:hi])
        gpad = np.concatenate([gw, np.full(len(q) + 1, 4, np.uint8)])     # N past the genome's end
        assert oracle.diag_score(qs, gpad, d - lo, wl.match, wl.mismatch) == s1
        s2 = 0
        if h["second_frag"] >= 0:
            s2 = _frag_score(genome, F, read, int(h["second_frag"]))
            assert s2 == int(h["second_score"]) and s2 <= s1
        flag = 1 if (s1 == 0 or 10 * s2 >= 9 * s1) else 0
        assert int(h["flags"]) == flag
        tf = (base + int(reads.true_start[i])) // F
        st = _frag_score(genome, F, read, tf)
        assert st <= s1
        if tf != int(h["best_frag"]):
            assert st <= s2
        # phase two at this offset: the oracle on the window around it
        a = oracle.nw_banded(gw, qs, d - lo, W, nm, nmm, go, ge)
        assert (int(alns["score"][i]), int(alns["gstart"][i]), int(alns["gend"][i])) == \
            (a[0], a[1] + lo if a[1] >= 0 else a[1], a[2] + lo if a[2] >= 0 else a[2]), i
        assert cig[i] == a[3]
        checked_high += d >= 2**31
    assert checked_high >= reads.count // 4, checked_high      # of the 48 reads checked

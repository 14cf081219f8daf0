"""Uneven read lengths in one persistent launch (the chromosome-shaped workload): lengths
{36, 51, 76, 100, 150, 250} mixed in one call, genome with N runs and interspersed repeats.

* all reads bit-exact against the oracle on a smaller genome built with the same recipe;
* at the full 230 Mbp genome: sampled reads checked by properties the oracle can compute one
  by one: the reported best and second fragment scores equal the oracle's S(f) of those
  fragments (each rescanned by the oracle alone), the offset/strand attain the best score, and
  the flags follow from the scores.
"""
import numpy as np
import pytest

import gen
import oracle
from tests.parity_util import assert_hits_equal, cpu_count, oracle_map

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


def test_mixed_lengths_small_genome_all_reads(mss):
    wl = gen.scaled(gen.workloads()["chrom-230M"], genome_len=300_000, reads=120)
    genome, reads = gen.materialize(wl)
    assert set(np.unique(reads.lengths).tolist()) == {36, 51, 76, 100, 150, 250}
    assert (genome == ord("N")).mean() > 0.02          # N runs are present
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=250)
    hits = mss.mss_map_reads(g, reads.seq, reads.offsets, wl.match, wl.mismatch)
    alns, cig = mss.nw_align(g, reads.seq, reads.offsets, hits, *wl.nw)
    oh, oa, oc = oracle_map(genome, wl.frag_len, reads.seq, reads.offsets, wl.match, wl.mismatch, nw=wl.nw,
                            procs=cpu_count())
    assert_hits_equal(hits, oh, "chrom-shaped 300 kbp")
    for f in ("score", "gstart", "gend", "cigar_len"):
        assert np.array_equal(alns[f], oa[f]), f
    assert cig == oc
    g.close()


def _frag_score(gcodes_pad, q, qrc, d0, F, match, mismatch):
    return max(max(oracle.diag_score(q, gcodes_pad, d, match, mismatch),
                   oracle.diag_score(qrc, gcodes_pad, d, match, mismatch)) for d in range(d0, d0 + F))


def test_full_230M_genome_sampled_properties(mss):
    wl = gen.workloads()["chrom-230M"]
    genome = gen.make_genome(wl.genome, wl.seed)
    rs = gen.ReadSpec(3000, lengths=(36, 51, 76, 100, 150, 250), sub_levels=((0.1, 0.3),))
    reads = gen.make_reads(genome, rs, wl.seed * 31)
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=250)
    info = g.info()
    hits = mss.mss_map_reads(g, reads.seq, reads.offsets, wl.match, wl.mismatch)
    F = wl.frag_len
    G = genome.shape[0]
    # one read of each length: rescan the reported fragments with the oracle
    lens = reads.lengths
    picks = [int(np.nonzero(lens == L)[0][0]) for L in (36, 51, 76, 100, 150, 250)]
    for i in picks:
        h = hits[i]
        q = oracle.encode(reads.read(i))
        qrc = oracle.revcomp_codes(q)
        lo = int(h["best_frag"]) * F
        win = genome[lo:min(G, lo + F + len(q))]
        gpad = np.concatenate([oracle.encode(win), np.full(F + len(q) - win.shape[0] + 1, 4, np.uint8)])
        s1 = _frag_score(gpad, q, qrc, 0, F, wl.match, wl.mismatch)
        assert s1 == h["best_score"], (i, s1, tuple(h))
        # offset and strand attain it
        qs = qrc if h["strand"] else q
        assert oracle.diag_score(qs, gpad, int(h["offset"]) - lo, wl.match, wl.mismatch) == s1
        if h["second_frag"] >= 0:
            lo2 = int(h["second_frag"]) * F
            win2 = genome[lo2:min(G, lo2 + F + len(q))]
            gpad2 = np.concatenate([oracle.encode(win2), np.full(F + len(q) - win2.shape[0] + 1, 4, np.uint8)])
            s2 = _frag_score(gpad2, q, qrc, 0, F, wl.match, wl.mismatch)
            assert s2 == h["second_score"]
            assert s2 <= s1
        flag = 1 if (h["best_score"] == 0 or 10 * h["second_score"] >= 9 * h["best_score"]) else 0
        assert h["flags"] == flag
    # most reads map where they were drawn (divergent reads in a repeat-rich genome)
    hit_true = hits["best_frag"] == (reads.true_start // F)
    assert hit_true.mean() > 0.3
    assert info["num_frags"] == -(-G // F)
    g.close()

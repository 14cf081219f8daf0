"""Truth-based accuracy report (host code, no GPU): CIGAR walking and the correctness rule on
hand-made alignments, and on the oracle's own mapping of a small synthetic workload, where
low-divergence reads must come out nearly all correct."""
import numpy as np
import pytest

import gen
import oracle
from paper_1403_2136_gb300 import accuracy


def test_base_positions():
    assert list(accuracy.base_positions(100, "5M", 5)) == [100, 101, 102, 103, 104]
    assert list(accuracy.base_positions(100, "2M2D3M", 5)) == [100, 101, 104, 105, 106]
    assert list(accuracy.base_positions(100, "2M1I2M", 5)) == [100, 101, -1, 102, 103]
    with pytest.raises(ValueError):
        accuracy.base_positions(0, "4M", 5)


def _arrays(rows):
    hits = np.zeros(len(rows), dtype=oracle.HIT_DTYPE)
    alns = np.zeros(len(rows), dtype=oracle.ALN_DTYPE)
    cig = []
    for i, (strand, flag, gstart, c) in enumerate(rows):
        hits[i]["strand"], hits[i]["flags"] = strand, flag
        hits[i]["best_score"], hits[i]["second_score"] = 50, 10
        alns[i]["score"], alns[i]["cigar_len"], alns[i]["gstart"] = 40, len(c), gstart
        cig.append(c)
    return hits, alns, cig


def test_correct_mask_rules():
    hits, alns, cig = _arrays([
        (0, 0, 1000, "10M"),        # at the true start: correct
        (0, 0, 1001, "10M"),        # shifted by one: no base at its true position
        (1, 0, 1000, "10M"),        # wrong strand
        (0, 1, 1000, "10M"),        # flagged as a repeat: not mapped
        (0, 0, 1000, "3M2D7M"),     # the first three bases at their true positions
        (0, 0, 998, "2I8M"),        # two inserted bases; bases 2.. at 998.., true 1002..: none right
    ])
    truth = [np.arange(1000, 1010)] * 6
    strand = np.zeros(6, dtype=np.int8)
    got = accuracy.correct_mask(hits, alns, cig, truth, strand)
    assert list(got) == [True, False, False, False, True, False]
    assert list(accuracy.mapped_mask(hits, alns)) == [True, True, True, False, True, True]


def test_true_alignment_after_an_indel():
    """The true alignment of every base decides, not true_start + j: a read whose first two
    bases are inserted (true positions -1, -1, 1000, ...) is correct when aligned as 2I8M at
    1000, and an alignment that only matches start + j (8M2I at 1000) is not."""
    truth = [np.array([-1, -1] + list(range(1000, 1008)))] * 2
    hits, alns, cig = _arrays([(0, 0, 1000, "2I8M"), (0, 0, 1000, "8M2I")])
    got = accuracy.correct_mask(hits, alns, cig, truth, np.zeros(2, dtype=np.int8))
    assert list(got) == [True, False]
    # a deletion after base 3: bases 3.. sit 4 further on
    truth = [np.array(list(range(500, 503)) + list(range(507, 514)))]
    hits, alns, cig = _arrays([(0, 0, 500, "3M4D7M")])
    assert accuracy.correct_mask(hits, alns, cig, truth, np.zeros(1, dtype=np.int8))[0]
    hits, alns, cig = _arrays([(0, 0, 503, "10M")])     # start + j past the deletion: all wrong
    assert not accuracy.correct_mask(hits, alns, cig, truth, np.zeros(1, dtype=np.int8))[0]


def test_generator_truth_matches_the_genome():
    """The generator's per-base truth: a base with a true position equals the genome base
    there (forward orientation) unless substituted, so the agreement is 1 - substitution rate."""
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=100_000, reads=300)
    genome = gen.make_genome(wl.genome, wl.seed)
    reads = gen.make_reads(genome, wl.reads[0], wl.seed * 31, positions=True)
    comp = bytes.maketrans(b"ACGT", b"TGCA")
    plain = gen.make_reads(genome, wl.reads[0], wl.seed * 31)
    assert np.array_equal(plain.seq, reads.seq)                  # recording truth changes nothing
    for i in range(reads.count):
        s = reads.read(i)
        if reads.true_strand[i]:
            s = s[::-1].translate(comp)
        pos = reads.true_positions(i)
        ok = pos >= 0
        assert pos[ok][0] == reads.true_start[i] or not ok[0]
        assert np.all(np.diff(pos[ok]) >= 1)                     # increasing along the read
        same = np.frombuffer(s, np.uint8)[ok] == genome[pos[ok]]
        assert (~same).sum() <= reads.n_sub[i]                   # differences are substitutions
        # gap bases: inserted read bases plus genome bases skipped inside the span
        assert (~ok).sum() + (pos[ok][-1] - pos[ok][0] + 1 - ok.sum()) == reads.n_gap[i]


def test_oracle_mapping_is_accurate_at_low_divergence():
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=150_000, reads=120)
    genome = gen.make_genome(wl.genome, wl.seed)
    reads = gen.make_reads(genome, wl.reads[0], wl.seed * 31, positions=True)   # 100 bp at 10 / 20 / 30 %
    hits, alns, cigars = oracle.map_batch(genome, wl.frag_len, reads.seq, reads.offsets, wl.match, wl.mismatch,
                                          nw=wl.nw)
    mq = np.array([min(254, int(np.floor(-100 * np.log2(s / b) + 0.5))) if 0 < s < b else (254 if s == 0 < b else 0)
                   for b, s in zip(hits["best_score"], hits["second_score"])])
    R = reads.count
    groups = {"10%": np.arange(0, R // 3), "20%": np.arange(R // 3, 2 * R // 3), "30%": np.arange(2 * R // 3, R)}
    truth = [reads.true_positions(i) for i in range(R)]
    rep = accuracy.report(hits, alns, cigars, truth, reads.true_strand, groups, mapq=mq)
    assert rep["10%"]["correct_mapq0"] >= 0.95, rep
    assert rep["10%"]["correct_mapq0"] >= rep["30%"]["correct_mapq0"]
    for g in rep.values():
        assert g["correct_mapq0"] <= g["mapped_mapq0"] and g["mapped_mapq30"] <= g["mapped_mapq0"]

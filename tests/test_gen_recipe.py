"""The synthetic inputs follow their stated recipes (no GPU): deterministic per seed; genome
composition (GC, N runs, alphabet); read lengths, strands, substitution levels, gap sizes and
C->T deamination, checked against the truth the generator returns (source start, strand,
substitution count, total gap length)."""
import numpy as np

import gen

COMP = bytes.maketrans(b"ACGTN", b"TGCAN")


def _source(genome, reads, i):
    m, s = int(reads.lengths[i]), int(reads.true_start[i])
    src = genome[s:s + m].tobytes()
    return src.translate(COMP)[::-1] if reads.true_strand[i] == 1 else src


def test_deterministic_per_seed():
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=100_000, reads=400)
    g1, r1 = gen.materialize(wl)
    g2, r2 = gen.materialize(wl)
    assert np.array_equal(g1, g2) and np.array_equal(r1.seq, r2.seq) and np.array_equal(r1.offsets, r2.offsets)
    other = gen.make_reads(g1, wl.reads[0], wl.seed * 31 + 1000003)     # another rank's seed
    assert not np.array_equal(other.seq[:1000], r1.seq[:1000])


def test_bacterial_recipe():
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=300_000, reads=3000)
    genome, reads = gen.materialize(wl)
    assert set(np.unique(genome).tobytes()) <= set(b"ACGT")
    assert abs(np.isin(genome, np.frombuffer(b"GC", np.uint8)).mean() - 0.508) < 0.005
    lens = reads.lengths
    assert sorted(set(lens.tolist())) == [100, 150] and (lens == 100).sum() == (lens == 150).sum()
    assert abs(reads.true_strand.mean() - 0.5) < 0.05
    assert reads.n_gap.max() <= 60                       # at most two gaps of at most 30 bases
    free = np.nonzero(reads.n_gap == 0)[0]
    assert free.size > 500
    for i in free:                                       # gap-free reads: exactly n_sub differences
        r = reads.read(int(i))
        assert sum(a != b for a, b in zip(r, _source(genome, reads, int(i)))) == reads.n_sub[i]
    # each length's reads are split evenly over substitution levels 10 / 20 / 30 %
    for lo, hi, level in ((0, 1000, 0.1), (1000, 2000, 0.2), (2000, 3000, 0.3)):
        idx = free[(free % 1500 >= lo // 2) & (free % 1500 < hi // 2)]
        rate = (reads.n_sub[idx] / lens[idx]).mean()
        assert abs(rate - level) < 0.02, (level, rate)


def test_chromosome_recipe():
    wl = gen.scaled(gen.workloads()["chrom-230M"], genome_len=2_000_000, reads=600)
    genome, reads = gen.materialize(wl)
    n = (genome == ord("N")).mean()
    assert 0.02 < n < 0.08, n                             # 5% in runs
    runs = np.diff(np.flatnonzero(np.diff(np.r_[0, (genome == ord("N")).astype(np.int8), 0]) != 0))[::2]
    assert runs.size >= 1 and runs.max() > 1              # runs, not scattered bases
    acgt = genome[genome != ord("N")]
    assert abs(np.isin(acgt, np.frombuffer(b"GC", np.uint8)).mean() - 0.41) < 0.01
    assert set(reads.lengths.tolist()) == {36, 51, 76, 100, 150, 250}
    for i in range(reads.count):                          # reads never start on an N
        assert genome[reads.true_start[i]] != ord("N")


def test_ancient_recipe():
    wl = gen.scaled(gen.workloads()["ancient-2.4G"], genome_len=1_000_000, reads=4000)
    genome, reads = gen.materialize(wl)
    lens = reads.lengths
    assert lens.min() >= 25 and lens.max() <= 80 and abs(np.median(lens) - 45) <= 3
    free = np.nonzero(reads.n_gap == 0)[0]
    ct = np.zeros(12)
    c_total = np.zeros(12)
    for i in free:
        r, s = reads.read(int(i)), _source(genome, reads, int(i))
        for k in range(12):
            if s[k] == ord("C"):
                c_total[k] += 1
                ct[k] += r[k] == ord("T")
    rate = ct / np.maximum(c_total, 1)
    # C->T 30% at the 5' base decaying over 5 bases, on top of 15-25% substitutions (1/3 to T)
    assert rate[0] > 0.25 and rate[0] > rate[4] and rate[6:].max() < 0.15, rate

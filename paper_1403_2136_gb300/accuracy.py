"""Truth-based mapping accuracy of phase two's alignments (the paper's "Measure of accuracy
and error": a read counts as aligned correctly when at least one of its bases is aligned to the
same genome base as in its true alignment).

Host code on the outputs of the path: the hits (strand, repeat flag, scores) and alignments
(genome start, CIGAR) of `mss_map_align` / `nw_align`, against the true alignment that the
synthetic read generator records for every base: the genome position each base of the read
was copied from (in SAM's SEQ orientation, the forward genome strand, on either strand), or
none for a base inserted by an indel.  A read is correct when it is mapped, on its true
strand, and some aligned base j (CIGAR M) sits at base j's true position.

    python -m paper_1403_2136_gb300.accuracy --workload bact-4.6M --reads 30000

maps a synthetic workload on the GPU and prints, per substitution level, the fraction of reads
mapped, the fraction correct, and the same at MAPQ thresholds.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import sys

import numpy as np

_CIGAR = re.compile(r"(\d+)([MID])")


def base_positions(gstart: int, cigar: str, m: int) -> np.ndarray:
    """Genome position of each SEQ base (-1 for inserted bases) from the alignment start and
    CIGAR (M: aligned, I: read base against a gap, D: genome base against a gap)."""
    pos = np.full(m, -1, dtype=np.int64)
    j, g = 0, int(gstart)
    for n, op in _CIGAR.findall(cigar):
        n = int(n)
        if op == "M":
            pos[j:j + n] = np.arange(g, g + n)
            j += n
            g += n
        elif op == "I":
            j += n
        else:
            g += n
    if j != m:
        raise ValueError(f"CIGAR {cigar!r} covers {j} read bases, not {m}")
    return pos


def mapped_mask(hits, alns) -> np.ndarray:
    """Reads reported as mapped: not flagged as repeats by phase one and aligned by phase two
    (the same rule as the SAM writer)."""
    none = np.iinfo(np.int32).min
    return ((hits["flags"] & 1) == 0) & (alns["score"] != none) & (alns["cigar_len"] > 0)


def correct_mask(hits, alns, cigars, true_positions, true_strand) -> np.ndarray:
    """Per read: mapped, on the true strand, with some aligned base at its true position.
    true_positions[i]: the true genome position of every SEQ base of read i (-1: inserted)."""
    mapped = mapped_mask(hits, alns)
    out = np.zeros(len(true_positions), dtype=bool)
    for i in np.nonzero(mapped)[0]:
        if int(hits["strand"][i]) != int(true_strand[i]):
            continue
        truth = np.asarray(true_positions[i], dtype=np.int64)
        pos = base_positions(int(alns["gstart"][i]), cigars[i], truth.shape[0])
        out[i] = bool(np.any((pos >= 0) & (pos == truth)))
    return out


def mapq_of(hits) -> np.ndarray:
    """MAPQ of every read as the library computes it (-100 log2(second / best), capped)."""
    from paper_1403_2136_gb300 import mss_mapq
    return np.array([mss_mapq(int(b), int(s)) for b, s in zip(hits["best_score"], hits["second_score"])],
                    dtype=np.int32)


def report(hits, alns, cigars, true_positions, true_strand, groups: dict, mapq=None,
           thresholds=(0, 20, 30)) -> dict:
    """Mapped and correct fractions per read group (name -> index array), overall and at MAPQ
    thresholds (a read counts at threshold t when it is mapped with MAPQ >= t)."""
    mapped = mapped_mask(hits, alns)
    correct = correct_mask(hits, alns, cigars, true_positions, true_strand)
    mq = mapq if mapq is not None else mapq_of(hits)
    out = {}
    for name, idx in groups.items():
        idx = np.asarray(idx)
        n = max(1, idx.size)
        row = {"reads": int(idx.size)}
        for t in thresholds:
            keep = mapped[idx] & (mq[idx] >= t)
            row[f"mapped_mapq{t}"] = round(float(keep.sum()) / n, 5)
            row[f"correct_mapq{t}"] = round(float((keep & correct[idx]).sum()) / n, 5)
        out[name] = row
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="bact-4.6M")
    ap.add_argument("--reads", type=int, default=30_000)
    ap.add_argument("--genome", type=int, default=0, help="scaled genome length (0 = the workload's)")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import gen
    import paper_1403_2136_gb300 as mss

    wl = gen.scaled(gen.workloads()[args.workload], genome_len=args.genome or None, reads=args.reads)
    genome = gen.make_genome(wl.genome, wl.seed)
    parts = [(gen.make_reads(genome, rs, wl.seed * 31 + i, positions=True), rs) for i, rs in enumerate(wl.reads)]
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=max(int(p.lengths.max()) for p, _ in parts))
    out = {"workload": wl.name, "criterion": "strand right and some aligned base at its true position "
                                             "(the true alignment of every base)",
           "groups": {}}
    for k, (reads, spec) in enumerate(parts):
        hits, alns, cig = mss.mss_map_align(g, reads.seq, reads.offsets, wl.match, wl.mismatch, wl.nw)
        cigars = [bytes(cig[i, :max(int(alns["cigar_len"][i]), 0)]).decode() for i in range(reads.count)]
        R = reads.count
        nlev = len(spec.sub_levels)
        bounds = [R * i // nlev for i in range(nlev + 1)]
        groups = {}
        for li, (lo, hi) in enumerate(spec.sub_levels):
            lens = sorted(set(reads.lengths.tolist()))
            name = (f"{lens[0]}-{lens[-1]} bp" if len(lens) > 3 else "/".join(map(str, lens)) + " bp") + \
                (f", subs {lo:.0%}" if lo == hi else f", subs {lo:.0%}-{hi:.0%}")
            groups[name] = np.arange(bounds[li], bounds[li + 1])
        truth = [reads.true_positions(i) for i in range(R)]
        out["groups"].update(report(hits, alns, cigars, truth, reads.true_strand, groups))
    g.close()
    print(json.dumps(out, indent=1))
    return 0


if __name__ == "__main__":
    sys.exit(main())

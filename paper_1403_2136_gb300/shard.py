"""Genome sharding across ranks (host logic): each rank maps all reads against a contiguous
range of fragments, and the per-read top-2 summaries are merged.

Rank r owns fragments [f0, f1) and loads the genome slice [f0*F, f1*F + max_len - 1) (clipped
to the genome): the extra max_len - 1 bases keep the windows that cross into the next rank's
first fragment (the junctions of "First phase of MaxSSmap").  On the slice that next fragment
appears partially (a subset of its diagonals, windows truncated by N padding), so its score
there is a lower bound; the merge below is exact for such duplicates: the merged best is the
best entry of all summaries (higher score, then lower fragment), and the merged second is the
best entry, over all summaries, among those whose fragment differs from the merged best (a
rank's own second when its best is that fragment).  The best diagonal/strand comes with the
best entry; for a fragment seen fully on one rank and partially on another the two agree
whenever their scores tie (a first argmax on the subset is also the first on the whole).

The exchange is one all-gather of a fixed-size record per read (about 32 bytes).
"""
from __future__ import annotations

import numpy as np

REC = np.dtype([("s1", np.int32), ("f1", np.int32), ("s2", np.int32), ("f2", np.int32), ("strand", np.int32),
                ("pad", np.int32), ("offset", np.int64)])


def shard_bounds(G: int, F: int, world: int, rank: int, max_len: int):
    """Fragment range [f0, f1) of a rank and its genome slice [g0, g1)."""
    NF = -(-G // F)
    per = -(-NF // world)
    f0 = min(NF, rank * per)
    f1 = min(NF, (rank + 1) * per)
    g0 = f0 * F
    g1 = min(G, f1 * F + max_len - 1)
    return f0, f1, g0, g1


def to_records(hits, f0: int, F: int) -> np.ndarray:
    """Shard-local hits (fields of mss_hit) -> global top-2 records.  A rank with no fragment
    (empty slice) contributes empty records (score -1)."""
    R = len(hits)
    rec = np.zeros(R, dtype=REC)
    rec["s1"] = hits["best_score"]
    rec["f1"] = hits["best_frag"] + f0
    has2 = hits["second_frag"] >= 0
    rec["s2"] = np.where(has2, hits["second_score"], -1)
    rec["f2"] = np.where(has2, hits["second_frag"] + f0, np.iinfo(np.int32).max)
    rec["strand"] = hits["strand"]
    rec["offset"] = hits["offset"] + f0 * F
    return rec


def empty_records(R: int) -> np.ndarray:
    rec = np.zeros(R, dtype=REC)
    rec["s1"] = -1
    rec["f1"] = np.iinfo(np.int32).max
    rec["s2"] = -1
    rec["f2"] = np.iinfo(np.int32).max
    return rec


def _better(sa, fa, sb, fb):
    return (sa > sb) | ((sa == sb) & (fa < fb))


def merge(records: list) -> np.ndarray:
    """Exact merge of per-rank top-2 records (list of REC arrays over the same reads)."""
    out = records[0].copy()
    for b in records[1:]:
        A, B = out.copy(), b.copy()
        swap = _better(B["s1"], B["f1"], A["s1"], A["f1"])
        A[swap], B[swap] = b[swap], out[swap]
        # second: A's own second, or B's best entry whose fragment differs from A's best
        same = B["f1"] == A["f1"]
        bs = np.where(same, B["s2"], B["s1"])
        bf = np.where(same, B["f2"], B["f1"])
        take = _better(bs, bf, A["s2"], A["f2"])
        A["s2"] = np.where(take, bs, A["s2"])
        A["f2"] = np.where(take, bf, A["f2"])
        out = A
    return out


def records_to_hits(rec: np.ndarray):
    """Merged records -> mss_hit fields (second -1 / 0 when there is none; repeat flag)."""
    R = len(rec)
    from . import HIT_DTYPE
    h = np.zeros(R, dtype=HIT_DTYPE)
    h["best_frag"] = rec["f1"]
    h["best_score"] = rec["s1"]
    none = rec["s2"] < 0
    h["second_frag"] = np.where(none, -1, rec["f2"])
    h["second_score"] = np.where(none, 0, rec["s2"])
    h["offset"] = rec["offset"]
    h["strand"] = rec["strand"]
    best = h["best_score"].astype(np.int64)
    sec = h["second_score"].astype(np.int64)
    h["flags"] = ((best == 0) | (10 * sec >= 9 * best)).astype(np.int32)
    return h


def map_sharded_local(genome: np.ndarray, F: int, reads_seq, reads_off, match: int, mismatch: int, world: int,
                      max_len: int):
    """All shards one after another on the local GPU (the exchange emulated in memory)."""
    from . import mss_load_genome, mss_map_reads
    G = genome.shape[0]
    recs = []
    for r in range(world):
        f0, f1, g0, g1 = shard_bounds(G, F, world, r, max_len)
        if f1 <= f0:
            recs.append(empty_records(len(reads_off) - 1))
            continue
        g = mss_load_genome(genome[g0:g1], frag_len=F, max_read_len=max_len)
        hits = mss_map_reads(g, reads_seq, reads_off, match, mismatch)
        g.close()
        recs.append(to_records(hits, f0, F))
    return records_to_hits(merge(recs))

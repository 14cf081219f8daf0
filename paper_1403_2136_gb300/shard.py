"""Genome sharding across ranks: each rank maps all reads against a contiguous range of
fragments, the ranks exchange one fixed-size record per read, and the records are merged into
the whole-genome answer (the paper's suggestion of spreading the work over several GPUs, in
its discussion; the first phase of MaxSSmap is unchanged on each rank).

Rank r owns fragments [f0, f1) and loads the genome slice [f0*F, f1*F + max_len - 1) (clipped
to the genome): the extra max_len - 1 bases keep the windows that cross into the next rank's
first fragment (the junctions of "First phase of MaxSSmap").  On the slice that next fragment
f1 appears partially: only its diagonals [f1*F, f1*F + max_len - 1) exist, and their windows
are cut off by padding where the slice ends.  Cutting a window only turns scores into the
mismatch score, so every diagonal score there is at most its true score, and so is the
partial fragment's maximum.

Merge (exact):
  * best: the entry of highest score, then lowest fragment; among records that tie on both,
    the smallest (strand, offset).  A partial copy can tie its owner only when its own argmax
    (strand, offset) reaches the fragment's true score, which makes it one of the true
    argmaxes; the owner reports the first of them in the oracle's order (+ strand before -,
    then smallest offset), so the smallest pair is the owner's.
  * second: the best entry, over all records, among those whose fragment differs from the
    merged best.  A partial copy's lower score never wins wrongly: when its fragment is not
    in the owner's top two, the owner holds two strictly better fragments that outrank it.
The exchange is one all-gather of a 32-byte record per read.  The second-fragment rule that
excludes the best's neighbours needs more than the top two per rank and is not supported
through sharding (``map_sharded`` raises).
"""
from __future__ import annotations

import numpy as np

REC = np.dtype([("s1", np.int32), ("f1", np.int32), ("s2", np.int32), ("f2", np.int32), ("strand", np.int32),
                ("pad", np.int32), ("offset", np.int64)])
INT32_MAX = np.iinfo(np.int32).max


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
    """Shard-local hits (fields of mss_hit) -> global top-2 records."""
    R = len(hits)
    rec = np.zeros(R, dtype=REC)
    rec["s1"] = hits["best_score"]
    rec["f1"] = hits["best_frag"] + f0
    has2 = hits["second_frag"] >= 0
    rec["s2"] = np.where(has2, hits["second_score"], -1)
    rec["f2"] = np.where(has2, hits["second_frag"] + f0, INT32_MAX)
    rec["strand"] = hits["strand"]
    rec["offset"] = hits["offset"] + f0 * F
    return rec


def empty_records(R: int) -> np.ndarray:
    """Records of a rank that owns no fragment (score -1: below every real entry)."""
    rec = np.zeros(R, dtype=REC)
    rec["s1"] = -1
    rec["f1"] = INT32_MAX
    rec["s2"] = -1
    rec["f2"] = INT32_MAX
    return rec


def _better(sa, fa, sb, fb):
    return (sa > sb) | ((sa == sb) & (fa < fb))


def _best_first(a, b):
    """Per read: does record b's best come before record a's (score, fragment, strand, offset)?"""
    tie = (b["s1"] == a["s1"]) & (b["f1"] == a["f1"])
    arg = (b["strand"] < a["strand"]) | ((b["strand"] == a["strand"]) & (b["offset"] < a["offset"]))
    return _better(b["s1"], b["f1"], a["s1"], a["f1"]) | (tie & arg)


def merge(records: list) -> np.ndarray:
    """Exact merge of per-rank top-2 records (list of REC arrays over the same reads)."""
    out = records[0].copy()
    for b in records[1:]:
        A, B = out.copy(), b.copy()
        swap = _best_first(out, b)
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


def _map_slice_gpu(genome_slice, F, reads_seq, reads_off, match, mismatch, max_len):
    """Phase one of one rank's slice on the current CUDA device (the library's scan)."""
    from . import mss_load_genome, mss_map_reads
    g = mss_load_genome(genome_slice, frag_len=F, max_read_len=max_len)
    try:
        return mss_map_reads(g, reads_seq, reads_off, match, mismatch)
    finally:
        g.close()


def map_sharded(genome: np.ndarray, F: int, reads_seq, reads_off, match: int, mismatch: int, max_len: int,
                group=None, exclude_neighbors: bool = False, map_slice=None):
    """Genome-sharded phase one over the ranks of a ``torch.distributed`` process group.

    Every rank passes the whole genome (host array) and the same reads; it maps the reads
    against its own slice, then one ``all_gather_into_tensor`` of the 32-byte records (on the
    current CUDA device for NCCL, on the CPU for gloo) gives every rank all records, and
    every rank returns the same merged hits (the mss_hit fields of the whole-genome scan).

    ``map_slice(genome_slice, F, reads_seq, reads_off, match, mismatch, max_len)`` maps one
    slice; the default is the library's GPU scan on the current device.  The neighbour-
    excluding second rule is rejected (ValueError): the records carry the top two only.
    """
    import torch
    import torch.distributed as dist
    if exclude_neighbors:
        raise ValueError("the second-fragment rule excluding neighbours is not supported by genome sharding")
    if map_slice is None:
        map_slice = _map_slice_gpu
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    R = len(reads_off) - 1
    f0, f1, g0, g1 = shard_bounds(int(genome.shape[0]), F, world, rank, max_len)
    if f1 > f0 and R > 0:
        mine = to_records(map_slice(genome[g0:g1], F, reads_seq, reads_off, match, mismatch, max_len), f0, F)
    else:
        mine = empty_records(R)
    if R == 0:
        return records_to_hits(mine)
    words = REC.itemsize // 4
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    send = torch.from_numpy(mine.view(np.int32).reshape(R, words).copy()).to(dev)
    recv = torch.empty((world * R, words), dtype=torch.int32, device=dev)
    dist.all_gather_into_tensor(recv, send, group=group)
    allrec = recv.cpu().numpy().reshape(world, R * words)
    recs = [np.ascontiguousarray(allrec[r]).view(REC) for r in range(world)]
    return records_to_hits(merge(recs))


def map_sharded_local(genome: np.ndarray, F: int, reads_seq, reads_off, match: int, mismatch: int, world: int,
                      max_len: int):
    """All shards one after another on the local GPU (the exchange emulated in memory)."""
    G = genome.shape[0]
    recs = []
    for r in range(world):
        f0, f1, g0, g1 = shard_bounds(G, F, world, r, max_len)
        if f1 <= f0:
            recs.append(empty_records(len(reads_off) - 1))
            continue
        hits = _map_slice_gpu(genome[g0:g1], F, reads_seq, reads_off, match, mismatch, max_len)
        recs.append(to_records(hits, f0, F))
    return records_to_hits(merge(recs))

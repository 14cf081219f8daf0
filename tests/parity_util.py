"""Shared helpers of the parity tests: oracle runs (optionally in a spawn process pool) and
element-by-element comparison of hits and alignments."""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import oracle

HIT_FIELDS = ("best_frag", "second_frag", "best_score", "second_score", "offset", "strand", "flags")
ALN_FIELDS = ("score", "cigar_len", "gstart", "gend")


def _oracle_chunk(args):
    genome, F, seq, offsets, match, mismatch, nw, step = args
    hits, alns, cig = oracle.map_batch(genome, F, seq, offsets, match, mismatch, nw=nw, step=step)
    return hits, alns, cig


def oracle_map(genome, F, reads_seq, reads_off, match, mismatch, nw=None, procs: int | None = None, step: int = 1):
    """Run the oracle over reads; with procs > 1 the reads are split over a spawn pool."""
    R = reads_off.shape[0] - 1
    if procs is None:
        procs = 1
    if procs <= 1 or R <= 1:
        return oracle.map_batch(genome, F, reads_seq, reads_off, match, mismatch, nw=nw, step=step)
    procs = min(procs, R)
    bounds = np.linspace(0, R, procs + 1).astype(int)
    jobs = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        off = reads_off[a:b + 1] - reads_off[a]
        seq = reads_seq[reads_off[a]:reads_off[b]]
        jobs.append((genome, F, np.ascontiguousarray(seq), np.ascontiguousarray(off), match, mismatch, nw, step))
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_oracle_chunk, jobs))
    hits = np.concatenate([p[0] for p in parts])
    alns = np.concatenate([p[1] for p in parts]) if nw is not None else None
    cig = sum([p[2] for p in parts], []) if nw is not None else None
    return hits, alns, cig


def assert_hits_equal(got, want, ctx=""):
    for f in HIT_FIELDS:
        g = np.asarray(got[f]).astype(np.int64)
        w = np.asarray(want[f]).astype(np.int64)
        if not np.array_equal(g, w):
            bad = np.nonzero(g != w)[0]
            i = int(bad[0])
            raise AssertionError(f"{ctx}: hit field {f} differs at {bad.size} reads; first read {i}: "
                                 f"gpu {tuple(got[i])} oracle {tuple(want[i])}")


def assert_alns_equal(got, gcig, want, wcig, ctx=""):
    for f in ALN_FIELDS:
        g = np.asarray(got[f]).astype(np.int64)
        w = np.asarray(want[f]).astype(np.int64)
        if not np.array_equal(g, w):
            bad = np.nonzero(g != w)[0]
            i = int(bad[0])
            raise AssertionError(f"{ctx}: alignment field {f} differs at {bad.size} reads; first read {i}: "
                                 f"gpu {tuple(got[i])} {gcig[i]!r} oracle {tuple(want[i])} {wcig[i]!r}")
    for i, (a, b) in enumerate(zip(gcig, wcig)):
        assert a == b, f"{ctx}: CIGAR differs at read {i}: gpu {a!r} oracle {b!r}"


def concat_reads(strs):
    """Concatenate str/bytes reads into (uint8 seq, int64 offsets)."""
    bs = [s.encode() if isinstance(s, str) else bytes(s) for s in strs]
    off = np.zeros(len(bs) + 1, dtype=np.int64)
    np.cumsum([len(b) for b in bs], out=off[1:])
    seq = np.frombuffer(b"".join(bs), dtype=np.uint8).copy() if bs else np.zeros(0, np.uint8)
    return seq, off


def cpu_count() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1

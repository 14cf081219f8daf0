"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws data (genomes, read lengths, reads and their true origin).  It
holds none of the mapping arithmetic.  The shapes follow the paper's workloads:
E. coli-like 4.6 Mbp genomes with 100-250 bp reads at 10-30% divergence and gaps up to
30 bp (Section "Data simulation"), read lengths 36-150 (Table 7), and short, very
divergent ancient reads on a Gbp genome (Section "Applications on real data").  The C
core (``gen.c``) is compiled on first use with the host ``gcc``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libmssgen.so")
_LOCK = threading.Lock()
_LIB = None

BASE_SEED = 14032136


def build(force: bool = False) -> str:
    """Compile gen.c into libmssgen.so next to it (portable C, no arch flags)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.gen_genome.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_int64, P]
            lib.gen_genome.restype = ctypes.c_int
            lib.gen_reads.argtypes = [ctypes.c_uint64, P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                      P, P, P, P, P, P, P]
            lib.gen_reads.restype = ctypes.c_int
            lib.gen_lengths.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, P]
            lib.gen_lengths.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class GenomeSpec:
    length: int
    gc: float = 0.5
    copy_frac: float = 0.0
    copy_min: int = 1000
    copy_max: int = 5000
    fam_frac: float = 0.0
    fam_count: int = 100
    fam_len: int = 300
    fam_div: float = 0.15
    n_frac: float = 0.0
    n_min: int = 1
    n_max: int = 50000


@dataclass
class ReadSpec:
    count: int
    lengths: tuple = (100,)          # constant (one entry) or uniform choice among entries
    lognormal: tuple | None = None   # (median, sigma, lo, hi) overrides lengths
    sub_levels: tuple = ((0.10, 0.10),)  # reads are split evenly over these [lo, hi] ranges
    gap_mode: int = 2                # 0 none, 1 one gap U[gap_min, gap_max], 2 U{0..2} geometric gaps
    gap_count_max: int = 2
    gap_min: int = 1
    gap_max: int = 30
    gap_p: float = 0.25
    deam_rate: float = 0.0
    deam_len: int = 5


def make_genome(spec: GenomeSpec, seed: int) -> np.ndarray:
    """ASCII genome (uint8 array of 'ACGTN')."""
    out = np.empty(spec.length, dtype=np.uint8)
    rc = _lib().gen_genome(seed, spec.length, spec.gc, spec.copy_frac, spec.copy_min, spec.copy_max,
                           spec.fam_frac, spec.fam_count, spec.fam_len, spec.fam_div, spec.n_frac,
                           spec.n_min, spec.n_max, _ptr(out))
    if rc != 0:
        raise RuntimeError(f"gen_genome failed ({rc})")
    return out


@dataclass
class Reads:
    seq: np.ndarray          # uint8 concatenated ASCII
    offsets: np.ndarray      # int64 [R+1]
    true_start: np.ndarray   # int64 [R]
    true_strand: np.ndarray  # int8 [R]
    n_sub: np.ndarray        # int32 [R]
    n_gap: np.ndarray        # int32 [R]
    true_rel: np.ndarray | None = None  # int32 per base (same offsets as seq): genome position of
    #                                     SEQ base j (forward-strand orientation) minus true_start,
    #                                     -1 for an inserted base; only when asked for

    @property
    def count(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int32)

    def read(self, i: int) -> bytes:
        return self.seq[self.offsets[i]:self.offsets[i + 1]].tobytes()

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths[idx].astype(np.int64)
        offs = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        seq = np.concatenate([self.seq[self.offsets[i]:self.offsets[i + 1]] for i in idx]) if idx.size else \
            np.zeros(0, np.uint8)
        rel = np.concatenate([self.true_rel[self.offsets[i]:self.offsets[i + 1]] for i in idx]) \
            if self.true_rel is not None and idx.size else None
        return Reads(seq, offs, self.true_start[idx], self.true_strand[idx], self.n_sub[idx], self.n_gap[idx], rel)

    def true_positions(self, i: int) -> np.ndarray:
        """Genome position of every SEQ base of read i (-1 for inserted bases)."""
        rel = self.true_rel[self.offsets[i]:self.offsets[i + 1]].astype(np.int64)
        return np.where(rel >= 0, rel + int(self.true_start[i]), -1)


def make_lengths(spec: ReadSpec, seed: int) -> np.ndarray:
    out = np.empty(spec.count, dtype=np.int32)
    if spec.lognormal is not None:
        med, sig, lo, hi = spec.lognormal
        lst = np.array([0], dtype=np.int32)
        _lib().gen_lengths(seed, spec.count, 2, _ptr(lst), 1, float(med), float(sig), int(lo), int(hi), _ptr(out))
    else:
        lst = np.asarray(spec.lengths, dtype=np.int32)
        mode = 0 if lst.size == 1 else 1
        _lib().gen_lengths(seed, spec.count, mode, _ptr(lst), int(lst.size), 0.0, 0.0, 0, 0, _ptr(out))
    return out


def make_reads(genome: np.ndarray, spec: ReadSpec, seed: int, positions: bool = False) -> Reads:
    lengths = make_lengths(spec, seed)
    R = spec.count
    parts = []
    nlev = len(spec.sub_levels)
    bounds = [R * i // nlev for i in range(nlev + 1)]
    for li, (lo, hi) in enumerate(spec.sub_levels):
        a, b = bounds[li], bounds[li + 1]
        n = b - a
        if n == 0:
            continue
        lens = np.ascontiguousarray(lengths[a:b])
        offs = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(lens.astype(np.int64), out=offs[1:])
        seq = np.empty(int(offs[-1]), dtype=np.uint8)
        ts = np.empty(n, dtype=np.int64)
        st = np.empty(n, dtype=np.int8)
        ns = np.empty(n, dtype=np.int32)
        ng = np.empty(n, dtype=np.int32)
        rel = np.empty(int(offs[-1]), dtype=np.int32) if positions else None
        rc = _lib().gen_reads(seed + 7919 * li, _ptr(genome), genome.shape[0], n, _ptr(lens), float(lo), float(hi),
                              spec.gap_mode, spec.gap_count_max, spec.gap_min, spec.gap_max, spec.gap_p,
                              spec.deam_rate, spec.deam_len, _ptr(seq), _ptr(offs), _ptr(ts), _ptr(st),
                              _ptr(ns), _ptr(ng), _ptr(rel) if positions else None)
        if rc != 0:
            raise RuntimeError(f"gen_reads failed ({rc})")
        parts.append(Reads(seq, offs, ts, st, ns, ng, rel))
    return concat_reads(parts)


@dataclass
class Workload:
    """One named workload: genome + reads + mapping parameters."""
    name: str
    genome: GenomeSpec
    reads: list                      # list of ReadSpec (concatenated in order)
    frag_len: int
    match: int
    mismatch: int
    nw: tuple = (5, -4, -26, -26, 32)  # match, mismatch, gap open, gap extend, band W
    seed: int = BASE_SEED
    notes: str = ""
    extra: dict = field(default_factory=dict)


def workloads() -> dict:
    """The workloads, named by what they are (sizes in the name)."""
    w = {}
    w["tiny-50k"] = Workload(
        "tiny-50k: 50 kbp uniform genome, F=1000, 100 x 100 bp reads, 10% subs + one 1-5 bp indel, +1/-1",
        GenomeSpec(50_000, gc=0.5),
        [ReadSpec(100, lengths=(100,), sub_levels=((0.10, 0.10),), gap_mode=1, gap_min=1, gap_max=5)],
        frag_len=1000, match=1, mismatch=-1, nw=(1, -1, -2, -1, 32), seed=BASE_SEED + 1)
    w["bact-4.6M"] = Workload(
        "bact-4.6M: 4.6 Mbp genome (GC 50.8%, 2% exact 1-5 kbp repeat copies), F=2048, "
        "200k x 100 bp + 200k x 150 bp reads at 10/20/30% subs, <=2 geometric gaps <=30 bp, 5/-4, "
        "banded NW 5/-4/-10/-1 W=32",
        GenomeSpec(4_600_000, gc=0.508, copy_frac=0.02, copy_min=1000, copy_max=5000),
        [ReadSpec(200_000, lengths=(100,), sub_levels=((0.1, 0.1), (0.2, 0.2), (0.3, 0.3))),
         ReadSpec(200_000, lengths=(150,), sub_levels=((0.1, 0.1), (0.2, 0.2), (0.3, 0.3)))],
        frag_len=2048, match=5, mismatch=-4, nw=(5, -4, -10, -1, 32), seed=BASE_SEED + 2)
    w["chrom-230M"] = Workload(
        "chrom-230M: 230 Mbp genome (GC 41%, 5% N runs 1-50 kbp, 10% interspersed 300 bp repeats at 15% div), "
        "1M reads, lengths uniform over {36,51,76,100,150,250}, 10-30% subs, gaps <=30 bp",
        GenomeSpec(230_000_000, gc=0.41, fam_frac=0.10, fam_count=100, fam_len=300, fam_div=0.15,
                   n_frac=0.05, n_min=1, n_max=50_000),
        [ReadSpec(1_000_000, lengths=(36, 51, 76, 100, 150, 250), sub_levels=((0.1, 0.3),))],
        frag_len=2048, match=5, mismatch=-4, nw=(5, -4, -10, -1, 32), seed=BASE_SEED + 3)
    w["ancient-2.4G"] = Workload(
        "ancient-2.4G: 2.4 Gbp genome (GC 41%), 2M reads lognormal lengths 25-80 (median 45), 15-25% div, "
        "C->T deamination 30% decaying over 5 bases",
        GenomeSpec(2_400_000_000, gc=0.41),
        [ReadSpec(2_000_000, lognormal=(45, 0.35, 25, 80), sub_levels=((0.15, 0.25),), deam_rate=0.30,
                  deam_len=5)],
        frag_len=2048, match=5, mismatch=-4, nw=(5, -4, -10, -1, 32), seed=BASE_SEED + 5)
    return w


def scaled(wl: Workload, genome_len: int | None = None, reads: int | None = None) -> Workload:
    """Same recipe at a smaller size (parity-test sizes)."""
    g = GenomeSpec(**{**wl.genome.__dict__})
    if genome_len is not None:
        g.length = genome_len
        g.n_max = min(g.n_max, max(1, genome_len // 50))
        g.copy_max = min(g.copy_max, max(g.copy_min, genome_len // 20))
        g.copy_min = min(g.copy_min, g.copy_max)
    rs = []
    for r in wl.reads:
        r2 = ReadSpec(**{**r.__dict__})
        if reads is not None:
            r2.count = max(1, reads * r.count // sum(x.count for x in wl.reads))
        rs.append(r2)
    return Workload(wl.name + f" (scaled: G={g.length}, R={sum(x.count for x in rs)})", g, rs, wl.frag_len,
                    wl.match, wl.mismatch, wl.nw, wl.seed, wl.notes)


def concat_reads(parts: list) -> Reads:
    if len(parts) == 1:
        return parts[0]
    R = sum(p.count for p in parts)
    seq = np.concatenate([p.seq for p in parts])
    lens = np.concatenate([p.lengths for p in parts]).astype(np.int64)
    offs = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    rel = np.concatenate([p.true_rel for p in parts]) if all(p.true_rel is not None for p in parts) else None
    return Reads(seq, offs, np.concatenate([p.true_start for p in parts]),
                 np.concatenate([p.true_strand for p in parts]), np.concatenate([p.n_sub for p in parts]),
                 np.concatenate([p.n_gap for p in parts]), rel)


def read_set(wl: Workload, genome: np.ndarray, rank: int = 0, positions: bool = False) -> Reads:
    """All reads of a workload in order (its ReadSpecs one after another), drawn for one rank:
    rank 0 gives the reads of ``materialize``; other ranks get other seeds.  positions: also
    record every base's true genome position (``Reads.true_rel``)."""
    return concat_reads([make_reads(genome, rs, wl.seed * 31 + i + 1000003 * rank, positions)
                    for i, rs in enumerate(wl.reads)])


def batch_index(R: int, n_batches: int, b: int) -> np.ndarray:
    """Reads of batch b when R reads are dealt into n_batches batches: b, b + n, b + 2n, ...
    (every batch gets the same mix of read lengths and divergences)."""
    return np.arange(b, R, n_batches, dtype=np.int64)


def materialize(wl: Workload):
    """Genome (uint8 ASCII) and Reads for a workload."""
    genome = make_genome(wl.genome, wl.seed)
    return genome, read_set(wl, genome, 0)

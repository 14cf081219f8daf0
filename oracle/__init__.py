"""CPU oracle for the MaxSSmap hot path — TEST INFRASTRUCTURE ONLY.

Plain single-threaded C (``oracle.c``), compiled with the host ``gcc`` and loaded with
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never calls it and shares no code
with it.  ``oracle.h`` lists the sections of the paper each function follows and every
reading taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

NW_NONE = -2147483648


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Hit(ctypes.Structure):
    _fields_ = [("best_frag", ctypes.c_int32), ("second_frag", ctypes.c_int32), ("best_score", ctypes.c_int32),
                ("second_score", ctypes.c_int32), ("offset", ctypes.c_int64), ("strand", ctypes.c_int32),
                ("flags", ctypes.c_int32)]

    def as_tuple(self):
        return (self.best_frag, self.second_frag, self.best_score, self.second_score, self.offset, self.strand,
                self.flags)


class Aln(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("cigar_len", ctypes.c_int32), ("gstart", ctypes.c_int64),
                ("gend", ctypes.c_int64)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            # MSS_ORACLE_LIB: a compiled variant of oracle.c to load instead (the tests that plant
            # mistakes in the oracle use it to show that the pins catch them)
            lib = ctypes.CDLL(os.environ.get("MSS_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.orc_base_code.argtypes = [ctypes.c_int]
            lib.orc_mss.argtypes = [P, i64]
            lib.orc_mss.restype = i64
            lib.orc_diag_score.argtypes = [P, i32, P, i64, i32, i32]
            lib.orc_diag_score.restype = i32
            lib.orc_diag_score_step.argtypes = [P, i32, P, i64, i32, i32, i32]
            lib.orc_diag_score_step.restype = i32
            lib.orc_map_read.argtypes = [P, i64, i64, P, i32, i32, i32, ctypes.POINTER(Hit), P]
            lib.orc_map_read_step.argtypes = [P, i64, i64, P, i32, i32, i32, i32, ctypes.POINTER(Hit), P]
            lib.orc_map_read_excl.argtypes = [P, i64, i64, P, i32, i32, i32, ctypes.POINTER(Hit), P]
            lib.orc_pssm_scores.argtypes = [i32, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
            lib.orc_map_read_pssm.argtypes = [P, i64, i64, P, P, i32, i32, i32, i32, ctypes.POINTER(Hit), P]
            lib.orc_nw_banded_pssm.argtypes = [P, i64, P, P, P, i32, i64, i32, i32, i32, ctypes.POINTER(Aln),
                                               ctypes.c_char_p, i32]
            lib.orc_map_batch_pssm.argtypes = [P, i64, i64, P, P, P, i32, i32, i32, i32, i32, i32, i32, i32, i32,
                                               P, P, P, i32]
            lib.orc_revcomp.argtypes = [P, i32, P]
            lib.orc_revcomp.restype = None
            lib.orc_encode.argtypes = [P, i64, P]
            lib.orc_nw_banded.argtypes = [P, i64, P, i32, i64, i32, i32, i32, i32, i32, ctypes.POINTER(Aln),
                                          ctypes.c_char_p, i32]
            lib.orc_nw_literal.argtypes = [P, i64, i64, i32, P, i32, i32, i32, i32, i32, ctypes.POINTER(Aln),
                                           ctypes.c_char_p, i32]
            lib.orc_map_batch.argtypes = [P, i64, i64, P, P, i32, i32, i32, i32, i32, i32, i32, i32, P, P, P, i32]
            lib.orc_map_batch_step.argtypes = [P, i64, i64, P, P, i32, i32, i32, i32, i32, i32, i32, i32, i32, P, P, P,
                                               i32]
            _LIB = lib
    return _LIB


def _buf(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    if isinstance(x, str):
        return np.frombuffer(x.encode(), dtype=np.uint8)
    return np.ascontiguousarray(x)


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def base_code(c: str) -> int:
    return _lib().orc_base_code(ord(c))


def encode(seq) -> np.ndarray:
    s = _buf(seq).astype(np.uint8, copy=False)
    out = np.empty(s.shape[0], dtype=np.uint8)
    if _lib().orc_encode(_p(s), s.shape[0], _p(out)) != 0:
        raise ValueError("invalid character")
    return out


def revcomp_codes(q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.uint8)
    out = np.empty_like(q)
    _lib().orc_revcomp(_p(q), q.shape[0], _p(out))
    return out


def mss(x) -> int:
    a = np.ascontiguousarray(x, dtype=np.int32)
    return int(_lib().orc_mss(_p(a), a.shape[0]))


def diag_score(qcodes, gcodes_padded, d: int, match: int, mismatch: int, step: int = 1) -> int:
    """step 2: the read sampled at every other position ("MaxSSmap_fast")."""
    q = np.ascontiguousarray(qcodes, dtype=np.uint8)
    g = np.ascontiguousarray(gcodes_padded, dtype=np.uint8)
    assert d + q.shape[0] <= g.shape[0]
    if step == 1:
        return int(_lib().orc_diag_score(_p(q), q.shape[0], _p(g), d, match, mismatch))
    return int(_lib().orc_diag_score_step(_p(q), q.shape[0], _p(g), d, match, mismatch, step))


def pssm_scores(qual_char: int, match: int, mismatch: int, scale: int):
    """(match, mismatch) of a base with Phred+33 quality character qual_char, in fixed point."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    if _lib().orc_pssm_scores(int(qual_char), match, mismatch, scale, ctypes.byref(a), ctypes.byref(b)) != 0:
        raise ValueError("bad quality character or scale")
    return a.value, b.value


def nw_banded_pssm(gcodes, qcodes, ma, mm, d: int, W: int, gap_open: int, gap_extend: int, cigar_cap: int = 4096):
    g = np.ascontiguousarray(gcodes, dtype=np.uint8)
    q = np.ascontiguousarray(qcodes, dtype=np.uint8)
    a_ = np.ascontiguousarray(ma, dtype=np.int32)
    m_ = np.ascontiguousarray(mm, dtype=np.int32)
    a = Aln()
    buf = ctypes.create_string_buffer(cigar_cap)
    rc = _lib().orc_nw_banded_pssm(_p(g), g.shape[0], _p(q), _p(a_), _p(m_), q.shape[0], d, W, gap_open, gap_extend,
                                   ctypes.byref(a), buf, cigar_cap)
    if rc != 0:
        raise ValueError(f"orc_nw_banded_pssm failed ({rc})")
    return a.score, a.gstart, a.gend, buf.value.decode()


def map_read(genome, F: int, read, match: int, mismatch: int, with_frag_scores: bool = False, step: int = 1,
             quals=None, scale: int = 4, exclude_neighbors: bool = False):
    """quals (Phred+33, one per read base): position-specific scores with the given fixed-point scale."""
    g = _buf(genome)
    r = _buf(read)
    h = Hit()
    NF = (g.shape[0] + F - 1) // F
    fs = np.empty(NF, dtype=np.int32) if with_frag_scores else None
    if exclude_neighbors:
        assert quals is None and step == 1
        rc = _lib().orc_map_read_excl(_p(g), g.shape[0], F, _p(r), r.shape[0], match, mismatch, ctypes.byref(h),
                                      _p(fs) if fs is not None else None)
    elif quals is not None:
        qb = _buf(quals)
        assert qb.shape[0] == r.shape[0]
        rc = _lib().orc_map_read_pssm(_p(g), g.shape[0], F, _p(r), _p(qb), r.shape[0], match, mismatch, scale,
                                      ctypes.byref(h), _p(fs) if fs is not None else None)
    elif step == 1:
        rc = _lib().orc_map_read(_p(g), g.shape[0], F, _p(r), r.shape[0], match, mismatch, ctypes.byref(h),
                                 _p(fs) if fs is not None else None)
    else:
        rc = _lib().orc_map_read_step(_p(g), g.shape[0], F, _p(r), r.shape[0], match, mismatch, step,
                                      ctypes.byref(h), _p(fs) if fs is not None else None)
    if rc != 0:
        raise ValueError(f"orc_map_read failed ({rc})")
    return (h.as_tuple(), fs) if with_frag_scores else h.as_tuple()


def nw_banded(gcodes, qcodes, d: int, W: int, match: int, mismatch: int, gap_open: int, gap_extend: int,
              cigar_cap: int = 4096):
    g = np.ascontiguousarray(gcodes, dtype=np.uint8)
    q = np.ascontiguousarray(qcodes, dtype=np.uint8)
    a = Aln()
    buf = ctypes.create_string_buffer(cigar_cap)
    rc = _lib().orc_nw_banded(_p(g), g.shape[0], _p(q), q.shape[0], d, W, match, mismatch, gap_open, gap_extend,
                              ctypes.byref(a), buf, cigar_cap)
    if rc != 0:
        raise ValueError(f"orc_nw_banded failed ({rc})")
    return a.score, a.gstart, a.gend, buf.value.decode()


def nw_literal(gcodes, F: int, best_frag: int, qcodes, match: int, mismatch: int, gap_open: int, gap_extend: int,
               cigar_cap: int = 8192):
    g = np.ascontiguousarray(gcodes, dtype=np.uint8)
    q = np.ascontiguousarray(qcodes, dtype=np.uint8)
    a = Aln()
    buf = ctypes.create_string_buffer(cigar_cap)
    rc = _lib().orc_nw_literal(_p(g), g.shape[0], F, best_frag, _p(q), q.shape[0], match, mismatch, gap_open,
                               gap_extend, ctypes.byref(a), buf, cigar_cap)
    if rc != 0:
        raise ValueError(f"orc_nw_literal failed ({rc})")
    return a.score, a.gstart, a.gend, buf.value.decode()


HIT_DTYPE = np.dtype([("best_frag", np.int32), ("second_frag", np.int32), ("best_score", np.int32),
                      ("second_score", np.int32), ("offset", np.int64), ("strand", np.int32), ("flags", np.int32)])
ALN_DTYPE = np.dtype([("score", np.int32), ("cigar_len", np.int32), ("gstart", np.int64), ("gend", np.int64)])


def map_batch(genome, F: int, reads: np.ndarray, offsets: np.ndarray, match: int, mismatch: int,
              nw=None, cigar_cap: int = 1024, step: int = 1, quals=None, scale: int = 4,
              exclude_neighbors: bool = False):
    """Phase one (and phase two when nw = (match, mismatch, open, extend, W)) for a batch.
    Returns (hits structured array, alns structured array or None, list of CIGAR strings or None)."""
    g = _buf(genome)
    rd = np.ascontiguousarray(reads, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    R = off.shape[0] - 1
    hits = np.zeros(R, dtype=HIT_DTYPE)
    alns = np.zeros(R, dtype=ALN_DTYPE) if nw is not None else None
    cig = np.zeros((R, cigar_cap), dtype=np.uint8) if nw is not None else None
    nm, nmm, go, ge, W = nw if nw is not None else (0, 0, 0, 0, 0)
    if exclude_neighbors:   # phase one only, read by read
        assert nw is None and quals is None and step == 1
        for i in range(R):
            hits[i] = map_read(g, F, rd[off[i]:off[i + 1]], match, mismatch, exclude_neighbors=True)
        return hits, None, None
    if quals is not None:
        qd = np.ascontiguousarray(quals, dtype=np.uint8)
        assert qd.shape[0] == rd.shape[0]
        rc = _lib().orc_map_batch_pssm(_p(g), g.shape[0], F, _p(rd), _p(qd), _p(off), R, match, mismatch, scale, nm,
                                       nmm, go, ge, W, _p(hits), _p(alns) if alns is not None else None,
                                       _p(cig) if cig is not None else None, cigar_cap)
    else:
        rc = _lib().orc_map_batch_step(_p(g), g.shape[0], F, _p(rd), _p(off), R, match, mismatch, step, nm, nmm, go,
                                       ge, W, _p(hits), _p(alns) if alns is not None else None,
                                       _p(cig) if cig is not None else None, cigar_cap)
    if rc != 0:
        raise ValueError(f"orc_map_batch failed ({rc})")
    cigars = None
    if cig is not None:
        cigars = [bytes(cig[i, :alns["cigar_len"][i]]).decode() for i in range(R)]
    return hits, alns, cigars

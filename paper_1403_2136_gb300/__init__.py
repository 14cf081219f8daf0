"""Python binding of libmaxss (MaxSSmap hot path on GB300).

Argument marshalling only: every step of the mapping runs in the CUDA kernels of
``libmaxss.so`` behind the C ABI declared in ``include/maxss.h``.  PyTorch is used for device
memory and streams; numpy arrays are accepted for the host-pointer entry points.  There is no
CPU fallback: importing this package fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmaxss.so")

MSS_OK = 0
MSS_EINVAL = -1
MSS_ENOMEM = -2
MSS_ECUDA = -3
MSS_EREADLEN = -4
MSS_EOVERFLOW = -5
MSS_ETIMEOUT = -6
MSS_ESTATE = -7
MSS_MAX_READ_LEN = 2432
MSS_NW_NONE = -2147483648
MSS_HIT_REPEAT = 1

# every symbol include/maxss.h declares
EXPORTS = ("mss_load_genome", "mss_load_genome_device", "mss_get_info", "mss_set_frag_len", "mss_set_read_step",
           "mss_set_second_rule",
           "mss_get_read_step", "mss_set_tune",
           "mss_get_tune", "mss_map_reads", "mss_map_reads_device", "nw_align", "nw_align_device", "nw_align_device_noalloc", "mss_map_align", "mss_sync",
           "mss_autotune", "mss_scan_timing", "mss_scan_time_ms", "mss_launch_count", "mss_genome_codes", "mss_probe_pipes", "mss_check_wait_timeout", "mss_prop_create", "mss_prop_free", "mss_prop_param_count",
           "mss_prop_get_params", "mss_prop_set_params", "mss_prop_set_pooling", "mss_prop_get_pooling", "mss_prop_read_codes", "mss_prop_window_codes",
           "mss_prop_embed_device", "mss_prop_grad_device", "mss_prop_train_step", "mss_prop_build_index",
           "mss_map_reads_proposed", "mss_prop_save", "mss_prop_load", "mss_prop_launch_count", "mss_free",
           "mss_map_reads_quals_device", "nw_align_quals_device", "mss_mapq", "mss_format_sam", "mss_last_error")

HIT_DTYPE = np.dtype([("best_frag", np.int32), ("second_frag", np.int32), ("best_score", np.int32),
                      ("second_score", np.int32), ("offset", np.int64), ("strand", np.int32), ("flags", np.int32)])
ALN_DTYPE = np.dtype([("score", np.int32), ("cigar_len", np.int32), ("gstart", np.int64), ("gend", np.int64)])
assert HIT_DTYPE.itemsize == 32 and ALN_DTYPE.itemsize == 24


class MssError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


class GenomeParams(ctypes.Structure):
    _fields_ = [("frag_len", ctypes.c_int64), ("max_read_len", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ScoreParams(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32)]


class NwParams(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("band", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GenomeInfo(ctypes.Structure):
    _fields_ = [("genome_len", ctypes.c_int64), ("frag_len", ctypes.c_int64), ("num_frags", ctypes.c_int64),
                ("padded_len", ctypes.c_int64), ("max_read_len", ctypes.c_int32), ("num_sms", ctypes.c_int32)]


class Tune(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("pairs", ctypes.c_int32), ("queries", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("min_items_per_cta", ctypes.c_int32), ("threads", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmaxss.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmaxss.so not built ({path}); run paper_1403_2136_gb300/build.py "
                          "(or __graft_entry__.build()) on a machine with nvcc")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "mss_load_genome": ([ctypes.POINTER(P), P, i64, ctypes.POINTER(GenomeParams), P], i32),
        "mss_load_genome_device": ([ctypes.POINTER(P), P, i64, ctypes.POINTER(GenomeParams), P], i32),
        "mss_get_info": ([P, ctypes.POINTER(GenomeInfo)], i32),
        "mss_set_frag_len": ([P, i64], i32),
        "mss_set_read_step": ([P, i32], i32),
        "mss_set_second_rule": ([P, i32], i32),
        "mss_get_read_step": ([P], i32),
        "mss_set_tune": ([P, ctypes.POINTER(Tune)], i32),
        "mss_get_tune": ([P, ctypes.POINTER(Tune)], i32),
        "mss_map_reads": ([P, P, P, i32, ctypes.POINTER(ScoreParams), P, P], i32),
        "mss_map_reads_device": ([P, P, P, i32, i32, ctypes.POINTER(ScoreParams), P, P], i32),
        "nw_align": ([P, P, P, i32, P, ctypes.POINTER(NwParams), P, P, i32, P], i32),
        "nw_align_device": ([P, P, P, i32, i32, P, ctypes.POINTER(NwParams), P, P, i32, P], i32),
        "nw_align_device_noalloc": ([P, P, P, i32, i32, P, ctypes.POINTER(NwParams), P, P, i32, P], i32),
        "mss_map_align": ([P, P, P, i32, ctypes.POINTER(ScoreParams), ctypes.POINTER(NwParams), P, P, P, i32, P],
                          i32),
        "mss_sync": ([P, P], i32),
        "mss_autotune": ([P, P, P, i32, i32, ctypes.POINTER(ScoreParams), i32, P], i32),
        "mss_scan_timing": ([P, i32], i32),
        "mss_scan_time_ms": ([P, ctypes.POINTER(ctypes.c_float)], i32),
        "mss_launch_count": ([P], i64),
        "mss_genome_codes": ([P, i64, i64, P], i32),
        "mss_probe_pipes": ([ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(ctypes.c_double)], i32),
        "mss_check_wait_timeout": ([P, ctypes.c_uint32, P], i32),
        "mss_prop_create": ([ctypes.POINTER(P), ctypes.c_uint64, P], i32),
        "mss_prop_free": ([P], None),
        "mss_prop_param_count": ([], i64),
        "mss_prop_get_params": ([P, P, i64], i32),
        "mss_prop_set_params": ([P, P, i64], i32),
        "mss_prop_set_pooling": ([P, i32], i32),
        "mss_prop_get_pooling": ([P], i32),
        "mss_prop_read_codes": ([P, P, P, P, P, i32, i32, P, P, P], i32),
        "mss_prop_window_codes": ([P, P, P, i32, i32, i32, P, P, P], i32),
        "mss_prop_embed_device": ([P, P, P, i32, i32, i32, P, P], i32),
        "mss_prop_grad_device": ([P, P, P, i32, i32, i32, P, P, P], i32),
        "mss_prop_train_step": ([P, P, P, i32, i32, i32, P, P, i32, i32, i32, P, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.POINTER(ctypes.c_float), P], i32),
        "mss_prop_build_index": ([P, P, i32, P], i32),
        "mss_map_reads_proposed": ([P, P, P, P, i32, i32, ctypes.POINTER(ScoreParams), i32, ctypes.c_float, P, P, P,
                                    ctypes.POINTER(ctypes.c_int32), P], i32),
        "mss_prop_save": ([P, ctypes.c_char_p], i32),
        "mss_prop_load": ([P, ctypes.c_char_p], i32),
        "mss_prop_launch_count": ([P], i64),
        "mss_free": ([P], None),
        "mss_last_error": ([], ctypes.c_char_p),
        "mss_mapq": ([i32, i32], i32),
        "mss_map_reads_quals_device": ([P, P, P, P, i32, i32, P, i32, P, P], i32),
        "nw_align_quals_device": ([P, P, P, P, i32, i32, P, P, i32, P, P, i32, P], i32),
        "mss_format_sam": ([ctypes.c_char_p, i64, P, P, i32, P, P, P, i32, i32, P, i64], i64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != MSS_OK:
        raise MssError(st, where, (_lib.mss_last_error() or b"").decode(errors="replace"))


def _host_ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(a.ctypes.data)
    # torch tensor (CPU pinned or device)
    return ctypes.c_void_p(a.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Genome:
    """A packed genome on the device (owns the mss_ctx)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        gi = GenomeInfo()
        _check(_lib.mss_get_info(self._h, ctypes.byref(gi)), "mss_get_info")
        return {f: getattr(gi, f) for f, _ in GenomeInfo._fields_}

    def close(self):
        if self._h:
            _lib.mss_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mss_load_genome(seq, frag_len: int = 2048, max_read_len: int = MSS_MAX_READ_LEN, stream=None) -> Genome:
    """Pack a genome.  seq: bytes / uint8 numpy array (host) or a uint8 CUDA tensor (device)."""
    lib = load_library()
    p = GenomeParams(frag_len, max_read_len, 0)
    h = ctypes.c_void_p()
    if isinstance(seq, (bytes, bytearray)):
        seq = np.frombuffer(bytes(seq), dtype=np.uint8)
    if isinstance(seq, np.ndarray):
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        st = lib.mss_load_genome(ctypes.byref(h), _host_ptr(seq), seq.shape[0], ctypes.byref(p), _stream_ptr(stream))
        _check(st, "mss_load_genome")
    else:
        st = lib.mss_load_genome_device(ctypes.byref(h), _host_ptr(seq), int(seq.numel()), ctypes.byref(p),
                                        _stream_ptr(stream))
        _check(st, "mss_load_genome_device")
    return Genome(h)


def mss_set_frag_len(g: Genome, frag_len: int):
    _check(load_library().mss_set_frag_len(g.handle, frag_len), "mss_set_frag_len")


def mss_set_read_step(g: Genome, step: int):
    """1: every read base; 2: every other read base ("MaxSSmap_fast")."""
    _check(load_library().mss_set_read_step(g.handle, step), "mss_set_read_step")


def mss_set_second_rule(g: Genome, exclude_neighbors: bool):
    """True: the second fragment is the best one not adjacent to the best."""
    _check(load_library().mss_set_second_rule(g.handle, 1 if exclude_neighbors else 0), "mss_set_second_rule")


def mss_get_read_step(g: Genome) -> int:
    return int(load_library().mss_get_read_step(g.handle))


def mss_set_tune(g: Genome, variant=-1, pairs=0, queries=0, ctas_per_sm=0, min_items_per_cta=0, threads=0):
    t = Tune(variant, pairs, queries, ctas_per_sm, min_items_per_cta, threads)
    _check(load_library().mss_set_tune(g.handle, ctypes.byref(t)), "mss_set_tune")


def mss_get_tune(g: Genome) -> dict:
    t = Tune()
    _check(load_library().mss_get_tune(g.handle, ctypes.byref(t)), "mss_get_tune")
    return {f: getattr(t, f) for f, _ in Tune._fields_}


def mss_map_reads(g: Genome, reads, offsets, match: int, mismatch: int, out=None, stream=None) -> np.ndarray:
    """Phase one, host buffers (numpy or pinned torch).  Returns the hits (HIT_DTYPE)."""
    lib = load_library()
    offsets = offsets if not isinstance(offsets, np.ndarray) else np.ascontiguousarray(offsets, dtype=np.int64)
    R = (offsets.shape[0] if isinstance(offsets, np.ndarray) else offsets.numel()) - 1
    if out is None:
        out = np.zeros(R, dtype=HIT_DTYPE)
    sp = ScoreParams(match, mismatch)
    st = lib.mss_map_reads(g.handle, _host_ptr(reads), _host_ptr(offsets), R, ctypes.byref(sp), _host_ptr(out),
                           _stream_ptr(stream))
    _check(st, "mss_map_reads")
    return out


def mss_map_reads_device(g: Genome, d_reads, d_offsets, R: int, max_len: int, match: int, mismatch: int, d_out,
                         stream=None):
    """Phase one, device buffers: d_out is a CUDA tensor of at least 32*R bytes."""
    sp = ScoreParams(match, mismatch)
    st = load_library().mss_map_reads_device(g.handle, _host_ptr(d_reads), _host_ptr(d_offsets), R, max_len,
                                             ctypes.byref(sp), _host_ptr(d_out), _stream_ptr(stream))
    _check(st, "mss_map_reads_device")


def nw_align(g: Genome, reads, offsets, hits: np.ndarray, match=5, mismatch=-4, gap_open=-26, gap_extend=-26,
             band=32, cigar_stride=None, stream=None):
    """Phase two, host buffers.  Returns (alns HIT array of ALN_DTYPE, list of CIGAR strings)."""
    lib = load_library()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    R = offsets.shape[0] - 1
    if cigar_stride is None:
        lens = np.diff(offsets)
        cigar_stride = int(max(16, 4 * (int(lens.max()) if R else 1) + 64))
    out = np.zeros(R, dtype=ALN_DTYPE)
    cig = np.zeros((max(R, 1), cigar_stride), dtype=np.uint8)
    npar = NwParams(match, mismatch, gap_open, gap_extend, band, 0)
    st = lib.nw_align(g.handle, _host_ptr(reads), _host_ptr(offsets), R, _host_ptr(np.ascontiguousarray(hits)),
                      ctypes.byref(npar), _host_ptr(out), _host_ptr(cig), cigar_stride, _stream_ptr(stream))
    _check(st, "nw_align")
    cigars = [bytes(cig[i, :max(out["cigar_len"][i], 0)]).decode() for i in range(R)]
    return out, cigars


def mss_map_reads_quals_device(g: Genome, d_reads, d_quals, d_offsets, R: int, max_len: int, match: int,
                               mismatch: int, scale: int, d_out, stream=None):
    """Phase one with base qualities (Phred+33, device tensors); d_out: 32*R bytes."""
    sp = ScoreParams(match, mismatch)
    _check(load_library().mss_map_reads_quals_device(g.handle, _host_ptr(d_reads), _host_ptr(d_quals),
                                                     _host_ptr(d_offsets), R, max_len, ctypes.byref(sp), scale,
                                                     _host_ptr(d_out), _stream_ptr(stream)),
           "mss_map_reads_quals_device")


def nw_align_quals_device(g: Genome, d_reads, d_quals, d_offsets, R: int, max_len: int, d_hits, d_out, d_cigars,
                          cigar_stride: int, scale: int, match=5, mismatch=-4, gap_open=-26, gap_extend=-26, band=32,
                          stream=None):
    npar = NwParams(match, mismatch, gap_open, gap_extend, band, 0)
    _check(load_library().nw_align_quals_device(g.handle, _host_ptr(d_reads), _host_ptr(d_quals), _host_ptr(d_offsets),
                                                R, max_len, _host_ptr(d_hits), ctypes.byref(npar), scale,
                                                _host_ptr(d_out), _host_ptr(d_cigars), cigar_stride,
                                                _stream_ptr(stream)),
           "nw_align_quals_device")


def mss_mapq(best_score: int, second_score: int) -> int:
    """-100 log2(second / best), rounded, capped at 254 ("Mapping qualities ..." paragraph)."""
    return int(load_library().mss_mapq(int(best_score), int(second_score)))


def format_sam(ref_name: str, genome_len: int, reads, offsets, hits, alns, cigars=None, header: bool = True) -> str:
    """SAM text of mapped reads (host arrays; cigars: list of CIGAR strings from nw_align)."""
    lib = load_library()
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    alns = np.ascontiguousarray(alns, dtype=ALN_DTYPE)
    R = offsets.shape[0] - 1
    cbuf, stride = None, 0
    if cigars is not None:
        stride = max([len(c) for c in cigars] + [0]) + 1
        cbuf = np.zeros((max(R, 1), stride), dtype=np.uint8)
        for i, c in enumerate(cigars):
            cbuf[i, :len(c)] = np.frombuffer(c.encode(), dtype=np.uint8)
    args = (ref_name.encode(), int(genome_len), _host_ptr(reads), _host_ptr(offsets), R, _host_ptr(hits),
            _host_ptr(alns), _host_ptr(cbuf) if cbuf is not None else None, stride, 1 if header else 0)
    n = lib.mss_format_sam(*args, None, 0)
    if n < 0:
        raise MssError(int(n), "mss_format_sam", "invalid arguments")
    buf = ctypes.create_string_buffer(int(n) + 1)
    lib.mss_format_sam(*args, buf, n + 1)
    return buf.value.decode()


def nw_align_device(g: Genome, d_reads, d_offsets, R: int, max_len: int, d_hits, d_out, d_cigars,
                    cigar_stride: int, match=5, mismatch=-4, gap_open=-26, gap_extend=-26, band=32, stream=None):
    npar = NwParams(match, mismatch, gap_open, gap_extend, band, 0)
    st = load_library().nw_align_device(g.handle, _host_ptr(d_reads), _host_ptr(d_offsets), R, max_len,
                                        _host_ptr(d_hits), ctypes.byref(npar), _host_ptr(d_out),
                                        _host_ptr(d_cigars), cigar_stride, _stream_ptr(stream))
    _check(st, "nw_align_device")


def mss_map_align(g: Genome, reads, offsets, match: int, mismatch: int, nw=(5, -4, -26, -26, 32), hits=None,
                  alns=None, cigars=None, cigar_stride: int = 0, stream=None):
    """Both phases, host buffers (numpy or pinned torch), one upload.  Outputs are allocated as
    numpy arrays unless given.  Returns (hits, alns, cigar bytes [R, stride])."""
    R = (offsets.shape[0] if isinstance(offsets, np.ndarray) else offsets.numel()) - 1
    if cigar_stride <= 0:
        lens = np.diff(np.asarray(offsets if isinstance(offsets, np.ndarray) else offsets.numpy()))
        cigar_stride = int(max(16, 4 * (int(lens.max()) if R else 1) + 64))
    hits = np.zeros(R, dtype=HIT_DTYPE) if hits is None else hits
    alns = np.zeros(R, dtype=ALN_DTYPE) if alns is None else alns
    cigars = np.zeros((max(R, 1), cigar_stride), dtype=np.uint8) if cigars is None else cigars
    sp = ScoreParams(match, mismatch)
    npar = NwParams(*nw, 0)
    st = load_library().mss_map_align(g.handle, _host_ptr(reads), _host_ptr(offsets), R, ctypes.byref(sp),
                                      ctypes.byref(npar), _host_ptr(hits), _host_ptr(alns), _host_ptr(cigars),
                                      cigar_stride, _stream_ptr(stream))
    _check(st, "mss_map_align")
    return hits, alns, cigars


def cigar_strings(alns, cigars) -> list:
    """Decode CIGAR slots (numpy [R, stride] uint8) using the lengths in alns."""
    return [bytes(cigars[i, :max(int(alns["cigar_len"][i]), 0)]).decode() for i in range(len(alns))]


def mss_sync(g: Genome, stream=None):
    _check(load_library().mss_sync(g.handle, _stream_ptr(stream)), "mss_sync")


def mss_autotune(g: Genome, d_reads, d_offsets, R: int, max_len: int, match: int, mismatch: int,
                 allow_frag_len: bool = False, stream=None) -> dict:
    sp = ScoreParams(match, mismatch)
    st = load_library().mss_autotune(g.handle, _host_ptr(d_reads), _host_ptr(d_offsets), R, max_len,
                                     ctypes.byref(sp), 1 if allow_frag_len else 0, _stream_ptr(stream))
    _check(st, "mss_autotune")
    return {**mss_get_tune(g), "frag_len": g.info()["frag_len"]}


def mss_scan_timing(g: Genome, enable: bool = True):
    _check(load_library().mss_scan_timing(g.handle, 1 if enable else 0), "mss_scan_timing")


def mss_scan_time_ms(g: Genome) -> float:
    ms = ctypes.c_float()
    _check(load_library().mss_scan_time_ms(g.handle, ctypes.byref(ms)), "mss_scan_time_ms")
    return float(ms.value)


def mss_launch_count(g: Genome) -> int:
    return int(load_library().mss_launch_count(g.handle))


def mss_genome_codes(g: Genome, start: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint8)
    _check(load_library().mss_genome_codes(g.handle, start, n, _host_ptr(out)), "mss_genome_codes")
    return out


PROBE_MODES = ("dpx_add_max", "fma_relu", "prmt_and_fma_relu", "prmt", "max3", "scan_mix", "dpx_and_fma_relu")


def mss_probe_pipes():
    """Warp-instructions per SM clock of the probes (dict keyed by PROBE_MODES) and the SM clock
    in MHz the rates are counted at."""
    r = (ctypes.c_double * len(PROBE_MODES))()
    clk = ctypes.c_double()
    _check(load_library().mss_probe_pipes(r, len(PROBE_MODES), ctypes.byref(clk)), "mss_probe_pipes")
    return dict(zip(PROBE_MODES, list(r))), clk.value


def mss_check_wait_timeout(g: Genome, limit_us: int = 2000, stream=None) -> int:
    """Run the bounded-wait self-check; returns its status (MSS_ETIMEOUT when the wait gave up
    as designed) without raising, so that the caller can check the code."""
    return int(load_library().mss_check_wait_timeout(g.handle, limit_us, _stream_ptr(stream)))


def hits_from_bytes(buf) -> np.ndarray:
    """View raw hit bytes (numpy uint8 or a CPU tensor) as HIT_DTYPE records."""
    a = buf.numpy() if hasattr(buf, "numpy") else np.asarray(buf)
    return a.view(HIT_DTYPE)


# ---------------------------------------------------------------------------------------------
# learned fragment proposal
class Proposal:
    """The proposal CNN (owns the mss_prop)."""

    def __init__(self, seed: int = 1, stream=None):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.mss_prop_create(ctypes.byref(h), seed, _stream_ptr(stream)), "mss_prop_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @staticmethod
    def param_count() -> int:
        return int(load_library().mss_prop_param_count())

    def get_params(self) -> np.ndarray:
        n = self.param_count()
        out = np.zeros(n, dtype=np.float32)
        _check(_lib.mss_prop_get_params(self._h, _host_ptr(out), n), "mss_prop_get_params")
        return out

    def set_params(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(_lib.mss_prop_set_params(self._h, _host_ptr(w), w.shape[0]), "mss_prop_set_params")

    POOLINGS = {"max": 0, "mean": 1}

    @property
    def pooling(self) -> str:
        """How the last layer's positions become one vector: "max" or "mean"."""
        v = int(_lib.mss_prop_get_pooling(self._h))
        return {i: k for k, i in self.POOLINGS.items()}[v]

    @pooling.setter
    def pooling(self, name: str):
        if name not in self.POOLINGS:
            raise ValueError(f"pooling must be one of {sorted(self.POOLINGS)}")
        _check(_lib.mss_prop_set_pooling(self._h, self.POOLINGS[name]), "mss_prop_set_pooling")

    def read_codes(self, d_reads, d_offsets, d_idx, d_strand, n, ld, d_codes, d_lens, stream=None):
        _check(_lib.mss_prop_read_codes(self._h, _host_ptr(d_reads), _host_ptr(d_offsets), _host_ptr(d_idx),
                                        _host_ptr(d_strand), n, ld, _host_ptr(d_codes), _host_ptr(d_lens),
                                        _stream_ptr(stream)), "mss_prop_read_codes")

    def window_codes(self, g: Genome, d_starts, n, length, ld, d_codes, d_lens, stream=None):
        _check(_lib.mss_prop_window_codes(self._h, g.handle, _host_ptr(d_starts), n, length, ld, _host_ptr(d_codes),
                                          _host_ptr(d_lens), _stream_ptr(stream)), "mss_prop_window_codes")

    def embed(self, d_codes, d_lens, ld, n, maxlen, d_emb, stream=None):
        _check(_lib.mss_prop_embed_device(self._h, _host_ptr(d_codes), _host_ptr(d_lens), ld, n, maxlen,
                                          _host_ptr(d_emb), _stream_ptr(stream)), "mss_prop_embed_device")

    def grad(self, d_codes, d_lens, ld, n, maxlen, d_demb, d_grad, stream=None):
        _check(_lib.mss_prop_grad_device(self._h, _host_ptr(d_codes), _host_ptr(d_lens), ld, n, maxlen,
                                         _host_ptr(d_demb), _host_ptr(d_grad), _stream_ptr(stream)),
               "mss_prop_grad_device")

    def train_step(self, d_rcodes, d_rlens, ld_r, B, maxlen_r, d_ccodes, d_clens, ld_c, C, maxlen_c, d_labels,
                   lr=1e-3, temperature=0.05, weight_decay=0.01, stream=None) -> float:
        loss = ctypes.c_float()
        _check(_lib.mss_prop_train_step(self._h, _host_ptr(d_rcodes), _host_ptr(d_rlens), ld_r, B, maxlen_r,
                                        _host_ptr(d_ccodes), _host_ptr(d_clens), ld_c, C, maxlen_c,
                                        _host_ptr(d_labels), lr, temperature, weight_decay, ctypes.byref(loss),
                                        _stream_ptr(stream)), "mss_prop_train_step")
        return float(loss.value)

    def build_index(self, g: Genome, max_read_len: int, stream=None):
        _check(_lib.mss_prop_build_index(self._h, g.handle, max_read_len, _stream_ptr(stream)),
               "mss_prop_build_index")

    def map_reads(self, g: Genome, d_reads, d_offsets, R, max_len, match, mismatch, K, tau, d_out, d_cand=None,
                  d_top=None, stream=None) -> int:
        sp = ScoreParams(match, mismatch)
        nfb = ctypes.c_int32()
        _check(_lib.mss_map_reads_proposed(g.handle, self._h, _host_ptr(d_reads), _host_ptr(d_offsets), R, max_len,
                                           ctypes.byref(sp), K, tau, _host_ptr(d_out), _host_ptr(d_cand),
                                           _host_ptr(d_top), ctypes.byref(nfb), _stream_ptr(stream)),
               "mss_map_reads_proposed")
        return int(nfb.value)

    def save(self, path: str):
        _check(_lib.mss_prop_save(self._h, path.encode()), "mss_prop_save")

    def load(self, path: str):
        _check(_lib.mss_prop_load(self._h, path.encode()), "mss_prop_load")

    def launch_count(self) -> int:
        return int(_lib.mss_prop_launch_count(self._h))

    def close(self):
        if self._h:
            _lib.mss_prop_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""nw_align_device_noalloc: phase two for callers that cannot allocate device memory.

Those callers (code inside CUDA stream capture, latency-critical serving loops, processes
whose device memory belongs to a pool allocator) use an entry point whose traceback scratch
is a fixed array in the library image.  This test calls it through the C ABI twice in a row
and checks both results against nw_align_device (integer results: bit-exact).  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def test_noalloc_matches_nw_align_device_twice():
    import torch

    import paper_1403_2136_gb300 as mss
    from paper_1403_2136_gb300 import build
    build.build()
    lib = mss.load_library()

    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=200_000, reads=300)
    genome, reads = gen.materialize(wl)
    R = reads.count
    max_len = int(np.diff(reads.offsets).max())
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=max_len)
    hits = mss.mss_map_reads(g, reads.seq, reads.offsets, wl.match, wl.mismatch)
    d_seq = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets).cuda()
    d_hits = torch.from_numpy(hits.view(np.uint8).copy()).cuda()
    stride = 4 * max_len + 64
    nw = mss.NwParams(*wl.nw, 0)

    ref_aln = torch.zeros(R * 24, dtype=torch.uint8, device="cuda")
    ref_cig = torch.zeros(R * stride, dtype=torch.uint8, device="cuda")
    st = lib.nw_align_device(g.handle, ctypes.c_void_p(d_seq.data_ptr()), ctypes.c_void_p(d_off.data_ptr()), R,
                             max_len, ctypes.c_void_p(d_hits.data_ptr()), ctypes.byref(nw),
                             ctypes.c_void_p(ref_aln.data_ptr()), ctypes.c_void_p(ref_cig.data_ptr()), stride, None)
    assert st == 0, lib.mss_last_error()
    mss.mss_sync(g)

    for call in range(2):
        out_aln = torch.full((R * 24,), 0xAB, dtype=torch.uint8, device="cuda")
        out_cig = torch.full((R * stride,), 0xCD, dtype=torch.uint8, device="cuda")
        st = lib.nw_align_device_noalloc(g.handle, ctypes.c_void_p(d_seq.data_ptr()),
                                         ctypes.c_void_p(d_off.data_ptr()), R, max_len,
                                         ctypes.c_void_p(d_hits.data_ptr()), ctypes.byref(nw),
                                         ctypes.c_void_p(out_aln.data_ptr()), ctypes.c_void_p(out_cig.data_ptr()),
                                         stride, None)
        assert st == 0, lib.mss_last_error()
        mss.mss_sync(g)
        a = out_aln.cpu().numpy().view(mss.ALN_DTYPE)
        b = ref_aln.cpu().numpy().view(mss.ALN_DTYPE)
        for f in ("score", "cigar_len", "gstart", "gend"):
            assert np.array_equal(a[f], b[f]), f"call {call}: field {f}"
        ca = out_cig.cpu().numpy().reshape(R, stride)
        cb = ref_cig.cpu().numpy().reshape(R, stride)
        for i in range(R):
            n = int(b["cigar_len"][i])
            assert n > 0 and bytes(ca[i, :n + 1]) == bytes(cb[i, :n + 1]), f"call {call}: CIGAR of read {i}"

    # sizes beyond what the context accepts are rejected with a message, nothing launched
    st = lib.nw_align_device_noalloc(g.handle, ctypes.c_void_p(d_seq.data_ptr()), ctypes.c_void_p(d_off.data_ptr()),
                                     R, max_len + 1, ctypes.c_void_p(d_hits.data_ptr()), ctypes.byref(nw),
                                     ctypes.c_void_p(ref_aln.data_ptr()), ctypes.c_void_p(ref_cig.data_ptr()), stride,
                                     None)
    assert st == mss.MSS_EREADLEN and lib.mss_last_error()
    g.close()

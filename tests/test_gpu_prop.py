"""GPU checks of the learned proposal against its oracle (oracle/prop_oracle.py) and against
the exact path:

* embeddings: BF16 tensor-core conv stack vs the fp64 oracle with the same rounding points
  (bounded in BF16 ulps: at most 1% of the coordinates off by more than one ulp);
* parameter gradients vs the oracle's backward pass (relative error of the whole vector and of
  every parameter block, 1e-2 / 1.5e-2);
* the mean-pooling option: embeddings, gradients and its checkpoint round trip;
* input codes (reads, both strands; genome windows) bit-exact;
* proposal + exact rescoring: with K = all fragments, and with every read falling back, the
  result equals the exhaustive scan bit for bit; with small K the rescored best/second equal
  the oracle's exact fragment scores over the candidates;
* top K consistent with the oracle's scores up to the embedding tolerance;
* a training step decreases the loss; checkpoints round-trip and reject corruption.
"""
import os
import tempfile

import numpy as np
import pytest

import gen
import oracle
from oracle import prop_oracle as po
from tests.parity_util import assert_hits_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mss():
    import torch
    assert torch.cuda.is_available()
    import paper_1403_2136_gb300 as m
    from paper_1403_2136_gb300 import build
    build.build()
    m.load_library()
    return m


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def random_params(seed, scale=1.0):
    w = po.unpack(np.zeros(po.param_count()))  # layout check
    rng = np.random.default_rng(seed)
    p = np.empty(po.param_count())
    o = 0
    n1 = po.TAPS * 4 * po.C
    p[o:o + n1] = rng.uniform(-1, 1, n1) * np.sqrt(6 / 28) * scale; o += n1
    p[o:o + po.C] = 0.01; o += po.C
    for _ in range(3):
        n = po.TAPS * po.C * po.C
        p[o:o + n] = rng.uniform(-1, 1, n) * np.sqrt(6 / (po.C * po.TAPS)) * scale; o += n
        p[o:o + po.C] = 0.01; o += po.C
    return p.astype(np.float32)


def test_embeddings_match_oracle(mss):
    import torch
    prop = mss.Proposal(seed=3)
    params = random_params(11)
    prop.set_params(params)
    rng = np.random.default_rng(12)
    lens = np.array([1, 7, 31, 100, 129, 250, 300, 64], dtype=np.int32)
    ld = 320
    codes = np.full((lens.size, ld), 4, np.uint8)
    for i, L in enumerate(lens):
        codes[i, :L] = rng.choice(5, size=L, p=[.24, .24, .24, .24, .04])
    d_emb = torch.zeros(lens.size * 128, dtype=torch.float32, device="cuda")
    prop.embed(dev(codes), dev(lens), ld, lens.size, int(lens.max()), d_emb)
    torch.cuda.synchronize()
    got = d_emb.cpu().numpy().reshape(-1, 128)
    for i, L in enumerate(lens):
        want, _ = po.forward(params.astype(np.float64), codes[i, :L])
        assert np.abs(got[i] - want).max() < 3e-3, (i, L, np.abs(got[i] - want).max())
        assert np.dot(got[i], want) > 0.99999
    prop.close()


def _bf16_ulp(x):
    """Spacing of BF16 numbers (8 significant bits) at |x|."""
    ax = np.maximum(np.abs(x), 1e-30)
    return np.exp2(np.floor(np.log2(ax)) - 7)


def test_embedding_coordinates_within_one_bf16_ulp(mss):
    """Tolerance from the rounding points: the oracle rounds the same values to BF16 at the
    same places as the kernels, so a coordinate can differ only where an FP32 sum of the
    tensor cores (accumulated in another order than the oracle's exact sum) falls on the
    other side of a BF16 rounding boundary; such a flip moves an activation by one BF16 ulp.
    Where such a flip moves the pooling's argmax the coordinate can move by more (measured on
    GB300: 0.35-0.49% of the coordinates above one ulp, 64-76% identical, at most 23 ulps,
    absolute differences at most 1.2e-3).  Bound: at most 1% of the coordinates off by more
    than one ulp, every coordinate within 2e-3, and the cosine to the oracle above 0.99999."""
    import torch
    prop = mss.Proposal(seed=6)
    params = random_params(41)
    prop.set_params(params)
    rng = np.random.default_rng(42)
    lens = rng.integers(20, 400, size=48).astype(np.int32)
    ld = 400
    codes = np.full((lens.size, ld), 4, np.uint8)
    for i, L in enumerate(lens):
        codes[i, :L] = rng.choice(5, size=L, p=[.24, .24, .24, .24, .04])
    d_emb = torch.zeros(lens.size * 128, dtype=torch.float32, device="cuda")
    prop.embed(dev(codes), dev(lens), ld, lens.size, int(lens.max()), d_emb)
    torch.cuda.synchronize()
    got = d_emb.cpu().numpy().reshape(-1, 128).astype(np.float64)
    want = np.stack([po.forward(params.astype(np.float64), codes[i, :L])[0] for i, L in enumerate(lens)])
    diff = np.abs(got - want)
    ulps = diff / _bf16_ulp(want)
    nz = np.abs(want) > 1e-6
    assert np.all(diff[~nz] < 1e-6), diff[~nz].max()
    over1 = float(np.mean(ulps[nz] > 1.0))
    stats = f"max {ulps[nz].max():.2f} ulp, {over1:.4%} of {nz.sum()} coordinates above 1 ulp, " \
            f"{float(np.mean(ulps[nz] <= 1e-3)):.2%} equal to 1e-3 ulp"
    assert over1 <= 0.01, stats
    assert diff.max() <= 2e-3, stats
    cos = np.sum(got * want, axis=1) / (np.linalg.norm(got, axis=1) * np.linalg.norm(want, axis=1))
    assert cos.min() > 0.99999, (cos.min(), stats)
    prop.close()


def test_gradients_match_oracle(mss):
    import torch
    prop = mss.Proposal(seed=4)
    params = random_params(21)
    prop.set_params(params)
    rng = np.random.default_rng(22)
    lens = np.array([40, 133, 77], dtype=np.int32)
    ld = 160
    codes = np.full((lens.size, ld), 4, np.uint8)
    for i, L in enumerate(lens):
        codes[i, :L] = rng.integers(0, 4, size=L)
    demb = rng.normal(size=(lens.size, 128)).astype(np.float32)
    d_grad = torch.zeros(po.param_count(), dtype=torch.float32, device="cuda")
    prop.grad(dev(codes), dev(lens), ld, lens.size, int(lens.max()), dev(demb), d_grad)
    torch.cuda.synchronize()
    got = d_grad.cpu().numpy().astype(np.float64)
    want = sum(po.backward(params.astype(np.float64), codes[i, :L], demb[i]) for i, L in enumerate(lens))
    # the same BF16 rounding points on both sides: only FP32 summation order differs (measured
    # on GB300: 2.3e-3 relative over the whole vector, at most 3.7e-3 per parameter block)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < 1e-2, rel
    # every block, not just the total
    o = 0
    for size in [po.TAPS * 4 * po.C, po.C] + [po.TAPS * po.C * po.C, po.C] * 3:
        g, w_ = got[o:o + size], want[o:o + size]
        if np.linalg.norm(w_) > 1e-6:
            assert np.linalg.norm(g - w_) / np.linalg.norm(w_) < 1.5e-2, (o, size)
        o += size
    prop.close()


def test_first_layer_keeps_fp32_weights(mss):
    """The first layer's weights are FP32 (the tensor-core kernel splits each into three
    exact BF16 parts).  Two one-path channels: channel 0 reads base A through tap 3 with
    weight 1 + 2^-9 + 2^-12 and bias 2^-9, whose exact sum 1 + 2^-8 + 2^-12 rounds to the BF16
    value 1 + 2^-7, while a BF16 weight (1) plus the bias would round to 1; channel 1 reads
    the same base with weight 1.  Layers 2-4 pass both channels on unchanged, so the
    embedding's ratio e0 / e1 is 1 + 2^-7 exactly, as in the oracle."""
    import torch
    C, T = po.C, po.TAPS
    p = np.zeros(po.param_count())
    p[(3 * 4 + 0) * C + 0] = 1 + 2 ** -9 + 2 ** -12
    p[(3 * 4 + 0) * C + 1] = 1.0
    p[T * 4 * C + 0] = 2 ** -9
    o = T * 4 * C + C
    for _ in range(3):
        p[o + (3 * C + 0) * C + 0] = 1.0
        p[o + (3 * C + 1) * C + 1] = 1.0
        o += T * C * C + C
    codes = np.array([[1, 2, 3, 1, 2, 0, 3, 3, 1, 2, 1, 3]], dtype=np.uint8)   # one A, at 5
    lens = np.array([12], dtype=np.int32)
    want, _ = po.forward(p, codes[0])
    assert want[0] / want[1] == 1 + 2 ** -7
    prop = mss.Proposal(seed=2)
    prop.set_params(p.astype(np.float32))
    d_emb = torch.zeros(128, dtype=torch.float32, device="cuda")
    prop.embed(dev(codes), dev(lens), 12, 1, 12, d_emb)
    torch.cuda.synchronize()
    got = d_emb.cpu().numpy().astype(np.float64)
    prop.close()
    assert np.abs(got - want).max() < 1e-6, (got[:3], want[:3])
    assert got[0] / got[1] == pytest.approx(1 + 2 ** -7, abs=1e-6)


def test_mean_pooling_matches_oracle(mss):
    """The mean-pooling option: embeddings (lengths 1 to 700, N bases, a sequence longer than
    a conv tile) against the oracle's mean pool with the same rounding points, the parameter
    gradient of a batch against the oracle's backward pass, the setting's checks, and its
    round trip through a checkpoint."""
    import torch
    prop = mss.Proposal(seed=7)
    assert prop.pooling == "max"
    with pytest.raises(ValueError):
        prop.pooling = "sum"
    assert mss.load_library().mss_prop_set_pooling(prop.handle, 2) == mss.MSS_EINVAL
    prop.pooling = "mean"
    assert prop.pooling == "mean"
    params = random_params(51)
    prop.set_params(params)
    rng = np.random.default_rng(52)
    lens = np.array([1, 2, 7, 31, 100, 129, 250, 700, 64, 333], dtype=np.int32)
    ld = 704
    codes = np.full((lens.size, ld), 4, np.uint8)
    for i, L in enumerate(lens):
        codes[i, :L] = rng.choice(5, size=L, p=[.24, .24, .24, .24, .04])
    d_emb = torch.zeros(lens.size * 128, dtype=torch.float32, device="cuda")
    prop.embed(dev(codes), dev(lens), ld, lens.size, int(lens.max()), d_emb)
    torch.cuda.synchronize()
    got = d_emb.cpu().numpy().reshape(-1, 128)
    p64 = params.astype(np.float64)
    for i, L in enumerate(lens):
        want, _ = po.forward(p64, codes[i, :L], pooling="mean")
        mx, _ = po.forward(p64, codes[i, :L])
        assert np.abs(got[i] - want).max() < 3e-3, (i, L, np.abs(got[i] - want).max())
        assert np.dot(got[i], want) > 0.99999
        if L > 1:
            assert np.abs(want - mx).max() > 1e-2     # the two poolings differ
    m = lens.size
    demb = rng.normal(size=(m, 128)).astype(np.float32)
    d_grad = torch.zeros(po.param_count(), dtype=torch.float32, device="cuda")
    prop.grad(dev(codes), dev(lens), ld, m, int(lens.max()), dev(demb), d_grad)
    torch.cuda.synchronize()
    g = d_grad.cpu().numpy().astype(np.float64)
    want = sum(po.backward(p64, codes[i, :L], demb[i], pooling="mean") for i, L in enumerate(lens))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-2
    o = 0
    for size in [po.TAPS * 4 * po.C, po.C] + [po.TAPS * po.C * po.C, po.C] * 3:
        gb, wb = g[o:o + size], want[o:o + size]
        if np.linalg.norm(wb) > 1e-6:
            assert np.linalg.norm(gb - wb) / np.linalg.norm(wb) < 1.5e-2, (o, size)
        o += size
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "mean.ckpt")
        prop.save(path)
        other = mss.Proposal(seed=8)
        assert other.pooling == "max"
        other.load(path)
        assert other.pooling == "mean"
        d_emb2 = torch.zeros_like(d_emb)
        other.embed(dev(codes), dev(lens), ld, lens.size, int(lens.max()), d_emb2)
        torch.cuda.synchronize()
        assert torch.equal(d_emb2, d_emb)
        # a file of the earlier format (magic "MSSPROP1", no pooling field) loads as max pooling
        import zlib
        hdr = np.array([po.param_count(), 5], dtype=np.int64).tobytes()
        body = np.concatenate([params, np.zeros(2 * po.param_count(), np.float32)]).tobytes()
        crc = (zlib.crc32(hdr + body) ^ 0xFFFFFFFF) & 0xFFFFFFFF
        v1 = os.path.join(td, "v1.ckpt")
        open(v1, "wb").write(b"MSSPROP1" + hdr + body + np.array([crc], np.uint32).tobytes())
        other.load(v1)
        assert other.pooling == "max" and np.array_equal(other.get_params(), params)
        other.close()
    prop.close()


def test_conv_many_items_per_cta(mss):
    """Batches with many more 128-position items than SMs: every persistent CTA of the conv
    kernels cycles its staging ring several times.  The embedding of a sequence does not depend
    on the batch it came in (bit for bit), sampled embeddings match the oracle, and the
    gradient of the whole batch matches the oracle's sum."""
    import torch
    prop = mss.Proposal(seed=5)
    params = random_params(31)
    prop.set_params(params)
    rng = np.random.default_rng(32)
    n = 300
    lens = rng.integers(1, 701, size=n).astype(np.int32)
    lens[:4] = [700, 1, 128, 129]
    ld = 704
    codes = np.full((n, ld), 4, np.uint8)
    for i, L in enumerate(lens):
        codes[i, :L] = rng.choice(5, size=L, p=[.24, .24, .24, .24, .04])
    d_emb = torch.zeros(n * 128, dtype=torch.float32, device="cuda")
    prop.embed(dev(codes), dev(lens), ld, n, int(lens.max()), d_emb)
    torch.cuda.synchronize()
    got = d_emb.cpu().numpy().reshape(n, 128)
    for lo in range(0, n, 7):
        hi = min(n, lo + 7)
        d_small = torch.zeros((hi - lo) * 128, dtype=torch.float32, device="cuda")
        prop.embed(dev(codes[lo:hi]), dev(lens[lo:hi]), ld, hi - lo, int(lens[lo:hi].max()), d_small)
        torch.cuda.synchronize()
        assert np.array_equal(d_small.cpu().numpy().reshape(-1, 128), got[lo:hi]), lo
    for i in [0, 1, 2, 3] + list(rng.choice(n, size=8, replace=False)):
        want, _ = po.forward(params.astype(np.float64), codes[i, :lens[i]])
        assert np.abs(got[i] - want).max() < 3e-3, (i, lens[i])
    m = 160
    demb = rng.normal(size=(m, 128)).astype(np.float32)
    d_grad = torch.zeros(po.param_count(), dtype=torch.float32, device="cuda")
    prop.grad(dev(codes[:m]), dev(lens[:m]), ld, m, int(lens[:m].max()), dev(demb), d_grad)
    torch.cuda.synchronize()
    g = d_grad.cpu().numpy().astype(np.float64)
    want = sum(po.backward(params.astype(np.float64), codes[i, :lens[i]], demb[i]) for i in range(m))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-2
    prop.close()


def test_codes(mss):
    import torch
    wl = gen.scaled(gen.workloads()["chrom-230M"], genome_len=30_000, reads=20)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=1024, max_read_len=250)
    prop = mss.Proposal(seed=1)
    n = reads.count
    ld = 256
    idx = np.arange(n, dtype=np.int32)
    for strand in (0, 1):
        st = np.full(n, strand, np.int8)
        d_codes = torch.zeros(n * ld, dtype=torch.uint8, device="cuda")
        d_lens = torch.zeros(n, dtype=torch.int32, device="cuda")
        prop.read_codes(dev(reads.seq), dev(reads.offsets), dev(idx), dev(st), n, ld, d_codes, d_lens)
        c = d_codes.cpu().numpy().reshape(n, ld)
        for i in range(n):
            q = oracle.encode(reads.read(i))
            if strand:
                q = oracle.revcomp_codes(q)
            assert np.array_equal(c[i, :q.size], q) and (c[i, q.size:] == 4).all()
    starts = np.array([0, 1000, 29_000, 29_990], dtype=np.int64)
    d_codes = torch.zeros(4 * 64, dtype=torch.uint8, device="cuda")
    d_lens = torch.zeros(4, dtype=torch.int32, device="cuda")
    prop.window_codes(g, dev(starts), 4, 50, 64, d_codes, d_lens)
    c = d_codes.cpu().numpy().reshape(4, 64)
    full = np.concatenate([oracle.encode(genome), np.full(200, 4, np.uint8)])
    for i, s in enumerate(starts):
        assert np.array_equal(c[i, :50], full[s:s + 50])
    prop.close()
    g.close()


def _proposal_setup(mss, K_frags=None, seed=5):
    import torch
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=40_000, reads=24)
    genome, reads = gen.materialize(wl)
    g = mss.mss_load_genome(genome, frag_len=1024, max_read_len=150)
    prop = mss.Proposal(seed=seed)
    prop.build_index(g, 150)
    return wl, genome, reads, g, prop


def test_proposed_with_all_fragments_equals_exhaustive(mss):
    import torch
    wl, genome, reads, g, prop = _proposal_setup(mss)
    NF = g.info()["num_frags"]
    R = reads.count
    d_out = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    nfb = prop.map_reads(g, dev(reads.seq), dev(reads.offsets), R, 150, 5, -4, NF, -1e30, d_out)
    assert nfb == 0
    got = mss.hits_from_bytes(d_out.cpu())
    want = mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4)
    assert_hits_equal(got, want, "K = NF")
    # the neighbour rule of the context applies to the rescored candidates as well
    mss.mss_set_second_rule(g, True)
    d_out.zero_()
    prop.map_reads(g, dev(reads.seq), dev(reads.offsets), R, 150, 5, -4, NF, -1e30, d_out)
    assert_hits_equal(mss.hits_from_bytes(d_out.cpu()), mss.mss_map_reads(g, reads.seq, reads.offsets, 5, -4),
                      "K = NF, neighbour rule")
    mss.mss_set_second_rule(g, False)
    # everything falls back: the exhaustive path
    d_out.zero_()
    nfb = prop.map_reads(g, dev(reads.seq), dev(reads.offsets), R, 150, 5, -4, 4, 1e30, d_out)
    assert nfb == R
    assert_hits_equal(mss.hits_from_bytes(d_out.cpu()), want, "all fallback")
    prop.close()
    g.close()


def test_proposed_small_k_rescoring_is_exact(mss):
    import torch
    wl, genome, reads, g, prop = _proposal_setup(mss)
    R, K, F = reads.count, 6, 1024
    d_out = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.zeros(R * K, dtype=torch.int32, device="cuda")
    prop.map_reads(g, dev(reads.seq), dev(reads.offsets), R, 150, 5, -4, K, -1e30, d_out, d_cand=d_cand)
    hits = mss.hits_from_bytes(d_out.cpu())
    cand = d_cand.cpu().numpy().reshape(R, K)
    for i in range(R):
        _, fs = oracle.map_read(genome, F, reads.read(i), 5, -4, with_frag_scores=True)
        cs = [(int(fs[f]), int(f)) for f in cand[i] if f >= 0]
        assert len(set(f for _, f in cs)) == len(cs)
        order = sorted(cs, key=lambda x: (-x[0], x[1]))
        assert hits["best_frag"][i] == order[0][1] and hits["best_score"][i] == order[0][0]
        if len(order) > 1:
            assert hits["second_frag"][i] == order[1][1] and hits["second_score"][i] == order[1][0]
    prop.close()
    g.close()


@pytest.mark.parametrize("F,match,mismatch", [(3000, 5, -4), (3000, 13, -4), (700, 1, -1)])
def test_rescoring_exact_multi_pass_fragments(mss, F, match, mismatch):
    """Candidate rescoring where a fragment takes several 2048-diagonal passes with a ragged
    last one (F = 3000, not a multiple of 16), where one pass covers less than a fragment
    (F = 700), with the int16 lanes (13 / -4 has no exact f16 byte form) and the f16 lanes,
    and with reads holding N and reads of one and two bases."""
    import torch
    from tests.parity_util import concat_reads
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=30_000, reads=10)
    genome, reads = gen.materialize(wl)
    strs = [bytes(reads.read(i)) for i in range(reads.count)]
    g_ascii = bytes(genome)
    strs += [g_ascii[5000:5120].replace(b"A", b"N", 7), b"G", b"TA", g_ascii[29_900:30_000]]
    seq, off = concat_reads(strs)
    R, K = len(strs), 5
    g = mss.mss_load_genome(genome, frag_len=F, max_read_len=150)
    prop = mss.Proposal(seed=9)
    prop.build_index(g, 150)
    d_out = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.zeros(R * K, dtype=torch.int32, device="cuda")
    prop.map_reads(g, dev(seq), dev(off), R, 150, match, mismatch, K, -1e30, d_out, d_cand=d_cand)
    hits = mss.hits_from_bytes(d_out.cpu())
    cand = d_cand.cpu().numpy().reshape(R, K)
    for i in range(R):
        q = np.frombuffer(strs[i], dtype=np.uint8)
        want, fs = oracle.map_read(genome, F, q, match, mismatch, with_frag_scores=True)
        cs = sorted([(int(fs[f]), int(f)) for f in cand[i] if f >= 0], key=lambda x: (-x[0], x[1]))
        assert hits["best_frag"][i] == cs[0][1] and hits["best_score"][i] == cs[0][0], (i, cs, hits[i])
        assert hits["second_frag"][i] == cs[1][1] and hits["second_score"][i] == cs[1][0], (i, cs, hits[i])
        # when the candidates hold the exhaustive best fragment, the best diagonal and strand are
        # the exhaustive scan's (the argmax rule inside one fragment)
        if want[0] == cs[0][1]:
            assert hits["offset"][i] == want[4] and hits["strand"][i] == want[5], i
    prop.close()
    g.close()


@pytest.mark.parametrize("R,K,genome_len", [(100, 64, 150_000), (70, 128, 150_000), (9_800, 64, 66_000),
                                             (33, 5, 20_000)])
def test_tensor_core_topk_matches_numpy(mss, R, K, genome_len):
    """The fused tensor-core scores + streaming top K against numpy on the same BF16
    embeddings (the GPU's own fp32 embeddings rounded to BF16): every returned fragment is
    among the K best (within FP32 accumulation error), the list is in score order, and ties
    between identical embeddings (two fragments with identical windows) go to the lower
    fragment.  Equal fp64 scores of different embeddings are not ties on the GPU: the FP32
    accumulation may separate them by an ulp.  Sizes: several
    fragment splits with the merge (100 reads), K = 128 (70 reads), one split per read block
    (9,800 reads = 154 blocks of 64), a ragged last tile of 128 fragments, NF below 128."""
    import torch
    F, ML = 512, 100
    wl = gen.scaled(gen.workloads()["chrom-230M"], genome_len=genome_len, reads=R)
    genome = gen.make_genome(wl.genome, wl.seed).copy()
    win = F + ML - 1
    f1, f2 = 3, 17                      # twin fragments: identical windows
    genome[f2 * F:f2 * F + win] = genome[f1 * F:f1 * F + win]
    reads = gen.make_reads(genome, gen.ReadSpec(R, lengths=(36, 51, 76, 100), sub_levels=((0.1, 0.2),)), wl.seed + 3)
    g = mss.mss_load_genome(genome, frag_len=F, max_read_len=ML)
    NF = g.info()["num_frags"]
    prop = mss.Proposal(seed=2)
    prop.build_index(g, ML)
    d_out = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.zeros(R * K, dtype=torch.int32, device="cuda")
    prop.map_reads(g, dev(reads.seq), dev(reads.offsets), R, ML, 5, -4, K, -1e30, d_out, d_cand=d_cand)
    cand = d_cand.cpu().numpy().reshape(R, K)
    # the same embeddings, computed by the library's own forward pass
    d_codes = torch.zeros(NF * win, dtype=torch.uint8, device="cuda")
    d_lens = torch.zeros(NF, dtype=torch.int32, device="cuda")
    prop.window_codes(g, dev(np.arange(NF, dtype=np.int64) * F), NF, win, win, d_codes, d_lens)
    d_ef = torch.zeros(NF * 128, dtype=torch.float32, device="cuda")
    prop.embed(d_codes, d_lens, win, NF, win, d_ef)
    n = 2 * R
    idx = np.repeat(np.arange(R, dtype=np.int32), 2)
    st = np.tile(np.array([0, 1], np.int8), R)
    d_rc = torch.zeros(n * ML, dtype=torch.uint8, device="cuda")
    d_rl = torch.zeros(n, dtype=torch.int32, device="cuda")
    prop.read_codes(dev(reads.seq), dev(reads.offsets), dev(idx), dev(st), n, ML, d_rc, d_rl)
    d_er = torch.zeros(n * 128, dtype=torch.float32, device="cuda")
    prop.embed(d_rc, d_rl, ML, n, ML, d_er)
    torch.cuda.synchronize()
    ef = po.bf16_round(d_ef.cpu().numpy().reshape(NF, 128))
    er = po.bf16_round(d_er.cpu().numpy().reshape(R, 2, 128))
    assert np.array_equal(ef[f1], ef[f2])
    sc = np.maximum(er[:, 0, :] @ ef.T, er[:, 1, :] @ ef.T)      # [R][NF], fp64
    Kc = min(K, NF)
    tol = 1e-5
    for i in range(R):
        got = cand[i]
        assert (got[Kc:] == -1).all()
        got = got[:Kc]
        assert len(set(got.tolist())) == Kc and (got >= 0).all() and (got < NF).all(), i
        kth = np.sort(sc[i])[::-1][Kc - 1]
        gs = sc[i][got]
        assert (gs >= kth - tol).all(), (i, gs.min(), kth)
        assert (np.diff(gs) <= tol).all(), i                       # score order
        for a in range(Kc - 1):  # identical embeddings score identically: lower fragment first
            if np.array_equal(ef[got[a]], ef[got[a + 1]]):
                assert got[a] < got[a + 1], (i, a)
        if f2 in got:
            assert f1 in got and list(got).index(f1) < list(got).index(f2), i
    prop.close()
    g.close()


def test_topk_consistent_with_oracle_scores(mss):
    import torch
    wl, genome, reads, g, prop = _proposal_setup(mss)
    params = prop.get_params().astype(np.float64)
    R, K, F = reads.count, 5, 1024
    NF = g.info()["num_frags"]
    d_out = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.zeros(R * K, dtype=torch.int32, device="cuda")
    prop.map_reads(g, dev(reads.seq), dev(reads.offsets), R, 150, 5, -4, K, -1e30, d_out, d_cand=d_cand)
    cand = d_cand.cpu().numpy().reshape(R, K)
    gcodes = np.concatenate([oracle.encode(genome), np.full(F + 200, 4, np.uint8)])
    ef = np.stack([po.forward(params, gcodes[f * F:f * F + F + 149])[0] for f in range(NF)])
    for i in range(0, R, 4):
        q = oracle.encode(reads.read(i))
        e1, _ = po.forward(params, q)
        e2, _ = po.forward(params, oracle.revcomp_codes(q))
        sc = np.maximum(ef @ e1, ef @ e2)
        kth = np.sort(sc)[::-1][K - 1]
        for f in cand[i]:
            assert sc[f] >= kth - 0.05, (i, f, sc[f], kth)
    prop.close()
    g.close()


def test_training_step_and_checkpoint(mss):
    import torch
    prop = mss.Proposal(seed=9)
    rng = np.random.default_rng(31)
    B, C, Lr, Lc = 16, 16, 80, 300
    rc = rng.integers(0, 4, size=(B, Lr)).astype(np.uint8)
    cc = rng.integers(0, 4, size=(C, Lc)).astype(np.uint8)
    for i in range(B):                      # read i is a substring of candidate i
        s = rng.integers(0, Lc - Lr)
        cc[i, s:s + Lr] = rc[i]
    rl = np.full(B, Lr, np.int32)
    cl = np.full(C, Lc, np.int32)
    lab = np.arange(B, dtype=np.int32)
    d = [dev(x) for x in (rc, rl, cc, cl, lab)]
    # the first step's loss equals the oracle's loss on the oracle's embeddings
    params = prop.get_params().astype(np.float64)
    er = np.stack([po.forward(params, rc[i])[0] for i in range(B)])
    ec = np.stack([po.forward(params, cc[j])[0] for j in range(C)])
    want_loss, _, _ = po.ce_loss(er, ec, lab, 0.1)
    losses = [prop.train_step(d[0], d[1], Lr, B, Lr, d[2], d[3], Lc, C, Lc, d[4], lr=3e-3, temperature=0.1)
              for _ in range(25)]
    assert abs(losses[0] - want_loss) < 5e-2 * max(1.0, abs(want_loss)), (losses[0], want_loss)
    # the fixed batch is learned (Adam at this rate then oscillates around the minimum)
    assert min(losses) < losses[0] * 0.5, losses
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "prop.ckpt")
        prop.save(path)
        before = prop.get_params()
        other = mss.Proposal(seed=123)
        other.load(path)
        assert np.array_equal(other.get_params(), before)
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0xFF
        open(path, "wb").write(bytes(raw))
        with pytest.raises(mss.MssError):
            other.load(path)
        other.close()
    prop.close()


def test_trainer_end_to_end_small(mss, capsys):
    """The training/evaluation driver runs end to end on small genomes: labels on one genome,
    training with hard negatives mined from the model's own top K, evaluation on held-out
    reads of another genome with the threshold chosen on one half and reported on the other;
    a threshold above every cosine sends every read to the exhaustive scan (exact)."""
    import json
    from paper_1403_2136_gb300 import proposal
    proposal.main(["--train-genome", "chrom-230M@300000", "--train-reads", "3000", "--steps", "30", "--batch", "64",
                   "--mine-every", "10", "--hard", "2", "--evals", "chrom-230M@400000:400", "--taus=-1e30,1e30"])
    out = capsys.readouterr().out.strip().splitlines()[-1]
    line = json.loads(out)
    # learning itself is pinned by the fixed-batch step test; here the trainer's end-to-end plumbing
    assert np.isfinite(line["loss_first"]) and np.isfinite(line["loss_last"])
    ev = line["evals"][0]
    assert ev["tau_chosen_on_validation"] == 1e30           # only the full fallback reaches 99.5%
    r_all, r_fallback = ev["test"]
    assert r_fallback["fallback_reads"] == ev["eval_reads"]
    assert r_fallback["top1_agreement"] == 1.0 and r_fallback["changed_mappings"] == 0
    assert 0.0 <= r_all["top1_agreement"] <= 1.0

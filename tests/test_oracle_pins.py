"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: brute-force enumeration
of every substring / every alignment on tiny inputs, closed forms printed in the paper,
invariants of the maximum scoring subsequence, and the paper's Figure 2 toy genome.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = "ACGTN"
COMP = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}


def revcomp(s: str) -> str:
    return "".join(COMP[c] for c in reversed(s))


def sub_score(a: str, b: str, match: int, mismatch: int) -> int:
    return match if (a == b and a != "N") else mismatch


# ---------------------------------------------------------------- maximum scoring subsequence
def brute_mss(x):
    """max over all contiguous runs x[i:j] (empty run allowed) — "Maximum scoring subsequence"."""
    best = 0
    for i in range(len(x) + 1):
        for j in range(i, len(x) + 1):
            best = max(best, sum(x[i:j]))
    return best


def test_mss_bruteforce():
    rng = np.random.default_rng(1)
    for _ in range(400):
        n = int(rng.integers(0, 14))
        x = rng.integers(-6, 7, size=n).tolist()
        assert oracle.mss(x) == brute_mss(x)


def test_mss_special_cases():
    assert oracle.mss([]) == 0                      # empty sequence: empty run
    assert oracle.mss([-3, -1, -7]) == 0            # all negative: empty run wins
    assert oracle.mss([2, 3, 4]) == 9               # all positive: whole sequence
    assert oracle.mss([5, -10, 4, 4]) == 8          # a dip resets the run
    assert oracle.mss([5, -1, 4]) == 8              # a small dip is bridged


# ---------------------------------------------------------------- one diagonal, tiny inputs
def brute_diag(read: str, gpad: str, d: int, match: int, mismatch: int, step: int = 1) -> int:
    """step 2: only read positions 0, 2, 4, ... take part ("MaxSSmap_fast")."""
    x = [sub_score(read[k], gpad[d + k], match, mismatch) for k in range(0, len(read), step)]
    return brute_mss(x)


@pytest.mark.parametrize("match,mismatch", [(1, -1), (5, -4), (3, 0), (2, -7)])
def test_diag_score_bruteforce(match, mismatch):
    rng = np.random.default_rng(2 + match)
    for _ in range(60):
        G = int(rng.integers(1, 40))
        m = int(rng.integers(1, 12))
        genome = "".join(rng.choice(list(ALPHA), p=[.22, .22, .22, .22, .12], size=G))
        read = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=m))
        gpad = genome + "N" * m
        q = oracle.encode(read)
        g = oracle.encode(gpad)
        for d in range(G):
            assert oracle.diag_score(q, g, d, match, mismatch) == brute_diag(read, gpad, d, match, mismatch)


# ---------------------------------------------------------------- whole phase one, tiny inputs
def brute_map(genome: str, F: int, read: str, match: int, mismatch: int, step: int = 1):
    """Phase one by enumeration: every strand, every diagonal of every fragment, every
    substring; fragment maximum with its first (strand, d); top two by sorting."""
    G = len(genome)
    NF = -(-G // F)
    Gp = NF * F
    m = len(read)
    gpad = genome + "N" * (Gp - G + m)
    reads = [read, revcomp(read)]
    frag = []
    for f in range(NF):
        cands = []
        for sg in range(2):
            for d in range(f * F, (f + 1) * F):
                cands.append((brute_diag(reads[sg], gpad, d, match, mismatch, step), sg, d))
        best = max(c[0] for c in cands)
        first = min((sg, d) for (s, sg, d) in cands if s == best)
        frag.append((best, first[0], first[1]))
    order = sorted(range(NF), key=lambda f: (-frag[f][0], f))
    b1 = order[0]
    b2 = order[1] if NF > 1 else -1
    s1 = frag[b1][0]
    s2 = frag[b2][0] if b2 >= 0 else 0
    repeat = 1 if (s1 == 0 or s2 / s1 >= 0.9) else 0
    return (b1, b2, s1, s2, frag[b1][2], frag[b1][1], repeat), [f[0] for f in frag]


@pytest.mark.parametrize("F", [1, 3, 5, 8, 16])
def test_map_read_bruteforce(F):
    rng = np.random.default_rng(10 + F)
    for trial in range(25):
        G = int(rng.integers(1, 48))
        m = int(rng.integers(1, 10))
        genome = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=G))
        if trial % 3 == 0 and G >= m:   # plant a (possibly reversed) copy so that ties and repeats occur
            s = int(rng.integers(0, G - m + 1))
            read = genome[s:s + m]
            if trial % 2:
                read = revcomp(read)
        else:
            read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        match, mismatch = [(1, -1), (5, -4), (2, -3)][trial % 3]
        want, wfs = brute_map(genome, F, read, match, mismatch)
        got, fs = oracle.map_read(genome, F, read, match, mismatch, with_frag_scores=True)
        assert got == want, (genome, F, read)
        assert fs.tolist() == wfs


# ---------------------------------------------------------------- MaxSSmap_fast (read step 2)
@pytest.mark.parametrize("match,mismatch", [(1, -1), (5, -4), (2, -7)])
def test_fast_diag_score_bruteforce(match, mismatch):
    """Every other read base: brute force over all runs of the sampled score sequence."""
    rng = np.random.default_rng(40 + match)
    for _ in range(60):
        G = int(rng.integers(1, 40))
        m = int(rng.integers(1, 13))
        genome = "".join(rng.choice(list(ALPHA), p=[.22, .22, .22, .22, .12], size=G))
        read = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=m))
        gpad = genome + "N" * m
        q, g = oracle.encode(read), oracle.encode(gpad)
        for d in range(G):
            assert oracle.diag_score(q, g, d, match, mismatch, step=2) == brute_diag(read, gpad, d, match, mismatch, 2)


def test_fast_equals_plain_scan_of_subsampled_sequences():
    """Sampling identity: diagonal d with step 2 is the plain diagonal d // 2 of the read's even
    positions against the genome positions of d's parity."""
    rng = np.random.default_rng(44)
    for _ in range(40):
        G = int(rng.integers(2, 60))
        m = int(rng.integers(1, 15))
        genome = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=G))
        read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        gpad = genome + "N" * (m + 2)
        q, g = oracle.encode(read), oracle.encode(gpad)
        qs = oracle.encode(read[::2])
        for d in range(G):
            gs = oracle.encode(gpad[d % 2::2])
            assert oracle.diag_score(q, g, d, 5, -4, step=2) == oracle.diag_score(qs, gs, d // 2, 5, -4)


@pytest.mark.parametrize("F", [1, 4, 7, 16])
def test_fast_map_read_bruteforce(F):
    rng = np.random.default_rng(50 + F)
    for trial in range(20):
        G = int(rng.integers(1, 48))
        m = int(rng.integers(1, 11))
        genome = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=G))
        if trial % 3 == 0 and G >= m:
            s0 = int(rng.integers(0, G - m + 1))
            read = genome[s0:s0 + m]
            if trial % 2:
                read = revcomp(read)
        else:
            read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        match, mismatch = [(1, -1), (5, -4), (2, -3)][trial % 3]
        want, wfs = brute_map(genome, F, read, match, mismatch, step=2)
        got, fs = oracle.map_read(genome, F, read, match, mismatch, with_frag_scores=True, step=2)
        assert got == want, (genome, F, read)
        assert fs.tolist() == wfs


def test_fast_exact_substring_scores_half_length():
    """An exact copy scores ceil(m / 2) * match at its diagonal with step 2."""
    rng = np.random.default_rng(46)
    genome = "".join(rng.choice(list("ACGT"), size=3000))
    for m in (1, 2, 7, 50, 101):
        s0 = 1234
        read = genome[s0:s0 + m]
        hit = oracle.map_read(genome, 500, read, 5, -4, step=2)
        assert hit[2] == 5 * ((m + 1) // 2)
        if m >= 50:  # long enough to be unique: found at its own diagonal, + strand
            assert hit[4] == s0 and hit[5] == 0


# ---------------------------------------------------------------- invariants
def test_exact_substring_scores_m_match():
    rng = np.random.default_rng(3)
    genome = "".join(rng.choice(list("ACGT"), size=3000))
    for m, d in [(50, 17), (100, 1234), (31, 2969)]:
        read = genome[d:d + m]
        hit = oracle.map_read(genome, 256, read, 5, -4)
        assert hit[2] == m * 5
        assert hit[4] == d and hit[5] == 0
        assert hit[0] == d // 256
        rc = oracle.map_read(genome, 256, revcomp(read), 5, -4)
        assert rc[2] == m * 5 and rc[4] == d and rc[5] == 1


def test_all_mismatch_diagonal_scores_zero():
    q = oracle.encode("A" * 20)
    g = oracle.encode("C" * 40)
    assert oracle.diag_score(q, g, 3, 5, -4) == 0
    hit = oracle.map_read("CG" * 45, 16, "A" * 12, 5, -4)   # reverse strand is T*12: no match either
    assert hit[2] == 0 and hit[3] == 0 and hit[6] == 1   # best == 0 -> unmapped


def test_fragment_score_is_max_over_its_diagonals():
    rng = np.random.default_rng(4)
    genome = "".join(rng.choice(list("ACGT"), size=500))
    read = "".join(rng.choice(list("ACGT"), size=40))
    F = 64
    hit, fs = oracle.map_read(genome, F, read, 1, -1, with_frag_scores=True)
    gpad = oracle.encode(genome + "N" * (len(fs) * F - len(genome) + 40))
    q = [oracle.encode(read), oracle.encode(revcomp(read))]
    for f in range(len(fs)):
        best = max(oracle.diag_score(q[s], gpad, d, 1, -1) for s in range(2) for d in range(f * F, (f + 1) * F))
        assert fs[f] == best
    assert hit[2] == max(fs)


def test_reverse_complement_symmetry():
    rng = np.random.default_rng(5)
    genome = "".join(rng.choice(list("ACGT"), size=2000))
    for d in (0, 333, 1900):
        read = list(genome[d:d + 60])
        for p in rng.choice(60, size=6, replace=False):   # a few substitutions keep it unique
            read[p] = {"A": "C", "C": "G", "G": "T", "T": "A"}[read[p]]
        read = "".join(read)
        a = oracle.map_read(genome, 100, read, 5, -4)
        b = oracle.map_read(genome, 100, revcomp(read), 5, -4)
        assert a[:5] == b[:5] and a[5] == 1 - b[5]


def test_junction_alignment_is_not_lost():
    """A read planted across a fragment border scores m*match in the fragment holding its
    start diagonal (windows run into the right neighbour: "First phase", Figure 1)."""
    rng = np.random.default_rng(6)
    genome = "".join(rng.choice(list("ACGT"), size=4000))
    F = 1000
    d = 2 * F - 30
    read = genome[d:d + 100]
    hit = oracle.map_read(genome, F, read, 1, -1)
    assert hit[0] == 1 and hit[2] == 100 and hit[4] == d


def test_planted_repeat_ties_go_to_lowest_fragment():
    rng = np.random.default_rng(7)
    genome = list(rng.choice(list("ACGT"), size=5000))
    src = 3100
    genome[700:900] = genome[src:src + 200]      # exact copy, earlier fragment
    genome = "".join(genome)
    read = genome[src + 20:src + 120]
    hit = oracle.map_read(genome, 512, read, 5, -4)
    assert hit[2] == hit[3] == 500
    assert hit[0] == 720 // 512 and hit[1] == (src + 20) // 512
    assert hit[6] == 1   # repeat


def test_single_fragment_has_no_second():
    hit = oracle.map_read("ACGTACGTAC", 64, "GTAC", 1, -1)
    assert hit[0] == 0 and hit[1] == -1 and hit[3] == 0


def test_ratio_flag_integer_form():
    """Mapped iff second/best < 0.9 ("First phase of MaxSSmap"); the oracle uses the exact
    integer form 10*second >= 9*best."""
    rng = np.random.default_rng(8)
    genome = "".join(rng.choice(list("ACGT"), size=1200))
    for t in range(40):
        read = "".join(rng.choice(list("ACGT"), size=int(rng.integers(8, 30))))
        h = oracle.map_read(genome, 100, read, 1, -1)
        b, s = h[2], h[3]
        assert h[6] == (1 if (b == 0 or s / b >= 0.9) else 0)


def test_lowercase_bases_are_bases():
    """Either case codes the same base (the genome and the reads may be soft-masked)."""
    assert list(oracle.encode("acgtn")) == list(oracle.encode("ACGTN")) == [0, 1, 2, 3, 4]
    rng = np.random.default_rng(22)
    genome = "".join(rng.choice(list("ACGT"), size=600))
    read = genome[210:250]
    up = oracle.map_read(genome, 100, read, 5, -4)
    assert up[2] == 200
    assert oracle.map_read(genome.lower(), 100, read.lower(), 5, -4) == up
    assert oracle.map_read(genome, 100, read[:20].lower() + read[20:], 5, -4) == up


def test_ratio_flag_boundary_is_inclusive():
    """second / best exactly 0.9 is not "below .9": the read is a repeat.  An exact 10-base
    copy (5 * 10 = 50) and a copy with its last base changed (the run of 9 scores 45)."""
    rng = np.random.default_rng(21)
    gen = list("".join(rng.choice(list("ACGT"), size=2000)))
    read = "ACGTTGCAAC"
    gen[150:160] = list(read)
    gen[1250:1260] = list(read[:9] + "A")
    h = oracle.map_read("".join(gen), 100, read, 5, -4)
    assert h[:4] == (1, 12, 50, 45) and h[6] == 1
    gen[1250:1260] = list(read[:8] + "GA")          # a run of 8: 40 / 50 = 0.8, mapped
    h = oracle.map_read("".join(gen), 100, read, 5, -4)
    assert h[2] == 50 and h[3] < 45 and h[6] == 0


# ---------------------------------------------------------------- Figure 2 toy genome
def _golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            d[k] = v
    return d


def test_figure2_toy_fragments():
    g = _golden("fig2_toy.txt")
    genome = g["genome"][0]
    F = int(g["frag_len"][0])
    frags = g["fragments"]
    assert -(-len(genome) // F) == len(frags)
    for f, s in enumerate(frags):
        hit, fs = oracle.map_read(genome, F, s, 1, -1, with_frag_scores=True)
        assert fs[f] == F          # the fragment's own bases score F*match in fragment f
        assert hit[2] == F
    # the transposed layout's first row is the first base of every fragment
    assert "".join(genome[f * F] for f in range(len(frags))) == g["transposed_row0"][0]
    # a read that starts in fragment 0 and runs into fragment 1 (junction) maps to fragment 0
    hit = oracle.map_read(genome, F, genome[1:5], 1, -1)
    assert hit[0] == 0 and hit[4] == 1 and hit[2] == 4


# ---------------------------------------------------------------- closed forms printed in the paper
def test_paper_closed_forms():
    # MAPQ threshold: -100 log2 0.9 = 15.2 ("Mapping qualities")
    assert round(-100 * math.log2(0.9), 1) == 15.2
    # strict threshold 62 <-> ratio 2^-0.62 ~ 0.651 (ancient DNA section)
    assert round(2 ** -0.62, 3) == 0.651
    # maximum read length: profile (m+16)*4*5 bytes in 49152 bytes of shared memory -> 2441,
    # largest multiple of 16 below it is 2432 ("Shared memory")
    cap = 49152 / (4 * 5) - 16
    assert int(cap) == 2441 and (int(cap) // 16) * 16 == 2432
    # OpenMP thread counts "about 1042, 104 and 11" for fragment lengths 4800, 48000, 480000 on
    # a ~5 Mbp genome: G/F rounded (the third, 10.4, is printed rounded up)
    assert round(5e6 / 4800) == 1042 and round(5e6 / 48000) == 104 and math.ceil(5e6 / 480000) == 11


# ---------------------------------------------------------------- phase two
def alignment_score(read, window, ops, match, mismatch, go, ge, pos=None):
    """pos = (ma, mm): position-specific match / mismatch scores of the read bases."""
    i = j = 0
    score = 0
    prev = None
    for op in ops:
        if op == "M":
            score += sub_score(read[i], window[j], *((pos[0][i], pos[1][i]) if pos else (match, mismatch)))
            i += 1
            j += 1
        elif op == "I":
            score += ge if prev == "I" else go
            i += 1
        else:
            score += ge if prev == "D" else go
            j += 1
        prev = op
    return score, i, j


def brute_glocal(read, window, match, mismatch, go, ge, pos=None):
    """Best glocal alignment by enumeration: every genome start, every op string."""
    m, L = len(read), len(window)
    best = None
    for js in range(L + 1):
        sub = window[js:]
        # enumerate op strings with exactly m read-consuming ops and up to len(sub) genome ops
        def rec(i, j, prev, score):
            nonlocal best
            if i == m:
                if best is None or score > best:
                    best = score
                # trailing genome bases are free: stop here
            if i < m and j < len(sub):
                sm, sx = (pos[0][i], pos[1][i]) if pos else (match, mismatch)
                rec(i + 1, j + 1, "M", score + sub_score(read[i], sub[j], sm, sx))
            if i < m:
                rec(i + 1, j, "I", score + (ge if prev == "I" else go))
            if j < len(sub) and i < m:   # a deletion must be followed by more read (trailing ones are free)
                rec(i, j + 1, "D", score + (ge if prev == "D" else go))
        rec(0, 0, None, 0)
    return best


def parse_cigar(c):
    ops, n = [], ""
    for ch in c:
        if ch.isdigit():
            n += ch
        else:
            ops += [ch] * int(n)
            n = ""
    return ops


def test_nw_bruteforce_tiny():
    rng = np.random.default_rng(9)
    for t in range(150):
        m = int(rng.integers(1, 6))
        L = int(rng.integers(0, 7))
        window = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=L))
        read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        match, mismatch, go, ge = [(5, -4, -26, -26), (5, -4, -10, -1), (2, -3, -4, -2), (1, -1, -2, -1)][t % 4]
        want = brute_glocal(read, window, match, mismatch, go, ge)
        got = oracle.nw_banded(oracle.encode(window) if L else np.zeros(0, np.uint8), oracle.encode(read), 0, 64,
                               match, mismatch, go, ge) if L else None
        if L == 0:
            continue   # empty window: the oracle reports no alignment (no genome to anchor the read)
        score, gs, ge_, cig = got
        assert score == want, (read, window, match, mismatch, go, ge)
        ops = parse_cigar(cig)
        s2, i, j = alignment_score(read, window[gs:], ops, match, mismatch, go, ge)
        assert s2 == score and i == m and gs + j == ge_


def test_nw_hand_worked():
    with open(os.path.join(GOLDEN, "nw_hand.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for r in rows:
        genome, read, d, W, ma, mm, go, ge, _, sc, cig, gs, gend = r
        got = oracle.nw_banded(oracle.encode(genome), oracle.encode(read), int(d), int(W), int(ma), int(mm),
                               int(go), int(ge))
        assert got == (int(sc), int(gs), int(gend), cig), r


def test_nw_banded_equals_unbanded_when_optimum_in_band():
    rng = np.random.default_rng(11)
    genome = "".join(rng.choice(list("ACGT"), size=3000))
    g = oracle.encode(genome)
    for t in range(20):
        d = int(rng.integers(100, 2700))
        read = list(genome[d:d + 120])
        for p in rng.choice(120, size=12, replace=False):
            read[p] = "ACGT"[(("ACGT".index(read[p])) + 1) % 4]
        cut = int(rng.integers(20, 100))
        k = int(rng.integers(1, 8))
        read = read[:cut] + read[cut + k:] if t % 2 else read[:cut] + list("ACGT"[:k % 4 + 1]) + read[cut:]
        q = oracle.encode("".join(read))
        a = oracle.nw_banded(g, q, d, 32, 5, -4, -10, -1)
        b = oracle.nw_banded(g, q, d, 400, 5, -4, -10, -1)
        assert a == b


def test_nw_band_edges_are_inclusive():
    """The band is |t| <= W for t = column - row - seed offset: a deletion of exactly W bases
    (t = +W after it) or an insertion of W bases (t = -W) still aligns inside band W, with
    the unbanded result; band W - 1 cannot reach it."""
    rng = np.random.default_rng(21)
    genome = "".join(rng.choice(list("ACGT"), size=400))
    g = oracle.encode(genome)
    W = 4
    for read, op in ((genome[100:140] + genome[140 + W:180 + W], "4D"), (genome[100:140] + "TTGA" + genome[140:180], "4I")):
        q = oracle.encode(read)
        inside = oracle.nw_banded(g, q, 100, W, 5, -4, -10, -1)
        assert inside == oracle.nw_banded(g, q, 100, 400, 5, -4, -10, -1)
        assert inside[0] == 80 * 5 - 10 - 3 and inside[3] == "40M" + op + "40M"
        assert oracle.nw_banded(g, q, 100, W - 1, 5, -4, -10, -1)[0] < inside[0]


def test_nw_literal_region():
    """Literal reading: region starts at the best fragment and spans ceil(m/F) fragments."""
    rng = np.random.default_rng(12)
    genome = "".join(rng.choice(list("ACGT"), size=600))
    F = 64
    read = genome[130:170]   # inside fragment 2 (128..191)
    sc, gs, ge, cig = oracle.nw_literal(oracle.encode(genome), F, 2, oracle.encode(read), 5, -4, -26, -26)
    assert (sc, gs, ge, cig) == (200, 130, 170, "40M")


# ---------------------------------------------------------------- base qualities (PSSM)
def pssm_py(qchar: int, match: int, mismatch: int, scale: int):
    """The paper's scores written out again in Python: x = 1 - 10^(-Q/10), match * x and
    mismatch * x / 3, times scale, rounded half away from zero."""
    x = 1.0 - 10.0 ** (-(qchar - 33) / 10.0)

    def rnd(v):
        return int(math.floor(v + 0.5)) if v >= 0 else -int(math.floor(-v + 0.5))
    return rnd(scale * match * x), rnd(scale * mismatch * x / 3.0)


def test_pssm_scores_closed_forms():
    # Q 40: x = 0.9999; Q 20: 0.99; Q 10: 0.9; Q 3: 0.4988; Q 0: 0 (scale 4, 5 / -4)
    assert oracle.pssm_scores(ord("I"), 5, -4, 4) == (20, -5)
    assert oracle.pssm_scores(ord("5"), 5, -4, 4) == (20, -5)      # 19.8, -5.28
    assert oracle.pssm_scores(ord("+"), 5, -4, 4) == (18, -5)      # 18.0, -4.8
    assert oracle.pssm_scores(ord("$"), 5, -4, 4) == (10, -3)      # 9.976, -2.66
    assert oracle.pssm_scores(ord("!"), 5, -4, 4) == (0, 0)
    assert oracle.pssm_scores(ord("?"), 3, -3, 1) == (3, -1)       # Q 30: 2.997, -0.999
    for q in range(33, 127):
        for (ma, mm, sc) in [(5, -4, 4), (1, -1, 8), (2, -3, 1)]:
            assert oracle.pssm_scores(q, ma, mm, sc) == pssm_py(q, ma, mm, sc)
    with pytest.raises(ValueError):
        oracle.pssm_scores(32, 5, -4, 4)


def brute_map_pssm(genome: str, F: int, read: str, quals: str, match: int, mismatch: int, scale: int):
    """Phase one with position-specific scores, by enumeration of every run on every diagonal."""
    G = len(genome)
    NF = -(-G // F)
    Gp = NF * F
    m = len(read)
    gpad = genome + "N" * (Gp - G + m)
    sc = [pssm_py(ord(c), match, mismatch, scale) for c in quals]
    strands = [(read, sc), (revcomp(read), sc[::-1])]
    frag = []
    for f in range(NF):
        cands = []
        for sg in range(2):
            r, p = strands[sg]
            for d in range(f * F, (f + 1) * F):
                x = [sub_score(r[k], gpad[d + k], p[k][0], p[k][1]) for k in range(m)]
                cands.append((brute_mss(x), sg, d))
        best = max(c[0] for c in cands)
        first = min((sg, d) for (v, sg, d) in cands if v == best)
        frag.append((best, first[0], first[1]))
    order = sorted(range(NF), key=lambda f: (-frag[f][0], f))
    b1 = order[0]
    b2 = order[1] if NF > 1 else -1
    s1 = frag[b1][0]
    s2 = frag[b2][0] if b2 >= 0 else 0
    repeat = 1 if (s1 == 0 or 10 * s2 >= 9 * s1) else 0
    return (b1, b2, s1, s2, frag[b1][2], frag[b1][1], repeat)


@pytest.mark.parametrize("F", [1, 4, 9])
def test_pssm_map_read_bruteforce(F):
    rng = np.random.default_rng(60 + F)
    for trial in range(20):
        G = int(rng.integers(1, 40))
        m = int(rng.integers(1, 9))
        genome = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=G))
        if trial % 3 == 0 and G >= m:
            s0 = int(rng.integers(0, G - m + 1))
            read = genome[s0:s0 + m]
            if trial % 2:
                read = revcomp(read)
        else:
            read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        quals = "".join(chr(33 + int(v)) for v in rng.integers(0, 42, size=m))
        match, mismatch, scale = [(5, -4, 4), (1, -1, 8), (2, -3, 2)][trial % 3]
        want = brute_map_pssm(genome, F, read, quals, match, mismatch, scale)
        got = oracle.map_read(genome, F, read, match, mismatch, quals=quals.encode(), scale=scale)
        assert got == want, (genome, F, read, quals)


def test_pssm_constant_quality_is_the_plain_scan_with_rounded_scores():
    """With every base at one quality the position-specific scores are constants, so the result
    is the plain scan's with those two scores."""
    rng = np.random.default_rng(66)
    genome = "".join(rng.choice(list("ACGTN"), p=[.24, .24, .24, .24, .04], size=3000))
    for qc in ("I", "+", "$"):
        ma, mm = pssm_py(ord(qc), 5, -4, 4)
        for _ in range(6):
            m = int(rng.integers(5, 60))
            s0 = int(rng.integers(0, 3000 - m))
            read = list(genome[s0:s0 + m].replace("N", "A"))
            for k in rng.integers(0, m, size=m // 6):
                read[k] = "ACGT"[(("ACGT".index(read[k])) + 1) % 4]
            read = "".join(read)
            got = oracle.map_read(genome, 256, read, 5, -4, quals=(qc * m).encode(), scale=4)
            want = oracle.map_read(genome, 256, read, ma, mm)
            assert got == want


def test_pssm_nw_bruteforce_tiny():
    rng = np.random.default_rng(67)
    for t in range(120):
        m = int(rng.integers(1, 6))
        L = int(rng.integers(1, 7))
        window = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=L))
        read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        quals = "".join(chr(33 + int(v)) for v in rng.integers(0, 42, size=m))
        sc = [pssm_py(ord(c), 5, -4, 4) for c in quals]
        ma, mm = [a for a, _ in sc], [b for _, b in sc]
        go, ge = [(-40, -4), (-104, -104), (-8, -4)][t % 3]
        want = brute_glocal(read, window, 0, 0, go, ge, pos=(ma, mm))
        score, gs, ge_, cig = oracle.nw_banded_pssm(oracle.encode(window), oracle.encode(read), ma, mm, 0, 64, go, ge)
        assert score == want, (read, window, quals)
        s2, i, j = alignment_score(read, window[gs:], parse_cigar(cig), 0, 0, go, ge, pos=(ma, mm))
        assert s2 == score and i == m and gs + j == ge_


# ---------------------------------------------------------------- second excluding the best's neighbours
def test_neighbour_exclusion_bruteforce():
    """The second is the best fragment f with |f - best| > 1 (ties to the lowest), checked on
    the brute-force fragment scores; with the neighbours allowed it is the plain second."""
    rng = np.random.default_rng(70)
    for trial in range(60):
        G = int(rng.integers(1, 60))
        F = int(rng.integers(1, 9))
        m = int(rng.integers(1, 9))
        genome = "".join(rng.choice(list(ALPHA), p=[.23, .23, .23, .23, .08], size=G))
        if trial % 2 == 0 and G >= m:
            s0 = int(rng.integers(0, G - m + 1))
            read = genome[s0:s0 + m]
        else:
            read = "".join(rng.choice(list(ALPHA), p=[.24, .24, .24, .24, .04], size=m))
        plain, fs = brute_map(genome, F, read, 2, -3)
        got = oracle.map_read(genome, F, read, 2, -3, exclude_neighbors=True)
        b1 = plain[0]
        others = [f for f in range(len(fs)) if abs(f - b1) > 1]
        if others:
            b2 = min(others, key=lambda f: (-fs[f], f))
            s2 = fs[b2]
        else:
            b2, s2 = -1, 0
        s1 = fs[b1]
        rep = 1 if (s1 == 0 or 10 * s2 >= 9 * s1) else 0
        assert got == (b1, b2, s1, s2, plain[4], plain[5], rep), (genome, F, read)


def test_pssm_batch_gap_costs_are_scaled():
    """Phase two with base qualities is in units of 1/scale, so its gap costs are scaled too
    ("Incorporating base qualities": match * x and mismatch * x / 3, here times scale 4).
    Hand-worked case: a 20-base read made of genome[60:70] + genome[72:82] (two genome bases
    deleted), every base at quality 'I' (Q 40, x = 0.9999): a match scores round(4 * 5 * x) = 20,
    and the best glocal alignment is 20 matches with one 2-base gap in the read:
    20 * 20 + 4 * (-10) + 4 * (-1) = 356.  With unscaled gaps it would be 389."""
    rng = np.random.default_rng(1403)
    genome = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 200)].copy()
    read = np.concatenate([genome[60:70], genome[72:82]])
    off = np.array([0, 20], dtype=np.int64)
    quals = np.full(20, ord("I"), dtype=np.uint8)
    assert oracle.pssm_scores(ord("I"), 5, -4, 4) == (20, -5)
    hits, alns, cig = oracle.map_batch(genome, 200, read, off, 5, -4, nw=(5, -4, -10, -1, 32), quals=quals, scale=4)
    assert int(hits["best_score"][0]) >= 10 * 20          # one half of the read lies on one diagonal
    assert int(alns["score"][0]) == 20 * 20 + 4 * (-10) + 4 * (-1) == 356
    assert cig[0] == "10M2D10M", cig[0]
    assert int(alns["gstart"][0]) == 60 and int(alns["gend"][0]) == 82

"""Pins of the proposal-network oracle (no GPU): the backward pass against finite
differences of the forward pass, the loss gradient against finite differences, and the
defining properties of the forward pass (unit norm, padding invariance, N = zero input)."""
import numpy as np

from oracle import prop_oracle as po


def small_params(seed=0, scale=0.2):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, size=po.param_count())


def test_embedding_is_unit_norm_and_nonnegative():
    w = small_params(1)
    codes = np.random.default_rng(2).integers(0, 5, size=40)
    e, _ = po.forward(w, codes)
    assert abs(np.linalg.norm(e) - 1.0) < 1e-5 or np.linalg.norm(e) < 1e-3
    assert (e >= 0).all()


def test_all_n_sequence_uses_only_biases():
    w = small_params(3)
    e_n, (acts, *_rest) = po.forward(w, np.full(30, 4))
    assert np.allclose(acts[0], 0)   # N is the zero one-hot


def test_backward_matches_finite_differences():
    w = small_params(4, scale=0.3)
    codes = np.random.default_rng(5).integers(0, 4, size=18)
    demb = np.random.default_rng(6).normal(size=po.C)
    g = po.backward(w, codes, demb, rounding=False)

    def f(wv):
        e, _ = po.forward(wv, codes, rounding=False)
        return float(np.dot(e, demb))

    rng = np.random.default_rng(7)
    # a few coordinates of every parameter block
    blocks = [(0, 7 * 4 * 128), (7 * 4 * 128, 7 * 4 * 128 + 128)]
    o = 7 * 4 * 128 + 128
    for _ in range(3):
        blocks += [(o, o + 7 * 128 * 128), (o + 7 * 128 * 128, o + 7 * 128 * 128 + 128)]
        o += 7 * 128 * 128 + 128
    for lo, hi in blocks:
        nz = [i for i in rng.integers(lo, hi, size=400) if abs(g[i]) > 1e-4][:4]
        for i in nz:
            h = 1e-5
            wp, wm = w.copy(), w.copy()
            wp[i] += h
            wm[i] -= h
            fd = (f(wp) - f(wm)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-4 + 1e-3 * abs(fd), (lo, i, fd, g[i])


def test_ce_loss_gradient():
    rng = np.random.default_rng(8)
    r = rng.normal(size=(5, 8))
    c = rng.normal(size=(7, 8))
    lab = rng.integers(0, 7, size=5)
    loss, dr, dc = po.ce_loss(r, c, lab, 0.5)
    h = 1e-6
    for i, j in [(0, 0), (3, 5), (4, 7)]:
        rp = r.copy(); rp[i, j] += h
        rm = r.copy(); rm[i, j] -= h
        fd = (po.ce_loss(rp, c, lab, 0.5)[0] - po.ce_loss(rm, c, lab, 0.5)[0]) / (2 * h)
        assert abs(fd - dr[i, j]) < 1e-6
    for i, j in [(0, 1), (6, 2)]:
        cp = c.copy(); cp[i, j] += h
        cm = c.copy(); cm[i, j] -= h
        fd = (po.ce_loss(r, cp, lab, 0.5)[0] - po.ce_loss(r, cm, lab, 0.5)[0]) / (2 * h)
        assert abs(fd - dc[i, j]) < 1e-6


def test_bf16_rounding_ties_to_even():
    assert po.bf16_round(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    assert po.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert po.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6

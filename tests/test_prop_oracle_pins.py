"""Pins of the proposal-network oracle (no GPU): the backward pass against finite
differences of the forward pass, the loss gradient against finite differences, and the
defining properties of the forward pass (unit norm, padding invariance, N = zero input)."""
import importlib.util
import os

import numpy as np
import pytest

if os.environ.get("MSS_PROP_ORACLE"):   # a variant with a planted mistake (tests/test_oracle_mutants.py)
    _spec = importlib.util.spec_from_file_location("prop_oracle_variant", os.environ["MSS_PROP_ORACLE"])
    po = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(po)
else:
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


@pytest.mark.parametrize("pooling", ["max", "mean"])
def test_backward_matches_finite_differences(pooling):
    w = small_params(4, scale=0.3)
    codes = np.random.default_rng(5).integers(0, 4, size=18)
    demb = np.random.default_rng(6).normal(size=po.C)
    g = po.backward(w, codes, demb, rounding=False, pooling=pooling)

    def f(wv):
        e, _ = po.forward(wv, codes, rounding=False, pooling=pooling)
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


def _one_path_params(w1v, wv, taps):
    """Every weight zero except one path: channel 0 of layer 1 reads base A through tap
    taps[0], and layer l (2..4) passes channel 0 on through tap taps[l - 1]; biases zero."""
    p = np.zeros(po.param_count())
    p[(taps[0] * 4 + 0) * po.C + 0] = w1v
    o = po.TAPS * 4 * po.C + po.C
    for l in range(3):
        p[o + (taps[l + 1] * po.C + 0) * po.C + 0] = wv[l]
        o += po.TAPS * po.C * po.C + po.C
    return p


def test_forward_fixed_by_hand():
    """The forward pass on a one-path network, worked out by hand: tap t at position p reads
    position p + t - 3 (zero outside the sequence), the max pool keeps the first maximum,
    the embedding is v / (|v| + 1e-6), and the stored values follow the rounding points
    (layer outputs rounded to BF16; layers 2-4 use BF16 weights, layer 1 FP32 ones)."""
    codes = np.array([1, 2, 0, 3, 1, 0, 2, 2, 1, 3, 3, 1, 0, 2])   # A at 2, 5 and 12; L = 14
    p = _one_path_params(1 + 2 ** -9, (1 + 2 ** -7, 1 + 2 ** -9, 1 + 2 ** -7), taps=(0, 0, 3, 3))
    e, (_, _, arg, v, nrm) = po.forward(p, codes)
    # two taps 0: position p sees base p - 6.  The A at 2 and 5 fire at 8 and 11 with equal
    # values (the first is kept); the A at 12 would fire at 18, outside the sequence.
    assert arg[0] == 8
    # bf16(1 + 2^-9) = 1 (layer 1 output); x (1 + 2^-7) exact; weight 1 + 2^-9 -> 1;
    # x (1 + 2^-7): 1 + 2^-6 + 2^-14 -> 1 + 2^-6
    assert v[0] == 1 + 2 ** -6 and np.all(v[1:] == 0)
    assert nrm == v[0] + 1e-6 and e[0] == v[0] / (v[0] + 1e-6) and np.all(e[1:] == 0)
    _, (_, _, arg_x, v_x, _) = po.forward(p, codes, rounding=False)
    assert arg_x[0] == 8 and abs(v_x[0] - (1 + 2 ** -9) ** 2 * (1 + 2 ** -7) ** 2) < 1e-12
    # values that cross rounding boundaries (BF16 steps of 2^-7 in [1, 2)), w = 1 + 2^-8 + 2^-9:
    # layer 1 (FP32 weight w): bf16(w) = 1 + 2^-7; layer 2 (x 1.75): 1.763671875 -> 1.765625;
    # layer 3 (BF16 weight bf16(w) = 1 + 2^-7): 1.779418... -> 1.78125; layer 4 x 1.
    # Skipping the layer-1 rounding would give 1.7578125 after layer 2, an FP32 layer-3
    # weight 1.7734375 after layer 3.
    w = 1 + 2 ** -8 + 2 ** -9
    p = _one_path_params(w, (1.75, w, 1.0), taps=(0, 0, 3, 3))
    _, (_, _, arg, v, _) = po.forward(p, codes)
    assert arg[0] == 8 and v[0] == 1.78125
    # two taps 6: position p sees base p + 6; only the A at 12 lands inside (at 6)
    p = _one_path_params(1.0, (1.0, 1.0, 1.0), taps=(6, 6, 3, 3))
    e, (_, _, arg, v, _) = po.forward(p, codes)
    assert arg[0] == 6 and v[0] == 1.0
    # N is no base: with the A at 12 replaced by N nothing fires and the embedding is zero
    codes_n = codes.copy()
    codes_n[12] = 4
    e, (_, _, _, v, nrm) = po.forward(p, codes_n)
    assert np.all(v == 0) and nrm == 1e-6 and np.all(e == 0)
    # T (code 3) is a base like the others: a T-reading path fires on the T at 3
    q = np.zeros(po.param_count())
    q[(3 * 4 + 3) * po.C + 0] = 1.0                       # layer 1, tap 3 (the position itself), base T
    o = po.TAPS * 4 * po.C + po.C
    for _ in range(3):
        q[o + (3 * po.C + 0) * po.C + 0] = 1.0
        o += po.TAPS * po.C * po.C + po.C
    _, (_, _, arg, v, _) = po.forward(q, codes)
    assert arg[0] == 3 and v[0] == 1.0


def test_mean_pool_fixed_by_hand():
    """Mean pooling on one-path networks: the pooled channel is the sum of the layer-4
    outputs over the sequence's positions divided by its length, the other channels are
    zero, and the embedding is the unit vector along channel 0."""
    codes = np.array([1, 2, 0, 3, 1, 0, 2, 2, 1, 3, 3, 1, 0, 2])   # A at 2, 5 and 12; L = 14
    # two taps 0: the A at 2 and 5 fire (value 1) at 8 and 11; the A at 12 falls outside
    p = _one_path_params(1.0, (1.0, 1.0, 1.0), taps=(0, 0, 3, 3))
    e, (_, _, _, v, nrm) = po.forward(p, codes, pooling="mean")
    assert v[0] == 2 / 14 and np.all(v[1:] == 0)
    assert nrm == v[0] + 1e-6 and e[0] == v[0] / (v[0] + 1e-6)
    # the max pool of the same network keeps one of the two: 1
    _, (_, _, _, vmax, _) = po.forward(p, codes)
    assert vmax[0] == 1.0
    # layer-2 weight 1.75: both firing positions carry 1.75, mean 3.5 / 14 = 0.25
    p = _one_path_params(1.0, (1.75, 1.0, 1.0), taps=(0, 0, 3, 3))
    _, (_, _, _, v, _) = po.forward(p, codes, pooling="mean")
    assert v[0] == 0.25
    # the layer-4 bias of channel 0 reaches the pooled value through the positions where
    # layer 4's output is positive (8 and 11), each with weight 1 / L: its gradient is 2 / 14
    # times the gradient at the pooled value (the normalisation's, pinned by finite
    # differences above), and the bias of a channel that never fires gets none
    demb = np.zeros(po.C)
    demb[0] = 1.0
    e, (_, _, _, v, nrm) = po.forward(p, codes, pooling="mean", rounding=False)
    g = po.backward(p, codes, demb, pooling="mean", rounding=False)
    o = po.TAPS * 4 * po.C + po.C + 2 * (po.TAPS * po.C * po.C + po.C) + po.TAPS * po.C * po.C
    dv0 = (1.0 - e[0] * e[0]) / nrm
    assert abs(g[o] - 2 / 14 * dv0) <= 1e-15, (g[o], 2 / 14 * dv0)
    assert np.all(g[o + 1:o + po.C] == 0)
    # the max pool routes the same gradient to one position only
    gmax = po.backward(p, codes, demb, rounding=False)
    _, (_, _, _, vm, nm) = po.forward(p, codes, rounding=False)
    em0 = vm[0] / nm
    assert abs(gmax[o] - (1.0 - em0 * em0) / nm) <= 1e-15

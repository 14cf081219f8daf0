"""CPU oracle of the learned fragment proposal — TEST INFRASTRUCTURE ONLY.

Plain numpy (fp64) statement of the proposal network and its training loss; loaded only by
tests.  The network: one-hot bases (N = all zero) -> 4 x [conv1d, kernel 7, "same" zero
padding, 128 channels, bias, ReLU] -> pool over positions -> L2 normalisation (+1e-6).
The pool is the maximum (first maximum kept) or, with pooling="mean", the mean over the
sequence's positions (the other reading of how a window's features become one vector).
Rounding points follow the documented precision of the path: layers 2..4 use BF16 weights,
the activations between layers are stored in BF16 (round to nearest even), accumulation is
exact here (fp64).  With rounding=False everything is fp64 (used by the finite-difference
pin of the backward pass).

Parameter layout (flat, as in the library): W1 [7][4][128], b1 [128], then for layers 2..4
W [7][128 in][128 out], b [128].
"""
from __future__ import annotations

import numpy as np

C = 128
TAPS = 7


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params: np.ndarray):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    w1 = p[o:o + TAPS * 4 * C].reshape(TAPS, 4, C); o += TAPS * 4 * C
    b1 = p[o:o + C]; o += C
    ws, bs = [], []
    for _ in range(3):
        ws.append(p[o:o + TAPS * C * C].reshape(TAPS, C, C)); o += TAPS * C * C
        bs.append(p[o:o + C]); o += C
    assert o == p.shape[0]
    return w1, b1, ws, bs


def param_count() -> int:
    return TAPS * 4 * C + C + 3 * (TAPS * C * C + C)


def _shift(a: np.ndarray, t: int) -> np.ndarray:
    """rows p -> a[p + t - 3] with zeros outside [0, L)"""
    L = a.shape[0]
    out = np.zeros_like(a)
    s = t - 3
    lo, hi = max(0, -s), min(L, L - s)
    if hi > lo:
        out[lo:hi] = a[lo + s:hi + s]
    return out


def forward(params, codes: np.ndarray, rounding: bool = True, pooling: str = "max"):
    """Embedding of one code sequence (values 0..3 bases, 4 = N).  Returns (emb, cache)."""
    assert pooling in ("max", "mean")
    w1, b1, ws, bs = unpack(params)
    x = np.asarray(codes, dtype=np.int64)
    L = x.shape[0]
    onehot = np.zeros((L, 4))
    ok = x < 4
    onehot[np.nonzero(ok)[0], x[ok]] = 1.0
    rnd = bf16_round if rounding else (lambda v: v)
    acts = [onehot]
    z = b1[None, :] + sum(_shift(onehot, t) @ w1[t] for t in range(TAPS))
    a = rnd(np.maximum(z, 0.0))
    acts.append(a)
    pres = [z]
    for l in range(3):
        W = rnd(ws[l]) if rounding else ws[l]
        z = bs[l][None, :] + sum(_shift(a, t) @ W[t] for t in range(TAPS))
        a = rnd(np.maximum(z, 0.0))
        acts.append(a)
        pres.append(z)
    if L > 0 and pooling == "mean":
        arg = np.zeros(C, dtype=np.int64)
        v = a.sum(axis=0) / L
    elif L > 0:
        arg = np.argmax(a, axis=0)          # first maximum
        v = a[arg, np.arange(C)]
    else:
        arg = np.zeros(C, dtype=np.int64)
        v = np.zeros(C)
    nrm = np.sqrt(np.sum(v * v)) + 1e-6
    e = v / nrm
    return e, (acts, pres, arg, v, nrm)


def backward(params, codes: np.ndarray, demb: np.ndarray, rounding: bool = True, pooling: str = "max") -> np.ndarray:
    """Gradient of <demb, emb(codes)> with respect to the flat parameters (fp64)."""
    w1, b1, ws, bs = unpack(params)
    e, (acts, pres, arg, v, nrm) = forward(params, codes, rounding, pooling)
    de = np.asarray(demb, dtype=np.float64)
    dv = (de - e * np.dot(e, de)) / nrm
    L = acts[0].shape[0]
    g = np.zeros_like(acts[4])
    if L > 0 and pooling == "mean":
        g[:, :] = dv[None, :] / L           # every position carries 1/L of the pooled value
    elif L > 0:
        g[arg, np.arange(C)] = dv
    grads_w, grads_b = [None] * 3, [None] * 3
    for l in range(2, -1, -1):     # layers 4, 3, 2
        gz = g * (acts[l + 2] > 0) if l == 2 else g * (acts[l + 2] > 0)
        a_in = acts[l + 1]
        W = bf16_round(ws[l]) if rounding else ws[l]
        grads_w[l] = np.stack([_shift(a_in, t).T @ gz for t in range(TAPS)])
        grads_b[l] = gz.sum(axis=0)
        # d a_in[p] = sum_t W[t] applied to gz[p - (t - 3)]
        g = np.zeros_like(a_in)
        for t in range(TAPS):
            s = t - 3
            contrib = gz @ W[t].T              # row p of gz contributes to a_in row p + s
            lo, hi = max(0, -s), min(L, L - s)
            if hi > lo:
                g[lo + s:hi + s] += contrib[lo:hi]
    gz1 = g * (acts[1] > 0)
    gw1 = np.stack([_shift(acts[0], t).T @ gz1 for t in range(TAPS)])
    gb1 = gz1.sum(axis=0)
    out = [gw1.ravel(), gb1]
    for l in range(3):
        out += [grads_w[l].ravel(), grads_b[l]]
    return np.concatenate(out)


def ce_loss(r: np.ndarray, c: np.ndarray, labels: np.ndarray, temperature: float):
    """Mean softmax cross-entropy of logits <r_i, c_j> / T against labels, and its gradients."""
    logits = r @ c.T / temperature
    m = logits.max(axis=1, keepdims=True)
    p = np.exp(logits - m)
    p /= p.sum(axis=1, keepdims=True)
    B = r.shape[0]
    loss = -np.log(p[np.arange(B), labels]).mean()
    d = p.copy()
    d[np.arange(B), labels] -= 1.0
    d /= B
    return loss, d @ c / temperature, d.T @ r / temperature

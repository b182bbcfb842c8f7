"""CPU FP64 oracle of the warm-start network (test infrastructure only).

The same encoder-decoder as the library's CUDA implementation, written with
plain numpy in float64: 3x3 convolutions (stride 1, zero padding 1) as sums
over the nine taps, ReLU, 2x2 average pooling, nearest 2x up-sampling, skip
additions, and the mean squared error; the backward pass by the chain rule,
layer by layer.  Parameter blob layout (shared reading with the library): per
layer the weights [cout][3][3][cin] then the bias [cout].

With bf16=True the oracle also rounds, to the nearest BF16 value (ties to
even), everything the library stores in BF16: the network input, the
weights, every stored activation (convolution outputs after bias and ReLU,
pooled, up-sampled and skip-added tensors; the linear head stays full
precision) and, backwards, the output gradient of the loss and every stored
activation gradient (data gradients of the convolutions, pooling and
up-sampling gradients, skip accumulations).  Sums themselves stay in
float64, so the two modes differ only by those roundings; parameter
gradients are never rounded.  This lets the tests compare the library's
layers element by element.

Pins (tests/test_oracle_cnn.py): the convolution against its definition
written as explicit loops on tiny inputs, every gradient against central
finite differences, and the BF16 rounding against the bit patterns of its
definition.  The network is resolution-generic here (any input side
divisible by 8) so that the pins run on small inputs.  stem = s (1 or 2)
gives the library's higher-resolution input variant: the first convolution
runs on the input of side 2^s x the rest's and its output is 2x2
average-pooled s times before the second convolution.
"""
from __future__ import annotations

import numpy as np

# (cin, cout, relu) of the 14 convolutions, in order
LAYERS = [(1, 32, 1), (32, 32, 1), (32, 64, 1), (64, 64, 1), (64, 128, 1), (128, 128, 1), (128, 256, 1),
          (256, 128, 1), (128, 128, 1), (128, 64, 1), (64, 64, 1), (64, 32, 1), (32, 32, 1), (32, 2, 0)]


def bf16_round(a):
    """Round to the nearest BF16 value, ties to even (BF16 keeps the upper 16
    bits of an IEEE float32): first to float32, then the low 16 bits of the
    float32 pattern are rounded away.  Finite inputs only."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def n_params():
    return sum(co * 9 * ci + co for ci, co, _ in LAYERS)


def unpack(blob):
    """[(W [cout, 9, cin], b [cout])] from the flat parameter blob."""
    out, off = [], 0
    for ci, co, _ in LAYERS:
        w = np.asarray(blob[off:off + co * 9 * ci], dtype=np.float64).reshape(co, 9, ci)
        off += co * 9 * ci
        b = np.asarray(blob[off:off + co], dtype=np.float64)
        off += co
        out.append((w, b))
    return out


def pack(grads):
    return np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])


def conv3x3(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{dy,dx,c} x[n, i+dy-1, j+dx-1, c] w[o, 3 dy + dx, c]."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((N, H, W, w.shape[0])) + b
    for t in range(9):
        dy, dx = divmod(t, 3)
        y += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + H, dx:dx + W], w[:, t])
    return y


def conv3x3_backward(x, w, gy):
    """Gradients (gx, gw, gb) of conv3x3 for the output gradient gy."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for t in range(9):
        dy, dx = divmod(t, 3)
        gw[:, t] = np.einsum("nhwo,nhwc->oc", gy, xp[:, dy:dy + H, dx:dx + W])
        gxp[:, dy:dy + H, dx:dx + W] += np.einsum("nhwo,oc->nhwc", gy, w[:, t])
    return gxp[:, 1:-1, 1:-1], gw, gy.sum(axis=(0, 1, 2))


def pool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(gy):
    N, H, W, C = gy.shape
    return gy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(params, x, bf16=False, stem=0):
    """x [N, H, W] pooled log densities -> (prediction [N, H / 2^stem, W / 2^stem, 2],
    saved tensors).  bf16: round what the library stores in BF16 (see the
    module docstring); stem: pools after the first convolution."""
    r = bf16_round if bf16 else (lambda a: a)
    P = unpack(params)
    if bf16:
        P = [(r(w), b) for w, b in P]
    s = {"x0": r(np.asarray(x, dtype=np.float64)[..., None])}

    def L(k, inp):
        y = conv3x3(inp, *P[k])
        if LAYERS[k][2]:
            return r(np.maximum(y, 0.0))
        return y                                  # the linear head: full precision

    s["a0f"] = L(0, s["x0"])                      # the first convolution at the input resolution
    a0 = s["a0f"]
    for _ in range(stem):
        a0 = r(pool2(a0))
    s["a0"] = a0
    s["e1"] = L(1, s["a0"]); s["p1"] = r(pool2(s["e1"]))
    s["a2"] = L(2, s["p1"]); s["e2"] = L(3, s["a2"]); s["p2"] = r(pool2(s["e2"]))
    s["a4"] = L(4, s["p2"]); s["e3"] = L(5, s["a4"]); s["p3"] = r(pool2(s["e3"]))
    s["bt"] = L(6, s["p3"]); s["u3"] = up2(s["bt"])
    s["z7"] = L(7, s["u3"]); s["d3"] = r(s["z7"] + s["e3"]); s["d3b"] = L(8, s["d3"]); s["u2"] = up2(s["d3b"])
    s["z9"] = L(9, s["u2"]); s["d2"] = r(s["z9"] + s["e2"]); s["d2b"] = L(10, s["d2"]); s["u1"] = up2(s["d2b"])
    s["z11"] = L(11, s["u1"]); s["d1"] = r(s["z11"] + s["e1"]); s["d1b"] = L(12, s["d1"])
    s["out"] = L(13, s["d1b"])
    return s["out"], s


def loss_and_grads(params, x, target, bf16=False, saved=None, stem=0):
    """Mean squared error over all outputs and its gradient blob.  bf16: the
    forward and backward roundings of the library (module docstring).
    saved: a dict that receives every stored activation gradient by name."""
    r = bf16_round if bf16 else (lambda a: a)
    P = unpack(params)
    if bf16:
        P = [(r(w), b) for w, b in P]
    out, s = forward(params, x, bf16=bf16, stem=stem)
    n = out.size
    loss = float(((out - target) ** 2).sum() / n)
    g = [None] * len(LAYERS)

    def back(k, gy, inp, act):
        if LAYERS[k][2]:
            gy = gy * (act > 0)
        gx, gw, gb = conv3x3_backward(inp, P[k][0], gy)
        g[k] = (gw, gb)
        return r(gx)

    gout = r(2.0 * (out - target) / n)
    gd1b = back(13, gout, s["d1b"], s["out"])
    gd1 = back(12, gd1b, s["d1"], s["d1b"])
    gu1 = back(11, gd1, s["u1"], s["z11"])
    gd2b = r(up2_backward(gu1))
    gd2 = back(10, gd2b, s["d2"], s["d2b"])
    gu2 = back(9, gd2, s["u2"], s["z9"])
    gd3b = r(up2_backward(gu2))
    gd3 = back(8, gd3b, s["d3"], s["d3b"])
    gu3 = back(7, gd3, s["u3"], s["z7"])
    gbt = r(up2_backward(gu3))
    gp3 = back(6, gbt, s["p3"], s["bt"])
    ge3 = r(r(pool2_backward(gp3)) + gd3)
    ga4 = back(5, ge3, s["a4"], s["e3"])
    gp2 = back(4, ga4, s["p2"], s["a4"])
    ge2 = r(r(pool2_backward(gp2)) + gd2)
    ga2 = back(3, ge2, s["a2"], s["e2"])
    gp1 = back(2, ga2, s["p1"], s["a2"])
    ge1 = r(r(pool2_backward(gp1)) + gd1)
    ga0 = back(1, ge1, s["a0"], s["e1"])
    for _ in range(stem):                          # back through the stem's pools
        ga0 = r(pool2_backward(ga0))
    back(0, ga0, s["x0"], s["a0f"])
    if saved is not None:
        saved.update(gout=gout, gd1b=gd1b, gd1=gd1, gu1=gu1, gd2b=gd2b, gd2=gd2, gu2=gu2, gd3b=gd3b, gd3=gd3,
                     gu3=gu3, gbt=gbt, gp3=gp3, ge3=ge3, ga4=ga4, gp2=gp2, ge2=ge2, ga2=ga2, gp1=gp1, ge1=ge1,
                     ga0=ga0)
    return loss, pack(g)


def he_init(seed):
    """A seeded parameter blob (He normal for ReLU layers, small linear head)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, relu in LAYERS:
        sd = np.sqrt(2.0 / (9 * ci)) if relu else 0.1 * np.sqrt(1.0 / (9 * ci))
        parts.append(rng.normal(0.0, sd, co * 9 * ci))
        parts.append(rng.normal(0.0, 0.05, co))
    return np.concatenate(parts)

"""GPU parity of the learned warm start (no counterpart in the paper).

The network's forward pass and its parameter gradients on the BF16 tensor
cores against the FP64 oracle network with the same parameters; the pooled
log-density input against the oracle's density texture; training lowers the
loss; a warm-started solve with an untrained (zero) field equals a cold one.

Tolerances follow from BF16 rounding: unit roundoff u = 2^-9 on the network
input, every weight and every stored activation (and, backwards, every stored
activation gradient).  14 convolutions plus 3 skip additions give about 40
independent roundings on the forward path, whose relative effects add like a
random walk: sqrt(40) * u = 1.2e-2 expected relative L2 error of the output;
the bound used is 3e-2 (2.5 sigma).  The backward path doubles the count and
adds ReLU mask flips where a pre-activation is within rounding of 0: 6e-2
per layer gradient, cosine similarity >= 0.998 over the whole blob.
Accumulation is FP32 throughout (its error, ~1e-6 relative, is negligible).
Those norm checks against the FP64 oracle stand beside element-wise checks
against the oracle's BF16 mode (below).
"""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from oracle import inim_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _P():
    import paper_2604_13880_gb300 as P
    return P


def _fields(B, seed, scale=1.0, res=64):
    """Smooth random log-density-like inputs [B, res, res] (sums of Gaussian bumps)."""
    rng = np.random.default_rng(seed)
    c = (np.arange(res) + 0.5) / res
    y, x = np.meshgrid(c, c, indexing="ij")
    out = np.zeros((B, res, res))
    for b in range(B):
        for _ in range(12):
            cx, cy, s, a = rng.uniform(0, 1), rng.uniform(0, 1), rng.uniform(0.03, 0.2), rng.normal(0, 1)
            out[b] += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
    return scale * (out + 0.05 * rng.normal(size=out.shape))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.fixture(scope="module")
def net():
    P = _P()
    c = P.inim_cnn_create(0)
    yield c
    c.close()


def test_params_roundtrip(net):
    P = _P()
    assert P.inim_cnn_num_params(net) == C.n_params() == P.inim_cnn_num_params()
    blob = C.he_init(5).astype(np.float32)
    P.inim_cnn_set_params(net, blob)
    assert np.array_equal(P.inim_cnn_get_params(net), blob)


@pytest.mark.parametrize("B,seed", [(1, 11), (3, 12)])
def test_forward_matches_oracle(net, B, seed):
    P = _P()
    blob = C.he_init(seed).astype(np.float32)
    P.inim_cnn_set_params(net, blob)
    x = _fields(B, seed)
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    yd = torch.empty((B, 64, 64, 2), dtype=torch.float32, device="cuda")
    P.inim_cnn_forward(net, xd, yd)
    got = yd.cpu().numpy().astype(np.float64)
    want, _ = C.forward(blob.astype(np.float64), x.astype(np.float32).astype(np.float64))
    assert np.isfinite(got).all()
    err = _rel(got, want)
    assert err < 3e-2 and _cos(got, want) > 0.999, (err, _cos(got, want))
    # each sample of the batch is computed independently
    if B > 1:
        y1 = torch.empty((1, 64, 64, 2), dtype=torch.float32, device="cuda")
        P.inim_cnn_forward(net, xd[1:2].contiguous(), y1)
        assert np.array_equal(y1.cpu().numpy()[0], got[1].astype(np.float32))


def test_gradients_match_oracle(net):
    P = _P()
    blob = C.he_init(21).astype(np.float32)
    P.inim_cnn_set_params(net, blob)
    B = 2
    x = _fields(B, 21)
    rng = np.random.default_rng(22)
    target = 0.3 * _fields(2 * B, 23).reshape(B, 2, 64, 64).transpose(0, 2, 3, 1) + 0.01 * rng.normal(size=(B, 64, 64, 2))
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    td = torch.as_tensor(target, dtype=torch.float32, device="cuda").contiguous()
    gd = torch.empty(C.n_params(), dtype=torch.float32, device="cuda")
    loss = P.inim_cnn_gradients(net, xd, td, gd)
    g = gd.cpu().numpy().astype(np.float64)
    want_loss, want = C.loss_and_grads(blob.astype(np.float64), x.astype(np.float32).astype(np.float64),
                                       target.astype(np.float32).astype(np.float64))
    assert abs(loss - want_loss) <= 2e-2 * want_loss, (loss, want_loss)
    assert _cos(g, want) > 0.998, _cos(g, want)
    off = 0
    for k, (ci, co, _) in enumerate(C.LAYERS):
        nw = co * 9 * ci
        ew = _rel(g[off:off + nw], want[off:off + nw])
        eb = _rel(g[off + nw:off + nw + co], want[off + nw:off + nw + co])
        assert ew < 6e-2 and eb < 6e-2, (k, ew, eb)
        off += nw + co


# Element-wise parity against the oracle in its BF16 mode (the same values
# rounded at the same places).  What remains is the order and precision of
# the sums (FP32 on the GPU, FP64 in the oracle), which moves stored values
# across BF16 rounding boundaries now and then and, backwards, flips a ReLU
# mask where a pre-activation is within rounding of zero.  The bounds below
# hold for an FP32-accumulating emulation of the same network with margins of
# 3-5x (forward: max |diff| <= 0.044 rms, worst 8x8 tile 0.042 relative;
# weight gradients: whole layer <= 0.0092 relative, at most 0.11% of the
# elements off by more than 0.1 rms, max 0.6 rms, per output channel at most
# 0.65 of the channel bound); a wrong tile, channel or layer breaks them.
def test_forward_elementwise_vs_bf16_oracle(net):
    P = _P()
    for B, seed in ((1, 11), (3, 12)):
        blob = C.he_init(seed).astype(np.float32)
        P.inim_cnn_set_params(net, blob)
        x = _fields(B, seed).astype(np.float32)
        xd = torch.as_tensor(x, device="cuda").contiguous()
        yd = torch.empty((B, 64, 64, 2), dtype=torch.float32, device="cuda")
        P.inim_cnn_forward(net, xd, yd)
        got = yd.cpu().numpy().astype(np.float64)
        want, _ = C.forward(blob.astype(np.float64), x.astype(np.float64), bf16=True)
        rms = float(np.sqrt((want ** 2).mean()))
        d = np.abs(got - want)
        assert d.max() <= 0.15 * rms, (B, d.max() / rms)
        dt = (got - want).reshape(B, 8, 8, 8, 8, 2)
        wt = want.reshape(B, 8, 8, 8, 8, 2)
        tile = np.sqrt((dt ** 2).sum(axis=(2, 4))) / np.sqrt((wt ** 2).sum(axis=(2, 4)))
        assert tile.max() <= 0.15, (B, tile.max())


def test_gradients_elementwise_vs_bf16_oracle(net):
    P = _P()
    blob = C.he_init(21).astype(np.float32)
    P.inim_cnn_set_params(net, blob)
    B = 2
    x = _fields(B, 21).astype(np.float32)
    rng = np.random.default_rng(22)
    target = (0.3 * _fields(2 * B, 23).reshape(B, 2, 64, 64).transpose(0, 2, 3, 1)
              + 0.01 * rng.normal(size=(B, 64, 64, 2))).astype(np.float32)
    xd = torch.as_tensor(x, device="cuda").contiguous()
    td = torch.as_tensor(target, device="cuda").contiguous()
    gd = torch.empty(C.n_params(), dtype=torch.float32, device="cuda")
    P.inim_cnn_gradients(net, xd, td, gd)
    g = gd.cpu().numpy().astype(np.float64)
    _, want = C.loss_and_grads(blob.astype(np.float64), x.astype(np.float64), target.astype(np.float64), bf16=True)
    off = 0
    for k, (ci, co, _) in enumerate(C.LAYERS):
        nw = co * 9 * ci
        gw, ww = g[off:off + nw].reshape(co, 9 * ci), want[off:off + nw].reshape(co, 9 * ci)
        rms = float(np.sqrt((ww ** 2).mean()))
        d = np.abs(gw - ww)
        assert np.linalg.norm(gw - ww) <= 0.05 * np.linalg.norm(ww), (k, "layer")
        assert (d > 0.1 * rms).mean() <= 0.01, (k, "fraction", (d > 0.1 * rms).mean())
        assert d.max() <= 2.0 * rms, (k, "max", d.max() / rms)
        # per output channel: a wrong channel (relative error ~1 or more) fails
        # unless its gradient is tiny; the emulation's worst channel (the
        # 8x8 bottleneck, where ReLU mask flips weigh most) reaches 0.65 of this
        ch_err = np.linalg.norm(gw - ww, axis=1)
        ch_ref = np.linalg.norm(ww, axis=1)
        assert np.all(ch_err <= 0.6 * ch_ref + 0.05 * rms * np.sqrt(9 * ci)), (k, "channel")
        gb, wb = g[off + nw:off + nw + co], want[off + nw:off + nw + co]
        assert np.linalg.norm(gb - wb) <= 0.05 * np.linalg.norm(wb), (k, "bias")
        off += nw + co


@pytest.mark.parametrize("in_res", [128, 256])
def test_stem_variant_matches_oracle(in_res):
    # the higher-resolution input: the first convolution at in_res, then
    # 2x2 pools down to 64^2; forward and gradients against the oracle with
    # the same stem, in its BF16 mode (two extra stored roundings per pool)
    P = _P()
    stem = {128: 1, 256: 2}[in_res]
    c = P.inim_cnn_create(0, in_res)
    assert c.in_res == in_res and P.inim_cnn_num_params(c) == C.n_params()
    blob = C.he_init(61).astype(np.float32)
    P.inim_cnn_set_params(c, blob)
    B = 2
    x = _fields(B, 61, res=in_res).astype(np.float32)
    rng = np.random.default_rng(62)
    target = (0.3 * _fields(2 * B, 63).reshape(B, 2, 64, 64).transpose(0, 2, 3, 1)
              + 0.01 * rng.normal(size=(B, 64, 64, 2))).astype(np.float32)
    xd = torch.as_tensor(x, device="cuda").contiguous()
    td = torch.as_tensor(target, device="cuda").contiguous()
    yd = torch.empty((B, 64, 64, 2), dtype=torch.float32, device="cuda")
    P.inim_cnn_forward(c, xd, yd)
    got = yd.cpu().numpy().astype(np.float64)
    want, _ = C.forward(blob.astype(np.float64), x.astype(np.float64), bf16=True, stem=stem)
    rms = float(np.sqrt((want ** 2).mean()))
    assert np.abs(got - want).max() <= 0.15 * rms, np.abs(got - want).max() / rms
    want64, _ = C.forward(blob.astype(np.float64), x.astype(np.float64), stem=stem)
    assert _rel(got, want64) < 3e-2 and _cos(got, want64) > 0.999
    gd = torch.empty(C.n_params(), dtype=torch.float32, device="cuda")
    loss = P.inim_cnn_gradients(c, xd, td, gd)
    g = gd.cpu().numpy().astype(np.float64)
    wl, wg = C.loss_and_grads(blob.astype(np.float64), x.astype(np.float64), target.astype(np.float64),
                              stem=stem)
    assert abs(loss - wl) <= 2e-2 * wl, (loss, wl)
    assert _cos(g, wg) > 0.998, _cos(g, wg)
    ci, co, _ = C.LAYERS[0]
    nw = co * 9 * ci                                  # the stem's convolution sees the full input
    assert _rel(g[:nw], wg[:nw]) < 6e-2 and _rel(g[nw:nw + co], wg[nw:nw + co]) < 6e-2
    # the wrong input size is refused
    with pytest.raises(ValueError):
        P.inim_cnn_forward(c, torch.zeros((B, 64, 64), device="cuda"), yd)
    c.close()


def test_training_lowers_loss():
    P = _P()
    c = P.inim_cnn_create(3)
    B = 8
    x = _fields(B, 31)
    # a learnable target: a smooth field derived from the input's gradient
    gy, gx = np.gradient(x, axis=(1, 2))
    t = 0.5 * np.stack([-gx, -gy], axis=-1) * 64 / 8
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    td = torch.as_tensor(t, dtype=torch.float32, device="cuda").contiguous()
    losses = [P.inim_cnn_train_step(c, xd, td, 1e-3) for _ in range(80)]
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])
    # the asynchronous form: no host wait inside the steps; the mean of their
    # losses is read once afterwards
    P.inim_cnn_loss_mean(c)                                   # resets the running sum
    for _ in range(10):
        assert P.inim_cnn_train_step(c, xd, td, 1e-3, wait=False) is None
    mean = P.inim_cnn_loss_mean(c)
    last = P.inim_cnn_train_step(c, xd, td, 1e-3)
    assert np.isfinite(mean) and 0 < mean < losses[0] and last <= 1.5 * mean, (mean, last)
    c.close()


def test_density_pooled_matches_oracle():
    P = _P()
    from paper_2604_13880_gb300 import synth
    mesh = synth.voronoi_map(60, 3000, seed=41, jitter=0.2)
    vals = synth.lognormal_values(60, seed=42)
    k, pool = 9, 8
    m = P.inim_map_create(mesh)
    out = np.empty((64, 64), np.float32)
    P.inim_density_pooled(m, mesh.verts_f32(), k, vals.astype(np.float32), pool, out)
    lab, cnt, _ = O.labels_scanline(mesh.verts_f32().astype(np.float64), mesh.ring_off, mesh.ring_idx,
                                    mesh.ring_region, mesh.n_regions, k)
    want = O.pooled_log_density(lab, cnt, vals.astype(np.float32).astype(np.float64), pool)
    # f32 density ratios and logs, 64 f32 additions per block
    assert np.abs(out - want).max() < 5e-5, np.abs(out - want).max()
    # device buffers give the same result
    xd = torch.as_tensor(mesh.verts_f32(), device="cuda")
    vd = torch.as_tensor(vals.astype(np.float32), device="cuda")
    od = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    P.inim_density_pooled(m, xd, k, vd, pool, od)
    torch.cuda.synchronize()
    assert np.array_equal(od.cpu().numpy(), out)
    m.close()


def test_zero_field_warm_start_equals_cold():
    # a network whose head is all zeros predicts a zero field: the warm-started
    # direct step must then follow the cold one exactly
    P = _P()
    from paper_2604_13880_gb300 import synth
    blob = C.he_init(7).astype(np.float32)
    ci, co, _ = C.LAYERS[-1]
    blob[-(co * 9 * ci + co):] = 0.0
    P.inim_warmstart_load(blob)
    mesh = synth.voronoi_map(40, 2000, seed=51)
    vals = synth.lognormal_values(40, seed=52)[None].astype(np.float32)
    m = P.inim_map_create(mesh)
    res = []
    for warm in (0, 1):
        p = P.params(log2_res=9, shape=0.5, max_iters=20, warm_start=warm)
        outs, stats, _ = P.inim_run_series([dict(map=m, values=vals, params=p)])
        res.append((outs[0], stats[0][0]))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1]["iters"] == res[1][1]["iters"]
    m.close()


def test_warm_start_argument_errors():
    P = _P()
    with pytest.raises(RuntimeError):
        P.inim_warmstart_load(np.zeros(10, np.float32))


@pytest.mark.slow
def test_trained_warm_start_beats_cold_start():
    # a network trained on fields the method itself generates (2048 maps of
    # 50-300 regions at 512^2) must start held-out maps closer to equal
    # density than the plain start and reach eps = 0.2 in fewer iterations
    from paper_2604_13880_gb300 import warmstart as W
    train_maps = W.generate_maps(range(50000, 52048), workers=8)
    test_maps = W.generate_maps(range(60000, 60064), workers=8)
    X, Y, _ = W.build_dataset(train_maps, eps_target=0.05, max_iters=512)
    net, hist = W.train(X, Y, epochs=15)
    assert hist["loss"][-1] < 0.5 * hist["loss"][0], hist["loss"]
    curve = W.eps_curve(net, test_maps, [1])
    assert curve["warm_mean"][0] < 0.8 * curve["cold_mean"][0], curve
    res = W.evaluate(net, test_maps, eps_target=0.2)
    assert res["warm"]["reached"] >= res["cold"]["reached"] - 1, res
    assert res["warm"]["iters_mean"] < 0.8 * res["cold"]["iters_mean"], res
    net.close()

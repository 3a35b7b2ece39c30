"""GPU parity of the U-Net surrogate (mlswlbm_unet_*) with the numpy
reference tests/unet_ref.py, stage by stage. Each stage is recomputed in
FP64 from the device's own BF16 inputs of that stage, so that one stage's
rounding does not feed the next comparison.

Tolerances:
- BF16 activations: the device accumulates in FP32 and rounds once to BF16
  (relative 2^-9); the bound is 2^-7 of the value plus 2^-9 of the layer's
  largest value, to cover the FP32 accumulation order.
- FP32 outputs and parameter gradients (FP32 atomics over pixels): 1e-3 of
  the largest entry of the layer.
- Halo rings hold the periodic images bit for bit.
"""
import numpy as np
import pytest

from tests import unet_ref as R

pytestmark = pytest.mark.gpu

N, SIDE, BATCH = 3, 128, 2
EXTRA = (0.5, -0.25)
IN_SCALE, OUT_SCALE = 1.0, 1.0


def _interior(t):
    return t[:, 1:-1, 1:-1, :].astype(np.float64)


def _halo_ok(t):
    """the halo ring equals the periodic image of the interior"""
    inner = t[:, 1:-1, 1:-1, :]
    want = np.pad(inner, ((0, 0), (1, 1), (1, 1), (0, 0)), mode="wrap")
    return np.array_equal(t.view(np.uint32), want.view(np.uint32))


def _close_bf16(got, want):
    scale = np.abs(want).max()
    err = np.abs(got - want) - (2.0 ** -7 * np.abs(want) + 2.0 ** -9 * scale)
    return err.max() <= 0, float(np.abs(got - want).max()), float(scale)


@pytest.fixture(scope="module")
def net():
    import torch
    from paper_2409_16659_gb300 import mlswlbm as B
    rng = np.random.default_rng(7)
    u = B.UNet(N, SIDE, SIDE, BATCH, extra=EXTRA, seed=3, in_scale=IN_SCALE, out_scale=OUT_SCALE)
    # random biases too, so that the bias path is exercised
    p = u.get_params()
    off = 0
    for _, ins, cout, _, _ in R.layer_table():
        cin = sum(c for _, c in ins)
        off += cout * 9 * cin
        p[off:off + cout] = 0.05 * rng.standard_normal(cout)
        off += cout
    u.set_params(p)
    h = 1.0 + 1e-2 * rng.standard_normal((BATCH, N, SIDE, SIDE))
    tgt = h + 1e-3 * rng.standard_normal(h.shape)
    hd = torch.from_numpy(h.astype(np.float32)).cuda()
    td = torch.from_numpy(tgt.astype(np.float32)).cuda()
    out = torch.empty_like(hd)
    u.predict(hd, out)
    torch.cuda.synchronize()
    fwd = {name: u.tensor(name) for name in R.OUTPUT_NAME.values() if name != "Y"}
    for name in ("X0", "P1", "P2", "P3", "U2", "U1", "U0"):
        fwd[name] = u.tensor(name)
    y = u.output().astype(np.float64)
    pred = out.cpu().numpy().astype(np.float64)
    loss = u.train_step(hd, td, 0.0)      # lr 0: gradients only
    grads = u.param_grads().astype(np.float64)
    bwd = {name: u.tensor(name, grad=True) for name in
           ("YG", "D0", "B0", "U0", "D1", "B1", "U1", "D2", "B2", "U2", "S3", "A3", "P3",
            "S2", "A2", "P2", "S1", "A1", "P1", "S0", "A0")}
    skips = [u.skip_grad(k) for k in range(3)]
    st = u.status()
    u.close()
    return dict(p=p, h=h, tgt=tgt, fwd=fwd, y=y, pred=pred, loss=loss, grads=grads, bwd=bwd,
                skips=skips, status=st)


def test_input_planes_and_halo(net):
    x0 = net["fwd"]["X0"]
    assert _halo_ok(x0)
    want = R.input_planes(net["h"].astype(np.float32), EXTRA, IN_SCALE)
    ok, err, scale = _close_bf16(_interior(x0), want)
    assert ok, (err, scale)


def test_every_forward_convolution_pooling_and_upsampling(net):
    fwd, P = net["fwd"], R.split_params(net["p"])
    assert net["status"] == 0
    for name in ("P1", "P2", "P3"):
        src = {"P1": "S0", "P2": "S1", "P3": "S2"}[name]
        assert _halo_ok(fwd[name])
        ok, err, sc = _close_bf16(_interior(fwd[name]), R.pool2(_interior(fwd[src])))
        assert ok, (name, err, sc)
    for name, src in (("U2", "S3"), ("U1", "D2"), ("U0", "D1")):
        # nearest upsampling copies BF16 values exactly
        assert np.array_equal(_interior(fwd[name]), R.up2(_interior(fwd[src]))), name
    for l, (lname, ins, cout, _, relu) in enumerate(R.layer_table()):
        w, b = P[l]
        xin = np.concatenate([_interior(fwd[nm]) for nm, _ in ins], axis=3)
        z = R.conv3(xin, R.bf16(w), b)
        if lname == "out":
            y = np.moveaxis(net["y"], 1, 3)            # [B][H][W][n]
            ref = z[..., :N]
            assert np.abs(y - ref).max() <= 1e-3 * np.abs(ref).max(), lname
            continue
        out = fwd[R.OUTPUT_NAME[lname]]
        assert _halo_ok(out), lname
        ok, err, sc = _close_bf16(_interior(out), np.maximum(z, 0.0))
        assert ok, (lname, err, sc)


def test_prediction_keeps_every_layer_mass(net):
    h, pred, y = net["h"].astype(np.float32).astype(np.float64), net["pred"], net["y"]
    s = R.sample_rms(h)[:, None, None, None]
    d = (y - y.mean(axis=(2, 3), keepdims=True)) * s / OUT_SCALE
    np.testing.assert_allclose(pred, h + d, rtol=0, atol=1e-6)
    np.testing.assert_allclose(pred.sum(axis=(2, 3)), h.sum(axis=(2, 3)), rtol=1e-6)


def test_loss_and_output_gradient(net):
    h = net["h"].astype(np.float32).astype(np.float64)
    t = net["tgt"].astype(np.float32).astype(np.float64)
    y = np.moveaxis(net["y"], 1, 3)
    ypad = np.zeros(y.shape[:3] + (R.C_OUT,))
    ypad[..., :N] = y
    L, g = R.loss_and_grad(ypad, h, t, N, OUT_SCALE)
    assert net["loss"] == pytest.approx(L, rel=1e-5)
    yg = net["bwd"]["YG"]
    assert _halo_ok(yg)
    ok, err, sc = _close_bf16(_interior(yg), g)
    assert ok, (err, sc)


def test_every_gradient_stage(net):
    fwd, bwd, P = net["fwd"], net["bwd"], R.split_params(net["p"])
    table = R.layer_table()
    G = R.split_params(net["grads"])
    dz_of = {"out": "YG"}
    dz_of.update({nm: R.OUTPUT_NAME[nm] for nm, *_ in table if nm != "out"})
    skip_name = {"S0": 0, "S1": 1, "S2": 2}
    for l, (lname, ins, cout, _, _) in enumerate(table):
        dz = _interior(bwd[dz_of[lname]])
        xin = np.concatenate([_interior(fwd[nm]) for nm, _ in ins], axis=3)
        # parameter gradients
        dw_ref, db_ref = R.conv3_weight_grad(dz, xin), dz.sum(axis=(0, 1, 2))
        dw, db = G[l]
        assert np.abs(dw - dw_ref).max() <= 1e-3 * np.abs(dw_ref).max(), (lname, "dW")
        assert np.abs(db - db_ref).max() <= 1e-3 * np.abs(db_ref).max() + 1e-12, (lname, "db")
        if lname == "e0a":
            continue
        # input gradients (before the masks and sums of the next stage)
        dx = R.conv3_input_grad(dz, R.bf16(P[l][0]))
        off = 0
        for nm, c in ins:
            part = dx[..., off:off + c]
            off += c
            if nm in ("U0", "U1", "U2", "P1", "P2", "P3"):
                got = bwd[nm]
            elif nm in skip_name and len(ins) == 2:
                got = net["skips"][skip_name[nm]]
            else:   # a ReLU output consumed only here: masked by its activation
                got = bwd[nm]
                part = part * (_interior(fwd[nm]) > 0)
            assert _halo_ok(got), (lname, nm)
            ok, err, sc = _close_bf16(_interior(got), part)
            assert ok, (lname, nm, err, sc)
    # upsampling and pooling gradients with their masks
    for dS, dU in (("D1", "U0"), ("D2", "U1"), ("S3", "U2")):
        want = R.up2_grad(_interior(bwd[dU])) * (_interior(fwd[dS]) > 0)
        ok, err, sc = _close_bf16(_interior(bwd[dS]), want)
        assert ok, (dS, err, sc)
    for S, dP, k in (("S2", "P3", 2), ("S1", "P2", 1), ("S0", "P1", 0)):
        want = (_interior(net["skips"][k]) + R.pool2_grad(_interior(bwd[dP]))) * (_interior(fwd[S]) > 0)
        ok, err, sc = _close_bf16(_interior(bwd[S]), want)
        assert ok, (S, err, sc)


def test_training_fits_a_known_linear_map():
    """A fixed smoothing of each layer (a 5-point average) as the change
    over a window: the loss falls by more than 10x in 300 Adam steps."""
    import torch
    from paper_2409_16659_gb300 import mlswlbm as B
    rng = np.random.default_rng(11)
    h = 1.0 + 1e-2 * rng.standard_normal((4, N, SIDE, SIDE))
    nb = (np.roll(h, 1, 2) + np.roll(h, -1, 2) + np.roll(h, 1, 3) + np.roll(h, -1, 3)) / 4.0
    tgt = h + 0.5 * (nb - h)
    hd = torch.from_numpy(h.astype(np.float32)).cuda()
    td = torch.from_numpy(tgt.astype(np.float32)).cuda()
    with B.UNet(N, SIDE, SIDE, 4, extra=EXTRA, seed=5, in_scale=IN_SCALE, out_scale=OUT_SCALE) as u:
        losses = [u.train_step(hd, td, 1e-3) for _ in range(300)]
        assert u.status() == 0
    assert np.isfinite(losses).all()
    assert np.mean(losses[-20:]) < 0.1 * losses[0], (losses[0], losses[-1])

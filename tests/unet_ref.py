"""Plain numpy reference of the U-Net surrogate's arithmetic (test helper).

Everything is FP64 from the given values. It covers:
- BF16 rounding (round to nearest, ties to even, as the device conversions);
- periodic 3 x 3 convolutions on NHWC arrays with weights [out][tap][in], tap = 3 (dy + 1) + (dx + 1),
  their input and weight gradients;
- 2 x 2 average pooling and nearest 2x upsampling with their adjoints;
- the network's layer table, its forward pass and its backward pass.

Shares no code with the CUDA path.
"""
import numpy as np

WIDTHS = (32, 64, 128, 256)   # channels of the four levels
C_IN = 16                     # input channels: n heights, parameter planes, zeros
C_OUT = 16                    # output channels: the first n are the change


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def from_bf16_bits(u16):
    return (np.asarray(u16, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def _roll(x, dy, dx):
    """x[b, y + dy, x + dx, :] at (b, y, x), periodic."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv3(x, w, b=None):
    """y[b,y,x,o] = sum_{t,c} w[o,t,c] x[b, y+dy_t, x+dx_t, c] (+ b[o])."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = 0.0
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        y = y + np.tensordot(_roll(x, dy, dx), w[:, t, :], axes=([3], [1]))
    if b is not None:
        y = y + np.asarray(b, dtype=np.float64)
    return y


def conv3_input_grad(dz, w):
    """dx[b,y,x,c] = sum_{t,o} w[o,t,c] dz[b, y-dy_t, x-dx_t, o] (adjoint of conv3)."""
    dz = np.asarray(dz, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dx_ = 0.0
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        dx_ = dx_ + np.tensordot(_roll(dz, -dy, -dx), w[:, t, :], axes=([3], [0]))
    return dx_


def conv3_weight_grad(dz, x):
    """dw[o,t,c] = sum_{b,y,x} dz[b,y,x,o] x[b, y+dy_t, x+dx_t, c]."""
    dz = np.asarray(dz, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    return np.stack([np.tensordot(dz, _roll(x, t // 3 - 1, t % 3 - 1), axes=([0, 1, 2], [0, 1, 2]))
                     for t in range(9)], axis=1)


def pool2(x):
    """2 x 2 average pooling."""
    x = np.asarray(x, dtype=np.float64)
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 0::2] + x[:, 1::2, 1::2])


def pool2_grad(dy):
    """Adjoint of pool2: every fine pixel gets a quarter of its coarse one."""
    return 0.25 * np.repeat(np.repeat(np.asarray(dy, dtype=np.float64), 2, axis=1), 2, axis=2)


def up2(x):
    """Nearest 2x upsampling."""
    return np.repeat(np.repeat(np.asarray(x, dtype=np.float64), 2, axis=1), 2, axis=2)


def up2_grad(dy):
    """Adjoint of up2: the sum of the four fine pixels of each coarse one."""
    dy = np.asarray(dy, dtype=np.float64)
    return dy[:, 0::2, 0::2] + dy[:, 0::2, 1::2] + dy[:, 1::2, 0::2] + dy[:, 1::2, 1::2]


# ---------------------------------------------------------------------------
# The network: 15 convolutions. LAYERS[l] = (input names, output name, relu).
# Inputs listed twice are concatenated along the channels (upsampled coarse
# features first, then the skip of the same level).
# ---------------------------------------------------------------------------
def layer_table():
    w0, w1, w2, w3 = WIDTHS
    return [
        # name, inputs (channels), output channels, level, relu
        ("e0a", [("X0", C_IN)], w0, 0, True),
        ("e0b", [("A0", w0)], w0, 0, True),
        ("e1a", [("P1", w0)], w1, 1, True),
        ("e1b", [("A1", w1)], w1, 1, True),
        ("e2a", [("P2", w1)], w2, 2, True),
        ("e2b", [("A2", w2)], w2, 2, True),
        ("e3a", [("P3", w2)], w3, 3, True),
        ("e3b", [("A3", w3)], w3, 3, True),
        ("d2a", [("U2", w3), ("S2", w2)], w2, 2, True),
        ("d2b", [("B2", w2)], w2, 2, True),
        ("d1a", [("U1", w2), ("S1", w1)], w1, 1, True),
        ("d1b", [("B1", w1)], w1, 1, True),
        ("d0a", [("U0", w1), ("S0", w0)], w0, 0, True),
        ("d0b", [("B0", w0)], w0, 0, True),
        ("out", [("D0", w0)], C_OUT, 0, False),
    ]


OUTPUT_NAME = {"e0a": "A0", "e0b": "S0", "e1a": "A1", "e1b": "S1", "e2a": "A2", "e2b": "S2",
               "e3a": "A3", "e3b": "S3", "d2a": "B2", "d2b": "D2", "d1a": "B1", "d1b": "D1",
               "d0a": "B0", "d0b": "D0", "out": "Y"}


def param_count():
    n = 0
    for _, ins, cout, _, _ in layer_table():
        cin = sum(c for _, c in ins)
        n += cout * 9 * cin + cout
    return n


def split_params(p):
    """Flat FP32 parameters -> per layer (w [out][9][in], b [out]); every
    layer's weights, then its bias, in the order of the table."""
    out, off = [], 0
    for _, ins, cout, _, _ in layer_table():
        cin = sum(c for _, c in ins)
        w = np.asarray(p[off:off + cout * 9 * cin], dtype=np.float64).reshape(cout, 9, cin)
        off += cout * 9 * cin
        b = np.asarray(p[off:off + cout], dtype=np.float64)
        off += cout
        out.append((w, b))
    return out


def sample_rms(h):
    """RMS over all layers and pixels of each sample's deviations from its
    layer means, [B]."""
    h = np.asarray(h, dtype=np.float64)
    d = h - h.mean(axis=(2, 3), keepdims=True)
    return np.sqrt((d * d).mean(axis=(1, 2, 3)))


def input_planes(h, extra, in_scale):
    """X0 [B][H][W][16]: (h_i - mean h_i) in_scale / s (s the sample's RMS
    deviation; all zero for a flat sample), then the parameter planes, then
    zeros. h [B][n][H][W]."""
    h = np.asarray(h, dtype=np.float64)
    B, n, H, W = h.shape
    s = sample_rms(h)
    k = np.where(s > 0, in_scale / np.where(s > 0, s, 1.0), 0.0)
    x = np.zeros((B, H, W, C_IN))
    for i in range(n):
        x[..., i] = (h[:, i] - h[:, i].mean(axis=(1, 2), keepdims=True)) * k[:, None, None]
    for j, v in enumerate(extra):
        x[..., n + j] = v
    return x


def forward(params, x0, rnd=bf16):
    """Forward pass from the input planes (already rounded as the device
    holds them). Every activation is rounded by `rnd` (FP64 in, as the
    device stores it; bf16 goes through FP32 like the device's FP32
    accumulators); returns (acts, y) with acts the stored tensors by name and y the
    FP64 output of the last convolution (before any rounding)."""
    P = split_params(params)
    acts = {"X0": np.asarray(x0, dtype=np.float64)}
    wb = [(np.asarray(rnd(w), dtype=np.float64), np.asarray(b, dtype=np.float64)) for w, b in P]
    for l, (name, ins, cout, lev, relu) in enumerate(layer_table()):
        if name == "e1a":
            acts["P1"] = np.asarray(rnd(pool2(acts["S0"])), dtype=np.float64)
        if name == "e2a":
            acts["P2"] = np.asarray(rnd(pool2(acts["S1"])), dtype=np.float64)
        if name == "e3a":
            acts["P3"] = np.asarray(rnd(pool2(acts["S2"])), dtype=np.float64)
        if name == "d2a":
            acts["U2"] = up2(acts["S3"])
        if name == "d1a":
            acts["U1"] = up2(acts["D2"])
        if name == "d0a":
            acts["U0"] = up2(acts["D1"])
        xin = np.concatenate([acts[nm] for nm, _ in ins], axis=3)
        w, b = wb[l]
        z = conv3(xin, w, b)
        if name == "out":
            return acts, z
        z = np.maximum(z, 0.0) if relu else z
        acts[OUTPUT_NAME[name]] = np.asarray(rnd(z), dtype=np.float64)
    raise AssertionError("no output layer")


def loss_and_grad(y, h, target, n, out_scale):
    """Mean squared error over the first n output channels against the
    change scaled by out_scale / s, and its gradient with respect to y
    (zero elsewhere)."""
    h = np.asarray(h, dtype=np.float64)
    s = sample_rms(h)
    k = np.where(s > 0, out_scale / np.where(s > 0, s, 1.0), 0.0)
    t = (np.asarray(target, dtype=np.float64) - h) * k[:, None, None, None]   # [B][n][H][W]
    t = np.moveaxis(t, 1, 3)                                     # [B][H][W][n]
    d = y[..., :n] - t
    cnt = d.size
    g = np.zeros_like(y)
    g[..., :n] = 2.0 * d / cnt
    return float((d * d).sum() / cnt), g


def backward(params, acts, gy, rnd=bf16):
    """Backward pass from the output gradient gy (FP64, [B][H][W][16]).

    The device stores every propagated gradient in BF16: `rnd` is applied
    where it rounds (the scaled output gradient, and each gradient tensor it
    writes). Returns (grads, dz) with grads[l] = (dW [out][9][in], db [out])
    and dz the stored gradients by the name of the tensor they belong to.
    """
    P = split_params(params)
    wq = [np.asarray(rnd(w), dtype=np.float64) for w, _ in P]
    table = layer_table()
    idx = {name: l for l, (name, *_r) in enumerate(table)}
    r = lambda a: np.asarray(rnd(a), dtype=np.float64)  # noqa: E731
    grads = [None] * len(table)
    dz = {}

    def layer(name, dzl):
        """weight and bias gradients of layer `name` from its output gradient
        dzl (after the ReLU mask), and the gradient of its input(s)"""
        l = idx[name]
        _, ins, cout, _, _ = table[l]
        xin = np.concatenate([acts[nm] for nm, _ in ins], axis=3)
        grads[l] = (conv3_weight_grad(dzl, xin), dzl.sum(axis=(0, 1, 2)))
        dx = conv3_input_grad(dzl, wq[l])
        parts, off = {}, 0
        for nm, c in ins:
            parts[nm] = dx[..., off:off + c]
            off += c
        return parts

    def mask(g, y):
        return g * (y > 0)

    dz["Y"] = r(gy)
    g = layer("out", dz["Y"])
    dz["D0"] = r(mask(g["D0"], acts["D0"]))
    g = layer("d0b", dz["D0"])
    dz["B0"] = r(mask(g["B0"], acts["B0"]))
    g = layer("d0a", dz["B0"])
    dz["U0"], skip0 = r(g["U0"]), r(g["S0"])
    dz["D1"] = r(mask(up2_grad(dz["U0"]), acts["D1"]))
    g = layer("d1b", dz["D1"])
    dz["B1"] = r(mask(g["B1"], acts["B1"]))
    g = layer("d1a", dz["B1"])
    dz["U1"], skip1 = r(g["U1"]), r(g["S1"])
    dz["D2"] = r(mask(up2_grad(dz["U1"]), acts["D2"]))
    g = layer("d2b", dz["D2"])
    dz["B2"] = r(mask(g["B2"], acts["B2"]))
    g = layer("d2a", dz["B2"])
    dz["U2"], skip2 = r(g["U2"]), r(g["S2"])
    dz["S3"] = r(mask(up2_grad(dz["U2"]), acts["S3"]))
    g = layer("e3b", dz["S3"])
    dz["A3"] = r(mask(g["A3"], acts["A3"]))
    g = layer("e3a", dz["A3"])
    dz["P3"] = r(g["P3"])
    dz["S2"] = r(mask(skip2 + pool2_grad(dz["P3"]), acts["S2"]))
    g = layer("e2b", dz["S2"])
    dz["A2"] = r(mask(g["A2"], acts["A2"]))
    g = layer("e2a", dz["A2"])
    dz["P2"] = r(g["P2"])
    dz["S1"] = r(mask(skip1 + pool2_grad(dz["P2"]), acts["S1"]))
    g = layer("e1b", dz["S1"])
    dz["A1"] = r(mask(g["A1"], acts["A1"]))
    g = layer("e1a", dz["A1"])
    dz["P1"] = r(g["P1"])
    dz["S0"] = r(mask(skip0 + pool2_grad(dz["P1"]), acts["S0"]))
    g = layer("e0b", dz["S0"])
    dz["A0"] = r(mask(g["A0"], acts["A0"]))
    layer("e0a", dz["A0"])
    return grads, dz


def flat_grads(grads):
    """Per-layer (dW, db) -> flat vector in the parameter order."""
    return np.concatenate([np.concatenate([dw.ravel(), db.ravel()]) for dw, db in grads])

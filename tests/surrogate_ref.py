"""Plain numpy reference of the convolutional surrogate's arithmetic (test
helper): BF16 rounding (round to nearest, ties to even, as the device
conversions), periodic K x K convolutions in NHWC with weights [d][in][out],
and their gradients, all in FP64 from the given BF16 values. Shares no code
with the CUDA path."""
import numpy as np

KS, KR = 5, 2
CH = (16, 32, 32, 16)


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def from_bf16_bits(u16):
    return (np.asarray(u16, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def split_params(w):
    """Weights [d][in][out] of the three layers and their biases."""
    ws, bs, off = [], [], 0
    for l in range(3):
        cnt = KS * KS * CH[l] * CH[l + 1]
        ws.append(np.asarray(w[off:off + cnt], dtype=np.float32).reshape(KS * KS, CH[l], CH[l + 1]))
        off += cnt
    for l in range(3):
        bs.append(np.asarray(w[off:off + CH[l + 1]], dtype=np.float32))
        off += CH[l + 1]
    return ws, bs


def _shifted(x, d, sign=1):
    """x[b, y + s dy, x + s dx] for offset d (periodic), s = sign."""
    dy, dx = d // KS - KR, d % KS - KR
    return np.roll(x, shift=(-sign * dy, -sign * dx), axis=(1, 2))


def conv(x, w):
    """out[b,y,x,o] = sum_{d,i} x[b, y+dy, x+dx, i] w[d,i,o] (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    out = 0.0
    for d in range(KS * KS):
        out = out + np.tensordot(_shifted(x, d), np.asarray(w[d], dtype=np.float64), axes=([3], [0]))
    return out


def conv_input_grad(dy, w):
    """dx[b,y,x,i] = sum_{d,o} dy[b, y-dy, x-dx, o] w[d,i,o]."""
    dy = np.asarray(dy, dtype=np.float64)
    out = 0.0
    for d in range(KS * KS):
        out = out + np.tensordot(_shifted(dy, d, -1), np.asarray(w[d], dtype=np.float64).T,
                                 axes=([3], [0]))
    return out


def conv_weight_grad(x, dy):
    """dw[d,i,o] = sum_{b,y,x} x[b, y+dy, x+dx, i] dy[b,y,x,o]."""
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    return np.stack([np.tensordot(_shifted(x, d), dy, axes=([0, 1, 2], [0, 1, 2]))
                     for d in range(KS * KS)])

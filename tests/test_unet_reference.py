"""Pins of the U-Net reference (tests/unet_ref.py) on the CPU, against what
the definitions fix, so that the reference the GPU kernels are held to is
itself checked:
- a periodic 3 x 3 convolution of a single unit input reproduces the
  weights, each tap at its own neighbour (closed form: this fixes the tap
  order and the sign of the offsets);
- the input and weight gradients are the adjoints of the convolution
  (<conv(x), z> = <x, conv_input_grad(z)> = <w, conv_weight_grad(z, x)>);
- pooling and upsampling: a constant stays constant, and each one's
  gradient is its adjoint;
- the whole backward pass against central differences of the loss in
  FP64 without rounding, on a 16 x 16 input;
- BF16 rounding goes to the nearest value, ties to even.
"""
import numpy as np

from tests import unet_ref as U


def test_convolution_of_a_unit_input_reproduces_the_taps():
    rng = np.random.default_rng(1)
    w = rng.standard_normal((5, 9, 3))
    x = np.zeros((1, 8, 8, 3))
    x[0, 4, 5, 2] = 1.0
    y = U.conv3(x, w)
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        # y[y0, x0] reads x[y0 + dy, x0 + dx]: the unit at (4, 5) reaches (4 - dy, 5 - dx)
        np.testing.assert_allclose(y[0, 4 - dy, 5 - dx], w[:, t, 2], rtol=0, atol=1e-15)
    assert np.count_nonzero(np.abs(y).sum(axis=3)) == 9
    # periodic: a unit in the corner reaches the opposite edges
    x = np.zeros((1, 8, 8, 3))
    x[0, 0, 0, 0] = 1.0
    y = U.conv3(x, w)
    np.testing.assert_allclose(y[0, 7, 7], w[:, 8, 0], atol=1e-15)   # dy = dx = +1


def test_gradients_are_the_adjoints_of_the_convolution():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 8, 4))
    w = rng.standard_normal((3, 9, 4))
    z = rng.standard_normal((2, 6, 8, 3))
    lhs = (U.conv3(x, w) * z).sum()
    assert abs(lhs - (x * U.conv3_input_grad(z, w)).sum()) <= 1e-10 * abs(lhs)
    assert abs(lhs - (w * U.conv3_weight_grad(z, x)).sum()) <= 1e-10 * abs(lhs)
    # the bias enters as a constant plane
    b = rng.standard_normal(3)
    np.testing.assert_allclose(U.conv3(x, w, b) - U.conv3(x, w), np.broadcast_to(b, z.shape))


def test_pooling_and_upsampling_with_their_adjoints():
    rng = np.random.default_rng(3)
    c = np.full((1, 8, 8, 2), 0.7)
    np.testing.assert_allclose(U.pool2(c), 0.7)
    np.testing.assert_allclose(U.up2(c), 0.7)
    x = rng.standard_normal((2, 8, 6, 3))
    np.testing.assert_allclose(U.pool2(U.up2(x)), x)
    y = rng.standard_normal((2, 4, 3, 3))
    assert abs((U.pool2(x) * y).sum() - (x * U.pool2_grad(y)).sum()) < 1e-12
    x2 = rng.standard_normal((2, 4, 3, 3))
    y2 = rng.standard_normal((2, 8, 6, 3))
    assert abs((U.up2(x2) * y2).sum() - (x2 * U.up2_grad(y2)).sum()) < 1e-12


def test_backward_pass_against_central_differences():
    rng = np.random.default_rng(4)
    n, side, scale_out = 3, 16, 40.0
    p = rng.standard_normal(U.param_count()) * 0.05
    h = 1.0 + 1e-2 * rng.standard_normal((1, n, side, side))
    tgt = h + 1e-3 * rng.standard_normal(h.shape)
    x0 = U.input_planes(h, [0.5, -0.25], 10.0)
    ident = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731

    def loss(q):
        _, y = U.forward(q, x0, rnd=ident)
        return U.loss_and_grad(y, h, tgt, n, scale_out)[0]

    acts, y = U.forward(p, x0, rnd=ident)
    L, gy = U.loss_and_grad(y, h, tgt, n, scale_out)
    grads, _ = U.backward(p, acts, gy, rnd=ident)
    g = U.flat_grads(grads)
    assert g.shape == p.shape
    # one weight and the bias of every layer, plus random entries
    offs, off = [], 0
    for _, ins, cout, _, _ in U.layer_table():
        cin = sum(c for _, c in ins)
        offs += [off + rng.integers(cout * 9 * cin), off + cout * 9 * cin]
        off += cout * 9 * cin + cout
    offs += list(rng.integers(0, p.size, 10))
    eps = 1e-6
    for k in offs:
        q = p.copy()
        q[k] += eps
        lp = loss(q)
        q[k] -= 2 * eps
        lm = loss(q)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(L)) + 1e-4 * abs(fd), (k, fd, g[k])


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5 - 2 ** -8, 3.14159], np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even (1.0)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, -2.5, 3.140625], np.float32)
    np.testing.assert_array_equal(U.bf16(v), want)
    bits = (U.bf16(v).view(np.uint32) >> 16).astype(np.uint16)
    np.testing.assert_array_equal(U.from_bf16_bits(bits), U.bf16(v))

"""Pins of the numpy reference for the surrogate's kernels (CPU): the
convolution equals its defining sum at sampled points, its input and weight
gradients are its adjoints (<conv(x, w), g> = <x, conv^T(g, w)> =
<w, dW(x, g)>), and BF16 rounding goes to the nearest value, ties to even."""
import numpy as np

from tests import surrogate_ref as R


def test_conv_is_its_defining_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 6, 8, 3))
    w = rng.standard_normal((25, 3, 4))
    out = R.conv(x, w)
    for b, y, xx, o in [(0, 0, 0, 0), (1, 2, 5, 3), (1, 5, 7, 1)]:
        v = sum(x[b, (y + d // 5 - 2) % 6, (xx + d % 5 - 2) % 8, i] * w[d, i, o]
                for d in range(25) for i in range(3))
        assert abs(v - out[b, y, xx, o]) < 1e-12


def test_gradients_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 8, 3))
    w = rng.standard_normal((25, 3, 4))
    g = rng.standard_normal((2, 6, 8, 4))
    a = (R.conv(x, w) * g).sum()
    assert np.isclose(a, (x * R.conv_input_grad(g, w)).sum(), rtol=1e-12)
    assert np.isclose(a, (w * R.conv_weight_grad(x, g)).sum(), rtol=1e-12)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5 - 2 ** -8, 3.14159], np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even (1.0)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, -2.5, 3.140625], np.float32)
    np.testing.assert_array_equal(R.bf16(v), want)
    bits = (R.bf16(v).view(np.uint32) >> 16).astype(np.uint16)
    np.testing.assert_array_equal(R.from_bf16_bits(bits), R.bf16(v))

"""Pins for the VGG16 oracle: the im2col convolution equals the convolution's
definition written as loops; identity kernels and pooling by hand."""
import numpy as np

from oracle import vgg as ov


def test_im2col_conv_equals_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 4, 3))
    W = rng.standard_normal((4, 27))
    b = rng.standard_normal(4)
    assert np.allclose(ov.conv3x3(x, W, b), ov.conv3x3_direct(x, W, b), rtol=1e-12, atol=1e-12)


def test_centre_tap_identity():
    x = np.random.default_rng(1).standard_normal((1, 6, 6, 2))
    W = np.zeros((2, 18))
    W[0, 4 * 2 + 0] = 1.0  # (kh, kw) = (1, 1), c = 0
    W[1, 4 * 2 + 1] = 1.0
    assert np.array_equal(ov.conv3x3(x, W, np.zeros(2)), x)


def test_maxpool_by_hand():
    x = np.arange(16, dtype=float).reshape(1, 4, 4, 1)
    assert np.array_equal(ov.maxpool2x2(x)[0, :, :, 0], [[5, 7], [13, 15]])

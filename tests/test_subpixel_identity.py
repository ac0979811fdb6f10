"""The decoder concat convs on the tensor cores never form the nearest-2x upsampled tensor:
for each output parity class (cx, cy) = (x mod 2, y mod 2) the 3x3 taps over the upsampled
tensor land on only 2 x 2 coarse pixels (coarse offset (c + k - 1) >> 1 per axis), so the
conv equals a 2x2 conv of the coarse tensor with the taps that share a coarse pixel summed.
This checks that identity in FP64 on random data, zero padding included -- the algebra the
kernel's weight blocks follow (the oracle itself convolves the upsampled tensor)."""
import numpy as np


def conv3x3_of_upsampled(x, w):
    """Definition: nearest 2x upsample of x (C, h, w), then a zero-padded 3x3 conv."""
    up = x.repeat(2, axis=1).repeat(2, axis=2)
    C, H, W = up.shape
    pad = np.zeros((C, H + 2, W + 2))
    pad[:, 1:-1, 1:-1] = up
    out = np.zeros((w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,chw->ohw", w[:, :, ky, kx], pad[:, ky:ky + H, kx:kx + W])
    return out


def subpixel(x, w):
    """Per class (cx, cy): a 2x2 conv of the coarse tensor with summed taps."""
    C, h, wd = x.shape
    pad = np.zeros((C, h + 2, wd + 2))
    pad[:, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], 2 * h, 2 * wd))
    for cy in range(2):
        for cx in range(2):
            acc = np.zeros((w.shape[0], h, wd))
            for dy in (cy - 1, cy):          # coarse row offsets this class reaches
                for dx in (cx - 1, cx):      # coarse column offsets
                    ws = np.zeros(w.shape[:2])
                    for ky in range(3):
                        for kx in range(3):
                            if (cy + ky - 1) >> 1 == dy and (cx + kx - 1) >> 1 == dx:
                                ws += w[:, :, ky, kx]
                    acc += np.einsum("oc,chw->ohw", ws, pad[:, 1 + dy:1 + dy + h, 1 + dx:1 + dx + wd])
            out[:, cy::2, cx::2] = acc
    return out


def test_upsampled_conv_is_a_summed_tap_2x2_conv_per_class():
    rng = np.random.default_rng(7)
    for C, O, h, wd in ((3, 2, 5, 7), (4, 3, 1, 1), (2, 5, 6, 3)):
        x = rng.standard_normal((C, h, wd))
        w = rng.standard_normal((O, C, 3, 3))
        ref = conv3x3_of_upsampled(x, w)
        got = subpixel(x, w)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max()), np.abs(got - ref).max()


def test_each_class_sums_nine_taps_over_four_coarse_pixels():
    """Every 3x3 tap is used exactly once per class, and each class's four coarse pixels
    take 4, 2, 2 and 1 taps (centre, two edges, corner)."""
    for cy in range(2):
        for cx in range(2):
            counts = {}
            for ky in range(3):
                for kx in range(3):
                    key = ((cy + ky - 1) >> 1, (cx + kx - 1) >> 1)
                    counts[key] = counts.get(key, 0) + 1
            assert sum(counts.values()) == 9
            assert sorted(counts.values()) == [1, 2, 2, 4]
            assert set(counts) == {(dy, dx) for dy in (cy - 1, cy) for dx in (cx - 1, cx)}

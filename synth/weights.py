"""Seeded U-Net weights in the library's weight-file layout.

Layout: a flat float32 array.  For every convolution in network order, its weight in
OIHW order followed by its bias; then the 1x1 head (weight OIHW, bias); then, when the
net has batch normalisation, (gamma, beta, mean, var) for each encoder convolution in
encoder order.  Network order is enc0a, enc0b, enc1a, enc1b, ..., the two bottleneck
convolutions, then dec(L-2)a, dec(L-2)b, ..., dec0a, dec0b.  A decoder "a" convolution
takes the skip tensor's channels first and the upsampled deeper tensor's channels after.
"""
from __future__ import annotations

import numpy as np


def unet_layer_shapes(ch, in_ch=5, out_ch=3):
    """[(name, cout, cin, k)] for the 3x3 convolutions in network order, then the head."""
    L = len(ch)
    shapes = []
    cin = in_ch
    for l in range(L):
        shapes.append((f"enc{l}a", ch[l], cin, 3))
        shapes.append((f"enc{l}b", ch[l], ch[l], 3))
        cin = ch[l]
    for l in range(L - 2, -1, -1):
        shapes.append((f"dec{l}a", ch[l], ch[l] + ch[l + 1], 3))
        shapes.append((f"dec{l}b", ch[l], ch[l], 3))
    shapes.append(("head", out_ch, ch[0], 1))
    return shapes


def n_weights(ch, in_ch=5, out_ch=3, has_bn=False):
    n = sum(co * ci * k * k + co for _, co, ci, k in unet_layer_shapes(ch, in_ch, out_ch))
    if has_bn:
        n += sum(4 * co for name, co, _, _ in unet_layer_shapes(ch, in_ch, out_ch)
                 if name.startswith("enc"))
    return n


def unet_weights(ch, seed=1, in_ch=5, out_ch=3, has_bn=False, bias_range=0.05):
    """He-normal N(0, 2/(k*k*cin)) weights, U(-bias_range, bias_range) biases (float32).

    With has_bn, the per-encoder-conv batch-norm statistics are drawn near identity:
    gamma U(0.8,1.2), beta U(-0.05,0.05), mean U(-0.1,0.1), var U(0.5,1.5).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    shapes = unet_layer_shapes(ch, in_ch, out_ch)
    for _, co, ci, k in shapes:
        std = np.sqrt(2.0 / (k * k * ci))
        parts.append(rng.normal(0.0, std, size=co * ci * k * k))
        parts.append(rng.uniform(-bias_range, bias_range, size=co))
    if has_bn:
        for name, co, _, _ in shapes:
            if name.startswith("enc"):
                parts.append(rng.uniform(0.8, 1.2, size=co))
                parts.append(rng.uniform(-0.05, 0.05, size=co))
                parts.append(rng.uniform(-0.1, 0.1, size=co))
                parts.append(rng.uniform(0.5, 1.5, size=co))
    return np.concatenate(parts).astype(np.float32)

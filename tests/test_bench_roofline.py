"""bench.py's roofline inputs: the U-Net's algorithmic FLOPs per pixel, and the DRAM traffic
that is reported only for the conv sources it was captured on (any change to them, or a
missing file, turns the figure into null)."""
import hashlib
import os
import shutil

import bench


def _tree(tmp_path):
    for rel in bench.CONV_TRAFFIC["sha256"]:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(bench.ROOT, rel), dst)


def test_traffic_follows_the_captured_sources(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    match = all(hashlib.sha256((tmp_path / rel).read_bytes()).hexdigest() == d
                for rel, d in bench.CONV_TRAFFIC["sha256"].items())
    assert bench.conv_traffic() == (bench.CONV_TRAFFIC["bytes_per_step"] if match else None)


def test_changed_or_missing_source_gives_null(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rel = next(iter(bench.CONV_TRAFFIC["sha256"]))
    with open(tmp_path / rel, "ab") as f:
        f.write(b"\n// changed\n")
    assert bench.conv_traffic() is None
    os.remove(tmp_path / rel)
    assert bench.conv_traffic() is None


def test_unet_flops_per_pixel_count_the_layer_plan():
    """The closed form equals a layer-by-layer count over the U-Net (Fig. 1): two 3x3 convs
    per encoder level (the first on the previous level's pooled output), two per decoder
    level (the first on the skip tensor concatenated with the upsampled deeper one), and
    the 1x1 head; 2 FLOPs per multiply-add, per full-resolution pixel."""
    for ch, in_ch in (((32, 64, 128, 256), 5), ((16, 32, 64), 5), ((8, 16), 3)):
        H = W = 2 ** (len(ch) + 2)
        macs, cin = 0, in_ch
        for l, c in enumerate(ch):                       # encoder
            px = (H >> l) * (W >> l)
            macs += 9 * cin * c * px + 9 * c * c * px
            cin = c
        for l in range(len(ch) - 2, -1, -1):             # decoder
            px = (H >> l) * (W >> l)
            macs += 9 * (ch[l] + ch[l + 1]) * ch[l] * px + 9 * ch[l] * ch[l] * px
        macs += ch[0] * 3 * H * W                        # head
        assert bench.unet_flops_per_px(ch, in_ch=in_ch) == 2.0 * macs / (H * W)
    assert bench.unet_flops_per_px((32, 64, 128, 256)) == 325632.0

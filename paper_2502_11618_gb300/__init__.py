"""GB300-native render path of "Real-time Neural Rendering of LiDAR Point Clouds"
(arXiv 2502.11618): uniform-grid culling, 1x1 projection into RGBDA, the depth-guided
filter and the U-Net, as hand-written sm_103a CUDA kernels behind the C ABI of
include/lnr.h.  This package is the thin Python binding of that library.
"""
from ._lib import (Renderer, LnrError, lib, SYMBOLS, FP32, BF16, FP8, STAGE_KEYS, STAGE_RGBDA_RAW,
                   STAGE_FILTERED, STAGE_UNET_IN, STAGE_CULL, LIB_PATH)

__all__ = ["Renderer", "LnrError", "lib", "SYMBOLS", "FP32", "BF16", "FP8", "STAGE_KEYS",
           "STAGE_RGBDA_RAW", "STAGE_FILTERED", "STAGE_UNET_IN", "STAGE_CULL", "LIB_PATH"]

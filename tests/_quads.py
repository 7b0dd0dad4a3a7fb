"""Row-major view of bf_forward's saved quads. The buffer keeps pixel (y, x)'s
quad at index ((y + (x mod 128)) mod H) * W + x for H >= 128 (row-major
below), the layout include/bf.h documents with bf_saved_bytes."""
import numpy as np


def rowmajor(sv):
    """[..., H, W, 4] quads as stored -> the same quads indexed by pixel."""
    a = sv.cpu().numpy() if hasattr(sv, "cpu") else np.asarray(sv)
    H, W = a.shape[-3], a.shape[-2]
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    sh = (xs & 127) if H >= 128 else 0
    idx = ((ys + sh) % H) * W + xs
    flat = a.reshape(a.shape[:-3] + (H * W, 4))
    return flat[..., idx, :]

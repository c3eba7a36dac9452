"""Oracle of the stereo-pair display composition -- TEST INFRASTRUCTURE.

Paper Sec. 3: post-processing turns the stereo pair into a display frame,
e.g. an anaglyph. Plain definitions in float32 numpy: colour anaglyph (L.r, R.g, R.b); grey
anaglyph (y(L), y(R), y(R)) with y = 0.299 r + 0.587 g + 0.114 b (the kernel
fuses the multiply-adds, so the grey mode agrees to a few ulps); side by side:
each output row is the left row followed by the right row.
"""
import numpy as np


def composite(L, R, mode):
    L = np.asarray(L, np.float32)
    R = np.asarray(R, np.float32)
    if mode == 0:
        return np.stack([L[..., 0], R[..., 1], R[..., 2]], axis=-1)
    if mode == 1:
        y = lambda a: (np.float32(0.299) * a[..., 0] + np.float32(0.587) * a[..., 1]) + np.float32(0.114) * a[..., 2]
        yl, yr = y(L), y(R)
        return np.stack([yl, yr, yr], axis=-1)
    if mode == 2:
        return np.concatenate([L, R], axis=1)
    raise ValueError(mode)

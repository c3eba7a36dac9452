"""Stereo display composition on the GPU vs the oracle (paper Sec. 3)."""
import numpy as np
import pytest

from oracle import post
from paper_1702_01530_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H", [(64, 48), (37, 23), (1, 1), (1920, 1080)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_composite_matches_oracle(W, H, mode):
    import torch
    from paper_1702_01530_gb300 import build
    build.build()
    rng = np.random.default_rng(W * 31 + H + mode)
    L = rng.random((H, W, 3), dtype=np.float32)
    R = rng.random((H, W, 3), dtype=np.float32)
    out = torch.empty((H, 2 * W if mode == 2 else W, 3), dtype=torch.float32, device="cuda")
    capi.rt_stereo_composite(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), W, H, mode, out)
    got = out.cpu().numpy()
    ref = post.composite(L, R, mode)
    if mode == 1:
        assert np.abs(got - ref).max() <= 4e-7
    else:
        assert np.array_equal(got, ref)

"""The blending network of Sec. 3.3 (a four-level U-Net), with seeded random
weights: the paper's trained weights are not available, so this exists to time
the whole per-frame path end to end, not to produce images worth looking at.

Its convolutions are PyTorch / cuDNN library calls in bfloat16; the
channels-last layout works too (convert the module and the input with
memory_format=torch.channels_last; the outputs are contiguous planes either
way).  The input assembly before it (`gvs.blend_features`) and the blend
after it (`gvs.blend`, Eqs. 4-5) are this library's kernels.

Output heads (readings; the paper gives no activations): w_k = sigmoid (Eq. 4
normalises by the sum over views anyway), w_BG = sigmoid, I_BG = sigmoid.
"""
from __future__ import annotations

import torch
import torch.nn as nn
import torch.nn.functional as F


def _block(cin: int, cout: int) -> nn.Sequential:
    return nn.Sequential(nn.Conv2d(cin, cout, 3, padding=1), nn.ReLU(inplace=True),
                         nn.Conv2d(cout, cout, 3, padding=1), nn.ReLU(inplace=True))


class BlendUNet(nn.Module):
    """Input [1, 9K + 1, H, W] (H, W divisible by 8); output planes w [K, H, W],
    w_BG [H, W], I_BG [3, H, W], each contiguous."""

    def __init__(self, n_views: int, widths=(32, 64, 128, 256), seed: int = 0):
        super().__init__()
        g = torch.random.fork_rng(devices=[])
        with g:
            torch.manual_seed(seed)
            self.K = n_views
            c_in = 9 * n_views + 1
            self.enc = nn.ModuleList()
            prev = c_in
            for w in widths:
                self.enc.append(_block(prev, w))
                prev = w
            self.dec = nn.ModuleList()
            for w_skip, w in zip(reversed(widths[:-1]), reversed(widths[:-1])):
                self.dec.append(_block(prev + w_skip, w))
                prev = w
            self.head = nn.Conv2d(prev, n_views + 4, 1)

    def forward(self, x: torch.Tensor):
        skips = []
        for i, blk in enumerate(self.enc):
            x = blk(x)
            if i < len(self.enc) - 1:
                skips.append(x)
                x = F.max_pool2d(x, 2)
        for blk in self.dec:
            x = F.interpolate(x, scale_factor=2.0, mode="nearest")
            x = blk(torch.cat([x, skips.pop()], dim=1))
        y = torch.sigmoid(self.head(x))[0]
        K = self.K
        return y[:K].contiguous(), y[K].contiguous(), y[K + 1:K + 4].contiguous()

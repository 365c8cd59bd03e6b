"""Plain CPU reference of the surrogate network's layers (PyTorch CPU, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the tests compare the
tensor-core convolutions, their backward passes and the training step of the
library against these definitions.  Inputs are taken exactly as the GPU sees
them (BF16 values widened to FP64); everything here is FP64.

Definitions (the library's documented network, include/lf_sur.h):
  conv(h, W)[p, o] = sum_{t, i} h[p + off_t, i] W[t, o, i],  off_t = (dy, dx),
  t = 3 (dy + 1) + (dx + 1), with h periodic in x and zero beyond y = 0, NY - 1.
"""
from __future__ import annotations

import numpy as np
import torch


def pad_xy(h: torch.Tensor) -> torch.Tensor:
    """[B, NY, NX, C] -> [B, NY + 2, NX + 2, C]: periodic columns, zero rows."""
    h = torch.cat([h[:, :, -1:], h, h[:, :, :1]], dim=2)
    z = torch.zeros_like(h[:, :1])
    return torch.cat([z, h, z], dim=1)


def conv3x3(h: torch.Tensor, W: torch.Tensor, bias=None) -> torch.Tensor:
    """h [B, NY, NX, CIN], W [9, COUT, CIN] -> [B, NY, NX, COUT] (FP64)."""
    B, NY, NX, _ = h.shape
    hp = pad_xy(h)
    out = 0
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        win = hp[:, 1 + dy:1 + dy + NY, 1 + dx:1 + dx + NX, :]
        out = out + torch.einsum("byxi,oi->byxo", win, W[t])
    if bias is not None:
        out = out + bias
    return out


def _store_bf16(a: torch.Tensor) -> torch.Tensor:
    """Value stored in BF16, gradient passed through unchanged."""
    return a + (a.to(torch.bfloat16).to(a.dtype) - a).detach()


def forward(x16: torch.Tensor, Ws, bs, x4=None, bf16_acts=False):
    """The network on normalised input x16 [B, NY, NX, 16] (channels 4.. zero);
    y = x4 + conv(h5)[..., :4] with x4 the unrounded input (x16[..., :4] when
    omitted).  With bf16_acts the activations are stored in BF16 between
    layers, as the documented network does.  Returns (y, h list, z list)."""
    st = _store_bf16 if bf16_acts else (lambda a: a)
    z1 = conv3x3(x16, Ws[0], bs[0])
    h = st(torch.relu(z1))
    hs, zs = [h], [z1]
    for l in range(1, 5):
        z = conv3x3(h, Ws[l], bs[l])
        h = st(h + torch.relu(z))
        hs.append(h)
        zs.append(z)
    z6 = conv3x3(h, Ws[5], bs[5])
    y = (x16[..., :4] if x4 is None else x4) + z6[..., :4]
    return y, hs, zs


def loss_and_grads(x16, y_target, Ws, bs, x4=None, bf16_acts=False):
    """MSE over all outputs and its gradients with respect to every weight and
    bias (autograd through the definitions above)."""
    Wt = [W.clone().requires_grad_(True) for W in Ws]
    bt = [b.clone().requires_grad_(True) for b in bs]
    y, _, _ = forward(x16, Wt, bt, x4=x4, bf16_acts=bf16_acts)
    loss = ((y - y_target) ** 2).mean()
    loss.backward()
    return float(loss.detach()), [W.grad for W in Wt], [b.grad for b in bt]


def bf16_round(a) -> np.ndarray:
    """Round FP32/FP64 values to the nearest BF16 (ties to even), as FP64."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()

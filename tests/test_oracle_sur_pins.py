"""Pins of the surrogate's CPU reference (oracle/sur_oracle.py): the tap-sum
convolution equals torch's conv2d with the lattice padding (periodic in x,
zero in y), and its autograd gradients equal central finite differences."""
import numpy as np
import torch
import torch.nn.functional as Fn

from oracle import sur_oracle as SO


def test_conv_matches_library_conv2d():
    g = torch.Generator().manual_seed(0)
    B, NY, NX, CI, CO = 2, 5, 7, 3, 4
    h = torch.randn((B, NY, NX, CI), generator=g, dtype=torch.float64)
    W = torch.randn((9, CO, CI), generator=g, dtype=torch.float64)
    ours = SO.conv3x3(h, W)
    # conv2d weight [CO, CI, 3, 3] with kernel index (dy + 1, dx + 1); NCHW input
    Wk = W.reshape(3, 3, CO, CI).permute(2, 3, 0, 1)
    x = h.permute(0, 3, 1, 2)
    x = Fn.pad(x, (1, 1, 0, 0), mode="circular")
    x = Fn.pad(x, (0, 0, 1, 1), mode="constant", value=0.0)
    ref = Fn.conv2d(x, Wk).permute(0, 2, 3, 1)
    assert torch.allclose(ours, ref, atol=1e-12)


def test_gradients_match_finite_differences():
    g = torch.Generator().manual_seed(1)
    B, NY, NX = 1, 3, 4
    shapes = [(16, 64), (64, 64), (64, 64), (64, 64), (64, 64), (64, 16)]
    Ws = [0.05 * torch.randn((9, co, ci), generator=g, dtype=torch.float64) for ci, co in shapes]
    bs = [0.05 * torch.randn((co,), generator=g, dtype=torch.float64) for _, co in shapes]
    x16 = torch.zeros((B, NY, NX, 16), dtype=torch.float64)
    x16[..., :4] = torch.randn((B, NY, NX, 4), generator=g, dtype=torch.float64)
    t = torch.randn((B, NY, NX, 4), generator=g, dtype=torch.float64)
    loss, gW, gb = SO.loss_and_grads(x16, t, Ws, bs)
    rng = np.random.default_rng(2)
    for l in (0, 2, 5):
        for _ in range(3):
            idx = tuple(int(rng.integers(0, n)) for n in Ws[l].shape)
            if l == 0 and idx[2] >= 4:
                continue
            eps = 1e-6
            Wp = [w.clone() for w in Ws]
            Wm = [w.clone() for w in Ws]
            Wp[l][idx] += eps
            Wm[l][idx] -= eps
            lp = float(((SO.forward(x16, Wp, bs)[0] - t) ** 2).mean())
            lm = float(((SO.forward(x16, Wm, bs)[0] - t) ** 2).mean())
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - float(gW[l][idx])) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, float(gW[l][idx]))

"""The surrogate's tensor-core kernels against the FP64 CPU reference
(oracle/sur_oracle.py), on BF16 inputs.  Products of BF16 values are exact in
FP32, so the accumulators differ from FP64 only by FP32 summation rounding;
BF16 outputs additionally carry one BF16 rounding (relative 2^-8)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import sur_oracle as SO  # noqa: E402
from paper_1102_3094_gb300 import lf  # noqa: E402

BF = torch.bfloat16


def _rand(shape, scale, g):
    return (scale * torch.randn(shape, generator=g, dtype=torch.float32)).to(BF)


@pytest.mark.parametrize("cin,cout,relu,use_resid", [(16, 64, 1, False), (64, 64, 1, True), (64, 16, 0, False)])
def test_conv3x3_forward(cin, cout, relu, use_resid):
    g = torch.Generator().manual_seed(cin * 100 + cout)
    B, NY, NX = 2, 5, 256
    h = _rand((B, NY, NX, cin), 1.0, g)
    W = _rand((9, cout, cin), 0.1, g)
    bias = (0.1 * torch.randn(cout, generator=g)).float()
    resid = _rand((B, NY, NX, cout), 1.0, g) if use_resid else None
    dev = "cuda"
    inp = lf.pad_nhwc(h).to(dev)
    out = torch.zeros((B, NY + 2, NX + 2, cout), dtype=BF, device=dev)
    zout = torch.zeros_like(out)
    res_d = lf.pad_nhwc(resid).to(dev) if use_resid else None
    x4 = torch.randn((B, NY, NX, 4), generator=g).float().to(dev) if cout == 16 else None
    y4 = torch.zeros((B, NY, NX, 4), dtype=torch.float32, device=dev) if cout == 16 else None
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    lf.lf_sur_conv3x3(B, NY, NX, cin, cout, inp, W.to(dev).contiguous(), bias.to(dev), relu, res_d, None, out,
                      None, zout, x4, y4, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    z_ref = SO.conv3x3(h.double(), W.double(), bias.double())
    ref = torch.relu(z_ref) if relu else z_ref
    if use_resid:
        ref = ref + resid.double()
    zo = zout.cpu().double()
    oo = out.cpu().double()
    # interior
    tol = 2.0 ** -7
    np.testing.assert_allclose(zo[:, 1:-1, 1:-1].numpy(), z_ref.numpy(), rtol=tol, atol=tol * 0.1)
    np.testing.assert_allclose(oo[:, 1:-1, 1:-1].numpy(), ref.numpy(), rtol=tol, atol=tol * 0.1)
    # halo: periodic columns, untouched (zero) rows
    assert torch.equal(oo[:, 1:-1, 0], oo[:, 1:-1, NX])
    assert torch.equal(oo[:, 1:-1, NX + 1], oo[:, 1:-1, 1])
    assert float(oo[:, 0].abs().max()) == 0.0 and float(oo[:, -1].abs().max()) == 0.0
    if cout == 16:
        y_ref = x4.cpu().double() + z_ref[..., :4]
        scale = (SO.conv3x3(h.double().abs(), W.double().abs()) [..., :4]).numpy() + 1.0
        assert np.all(np.abs(y4.cpu().double().numpy() - y_ref.numpy()) <= 1e-5 * scale)

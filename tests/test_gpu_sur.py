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


@pytest.mark.parametrize("cin,cout,relu,use_resid,shape", [
    (16, 64, 1, False, (2, 5, 256)), (64, 64, 1, True, (2, 5, 256)), (64, 16, 0, False, (2, 5, 256)),
    (64, 64, 1, True, (3, 121, 256)),     # more row runs than SMs: CTAs march over several
    (16, 64, 1, False, (1, 1, 128)),      # one row: prologue and drain only
    # the residual is the layer's own input (the surrogate's residual layers):
    # it is read from the input rows already in shared memory
    (64, 64, 1, "self", (2, 5, 256)), (64, 64, 1, "self", (3, 121, 256)), (64, 64, 0, "self", (1, 1, 128)),
    (64, 64, 1, "self", (2, 2, 128)),
])
def test_conv3x3_forward(cin, cout, relu, use_resid, shape):
    g = torch.Generator().manual_seed(cin * 100 + cout)
    B, NY, NX = shape
    h = _rand((B, NY, NX, cin), 1.0, g)
    W = _rand((9, cout, cin), 0.1, g)
    bias = (0.1 * torch.randn(cout, generator=g)).float()
    resid = h if use_resid == "self" else _rand((B, NY, NX, cout), 1.0, g) if use_resid else None
    dev = "cuda"
    inp = lf.pad_nhwc(h).to(dev)
    out = torch.zeros((B, NY + 2, NX + 2, cout), dtype=BF, device=dev)
    zout = torch.zeros_like(out)
    res_d = inp if use_resid == "self" else lf.pad_nhwc(resid).to(dev) if use_resid else None
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


@pytest.mark.parametrize("cin,cout,shape", [
    (16, 64, (2, 3, 128)), (64, 64, (2, 3, 128)), (64, 16, (2, 3, 128)),
    (64, 64, (3, 41, 256)), (16, 64, (3, 41, 256)), (64, 16, (3, 41, 256)),   # runs cross images and blocks
])
def test_conv3x3_weight_gradient(cin, cout, shape):
    g_ = torch.Generator().manual_seed(7 * cin + cout)
    B, NY, NX = shape
    h = _rand((B, NY, NX, cin), 1.0, g_)
    gr = _rand((B, NY, NX, cout), 1.0, g_)
    dev = "cuda"
    dW = torch.zeros((9, cout, cin), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    lf.lf_sur_conv3x3_wgrad(B, NY, NX, cin, cout, lf.pad_nhwc(h).to(dev), lf.pad_nhwc(gr).to(dev), dW, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    hp = SO.pad_xy(h.double())
    ref = torch.zeros((9, cout, cin), dtype=torch.float64)
    absr = torch.zeros_like(ref)
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        win = hp[:, 1 + dy:1 + dy + NY, 1 + dx:1 + dx + NX, :]
        ref[t] = torch.einsum("byxi,byxo->oi", win, gr.double())
        absr[t] = torch.einsum("byxi,byxo->oi", win.abs(), gr.double().abs())
    assert np.all(np.abs(dW.cpu().double().numpy() - ref.numpy()) <= 1e-5 * absr.numpy() + 1e-30)


def _oracle_params(p):
    """split the flat FP32 parameter vector into BF16-rounded weights and FP32 biases"""
    Ws, bs, off = [], [], 0
    for cin, cout in [(16, 64), (64, 64), (64, 64), (64, 64), (64, 64), (64, 16)]:
        n = 9 * cout * cin
        Ws.append(torch.tensor(SO.bf16_round(p[off:off + n]).reshape(9, cout, cin)))
        off += n
        bs.append(torch.tensor(p[off:off + cout].astype(np.float64)))
        off += cout
    return Ws, bs


def test_network_gradients_match_oracle():
    B, NY, NX = 2, 6, 128
    g_ = torch.Generator().manual_seed(3)
    x = torch.randn((B, 4, NY, NX), generator=g_).float()
    y = x + 0.1 * torch.randn((B, 4, NY, NX), generator=g_).float()
    sur = lf.Surrogate(NY, NX, B, scale=[1, 1, 1, 1], offset=[0, 0, 0, 0], seed=11)
    p = sur.get_params()
    p[-16:] = 0.05 * np.random.default_rng(1).standard_normal(16)      # nonzero last bias
    sur.set_params(p)
    p = sur.get_params()
    loss_gpu, g_gpu = sur.grads(x.cuda(), y.cuda())
    Ws, bs = _oracle_params(p)
    x4 = x.permute(0, 2, 3, 1).double()
    x16 = torch.zeros((B, NY, NX, 16), dtype=torch.float64)
    x16[..., :4] = torch.tensor(SO.bf16_round(x4.numpy()))
    t4 = y.permute(0, 2, 3, 1).double()
    loss_ref, gW, gb = SO.loss_and_grads(x16, t4, Ws, bs, x4=x4, bf16_acts=True)
    assert abs(loss_gpu / loss_ref - 1) < 1e-3, (loss_gpu, loss_ref)
    off = 0
    for l, (gw_r, gb_r) in enumerate(zip(gW, gb)):
        n = gw_r.numel()
        gw_g = torch.tensor(g_gpu[off:off + n].astype(np.float64)).reshape(gw_r.shape)
        off += n
        gb_g = torch.tensor(g_gpu[off:off + gb_r.numel()].astype(np.float64))
        off += gb_r.numel()
        for a, b_, name in ((gw_g, gw_r, "W"), (gb_g, gb_r, "b")):
            if l == 0 and name == "W":
                b_ = b_[..., :4].contiguous()
                a = a[..., :4].contiguous()
            rel = float((a - b_).norm() / b_.norm())
            cos = float((a * b_).sum() / (a.norm() * b_.norm()))
            assert rel < 0.05 and cos > 0.998, (l, name, rel, cos)
    sur.close()


def _trajectory_pairs(nx, ny, K, npairs, seed):
    sim = lf.Lattice(nx=nx, ny=ny, precision="fp32", xi=0.01, seed=seed)
    sim.step(200)
    xs, ys = [], []
    def state():
        return torch.stack([sim.get(n, "fp32", device=True) for n in ("phi", "T", "ux", "uy")])
    prev = state()
    for _ in range(npairs):
        sim.step(K)
        cur = state()
        xs.append(prev)
        ys.append(cur)
        prev = cur
    sim.close()
    return torch.stack(xs), torch.stack(ys)


def test_training_lowers_the_loss():
    NY, NX, K = 64, 128, 10
    x, y = _trajectory_pairs(NX, NY, K, 24, seed=5)
    flat = x.permute(1, 0, 2, 3).reshape(4, -1)
    scale = flat.std(dim=1).clamp_min(1e-3).cpu().numpy()
    offset = flat.mean(dim=1).cpu().numpy()
    sur = lf.Surrogate(NY, NX, 8, scale=scale, offset=offset, seed=3)
    l0 = sur.loss(x[:8], y[:8])
    for it in range(60):
        i = (it * 8) % 24
        sur.train_step(x[i:i + 8].contiguous(), y[i:i + 8].contiguous(), 1e-3)
    l1 = sur.loss(x[:8], y[:8])
    assert np.isfinite(l1) and l1 < 0.7 * l0, (l0, l1)
    sur.close()


def test_interleaved_run_falls_back_to_plain():
    NY, NX, K = 64, 128, 10
    sur = lf.Surrogate(NY, NX, 1, scale=[0.3, 0.3, 0.01, 0.01], offset=[0, 0.8, 0, 0], seed=3)
    a = lf.Lattice(nx=NX, ny=NY, precision="fp32", xi=0.01, seed=9)
    b = lf.Lattice(nx=NX, ny=NY, precision="fp32", xi=0.01, seed=9)
    a.step(100)
    b.step(100)
    rep = sur.run(a, K, 6, 1, 1e-9)           # every surrogate window checked and rejected
    b.step(6 * K)
    assert rep["windows_done"] == 6 and rep["shadow_checks"] == 3 and rep["fallbacks"] == 3
    assert a.step_count == b.step_count
    pa, pb = a.get("phi", "fp32"), b.get("phi", "fp32")
    assert np.abs(pa - pb).max() <= 1e-4 * np.abs(pb).max()
    # last layer zero: the network maps the state to itself (a usable
    # prediction); with no threshold every such prediction is kept
    p = sur.get_params()
    p[-(9 * 16 * 64 + 16):] = 0.0
    sur.set_params(p)
    before = a.get("phi", "fp32")
    rep2 = sur.run(a, K, 4, 1, 1e30)
    assert rep2["fallbacks"] == 0 and rep2["rejected"] == 0
    assert rep2["surrogate_windows"] == 2 and rep2["shadow_checks"] == 2 and rep2["windows_done"] == 4
    assert np.isfinite(a.get("phi", "fp32")).all() and not np.array_equal(a.get("phi", "fp32"), before)
    for o in (a, b, sur):
        o.close()

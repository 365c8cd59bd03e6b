"""lf_diag_sums_noalloc: the diagnostics sums for callers that cannot
allocate device memory at the call (inside graph capture, allocation-free
loops, frameworks that own all device memory).  Its output must match the
allocating entry points (lf_diag, lf_diag_layers) on the same state, on two
calls in a row (the calls share one scratch array in the library).  This file
is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1102_3094_gb300 import lf  # noqa: E402

TOL = 1e-12


def _fields(sim, dt):
    phi = sim.get("phi", dt, device=True)
    T = sim.get("T", dt, device=True)
    mom = torch.zeros((4,) + sim.shape, dtype=phi.dtype, device=phi.device)
    for i, name in enumerate(("rho", "ux", "uy", "uz")):
        if name == "uz" and len(sim.shape) == 2:
            continue
        mom[i] = sim.get(name, dt, device=True)
    return phi, T, mom


@pytest.mark.parametrize("case", [dict(d=2, nx=70, ny=37, precision="fp32"),
                                  dict(d=2, nx=64, ny=64, precision="fp64"),
                                  dict(d=3, nx=20, ny=12, nz=9, precision="fp32")])
def test_noalloc_matches_allocating_diagnostics(case):
    sim = lf.Lattice(xi=0.01, **case)
    sim.step(40)
    torch.cuda.synchronize()
    ref = sim.diag()
    ref_layers = sim.layers()
    dt = case["precision"]
    phi, T, mom = _fields(sim, dt)
    d = case["d"]
    L = sim.shape[0]
    want = np.array([ref["mass"], ref["phi_sum"], *ref["mom"], *ref["grad2"], ref["free_energy"],
                     ref["umax"] ** 2])
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((10 + L,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lf.lf_diag_sums_noalloc(d, case["nx"], case["ny"], case.get("nz", 1), 1,
                                     lf.LF_FP64 if dt == "fp64" else lf.LF_FP32, phi.data_ptr(), T.data_ptr(),
                                     mom.data_ptr(), 1.0, -0.025, 0.02, 1.0, out.data_ptr(), stream.cuda_stream)
        assert rc == 0, (call, lf.strerror(rc))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = np.maximum(np.abs(want), 1e-300)
        assert np.all(np.abs(got[:10] - want) <= TOL * np.maximum(scale, np.abs(want).max() * 1e-3)), (call, got[:10], want)
        np.testing.assert_allclose(got[10:], ref_layers, rtol=TOL, atol=TOL)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    rc = lf.lf_diag_sums_noalloc(2, 8, 4097, 1, 1, lf.LF_FP64, p, p, p, 1.0, -0.025, 0.02, 1.0, p, 0)
    assert rc == lf.LF_EINVAL
    rc = lf.lf_diag_sums_noalloc(3, 8, 8, 5000, 1, lf.LF_FP32, p, p, p, 1.0, -0.025, 0.02, 1.0, p, 0)
    assert rc == lf.LF_EINVAL
    # an extent whose product with the others wraps to a small number
    rc = lf.lf_diag_sums_noalloc(2, (1 << 62) + 1, 4, 1, 1, lf.LF_FP64, p, p, p, 1.0, -0.025, 0.02, 1.0, p, 0)
    assert rc == lf.LF_EINVAL

"""Implicit temperature step (lf_set_t_solver) against the FP64 reference
(oracle/t_implicit.py): one backward-Euler step of T per time step, the phi
and f update of the same step unchanged (it uses T(t))."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from oracle import t_implicit as TI  # noqa: E402
from paper_1102_3094_gb300 import lf  # noqa: E402

from test_gpu_step import TOL, make_pair, relerr, to_oracle_f  # noqa: E402

CASES = [
    dict(nx=64, ny=48, xi=5.0),                              # held wall layers
    dict(nx=40, ny=33, t_wall_mode=1, xi=30.0),              # halfway ghosts
    dict(nx=48, ny=20, walls=0, xi=2.0),                     # fully periodic
    dict(nx=36, ny=3, xi=100.0),                             # one unknown layer
    dict(d=3, nx=12, ny=10, nz=9, xi=4.0),                   # 3D, walls along z
    dict(d=3, nx=8, ny=6, nz=10, walls=0, xi=1.5),           # 3D periodic
    dict(d=3, nx=10, ny=12, nz=7, t_wall_mode=1, xi=20.0),   # 3D halfway
]


def _oracle_step(cfg, st, xi):
    """phi and f by the oracle with the temperature frozen, T by the implicit reference."""
    cfg0 = type(cfg).from_buffer_copy(cfg)
    cfg0.xi = 0.0
    cfg0.nsub = 1
    out = O.step(O.State(cfg0, st.f, st.phi, st.T))
    Tn = TI.implicit_step(st.T, xi, cfg.T_w, cfg.walls, cfg.t_wall_mode, cfg.stencil)   # wall normal on axis 0
    return out.phi, Tn, out.f


@pytest.mark.parametrize("stencil", ["compact", "isotropic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(str(c.get(k, "")) for k in ("nx", "ny", "nz")) + str(c))
def test_implicit_temperature_step(case, prec, stencil):
    sim, cfg, st = make_pair(case, prec, stencil=stencil)
    sim.set_t_solver("implicit")
    sim.step(1)
    phi_w, T_w, f_w = _oracle_step(cfg, st, case["xi"])
    d = case.get("d", 2)
    tol = TOL[prec]
    assert relerr(sim.get("T"), T_w) < tol, relerr(sim.get("T"), T_w)
    assert relerr(sim.get("phi"), phi_w) < tol
    assert relerr(to_oracle_f(sim.get("pop"), d), f_w) < tol
    sim.close()


@pytest.mark.parametrize("stencil", ["compact", "isotropic"])
def test_implicit_multistep_fp64(stencil):
    case = dict(nx=32, ny=24, xi=8.0)
    sim, cfg, st = make_pair(case, "fp64", stencil=stencil)
    sim.set_t_solver("implicit")
    for _ in range(10):
        phi, T, f = _oracle_step(cfg, st, case["xi"])
        st = O.State(cfg, f, phi, T)
    sim.step(10)
    assert relerr(sim.get("T"), st.T) < 1e-11
    assert relerr(sim.get("phi"), st.phi) < 1e-11
    sim.close()


def test_unsupported_size_is_refused():
    sim = lf.Lattice(nx=37, ny=16, precision="fp32", xi=2.0)    # 37 is a prime above 31
    with pytest.raises(lf.LFError) as ei:
        sim.set_t_solver("implicit")
    assert ei.value.code == lf.LF_EINVAL
    sim.set_t_solver("explicit")
    sim.close()

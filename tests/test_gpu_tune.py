"""The autotuner (lf_tune, include/lf.h): it leaves the context's state
untouched, picks one of the variants that compute the same step, the step it
picks still matches the FP64 oracle, and a second call with the same lattice
key returns the cached choice."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1102_3094_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1102_3094_gb300 import lf  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-6}
VARIANTS = {lf.LF_VARIANT_MARCH, lf.LF_VARIANT_TILE, lf.LF_VARIANT_MARCH2, lf.LF_VARIANT_SPLIT3}

CASES = [
    (dict(nx=130, ny=70, xi=0.01), "fp32", "compact"),
    (dict(nx=64, ny=40, xi=0.5), "fp64", "compact"),
    (dict(nx=64, ny=32, xi=0.01), "fp32", "isotropic"),
    (dict(d=3, nx=20, ny=16, nz=12, xi=0.01), "fp32", "compact"),
    (dict(d=3, nx=14, ny=11, nz=9, xi=0.3, t_wall_mode=1), "fp32", "isotropic"),
]


def _to_oracle_f(f_lib, d):
    e, _ = lf.lf_lattice(d)
    eo, _ = O.velocity_set(d)
    out = np.empty_like(f_lib)
    for i, v in enumerate(e):
        out[int(np.where((eo == v).all(1))[0][0])] = f_lib[i]
    return out


def _relerr(got, want):
    s = np.abs(want).max()
    return np.abs(got - want).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("case,prec,stencil", CASES, ids=lambda v: str(v))
def test_tune_keeps_state_and_parity(case, prec, stencil):
    d = case.get("d", 2)
    sim = lf.Lattice(precision=prec, stencil=stencil, **case)
    dt = np.float64 if prec == "fp64" else np.float32
    phi, T, r = synth.random_state(sim.shape, sim.Q, 5, dtype=dt)
    _, w = lf.lf_lattice(d)
    if case.get("t_wall_mode", 0) == 0:
        T[0] = 0.5
        T[-1] = 0.5
    sim.set("phi", phi)
    sim.set("T", T)
    sim.set("pop", (w.reshape((-1,) + (1,) * len(sim.shape)) * (1 + r)).astype(dt))
    before = {k: sim.get(k) for k in ("phi", "T", "pop")}
    variant, param, ms = sim.tune(reps=2)
    assert variant in VARIANTS and param >= 0 and ms > 0
    for k, v in before.items():
        np.testing.assert_array_equal(sim.get(k), v, err_msg=k)
    assert sim.step_count == 0
    cfg = O.make_cfg(d=d, nx=case["nx"], ny=case["ny"], nz=case.get("nz", 1), xi=case["xi"],
                     t_wall_mode=case.get("t_wall_mode", 0), stencil=int(stencil == "isotropic"))
    st = O.State(cfg, _to_oracle_f(before["pop"], d), before["phi"], before["T"])
    sim.step(1)
    ref = O.step(st)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", _to_oracle_f(sim.get("pop"), d), ref.f)):
        assert _relerr(got, want) < TOL[prec], (name, variant, param, _relerr(got, want))
    # a second lattice with the same key takes the cached choice
    other = lf.Lattice(precision=prec, stencil=stencil, seed=9, **case)
    assert other.tune(reps=2) == (variant, param, ms)
    other.close()
    sim.close()

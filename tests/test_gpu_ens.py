"""Batched ensembles (include/lf_ens.h): every run of an ensemble, advanced
by the graph-replayed persistent launch, must equal the same run advanced
alone by lf_step with the same kernel and row split, bit for bit (the per-site
arithmetic is shared code)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1102_3094_gb300 import lf  # noqa: E402

MEMBERS = [
    dict(nx=64, ny=64, xi=0.01, tau=1.0, seed=11),
    dict(nx=96, ny=80, xi=0.5, tau=0.6, seed=12),            # 3 temperature sub-steps
    dict(nx=130, ny=70, xi=1e-3, tau=3.0, seed=13),
    dict(nx=40, ny=24, xi=math.inf, tau=1.0, seed=14),       # instantaneous quench
    dict(nx=33, ny=17, xi=0.2, tau=0.8, seed=15, walls=0),   # periodic
    dict(nx=128, ny=128, xi=1.0, tau=1.0, seed=16, t_wall_mode=1),   # 5 sub-steps, halfway T
]


def _alone(m, phases):
    """The run advanced alone: phases = [(steps, march2 param), ...]."""
    kw = {k: v for k, v in m.items()}
    sim = lf.Lattice(precision="fp32", **kw)
    for steps, rows in phases:
        sim.set_variant("march2", rows)
        sim.step(steps)
    return sim


def _compare(ens, steps, before=None):
    """before: (steps, shape param per run) taken before the current shapes."""
    for r, m in enumerate(MEMBERS):
        phases = [(steps, ens.param(r))]
        if before is not None:
            phases = [(before[0], before[1][r]), (steps - before[0], ens.param(r))]
        ref = _alone(m, phases)
        run = ens.run(r)
        for name in ("phi", "T", "pop"):
            np.testing.assert_array_equal(run.get(name, "fp32"), ref.get(name, "fp32"), err_msg=f"run {r} {name}")
        assert run.step_count == ref.step_count == steps
        ref.close()


def test_ensemble_equals_single_runs():
    ens = lf.Ensemble(MEMBERS)
    ens.step(7)          # odd: single-step graphs and the two-step graph
    ens.step(10)
    _compare(ens, 17)
    d = ens.run(1).diag()
    assert d["rc"] == 0 and d["mach"] < 0.1
    ens.close()


def test_ensemble_after_tuning():
    ens = lf.Ensemble(MEMBERS)
    ens.step(3)
    params0 = [ens.param(r) for r in range(len(MEMBERS))]
    ens.tune(reps=3)
    rows = [ens.rows(r) for r in range(len(MEMBERS))]
    assert all(r >= 1 for r in rows)
    ens.step(6)
    _compare(ens, 9, before=(3, params0))
    ens.close()


def test_ensemble_run_refuses_lf_step():
    ens = lf.Ensemble(MEMBERS[:2])
    ctx = lf.lf_ens_run(ens.ens, 0)
    with pytest.raises(lf.LFError) as ei:
        lf.lf_step(ctx, 1)
    assert ei.value.code == lf.LF_EINVAL
    ens.close()


ISO_MEMBERS = [
    dict(nx=64, ny=64, xi=0.01, tau=1.0, seed=21, stencil="isotropic"),
    dict(nx=96, ny=80, xi=0.5, tau=0.6, seed=22, stencil="isotropic", t_wall_mode=1),   # 3 sub-steps, halfway T
    dict(nx=130, ny=70, xi=1e-3, tau=3.0, seed=23),                                    # compact, in the same launch
    dict(nx=33, ny=17, xi=0.2, tau=0.8, seed=24, walls=0, stencil="isotropic"),         # periodic, ragged strips
]


def test_isotropic_runs_in_an_ensemble_equal_single_runs():
    """Runs with the isotropic stencils (two-lane isotropic march items) and a
    compact run (packed march items) in one ensemble, each equal bit for bit
    to the run stepped alone with the ensemble's shape."""
    ens = lf.Ensemble(ISO_MEMBERS)
    ens.tune(reps=2)                     # shapes of every (lattice, stencil) class
    ens.step(5)
    ens.step(6)
    for r, m in enumerate(ISO_MEMBERS):
        ref = lf.Lattice(precision="fp32", **m)
        ref.set_variant("march2", ens.param(r))
        ref.step(11)
        run = ens.run(r)
        for name in ("phi", "T", "pop"):
            np.testing.assert_array_equal(run.get(name, "fp32"), ref.get(name, "fp32"), err_msg=f"run {r} {name}")
        ref.close()
    ens.close()


# ---- every member against the FP64 oracle ----------------------------------
from oracle import oracle as O  # noqa: E402
from paper_1102_3094_gb300 import synth  # noqa: E402

ORACLE_MEMBERS = [
    dict(nx=64, ny=40, xi=0.01, tau=1.0, seed=31),                                  # compact, walls
    dict(nx=70, ny=37, xi=0.5, tau=0.6, seed=32, t_wall_mode=1),                    # 3 sub-steps, halfway T
    dict(nx=33, ny=17, xi=math.inf, tau=3.0, seed=33),                              # instantaneous quench
    dict(nx=41, ny=23, xi=0.2, tau=0.6, seed=34, walls=0),                          # periodic, 2 sub-steps
    dict(nx=56, ny=30, xi=0.01, tau=3.0, seed=35, stencil="isotropic"),             # isotropic row-march items
    dict(nx=47, ny=29, xi=0.7, tau=0.6, seed=36, stencil="isotropic", walls=0),     # isotropic, periodic, 4 sub-steps
    dict(nx=120, ny=3, xi=0.01, tau=1.0, seed=37),                                  # thinner than the halo
]


def _oracle_cfg(m):
    return O.make_cfg(d=2, nx=m["nx"], ny=m["ny"], walls=m.get("walls", 1), t_wall_mode=m.get("t_wall_mode", 0),
                      xi=m["xi"], tau=m["tau"], seed=m["seed"], stencil=int(m.get("stencil") == "isotropic"))


def _to_oracle_f(f_lib):
    e, _ = lf.lf_lattice(2)
    eo, _ = O.velocity_set(2)
    out = np.empty_like(f_lib)
    for i, v in enumerate(e):
        out[int(np.where((eo == v).all(1))[0][0])] = f_lib[i]
    return out


def _relerr(got, want):
    s = np.abs(want).max()
    return np.abs(got - want).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("tuned", [False, True])
def test_ensemble_members_match_oracle_one_step(tuned):
    """Every member of a mixed ensemble (both stencils, n_sub > 1, xi = inf,
    periodic and walled, tau = 0.6 .. 3, a lattice thinner than the halo),
    set to a random state, advanced by one batched step and compared element
    by element with one FP64 oracle step from the same (FP32-rounded) state:
    within 2e-6 max-norm relative error on f, phi and T."""
    ens = lf.Ensemble(ORACLE_MEMBERS)
    if tuned:
        ens.tune(reps=2)
    states = []
    _, w = lf.lf_lattice(2)
    for r, m in enumerate(ORACLE_MEMBERS):
        run = ens.run(r)
        phi, T, rr = synth.random_state(run.shape, 9, 100 + r, dtype=np.float32)
        if m.get("walls", 1) and m.get("t_wall_mode", 0) == 0:
            T[0] = 0.5
            T[-1] = 0.5
        f = (w.reshape(-1, 1, 1) * (1 + rr)).astype(np.float32)
        run.set("phi", phi)
        run.set("T", T)
        run.set("pop", f)
        states.append(O.State(_oracle_cfg(m), _to_oracle_f(run.get("pop")), run.get("phi"), run.get("T")))
    ens.step(1)
    for r, m in enumerate(ORACLE_MEMBERS):
        run = ens.run(r)
        want = O.step(states[r])
        for name, got, ref in (("phi", run.get("phi"), want.phi), ("T", run.get("T"), want.T),
                               ("pop", _to_oracle_f(run.get("pop")), want.f)):
            assert _relerr(got, ref) < 2e-6, (r, m, name, _relerr(got, ref))
    ens.close()


def test_ensemble_members_match_oracle_many_steps():
    """The same members from their initial quench, 40 batched steps, against
    40 FP64 oracle steps from the FP32-rounded initial state; FP32 rounding
    accumulates over the steps, so the bound is 40 x the one-step 2e-6."""
    ens = lf.Ensemble(ORACLE_MEMBERS)
    starts = []
    for r, m in enumerate(ORACLE_MEMBERS):
        run = ens.run(r)
        starts.append(O.State(_oracle_cfg(m), _to_oracle_f(run.get("pop")), run.get("phi"), run.get("T")))
    ens.step(40)
    for r, m in enumerate(ORACLE_MEMBERS):
        run = ens.run(r)
        want = O.run(starts[r], 40)
        for name, got, ref in (("phi", run.get("phi"), want.phi), ("T", run.get("T"), want.T),
                               ("pop", _to_oracle_f(run.get("pop")), want.f)):
            assert _relerr(got, ref) < 40 * 2e-6, (r, m, name, _relerr(got, ref))
    ens.close()


def test_prune_retires_nonfinite_runs():
    """A run that diverges (tau = 0.6 with an instantaneous quench: the method
    itself goes non-finite at these parameters) is retired by lf_ens_prune:
    its step count stops, while the other runs keep stepping and still equal
    the same runs stepped alone."""
    members = [dict(nx=64, ny=64, xi=math.inf, tau=0.6, seed=41),
               dict(nx=70, ny=37, xi=0.01, tau=1.0, seed=42),
               dict(nx=48, ny=40, xi=0.5, tau=3.0, seed=43, stencil="isotropic")]
    ens = lf.Ensemble(members)
    ens.step(600)
    nonfinite = [bool(ens.run(r).diag()["nonfinite"]) for r in range(len(members))]
    assert nonfinite[0] and not nonfinite[1] and not nonfinite[2]
    assert ens.prune() == 2
    assert [ens.active(r) for r in range(3)] == [False, True, True]
    ens.step(7)
    assert ens.run(0).step_count == 600
    for r in (1, 2):
        assert ens.run(r).step_count == 607
        ref = lf.Lattice(precision="fp32", **members[r])
        ref.set_variant("march2", ens.param(r))
        ref.step(607)
        for name in ("phi", "T", "pop"):
            np.testing.assert_array_equal(ens.run(r).get(name, "fp32"), ref.get(name, "fp32"), err_msg=f"{r} {name}")
        ref.close()
    ens.close()

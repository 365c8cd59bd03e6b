"""GPU parity of the fused step kernels against the FP64 oracle, through the
C ABI.  Tolerances (max-norm relative error per field, on f (full, not the
deviations), phi, T, mu, F): 1e-12 in FP64, 2e-6 in FP32, from an identical
state, one step."""
import math
import os
import tempfile

import numpy as np
import pytest

from oracle import diag as D
from oracle import oracle as O
from paper_1102_3094_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1102_3094_gb300 import lf  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-6}


def relerr(got, want):
    s = np.abs(want).max()
    return np.abs(got - want).max() / (s if s > 0 else 1.0)


def perm_to_oracle(d):
    """index in the oracle's order for each library population."""
    e, _ = lf.lf_lattice(d)
    eo, _ = O.velocity_set(d)
    return [int(np.where((eo == v).all(1))[0][0]) for v in e]


def to_oracle_f(f_lib, d):
    out = np.empty_like(f_lib)
    for i, j in enumerate(perm_to_oracle(d)):
        out[j] = f_lib[i]
    return out


VARIANTS = {"march": ("march", 0), "march-h5": ("march", 5), "tile": ("tile", 0),
            "march2": ("march2", 0), "march2-h5": ("march2", 5), "march2-h1": ("march2", 1),
            "march2-n64": ("march2", 1 << 16), "march-h1": ("march", 1), "march-n64-h3": ("march", (1 << 16) | 3)}


def make_pair(case, prec, seed=11, variant="march", stencil="compact"):
    """A GPU lattice and an oracle config with the same parameters, the GPU set
    to a random state; returns (sim, cfg, oracle_state_read_back)."""
    kw = dict(synth.BASE)
    kw.update(case)
    d = kw.get("d", 2)
    sim = lf.Lattice(precision=prec, **{k: v for k, v in kw.items() if k not in ("d",)}, d=d, stencil=stencil)
    sim.set_variant(*VARIANTS[variant])
    cfg = O.make_cfg(stencil=int(stencil == "isotropic"), d=d, nx=kw["nx"], ny=kw["ny"], nz=kw.get("nz", 1), walls=kw["walls"],
                     t_wall_mode=kw["t_wall_mode"], hydro=kw["hydro"], b=kw["b"], kappa=kw["kappa"],
                     c=kw["c"], Gamma=kw["Gamma"], Tc=kw["Tc"], T0=kw["T0"], T_w=kw["T_w"], xi=kw["xi"],
                     tau=kw["tau"], n0=kw["n0"], phi_amp=kw["phi_amp"], seed=kw.get("seed", 1))
    dt = np.float64 if prec == "fp64" else np.float32
    phi, T, r = synth.random_state(sim.shape, sim.Q, seed, dtype=dt)
    _, w = lf.lf_lattice(d)
    f = (w.reshape((-1,) + (1,) * len(sim.shape)) * (1 + r)).astype(dt)
    if kw["walls"] and kw["t_wall_mode"] == 0:
        T[0] = kw["T_w"]
        T[-1] = kw["T_w"]
    sim.set("phi", phi)
    sim.set("T", T)
    sim.set("pop", f)
    st = O.State(cfg, to_oracle_f(sim.get("pop"), d), sim.get("phi"), sim.get("T"))
    return sim, cfg, st


CASES = [
    dict(nx=64, ny=64, xi=0.01),                                  # whole tiles
    dict(nx=70, ny=37, xi=0.01),                                  # ragged in x and y
    dict(nx=5, ny=3, xi=0.01),                                    # smaller than one tile and the halo
    dict(nx=48, ny=20, walls=0, xi=0.01),                         # fully periodic
    dict(nx=33, ny=17, t_wall_mode=1, xi=0.5),                    # halfway T ghost, 3 T sub-steps
    dict(nx=40, ny=24, hydro=0, xi=0.1),                          # no hydrodynamics
    dict(nx=130, ny=70, tau=0.6, xi=1e-3),                        # several tiles, low viscosity
    dict(nx=36, ny=30, xi=math.inf, tau=3.0),                     # instantaneous quench
    dict(nx=3, ny=2, xi=0.01),                                    # thinner than every halo: the
    dict(nx=2, ny=3, walls=0, xi=0.01),                           # index maps' general path
]


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(str(c[k]) for k in ("nx", "ny")) + str(c))
def test_aux_and_step_parity(case, prec, variant):
    sim, cfg, st = make_pair(case, prec, variant=variant)
    _check_aux_and_step(sim, st, prec)


@pytest.mark.parametrize("variant", ["march", "march-h5", "march-h1", "march-n64-h3", "march2", "march2-h5", "march2-h1",
                                     "march2-n64", "tile"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(str(c[k]) for k in ("nx", "ny")) + str(c))
def test_isotropic_stencil_parity(case, prec, variant):
    """Isotropic 9-point stencils: the row march with sliding row sums, one
    lane (LF_VARIANT_MARCH) and, in FP32, two packed lanes (LF_VARIANT_MARCH2;
    FP64 runs the one-lane march), segments of the model's height and of 5, 1
    and 3 rows, 128- and 64-thread strips; and the tile kernel."""
    sim, cfg, st = make_pair(case, prec, variant=variant, stencil="isotropic")
    _check_aux_and_step(sim, st, prec)


@pytest.mark.parametrize("variant", ["march", "tile"])
def test_isotropic_multistep_fp64(variant):
    """200 coupled steps with the isotropic stencils: walls with the halfway T
    ghost and nsub = 2, then a fully periodic lattice."""
    for kw in (dict(nx=64, ny=48, t_wall_mode=1, xi=0.3), dict(nx=40, ny=36, walls=0, xi=0.01)):
        sim = lf.Lattice(precision="fp64", **kw)
        sim.set_stencil("isotropic")
        sim.set_variant(*VARIANTS[variant])
        st = O.init(O.make_cfg(stencil=1, **kw))
        sim.step(200)
        ref = O.run(st, 200)
        for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                                ("f", to_oracle_f(sim.get("pop"), 2), ref.f)):
            assert relerr(got, want) < 1e-10, (kw, name, relerr(got, want))
        sim.close()


def test_isotropic_stencil_refusals():
    # parameters of the paper's 3D runs: unstable with the 7-point Laplacian only
    fig3 = dict(d=3, nx=16, ny=16, nz=24, b=0.1, kappa=-0.03, c=0.03, Gamma=0.1, Tc=0.005, T0=0.0055,
                T_w=0.0045, phi_amp=0.01, precision="fp32")
    with pytest.raises(lf.LFError):
        lf.Lattice(**fig3)
    sim = lf.Lattice(stencil="isotropic", **fig3)
    with pytest.raises(lf.LFError):
        sim.set_stencil("compact")             # unstable: the context keeps its stencil
    sim.step(10)
    assert sim.diag()["rc"] == 0
    sim.close()
    sim = lf.Lattice(nx=32, ny=32, precision="fp64", xi=0.5)
    sim.set_stencil("isotropic")
    # switching back restores the compact step exactly
    sim.set_stencil("compact")
    st = O.State(O.make_cfg(nx=32, ny=32, xi=0.5), to_oracle_f(sim.get("pop"), 2), sim.get("phi"), sim.get("T"))
    sim.step(1)
    assert relerr(sim.get("phi"), O.step(st).phi) < 1e-12
    sim.close()


def _check_aux_and_step(sim, st, prec):
    tol = TOL[prec]
    d = 2
    ax = O.aux(st)
    checks = {"mu": (sim.get("mu"), ax["mu"]), "Fx": (sim.get("Fx"), ax["F"][0]),
              "Fy": (sim.get("Fy"), ax["F"][1]), "rho": (sim.get("rho"), ax["n"]),
              "ux": (sim.get("ux"), ax["u"][0]), "uy": (sim.get("uy"), ax["u"][1])}
    for k, (g, w) in checks.items():
        if np.abs(w).max() == 0:
            assert np.abs(g).max() == 0, k
            continue
        assert relerr(g, w) < tol, (k, relerr(g, w))
    sim.step(1)
    ref = O.step(st)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), d), ref.f)):
        assert relerr(got, want) < tol, (name, relerr(got, want))
    sim.close()


CASES3 = [
    dict(d=3, nx=12, ny=10, nz=9, xi=0.01),                        # walls along z, one tile
    dict(d=3, nx=40, ny=12, nz=20, xi=0.01),                       # several tiles, ragged in x and y
    dict(d=3, nx=9, ny=7, nz=6, walls=0, xi=0.01),                 # fully periodic, smaller than the halo
    dict(d=3, nx=14, ny=11, nz=8, t_wall_mode=1, xi=0.4),          # halfway T ghost, 3 sub-steps
    dict(d=3, nx=10, ny=9, nz=7, hydro=0, xi=0.1),                 # no hydrodynamics
    dict(d=3, nx=36, ny=17, nz=5, tau=0.6, xi=1e-3),               # thin in z
    dict(d=3, nx=3, ny=2, nz=2, xi=0.01),                          # thinner than every halo: the
    dict(d=3, nx=2, ny=3, nz=3, walls=0, xi=0.01),                 # index maps' general path
]


VARIANTS3 = {"fused": ("march", 0), "split3": ("split3", 0), "split3-z3": ("split3", 3),
             "split3-60x4": ("split3", 1 << 16), "split3-scalar-z5": ("split3", (2 << 16) | 5),
             "split3-phi1": ("split3", 1 << 20), "split3-phi7-z5": ("split3", (7 << 20) | 5)}


@pytest.mark.parametrize("variant", list(VARIANTS3))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES3, ids=lambda c: "x".join(str(c[k]) for k in ("nx", "ny", "nz")) + str(c))
def test_aux_and_step_parity_3d(case, prec, variant):
    sim, cfg, st = make_pair(case, prec)
    sim.set_variant(*VARIANTS3[variant])
    _check_aux_and_step_3d(sim, st, prec)


# force-pass forms of the isotropic three-pass step ((param >> 16) & 15)
VARIANTS3_ISO = {"split3": ("split3", 0), "split3-z3": ("split3", 3), "split3-phi1": ("split3", 1 << 20),
                 "split3-28x28": ("split3", 1 << 16), "split3-28x28-z5": ("split3", (1 << 16) | 5),
                 "split3-1cta-z5": ("split3", (3 << 16) | 5), "split3-phi5": ("split3", 5 << 20),
                 "split3-x2": ("split3", 4 << 16), "split3-x2-z3": ("split3", (4 << 16) | 3),
                 "split3-x2-z8": ("split3", (4 << 16) | 8),
                 "split3-phiasync": ("split3", 1 << 28), "split3-phiasync-z1": ("split3", (1 << 28) | (1 << 20)),
                 "fused": ("march", 0)}


@pytest.mark.parametrize("variant", list(VARIANTS3_ISO))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES3, ids=lambda c: "x".join(str(c[k]) for k in ("nx", "ny", "nz")) + str(c))
def test_isotropic_stencil_parity_3d(case, prec, variant):
    """Isotropic 19-point stencils: the three-pass step with each force-pass
    form (sliding sums on 28x12 and 28x28 tiles, on two z-lanes in packed FP32x2
    (one lane in FP64); segments of 3, 5 and 8 planes as well), the phi pass
    with segments of 16, 5 and 1 planes, and the fused plane march."""
    sim, cfg, st = make_pair(case, prec, stencil="isotropic")
    sim.set_variant(*VARIANTS3_ISO[variant])
    _check_aux_and_step_3d(sim, st, prec)


def test_isotropic_multistep_3d_fp64():
    kw = dict(d=3, nx=20, ny=16, nz=18, xi=0.3, t_wall_mode=1)
    sim = lf.Lattice(precision="fp64", stencil="isotropic", **kw)
    st = O.init(O.make_cfg(stencil=1, **kw))
    sim.step(50)
    ref = O.run(st, 50)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 3), ref.f)):
        assert relerr(got, want) < 1e-10, (name, relerr(got, want))
    sim.close()


def _check_aux_and_step_3d(sim, st, prec):
    """Components of F and u are measured against the largest component of
    their vector: on a lattice two sites thick a y-derivative is zero, exactly
    on the GPU and up to rounding (1e-19) in the oracle's 19-point sums."""
    tol = TOL[prec]
    ax = O.aux(st)
    for k, (g, w) in {"mu": (sim.get("mu"), ax["mu"]), "rho": (sim.get("rho"), ax["n"])}.items():
        assert relerr(g, w) < tol, (k, relerr(g, w))
    for vec, key in (("F", "F"), ("u", "u")):
        scale = max(np.abs(c).max() for c in ax[key])
        for a, name in enumerate(("x", "y", "z")):
            g, w = sim.get(vec + name), ax[key][a]
            if scale == 0:
                assert np.abs(g).max() == 0, vec + name
                continue
            err = np.abs(g - w).max() / scale
            assert err < tol, (vec + name, err)
    sim.step(1)
    ref = O.step(st)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 3), ref.f)):
        assert relerr(got, want) < tol, (name, relerr(got, want))
    sim.close()


@pytest.mark.parametrize("variant", ["march", "split3"])
def test_multistep_3d_fp64(variant):
    sim = lf.Lattice(d=3, nx=20, ny=16, nz=18, precision="fp64", xi=0.01)
    sim.set_variant(variant, 0)
    st = O.init(O.make_cfg(d=3, nx=20, ny=16, nz=18, xi=0.01))
    sim.step(50)
    ref = O.run(st, 50)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 3), ref.f)):
        assert relerr(got, want) < 1e-10, (name, relerr(got, want))
    d = sim.diag()
    assert d["rc"] == 0 and abs(d["mass"] - 20 * 16 * 18) < 1e-9
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_init_matches_generator(prec):
    sim = lf.Lattice(nx=70, ny=37, precision=prec, seed=123)
    cfg = O.make_cfg(nx=70, ny=37, seed=123)
    st = O.init(cfg)
    if prec == "fp64":
        np.testing.assert_array_equal(sim.get("phi"), st.phi)
        np.testing.assert_array_equal(sim.get("T"), st.T)
    else:
        np.testing.assert_array_equal(sim.get("phi", "fp32"), st.phi.astype(np.float32))
        np.testing.assert_array_equal(sim.get("T", "fp32"), st.T.astype(np.float32))
    np.testing.assert_allclose(to_oracle_f(sim.get("pop"), 2), st.f, rtol=0, atol=0)
    sim.close()


def test_multistep_fp64_small64():
    """200 coupled steps of the 64 x 64 case from the seeded initial state."""
    sim = lf.Lattice(nx=64, ny=64, precision="fp64")
    st = O.init(O.make_cfg(nx=64, ny=64))
    sim.step(200)
    ref = O.run(st, 200)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 2), ref.f)):
        assert relerr(got, want) < 1e-10, (name, relerr(got, want))
    sim.close()


@pytest.mark.parametrize("tuned", [False, True])
def test_full_size_one_step_fp32(tuned):
    """The 1024 x 1024 FP32 workload, in the launch configuration the benchmark
    times (the autotuner's choice, as the benchmark takes it, and the library's
    default): one step from the seeded state, every site against the oracle."""
    kw = synth.WORKLOADS["prec1024"]
    sim = lf.Lattice(nx=1024, ny=1024, precision="fp32", xi=kw["xi"])
    if tuned:
        sim.tune(reps=5)
    cfg = O.make_cfg(nx=1024, ny=1024, xi=kw["xi"])
    sim.step(3)            # leave the trivial initial populations
    st = O.State(cfg, to_oracle_f(sim.get("pop"), 2), sim.get("phi"), sim.get("T"))
    sim.step(1)
    ref = O.step(st)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 2), ref.f)):
        assert relerr(got, want) < 2e-6, (name, relerr(got, want))
    sim.close()


@pytest.mark.parametrize("tuned", [False, True])
@pytest.mark.parametrize("xi", [1e-3, 0.1])
def test_full_size_one_step_isotropic_fp32(tuned, xi):
    """The same 1024 x 1024 workload with the isotropic 9-point stencils (the
    two 2D configurations that run their 50k steps), in the library's default
    configuration (the packed isotropic march) and the autotuner's choice:
    one step from the seeded state, every site against the oracle."""
    sim = lf.Lattice(nx=1024, ny=1024, precision="fp32", xi=xi, stencil="isotropic")
    if tuned:
        sim.tune(reps=5)
    cfg = O.make_cfg(nx=1024, ny=1024, xi=xi, stencil=1)
    sim.step(3)
    st = O.State(cfg, to_oracle_f(sim.get("pop"), 2), sim.get("phi"), sim.get("T"))
    sim.step(1)
    ref = O.step(st)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 2), ref.f)):
        assert relerr(got, want) < 2e-6, (name, relerr(got, want))
    sim.close()


def _sampled_window_parity(sim, d, okw, centres, half=8):
    """One step of `sim` checked on sub-lattices: around each sampled centre
    (x0 in 2D, (x0, y0) in 3D) the oracle steps a 2*half-wide window, periodic
    along x (and y), over the whole wall-normal extent.  The step reaches 4 sites
    (phi -> psi -> lam, grad psi -> P -> F -> u -> div(phi u)), so the window's
    own wrap cannot reach its core |x - x0| < half - 4, which is compared site by
    site with the GPU step (FP32 tolerance)."""
    torch_ = sim.torch
    perm = perm_to_oracle(d)
    before = {k: sim.get(k, device=True) for k in ("pop", "phi", "T")}
    sim.step(1)
    after = {k: sim.get(k, device=True) for k in ("pop", "phi", "T")}
    nx, ny = sim.shape[-1], sim.shape[-2]
    w = 2 * half
    core = slice(half - 4, half + 4)
    for c in centres:
        ix = torch_.tensor([(c[0] - half + i) % nx for i in range(w)], device=sim.device)
        iy = torch_.tensor([(c[1] - half + i) % ny for i in range(w)], device=sim.device) if d == 3 else None

        def win(t):
            t = torch_.index_select(t, t.dim() - 1, ix)
            if d == 3:
                t = torch_.index_select(t, t.dim() - 2, iy)
            return t.cpu().numpy()

        f0 = win(before["pop"])
        fo = np.empty_like(f0)
        for i, j in enumerate(perm):
            fo[j] = f0[i]
        shp = dict(nx=w, ny=w, nz=sim.shape[0]) if d == 3 else dict(nx=w, ny=ny)
        cfg = O.make_cfg(d=d, **shp, **okw)
        ref = O.step(O.State(cfg, fo, win(before["phi"]), win(before["T"])))
        f1 = to_oracle_f(win(after["pop"]), d)
        sel = (Ellipsis, core, core) if d == 3 else (Ellipsis, core)
        for name, got, want in (("phi", win(after["phi"]), ref.phi), ("T", win(after["T"]), ref.T),
                                ("f", f1, ref.f)):
            assert relerr(got[sel], want[sel]) < 2e-6, (c, name, relerr(got[sel], want[sel]))


@pytest.mark.parametrize("tuned", [False, True])
def test_cube384_sampled_windows_fp32(tuned):
    """The 384^3 FP32 workload in the launch configuration the benchmark times
    (the three-pass step with the autotuner's shape, as the benchmark takes it,
    and with the library's default shape; seed 1): one step, checked on six
    8 x 8 columns of all 384 planes against the oracle on 16 x 16 x 384 windows."""
    kw = synth.WORKLOADS["cube384"]
    sim = lf.Lattice(d=3, nx=384, ny=384, nz=384, precision="fp32", xi=kw["xi"], tau=kw["tau"], seed=1)
    if tuned:
        sim.tune(reps=3)
    sim.step(3)            # leave the trivial initial populations
    rng = np.random.default_rng(21)
    centres = [tuple(int(v) for v in rng.integers(0, 384, 2)) for _ in range(5)] + [(0, 383)]
    _sampled_window_parity(sim, 3, dict(xi=kw["xi"], tau=kw["tau"]), centres)
    sim.close()


def test_cube384_isotropic_tau3_sampled_windows_fp32():
    """The configuration the benchmark times beside its main line (384^3, tau = 3,
    isotropic 19-point stencils, the autotuner's shape): one step, checked on six
    8 x 8 columns of all 384 planes against the oracle on 16 x 16 x 384 windows."""
    kw = synth.WORKLOADS["cube384"]
    sim = lf.Lattice(d=3, nx=384, ny=384, nz=384, precision="fp32", xi=kw["xi"], tau=3.0, seed=1,
                     stencil="isotropic")
    sim.tune(reps=3)
    sim.step(3)            # leave the trivial initial populations
    rng = np.random.default_rng(23)
    centres = [tuple(int(v) for v in rng.integers(0, 384, 2)) for _ in range(5)] + [(383, 0)]
    _sampled_window_parity(sim, 3, dict(xi=kw["xi"], tau=3.0, stencil=1), centres)
    sim.close()


def test_largest_2d_lattice_fp32():
    """The largest 2D FP32 lattice the library accepts with 32-bit element
    indices (9 x pitch x ny < 2^31: 16384 x 14563, 238.6 M sites), one step of
    the default kernel checked on sampled 16-column windows of all rows, with the
    wrap at x = 0 among them."""
    nx, ny = 16384, 14563
    assert 9 * nx * ny < 2 ** 31 <= 9 * nx * (ny + 1)
    sim = lf.Lattice(nx=nx, ny=ny, precision="fp32", xi=0.01)
    sim.step(2)
    rng = np.random.default_rng(22)
    centres = [(int(v),) for v in rng.integers(0, nx, 3)] + [(0,), (nx - 3,)]
    _sampled_window_parity(sim, 2, dict(xi=0.01), centres)
    d = sim.diag()
    assert d["rc"] == 0 and abs(d["mass"] / (nx * ny) - 1) < 1e-6
    sim.close()


@pytest.mark.parametrize("tuned", [False, True])
def test_isotropic_4096_sampled_windows_fp32(tuned):
    """The 2D isotropic step at 4096^2 (the size of the benchmark's isotropic
    4096^2 line), in the default packed isotropic march (lanes of about 158 rows:
    longer than any smaller case) and the autotuner's choice: one step checked on
    sampled 16-column windows of all rows, the wrap at x = 0 among them."""
    n = 4096
    sim = lf.Lattice(nx=n, ny=n, precision="fp32", xi=1e-3, stencil="isotropic")
    if tuned:
        sim.tune(reps=3)
    sim.step(3)
    rng = np.random.default_rng(41)
    centres = [(int(v),) for v in rng.integers(0, n, 3)] + [(0,), (n - 3,)]
    _sampled_window_parity(sim, 2, dict(xi=1e-3, stencil=1), centres)
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_resume_bit_identical(prec):
    a = lf.Lattice(nx=70, ny=37, precision=prec)
    a.step(10)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ck.bin")
        a.save(path)
        a.step(15)
        b = lf.Lattice(nx=70, ny=37, precision=prec, seed=99)
        b.load(path)
        assert b.step_count == 10
        b.step(15)
    dt = "fp64" if prec == "fp64" else "fp32"
    for name in ("phi", "T", "pop"):
        np.testing.assert_array_equal(a.get(name, dt), b.get(name, dt))
    assert a.step_count == b.step_count == 25
    a.close()
    b.close()


def test_checkpoint_refuses_another_scheme():
    """A checkpoint written with one stencil or temperature solver does not
    load into a context set to the other (LF_EIO, state kept); once the
    context is set like the writer, it loads and resumes bit for bit."""
    a = lf.Lattice(nx=40, ny=24, precision="fp32", xi=0.5, stencil="isotropic")
    a.set_t_solver("implicit")
    a.step(4)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "iso_impl.lfck")
        a.save(path)
        a.step(3)
        b = lf.Lattice(nx=40, ny=24, precision="fp32", xi=0.5)
        phi0 = b.get("phi", "fp32")
        for stencil, solver in (("compact", "explicit"), ("isotropic", "explicit"), ("compact", "implicit")):
            b.set_stencil(stencil)
            b.set_t_solver(solver)
            with pytest.raises(lf.LFError) as ei:
                b.load(path)
            assert ei.value.code == lf.LF_EIO, (stencil, solver)
            np.testing.assert_array_equal(b.get("phi", "fp32"), phi0)
        b.set_stencil("isotropic")
        b.set_t_solver("implicit")
        b.load(path)
        b.step(3)
    for name in ("phi", "T", "pop"):
        np.testing.assert_array_equal(a.get(name, "fp32"), b.get(name, "fp32"))
    a.close()
    b.close()


def test_bounded_wait_reports_timeout_and_recovers(monkeypatch):
    """A blocking call whose wait for the stream runs out returns LF_ETIMEOUT
    (here: a 1 us limit behind ~100 queued steps) without breaking the context;
    after the stream drains, the same call succeeds and sees the finished state."""
    sim = lf.Lattice(nx=2048, ny=2048, precision="fp32", xi=1e-3)
    sim.step(1)
    torch.cuda.synchronize()
    out = torch.empty(sim.shape, dtype=torch.float32, device=sim.device)
    monkeypatch.setenv("LF_WAIT_TIMEOUT_S", "1e-6")
    sim.step(100)
    with pytest.raises(lf.LFError) as ei:
        lf.lf_fields(sim.ctx, lf.FIELDS["phi"], out.data_ptr(), out.numel() * 4, True)
    assert ei.value.code == lf.LF_ETIMEOUT
    monkeypatch.delenv("LF_WAIT_TIMEOUT_S")
    torch.cuda.synchronize()
    a = sim.get("phi", "fp32")
    lf.lf_fields(sim.ctx, lf.FIELDS["phi"], out.data_ptr(), out.numel() * 4, True)
    np.testing.assert_array_equal(out.cpu().numpy(), a)
    assert lf.lf_step_count(sim.ctx) == 101 and sim.diag()["rc"] == 0
    sim.close()


def test_checkpoint_failures_leave_the_context_intact():
    """lf_save to a path that cannot be written, lf_load of a checkpoint of
    another lattice, a truncated file and a file with a wrong header all return
    LF_EIO; the context keeps its state and steps on."""
    a = lf.Lattice(nx=40, ny=24, precision="fp32")
    a.step(3)
    phi0 = a.get("phi", "fp32")
    with tempfile.TemporaryDirectory() as tmp:
        with pytest.raises(lf.LFError) as ei:
            a.save(os.path.join(tmp, "no_such_dir", "c.lfck"))
        assert ei.value.code == lf.LF_EIO
        good = os.path.join(tmp, "good.lfck")
        a.save(good)
        other = lf.Lattice(nx=40, ny=26, precision="fp32")
        other_path = os.path.join(tmp, "other.lfck")
        other.save(other_path)
        other.close()
        raw = open(good, "rb").read()
        trunc = os.path.join(tmp, "trunc.lfck")
        open(trunc, "wb").write(raw[: len(raw) // 2])
        bad_magic = os.path.join(tmp, "magic.lfck")
        open(bad_magic, "wb").write(b"XXXXXXXX" + raw[8:])
        for path in (other_path, trunc, bad_magic, os.path.join(tmp, "missing.lfck")):
            with pytest.raises(lf.LFError) as ei:
                a.load(path)
            assert ei.value.code == lf.LF_EIO, path
            np.testing.assert_array_equal(a.get("phi", "fp32"), phi0)
        a.load(good)
        np.testing.assert_array_equal(a.get("phi", "fp32"), phi0)
    a.step(2)
    assert a.diag()["rc"] == 0 and lf.lf_step_count(a.ctx) == 5
    a.close()


def test_nonfinite_is_reported():
    sim = lf.Lattice(nx=40, ny=24, precision="fp32")
    phi = sim.get("phi", "fp32")
    phi[5, 7] = np.nan
    sim.set("phi", phi)
    sim.step(1)
    torch.cuda.synchronize()
    with pytest.raises(lf.LFError) as ei:
        sim.step(1)
    assert ei.value.code == lf.LF_ENONFINITE
    assert sim.diag()["rc"] == lf.LF_ENONFINITE
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_conservation_2000_steps(prec):
    sim = lf.Lattice(nx=64, ny=64, precision=prec)
    d0 = sim.diag()
    sim.step(2000)
    d1 = sim.diag()
    assert d1["rc"] == 0
    tol_m = 1e-12 if prec == "fp64" else 1e-6
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < tol_m
    assert abs(d1["phi_sum"] - d0["phi_sum"]) < (1e-11 if prec == "fp64" else 2e-3)
    assert d1["mach"] < 0.1
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fields_through_pinned_host_buffers(prec):
    """Pinned host buffers are read and written in place by the conversion
    kernels (no staging copy); the result equals the pageable and the device
    paths exactly, in both directions and for both element sizes."""
    sim = lf.Lattice(nx=70, ny=37, precision=prec, xi=0.05, seed=5)
    sim.step(3)
    for name in ("pop", "phi", "T"):
        for dt in (np.float32, np.float64):
            ref = sim.get(name, dt)
            tdt = torch.float32 if dt == np.float32 else torch.float64
            pin = torch.empty(ref.shape, dtype=tdt, pin_memory=True)
            lf.lf_fields(sim.ctx, lf.FIELDS[name], pin.data_ptr(), pin.numel() * pin.element_size(), False)
            np.testing.assert_array_equal(pin.numpy(), ref)
            dev = sim.get(name, dt, device=True)
            np.testing.assert_array_equal(dev.cpu().numpy(), ref)
    # writing through a pinned buffer stores what the pageable path stores
    native = np.float64 if prec == "fp64" else np.float32
    for name in ("pop", "phi", "T"):
        v = sim.get(name, native) * native(0.5)
        sim.set(name, v)
        a = sim.get(name, native)
        sim.set(name, v * native(3))
        pin = torch.from_numpy(v.copy()).pin_memory()
        lf.lf_fields_set(sim.ctx, lf.FIELDS[name], pin.data_ptr(), pin.numel() * pin.element_size(), False)
        np.testing.assert_array_equal(sim.get(name, native), a)
    sim.close()


def _random_case(rng):
    """A random configuration: lattice (ragged sizes), walls and T wall rule,
    hydrodynamics, stencil, step variant and parameters inside the stability
    limits."""
    d = int(rng.choice([2, 3]))
    case = dict(d=d, nx=int(rng.integers(3, 70)), ny=int(rng.integers(3, 50)),
                walls=int(rng.integers(0, 2)), t_wall_mode=int(rng.integers(0, 2)), hydro=int(rng.integers(0, 2)),
                b=float(rng.uniform(0.0, 1.5)), kappa=float(rng.uniform(-0.05, 0.05)), c=float(rng.uniform(0.0, 0.04)),
                Gamma=float(rng.uniform(0.01, 0.08)), Tc=1.0, T0=float(rng.uniform(0.6, 1.3)),
                T_w=float(rng.uniform(0.4, 0.9)), tau=float(rng.uniform(0.6, 3.0)),
                xi=float(rng.choice([0.0, 1e-3, 0.05, 0.3, 2.0, math.inf])))
    if d == 3:
        case.update(nx=int(rng.integers(3, 30)), ny=int(rng.integers(3, 24)), nz=int(rng.integers(3, 24)))
    stencil = str(rng.choice(["compact", "isotropic"]))
    variant = str(rng.choice(["march", "tile", "march2"] if d == 2 else ["march", "split3"]))
    return case, stencil, variant


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(24))
def test_random_configurations_one_step(seed, prec):
    """Seeded random configurations (every switch of the step drawn at random)
    against the oracle, one step from a random state."""
    rng = np.random.default_rng(1000 + seed)
    case, stencil, variant = _random_case(rng)
    try:
        sim, cfg, st = make_pair(case, prec, seed=seed, stencil=stencil)
    except lf.LFError as ex:                       # outside the stability limits of the explicit schemes
        assert ex.code == lf.LF_EUNSTABLE, (case, ex)
        return
    if case["d"] == 3:
        sim.set_variant(*{"march": ("march", 0), "split3": ("split3", 0)}[variant])
    else:
        sim.set_variant(*VARIANTS[variant])
    sim.step(1)
    ref = O.step(st)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), case["d"]), ref.f)):
        assert relerr(got, want) < TOL[prec], (case, stencil, variant, name, relerr(got, want))
    sim.close()


PAPER = dict(b=0.1, kappa=-0.03, c=0.03, Gamma=0.1, Tc=0.005, T0=0.0055, T_w=0.0045, phi_amp=0.01)


@pytest.mark.parametrize("stencil", ["compact", "isotropic"])
@pytest.mark.parametrize("hydro,tau,xi", [(0, 1.0, 1e-2), (1, 5.0, 1e-3), (1, 5.0, 1.0)])
def test_paper_parameters_multistep_fp64(stencil, hydro, tau, xi):
    """The paper's own parameters (Sec. 3: b = 0.1, kappa = -c = -0.03, Tc = 0.005,
    Gamma = 0.1, T_w = 0.9 Tc; here T0 = 1.1 Tc), where a = (T - Tc)/Tc amplifies
    temperature differences 200-fold: 300 FP64 steps from the seeded state, walls,
    with and without hydrodynamics, against the oracle."""
    kw = dict(PAPER, nx=96, ny=64, hydro=hydro, tau=tau, xi=xi, seed=3)
    sim = lf.Lattice(precision="fp64", stencil=stencil, **kw)
    st = O.init(O.make_cfg(stencil=int(stencil == "isotropic"), **kw))
    sim.step(300)
    ref = O.run(st, 300)
    for name, got, want in (("phi", sim.get("phi"), ref.phi), ("T", sim.get("T"), ref.T),
                            ("f", to_oracle_f(sim.get("pop"), 2), ref.f)):
        assert relerr(got, want) < 1e-10, (name, relerr(got, want))
    sim.close()



def test_checked_mode_guard_bands(monkeypatch):
    """Checked mode (LF_CHECKED=1): every step kind on odd sizes leaves the guard
    bands around the device buffers intact; a byte changed in a guard band
    (written here into the front band of the workspace through the torch
    tensor that holds it) makes the next lf_step return LF_ECORRUPT."""
    monkeypatch.setenv("LF_CHECKED", "1")
    cases = [(dict(nx=37, ny=29, xi=0.5), "march2", "compact"), (dict(nx=37, ny=29, xi=0.5), "march", "compact"),
             (dict(nx=5, ny=3, xi=0.01, t_wall_mode=1), "tile", "isotropic"),
             (dict(nx=70, ny=37, xi=0.5, t_wall_mode=1), "march2", "isotropic"),
             (dict(d=3, nx=13, ny=11, nz=7, xi=0.4), "split3", "compact"),
             (dict(d=3, nx=13, ny=11, nz=7, xi=0.4, walls=0), "march", "isotropic")]
    for kw, variant, stencil in cases:
        for prec in ("fp32", "fp64"):
            sim = lf.Lattice(precision=prec, stencil=stencil, **kw)
            sim.set_variant(variant, 0)
            sim.step(3)
            sim.diag()
            sim.set("phi", sim.get("phi"))
            sim.step(2)
            sim.step(0)                                 # reports what the last steps left
            assert sim.diag()["rc"] == 0
            sim.close()
    sim = lf.Lattice(nx=64, ny=48, precision="fp32")
    sim.step(1)
    base = sim.params.workspace - sim.ws.data_ptr()     # the front guard band starts here
    sim.ws[base + 100] = 0
    sim.step(1)                                        # its guard check sees the change
    torch.cuda.synchronize()
    with pytest.raises(lf.LFError) as ei:
        sim.step(1)
    assert ei.value.code == lf.LF_ECORRUPT
    sim.close()


@pytest.mark.parametrize("stencil,steps", [("compact", 100), ("isotropic", 500)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_conservation_3d(prec, stencil, steps):
    """D3Q19 with walls along z, the default three-pass step: total mass and
    sum(phi) (FP64 to round-off; FP32 to its storage precision).  With the
    compact stencils these parameters diverge after about 150 steps, in the
    oracle as well, so that run stops at 100."""
    sim = lf.Lattice(d=3, nx=32, ny=24, nz=20, precision=prec, stencil=stencil, xi=0.01, tau=0.8)
    d0 = sim.diag()
    sim.step(steps)
    d1 = sim.diag()
    assert d1["rc"] == 0
    tol_m = 1e-12 if prec == "fp64" else 1e-6
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < tol_m
    assert abs(d1["phi_sum"] - d0["phi_sum"]) < (1e-10 if prec == "fp64" else 5e-3)
    assert d1["mach"] < 0.1
    sim.close()


def test_pass_times_of_the_three_pass_step():
    """lf_set_pass_timing / lf_pass_times: three positive pass durations for a
    three-pass 3D step, none with the timing off, for a 2D step or for the
    fused variant; the step's result is that of the untimed step."""
    kw = dict(d=3, nx=40, ny=12, nz=20, xi=0.01)
    a = lf.Lattice(precision="fp32", **kw)
    b = lf.Lattice(precision="fp32", **kw)
    a.set_pass_timing(True)
    a.step(2)
    b.step(2)
    ms = a.pass_times()
    assert len(ms) == 3 and all(t > 0 for t in ms), ms
    for name in ("phi", "T", "pop"):
        np.testing.assert_array_equal(a.get(name, "fp32"), b.get(name, "fp32"))
    a.set_pass_timing(False)
    a.step(1)
    assert a.pass_times() == []
    a.set_pass_timing(True)
    a.set_variant("march", 0)                # the fused plane march: one kernel
    a.step(1)
    assert a.pass_times() == []
    a.close()
    b.close()
    c = lf.Lattice(nx=64, ny=32, precision="fp32", xi=0.01)
    c.set_pass_timing(True)
    c.step(1)
    assert c.pass_times() == []
    c.close()

"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/*.h declares, and its pure host logic (lattice tables, the
temperature sub-step rule, argument and stability validation) agrees with the
oracle and the documented rules."""
import ctypes as C
import glob
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1102_3094_gb300 import _build, lf
    _build.build()
    return lf


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lf\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function(L):
    names = _declared_functions()
    assert len(names) >= 15
    lib = C.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("d", [2, 3])
def test_lattice_matches_oracle_set(L, d):
    e, w = L.lf_lattice(d)
    eo, wo = O.velocity_set(d)
    got = {tuple(v): x for v, x in zip(e.tolist(), w)}
    want = {tuple(v): x for v, x in zip(eo.tolist(), wo)}
    assert got.keys() == want.keys()
    for k in got:
        assert got[k] == pytest.approx(want[k], abs=1e-16)


def test_nsub_rule_matches_oracle(L):
    for d in (2, 3):
        for xi in [0.0, 1e-4, 1e-3, 0.01, 0.1, 0.13, 0.2, 0.2000001, 0.25, 0.5, 1.0, 3.7, 100.0, math.inf]:
            assert L.lf_nsub(xi, d) == O.nsub_for(xi, d), (xi, d)


def _args(L, **kw):
    g = L.lf_grid(d=2, nx=64, ny=64, nz=1)
    w = L.lf_walls(walls=1, t_wall_mode=0, T_w=0.5)
    p = L.lf_params(b=1.0, kappa=-0.025, c=0.02, Gamma=0.05, Tc=1.0, T0=1.1, xi=0.01, tau=1.0, n0=1.0,
                    phi_amp=0.05, seed=1, precision=0, hydro=1, ideal_mode=0)
    for k, v in kw.items():
        for s in (g, w, p):
            if hasattr(s, k):
                setattr(s, k, v)
    return g, w, p


@pytest.mark.parametrize("kw,code", [
    (dict(tau=0.5), -2), (dict(tau=0.3), -2), (dict(Gamma=5.0), -2),
    (dict(d=4), -1), (dict(nx=0), -1), (dict(nz=2), -1), (dict(precision=7), -1),
    (dict(ideal_mode=1), -1), (dict(Tc=0.0), -1), (dict(xi=-1.0), -1), (dict(xi=float("nan")), -1),
    (dict(ny=1), -1), (dict(walls=2), -1), (dict(t_wall_mode=3), -1), (dict(b=float("inf")), -1),
    (dict(stencil=2), -1), (dict(stencil=-1), -1),
])
def test_validation_codes(L, kw, code):
    g, w, p = _args(L, **kw)
    n = C.c_size_t()
    rc = L.lib().lf_workspace_bytes(C.byref(g), C.byref(w), C.byref(p), C.byref(n))
    assert rc == code
    ctx = C.c_void_p()
    assert L.lib().lf_create(C.byref(g), C.byref(w), C.byref(p), C.byref(ctx)) == code
    assert not ctx.value


@pytest.mark.parametrize("d", [2, 3])
def test_stability_limit_follows_the_stencil(L, d):
    """The explicit phi update is checked against the largest Laplacian
    eigenvalue of the chosen stencils: 4d (compact) or 16/3 (isotropic).  At
    the parameters of the paper's runs (b = 0.1, kappa = -c = -0.03, Gamma =
    0.1, T_w = 0.9 Tc) the 3D compact step is unstable and the isotropic one
    is not; a larger Gamma makes both unstable."""
    kw = dict(d=d, nz=24 if d == 3 else 1, b=0.1, kappa=-0.03, c=0.03, Gamma=0.1, Tc=0.005, T0=0.0055,
              T_w=0.0045)
    n = C.c_size_t()

    def rc(**more):
        g, w, p = _args(L, **dict(kw, **more))
        return L.lib().lf_workspace_bytes(C.byref(g), C.byref(w), C.byref(p), C.byref(n))

    assert rc(stencil=0) == (-2 if d == 3 else 0)
    assert rc(stencil=1) == 0
    assert rc(stencil=1, Gamma=1.0) == -2


def test_largest_lattice_accepted(L):
    """Element indices of one population field stay below 2^31: 9 x pitch x ny
    for 2D (pitch = nx rounded up to 32), 19 x pitch x ny x nz for 3D."""
    n = C.c_size_t()

    def rc(**kw):
        g, w, p = _args(L, **kw)
        return L.lib().lf_workspace_bytes(C.byref(g), C.byref(w), C.byref(p), C.byref(n))

    assert rc(nx=16384, ny=14560, precision=1) == 0
    assert rc(nx=16384, ny=14564, precision=1) == -1
    assert rc(nx=16383, ny=14560, precision=1) == 0          # pitch 16384 as well
    assert rc(d=3, nx=416, ny=416, nz=653, precision=1) == 0     # 19 * 416 * 416 * 653 < 2^31
    assert rc(d=3, nx=416, ny=416, nz=654, precision=1) == -1


def test_workspace_bytes_scale(L):
    g, w, p = _args(L)
    b64 = L.lf_workspace_bytes(g, w, p)
    p.precision = 1
    b32 = L.lf_workspace_bytes(g, w, p)
    # two copies of 9 populations + phi + T, plus 8 aux planes, in the state precision
    assert b64 > 2 * 11 * 64 * 64 * 8 and b32 < b64


def test_strerror_covers_codes(L):
    for c in range(0, -9, -1):
        assert L.strerror(c) != "unknown error"


@pytest.mark.parametrize("kw", [dict(precision=0), dict(precision=1, d=3, nz=8), dict(precision=1, ny=1, walls=0),
                                dict(precision=1, stencil=2)])
def test_ensemble_refuses_bad_runs_before_allocating(L, kw):
    """Ensembles take 2D FP32 runs with ny >= 2: anything else is refused
    (LF_EINVAL) by the argument checks, before any device allocation."""
    g, w, p = _args(L, **kw)
    with pytest.raises(L.LFError) as ei:
        L.lf_ens_create([g], [w], [p])
    assert ei.value.code == -1


def test_checked_mode_adds_guard_bands(L, monkeypatch):
    """LF_CHECKED=1 grows the workspace by the ten 64 KiB guard bands."""
    g, w, p = _args(L)
    plain = L.lf_workspace_bytes(g, w, p)
    monkeypatch.setenv("LF_CHECKED", "1")
    assert L.lf_workspace_bytes(g, w, p) == plain + 10 * 64 * 1024


def test_convolution_calls_refuse_bad_arguments(L):
    """The surrogate's convolution entry points check their arguments before
    any CUDA call (shapes the tensor-core kernels take, 16-byte alignment of
    every buffer that TMA or vector accesses read, required outputs, scratch
    size); the pointers below are never dereferenced."""
    lib = L._sur2_lib()
    EINVAL = L.LF_EINVAL
    p = C.c_void_p(0x10000)             # 16-byte aligned, never dereferenced
    q = C.c_void_p(0x10008)             # 8-byte aligned only
    conv = lib.lf_sur_conv3x3

    def c(B=2, NY=8, NX=256, cin=64, cout=64, inp=p, w=p, out=p, resid=None, mask=None, out2=None, zout=None,
          x4=None, y4=None, err=p):
        return conv(B, NY, NX, cin, cout, inp, w, None, 1, resid, mask, out, out2, zout, x4, y4, err, None)

    assert c(NX=200) == EINVAL            # NX not a multiple of the 128-pixel tile
    assert c(NX=0) == EINVAL
    assert c(B=0) == EINVAL
    assert c(cin=32) == EINVAL            # (cin, cout) outside the three layer shapes
    assert c(cin=16, cout=16) == EINVAL
    assert c(inp=q) == EINVAL             # TMA and vector accesses need 16-byte alignment
    assert c(resid=q) == EINVAL
    assert c(out=None) == EINVAL          # nothing to write
    assert c(mask=p) == EINVAL            # a mask needs out2
    assert c(cout=16, cin=64, out=None, y4=p) == EINVAL   # y4 needs x4
    assert c(err=None) == EINVAL

    sc = lib.lf_sur_wgrad_scratch_floats
    assert sc(64, 64) == 3 * (2 * 152 // 3) * 3 * 64 * 64     # three tap groups by dy
    assert sc(16, 64) == (2 * 152) * 9 * 64 * 16              # one group of nine taps
    assert sc(64, 16) == (2 * 152) * 9 * 64 * 16
    assert sc(32, 64) == 0
    wg = lib.lf_sur_conv3x3_wgrad
    assert wg(2, 8, 256, 64, 64, p, p, p, sc(64, 64) - 1, p, p, None) == EINVAL   # scratch too small
    assert wg(2, 8, 200, 64, 64, p, p, p, sc(64, 64), p, p, None) == EINVAL
    assert wg(2, 8, 256, 64, 64, q, p, p, sc(64, 64), p, p, None) == EINVAL
    assert wg(2, 8, 256, 64, 32, p, p, p, 1 << 30, p, p, None) == EINVAL

"""Python face of the plain FP64 CPU oracle (``lf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module; the GPU library never does.  It shares no
code with the CUDA path.

The C file states the time step of arXiv:1102.3094 Sec. 2 site by site.  This
wrapper compiles it on first use (gcc, OpenMP, ``-ffp-contract=off``), passes
numpy FP64 arrays in and out, and holds the one piece of host logic the C code
takes as input: the number of temperature sub-steps.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lf_oracle.c into liboracle.so beside it (plain gcc, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrCfg(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("walls", C.c_int), ("t_wall_mode", C.c_int), ("hydro", C.c_int),
        ("nsub", C.c_int), ("stencil", C.c_int),
        ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
        ("b", C.c_double), ("kappa", C.c_double), ("c", C.c_double), ("Gamma", C.c_double),
        ("Tc", C.c_double), ("T0", C.c_double), ("T_w", C.c_double), ("xi", C.c_double),
        ("tau", C.c_double), ("n0", C.c_double), ("phi_amp", C.c_double),
        ("seed", C.c_uint64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
            ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
            cp = C.POINTER(OrCfg)
            lib.or_velocity_set.argtypes = [C.c_int, ip, dp]
            lib.or_velocity_set.restype = C.c_int
            lib.or_splitmix64.argtypes = [C.c_uint64, C.c_int64, up]
            lib.or_init.argtypes = [cp, dp, dp, dp]
            lib.or_step.argtypes = [cp, dp, dp, dp, dp, dp, dp]
            lib.or_run.argtypes = [cp, C.c_int64, dp, dp, dp]
            lib.or_aux.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp]
            lib.or_feq.argtypes = [C.c_int, C.c_double, dp, dp]
            lib.or_guo.argtypes = [C.c_int, C.c_double, dp, dp, dp]
            lib.or_collide_site.argtypes = [C.c_int, C.c_double, dp, dp, dp]
            lib.or_threads.argtypes = []
            lib.or_threads.restype = C.c_int
            for fn in ("or_init", "or_step", "or_run", "or_aux", "or_feq", "or_guo",
                       "or_collide_site", "or_splitmix64"):
                getattr(lib, fn).restype = None
            _lib = lib
    return _lib


# --------------------------------------------------------------------------
# Configuration
# --------------------------------------------------------------------------
def nsub_for(xi: float, d: int) -> int:
    """Temperature sub-steps: explicit Euler of d_t T = xi nabla^2 T with the
    (2d+1)-point Laplacian is stable for xi*dt <= 1/(2d); the oracle keeps a
    20% margin, i.e. the smallest nsub with xi/nsub <= 0.8/(2d)."""
    if math.isinf(xi) or xi <= 0.0:
        return 1
    return max(1, math.ceil(xi / (0.8 / (2 * d)) - 1e-12))


def make_cfg(d=2, nx=64, ny=64, nz=1, walls=1, t_wall_mode=0, hydro=1, b=1.0,
             kappa=-0.025, c=0.02, Gamma=0.05, Tc=1.0, T0=1.1, T_w=0.5, xi=0.01,
             tau=1.0, n0=1.0, phi_amp=0.05, seed=1, nsub=None, stencil=0) -> OrCfg:
    if d == 2:
        nz = 1
    cfg = OrCfg()
    cfg.d, cfg.walls, cfg.t_wall_mode, cfg.hydro = d, walls, t_wall_mode, hydro
    cfg.nsub = nsub_for(xi, d) if nsub is None else nsub
    cfg.stencil = stencil
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.b, cfg.kappa, cfg.c, cfg.Gamma = b, kappa, c, Gamma
    cfg.Tc, cfg.T0, cfg.T_w, cfg.xi = Tc, T0, T_w, xi
    cfg.tau, cfg.n0, cfg.phi_amp, cfg.seed = tau, n0, phi_amp, seed
    return cfg


def shape_of(cfg: OrCfg):
    """Field shape (z, y, x) with x fastest; (ny, nx) in two dimensions."""
    return (int(cfg.ny), int(cfg.nx)) if cfg.d == 2 else (int(cfg.nz), int(cfg.ny), int(cfg.nx))


def velocity_set(d: int):
    """(e[Q,3] int, w[Q]) in the oracle's own enumeration order."""
    lib = _load()
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19, np.float64)
    q = lib.or_velocity_set(d, e.reshape(-1), w)
    return e[:q].copy(), w[:q].copy()


def threads() -> int:
    """OpenMP threads the oracle's loops run on."""
    return int(_load().or_threads())


def splitmix64(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, np.uint64)
    _load().or_splitmix64(seed, count, out)
    return out


# --------------------------------------------------------------------------
# State
# --------------------------------------------------------------------------
class State:
    """f[Q, *shape], phi[*shape], T[*shape] as FP64 numpy arrays."""

    def __init__(self, cfg: OrCfg, f, phi, T):
        self.cfg, self.f, self.phi, self.T = cfg, f, phi, T

    def copy(self):
        return State(self.cfg, self.f.copy(), self.phi.copy(), self.T.copy())


def init(cfg: OrCfg) -> State:
    shp = shape_of(cfg)
    Q = velocity_set(cfg.d)[0].shape[0]
    f = np.zeros((Q,) + shp)
    phi = np.zeros(shp)
    T = np.zeros(shp)
    _load().or_init(C.byref(cfg), f.reshape(-1), phi.reshape(-1), T.reshape(-1))
    return State(cfg, f, phi, T)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def step(st: State) -> State:
    """One step t -> t+1 (returns a new State)."""
    f, phi, T = _c(st.f), _c(st.phi), _c(st.T)
    f2, p2, t2 = np.empty_like(f), np.empty_like(phi), np.empty_like(T)
    _load().or_step(C.byref(st.cfg), f.reshape(-1), phi.reshape(-1), T.reshape(-1),
                    f2.reshape(-1), p2.reshape(-1), t2.reshape(-1))
    return State(st.cfg, f2, p2, t2)


def run(st: State, nsteps: int) -> State:
    out = State(st.cfg, _c(st.f).copy(), _c(st.phi).copy(), _c(st.T).copy())
    _load().or_run(C.byref(st.cfg), nsteps, out.f.reshape(-1), out.phi.reshape(-1),
                   out.T.reshape(-1))
    return out


def aux(st: State):
    """dict of mu, F[3], n, u[3] at time t (u includes the half-force shift)."""
    shp = shape_of(st.cfg)
    N = int(np.prod(shp))
    mu, n = np.empty(N), np.empty(N)
    F, u = np.empty(3 * N), np.empty(3 * N)
    _load().or_aux(C.byref(st.cfg), _c(st.f).reshape(-1), _c(st.phi).reshape(-1),
                   _c(st.T).reshape(-1), mu, F, n, u)
    return {"mu": mu.reshape(shp), "F": F.reshape((3,) + shp), "n": n.reshape(shp),
            "u": u.reshape((3,) + shp)}


def feq(d: int, n: float, u) -> np.ndarray:
    Q = velocity_set(d)[0].shape[0]
    out = np.zeros(19)
    _load().or_feq(d, n, _c(np.resize(np.asarray(u, float), 3)), out)
    return out[:Q]


def guo(d: int, tau: float, u, F) -> np.ndarray:
    Q = velocity_set(d)[0].shape[0]
    out = np.zeros(19)
    _load().or_guo(d, tau, _c(np.resize(np.asarray(u, float), 3)),
                   _c(np.resize(np.asarray(F, float), 3)), out)
    return out[:Q]


def collide_site(d: int, tau: float, fi, F) -> np.ndarray:
    Q = velocity_set(d)[0].shape[0]
    out = np.zeros(19)
    fin = np.zeros(19)
    fin[:Q] = fi
    _load().or_collide_site(d, tau, fin, _c(np.resize(np.asarray(F, float), 3)), out)
    return out[:Q]

"""Thin Python binding of the C ABI in include/lf.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``liblf.so``.  Device buffers are torch tensors (``data_ptr()``) and the stream
is a torch CUDA stream; torch is used for nothing else.  Importing this module
does not load the library; the first call does, and raises if it is missing
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblf.so")

LF_OK, LF_EINVAL, LF_EUNSTABLE, LF_ENOMEM, LF_ECUDA, LF_ENONFINITE, LF_ETIMEOUT, LF_EIO = 0, -1, -2, -3, -4, -5, -6, -7
LF_ECORRUPT = -8
LF_FP64, LF_FP32 = 0, 1
LF_TWALL_LAYERS, LF_TWALL_HALFWAY = 0, 1
FIELDS = {"phi": 0, "T": 1, "rho": 2, "ux": 3, "uy": 4, "uz": 5, "pop": 6, "mu": 7, "Fx": 8, "Fy": 9, "Fz": 10}


class LFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class lf_grid(C.Structure):
    _fields_ = [("d", C.c_int), ("pad_", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64)]


class lf_walls(C.Structure):
    _fields_ = [("walls", C.c_int), ("t_wall_mode", C.c_int), ("T_w", C.c_double)]


class lf_params(C.Structure):
    _fields_ = [("b", C.c_double), ("kappa", C.c_double), ("c", C.c_double), ("Gamma", C.c_double),
                ("Tc", C.c_double), ("T0", C.c_double), ("xi", C.c_double), ("tau", C.c_double),
                ("n0", C.c_double), ("phi_amp", C.c_double), ("seed", C.c_uint64),
                ("precision", C.c_int), ("hydro", C.c_int), ("ideal_mode", C.c_int), ("stencil", C.c_int),
                ("stream", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


class lf_diag_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("mass", C.c_double), ("phi_sum", C.c_double), ("mom", C.c_double * 3),
                ("umax", C.c_double), ("mach", C.c_double), ("free_energy", C.c_double),
                ("grad2", C.c_double * 3), ("orient_s", C.c_double), ("k_peak", C.c_double),
                ("s_peak", C.c_double), ("nonfinite", C.c_int), ("pad_", C.c_int)]

    def as_dict(self):
        return {"step": self.step, "mass": self.mass, "phi_sum": self.phi_sum, "mom": list(self.mom),
                "umax": self.umax, "mach": self.mach, "free_energy": self.free_energy,
                "grad2": list(self.grad2), "orient_s": self.orient_s, "k_peak": self.k_peak,
                "s_peak": self.s_peak, "nonfinite": self.nonfinite}


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded liblf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it first (__graft_entry__.build()); "
                                   "there is no CPU fallback")
            L = C.CDLL(LIB_PATH)
            vp, sz, i64 = C.c_void_p, C.c_size_t, C.c_int64
            L.lf_lattice.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.lf_nsub.argtypes = [C.c_double, C.c_int]
            L.lf_workspace_bytes.argtypes = [C.POINTER(lf_grid), C.POINTER(lf_walls), C.POINTER(lf_params),
                                             C.POINTER(sz)]
            L.lf_create.argtypes = [C.POINTER(lf_grid), C.POINTER(lf_walls), C.POINTER(lf_params), C.POINTER(vp)]
            L.lf_step.argtypes = [vp, i64]
            L.lf_fields.argtypes = [vp, C.c_int, vp, sz, C.c_int]
            L.lf_fields_set.argtypes = [vp, C.c_int, vp, sz, C.c_int]
            L.lf_diag.argtypes = [vp, C.POINTER(lf_diag_t)]
            L.lf_diag_layers.argtypes = [vp, C.POINTER(C.c_double), i64]
            L.lf_structure_factor.argtypes = [vp, C.POINTER(C.c_double), i64]
            L.lf_save.argtypes = [vp, C.c_char_p]
            L.lf_load.argtypes = [vp, C.c_char_p]
            L.lf_set_kernel_variant.argtypes = [vp, C.c_int, C.c_int]
            L.lf_set_kernel_variant.restype = C.c_int
            L.lf_set_t_solver.argtypes = [vp, C.c_int]
            L.lf_set_t_solver.restype = C.c_int
            L.lf_set_stencil.argtypes = [vp, C.c_int]
            L.lf_set_stencil.restype = C.c_int
            L.lf_tune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.lf_tune.restype = C.c_int
            L.lf_step_count.argtypes = [vp]
            L.lf_step_count.restype = i64
            L.lf_set_pass_timing.argtypes = [vp, C.c_int]
            L.lf_set_pass_timing.restype = C.c_int
            L.lf_pass_times.argtypes = [vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]
            L.lf_pass_times.restype = C.c_int
            L.lf_destroy.argtypes = [vp]
            L.lf_destroy.restype = None
            L.lf_strerror.argtypes = [C.c_int]
            L.lf_strerror.restype = C.c_char_p
            for fn in ("lf_lattice", "lf_nsub", "lf_workspace_bytes", "lf_create", "lf_step", "lf_fields",
                       "lf_fields_set", "lf_diag", "lf_diag_layers", "lf_structure_factor", "lf_save", "lf_load"):
                getattr(L, fn).restype = C.c_int
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().lf_strerror(code).decode()


def _ok(rc: int, where: str) -> int:
    if rc < 0:
        raise LFError(rc, where)
    return rc


# ------------------------------------------------------------------ calls
def lf_lattice(d: int):
    e = (C.c_int * 57)()
    w = (C.c_double * 19)()
    q = _ok(lib().lf_lattice(d, e, w), "lf_lattice")
    return np.array(e[: 3 * q], dtype=np.int32).reshape(q, 3), np.array(w[:q])


def lf_nsub(xi: float, d: int) -> int:
    return _ok(lib().lf_nsub(xi, d), "lf_nsub")


def lf_workspace_bytes(grid, walls, params) -> int:
    n = C.c_size_t()
    _ok(lib().lf_workspace_bytes(C.byref(grid), C.byref(walls), C.byref(params), C.byref(n)), "lf_workspace_bytes")
    return n.value


def lf_create(grid, walls, params) -> C.c_void_p:
    ctx = C.c_void_p()
    _ok(lib().lf_create(C.byref(grid), C.byref(walls), C.byref(params), C.byref(ctx)), "lf_create")
    return ctx


def lf_step(ctx, nsteps: int) -> None:
    _ok(lib().lf_step(ctx, nsteps), "lf_step")


def lf_fields(ctx, which: int, dst_ptr: int, nbytes: int, dst_on_device: bool) -> None:
    _ok(lib().lf_fields(ctx, which, C.c_void_p(dst_ptr), nbytes, int(dst_on_device)), "lf_fields")


def lf_fields_set(ctx, which: int, src_ptr: int, nbytes: int, src_on_device: bool) -> None:
    _ok(lib().lf_fields_set(ctx, which, C.c_void_p(src_ptr), nbytes, int(src_on_device)), "lf_fields_set")


def lf_diag(ctx) -> lf_diag_t:
    out = lf_diag_t()
    rc = lib().lf_diag(ctx, C.byref(out))
    if rc < 0 and rc != LF_ENONFINITE:
        raise LFError(rc, "lf_diag")
    return out, rc


def lf_diag_layers(ctx, L: int) -> np.ndarray:
    out = np.zeros(L)
    _ok(lib().lf_diag_layers(ctx, out.ctypes.data_as(C.POINTER(C.c_double)), L), "lf_diag_layers")
    return out


def lf_structure_factor(ctx, nb: int) -> np.ndarray:
    out = np.zeros(nb)
    _ok(lib().lf_structure_factor(ctx, out.ctypes.data_as(C.POINTER(C.c_double)), nb), "lf_structure_factor")
    return out


def lf_save(ctx, path: str) -> None:
    _ok(lib().lf_save(ctx, path.encode()), "lf_save")


def lf_load(ctx, path: str) -> None:
    _ok(lib().lf_load(ctx, path.encode()), "lf_load")


LF_VARIANT_MARCH, LF_VARIANT_TILE, LF_VARIANT_MARCH2, LF_VARIANT_SPLIT3 = 0, 1, 2, 3
LF_STENCIL_COMPACT, LF_STENCIL_ISOTROPIC = 0, 1


def lf_set_kernel_variant(ctx, variant: int, param: int = 0) -> None:
    _ok(lib().lf_set_kernel_variant(ctx, variant, param), "lf_set_kernel_variant")


def lf_tune(ctx, reps: int = 5):
    """Runs the autotuner (include/lf.h); returns (variant, param, ms per step)."""
    v, p, ms = C.c_int(), C.c_int(), C.c_double()
    _ok(lib().lf_tune(ctx, reps, C.byref(v), C.byref(p), C.byref(ms)), "lf_tune")
    return v.value, p.value, ms.value


def lf_step_count(ctx) -> int:
    return lib().lf_step_count(ctx)


def lf_set_pass_timing(ctx, enable: bool) -> int:
    return lib().lf_set_pass_timing(ctx, int(bool(enable)))


def lf_pass_times(ctx):
    """(rc, [ms of the passes of the last step])."""
    ms = (C.c_float * 3)()
    n = C.c_int(0)
    rc = lib().lf_pass_times(ctx, ms, 3, C.byref(n))
    return rc, [float(ms[i]) for i in range(n.value)]


def lf_destroy(ctx) -> None:
    lib().lf_destroy(ctx)


# ------------------------------------------------------- convenience wrapper
class Lattice:
    """One simulation context.  Wraps the C calls above; holds the workspace
    tensor (device memory from torch) and the stream the library enqueues on."""

    def __init__(self, d=2, nx=64, ny=64, nz=1, walls=1, t_wall_mode=0, T_w=0.5, b=1.0, kappa=-0.025,
                 c=0.02, Gamma=0.05, Tc=1.0, T0=1.1, xi=0.01, tau=1.0, n0=1.0, phi_amp=0.05, seed=1,
                 precision="fp64", hydro=1, stream=None, device=None, use_torch_workspace=True,
                 stencil="compact"):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda:0")
        if d == 2:
            nz = 1
        self.grid = lf_grid(d=d, nx=nx, ny=ny, nz=nz)
        self.walls = lf_walls(walls=walls, t_wall_mode=t_wall_mode, T_w=T_w)
        self.prec = LF_FP64 if precision in ("fp64", LF_FP64) else LF_FP32
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = lf_params(b=b, kappa=kappa, c=c, Gamma=Gamma, Tc=Tc, T0=T0, xi=xi, tau=tau, n0=n0,
                                phi_amp=phi_amp, seed=seed, precision=self.prec, hydro=hydro, ideal_mode=0,
                                stencil={"compact": LF_STENCIL_COMPACT, "isotropic": LF_STENCIL_ISOTROPIC}[stencil],
                                stream=self.stream.cuda_stream, workspace=None, workspace_bytes=0)
        self.ws = None
        if use_torch_workspace:
            nbytes = lf_workspace_bytes(self.grid, self.walls, self.params)
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.ws.data_ptr()
            off = (-base) % 256
            self.params.workspace = base + off
            self.params.workspace_bytes = nbytes
        self.ctx = lf_create(self.grid, self.walls, self.params)
        self.Q = 9 if d == 2 else 19
        self.shape = (ny, nx) if d == 2 else (nz, ny, nx)
        self.N = int(np.prod(self.shape))

    # -- state access -------------------------------------------------------
    def _dtype(self, dtype):
        return np.float64 if dtype in (None, "fp64", np.float64) else np.float32

    def get(self, name: str, dtype=None, device=False):
        """Field as a numpy array (host) or a torch tensor (device=True)."""
        which = FIELDS[name]
        shp = ((self.Q,) + self.shape) if name == "pop" else self.shape
        npdt = self._dtype(dtype)
        if device:
            tdt = self.torch.float64 if npdt == np.float64 else self.torch.float32
            out = self.torch.empty(shp, dtype=tdt, device=self.device)
            lf_fields(self.ctx, which, out.data_ptr(), out.numel() * out.element_size(), True)
            return out
        out = np.empty(shp, dtype=npdt)
        lf_fields(self.ctx, which, out.ctypes.data, out.nbytes, False)
        return out

    def set(self, name: str, value):
        which = FIELDS[name]
        if hasattr(value, "data_ptr"):
            v = value.contiguous()
            lf_fields_set(self.ctx, which, v.data_ptr(), v.numel() * v.element_size(), True)
        else:
            v = np.ascontiguousarray(value)
            lf_fields_set(self.ctx, which, v.ctypes.data, v.nbytes, False)

    def step(self, n: int = 1):
        lf_step(self.ctx, n)

    def set_variant(self, variant: str = "march", param: int = 0):
        code = {"march": LF_VARIANT_MARCH, "tile": LF_VARIANT_TILE, "march2": LF_VARIANT_MARCH2,
                "split3": LF_VARIANT_SPLIT3}[variant]
        lf_set_kernel_variant(self.ctx, code, param)

    def set_t_solver(self, solver: str = "explicit"):
        code = {"explicit": 0, "implicit": 1}[solver]
        _ok(lib().lf_set_t_solver(self.ctx, code), "lf_set_t_solver")

    def tune(self, reps: int = 5):
        """Autotune the kernel variant and shape; returns (variant, param, ms)."""
        return lf_tune(self.ctx, reps)

    def set_stencil(self, stencil: str = "compact"):
        code = {"compact": LF_STENCIL_COMPACT, "isotropic": LF_STENCIL_ISOTROPIC}[stencil]
        _ok(lib().lf_set_stencil(self.ctx, code), "lf_set_stencil")

    def diag(self):
        d, rc = lf_diag(self.ctx)
        out = d.as_dict()
        out["rc"] = rc
        return out

    def layers(self):
        return lf_diag_layers(self.ctx, self.shape[0])

    def structure_factor(self):
        return lf_structure_factor(self.ctx, min(self.shape) // 2 + 1)

    def save(self, path):
        lf_save(self.ctx, path)

    def load(self, path):
        lf_load(self.ctx, path)

    @property
    def step_count(self):
        return lf_step_count(self.ctx)

    def set_pass_timing(self, enable: bool = True):
        """CUDA events at the pass boundaries of every later three-pass 3D step."""
        _ok(lf_set_pass_timing(self.ctx, enable), "lf_set_pass_timing")

    def pass_times(self):
        """Milliseconds of the passes (A, B, C) of the last step, [] if it recorded none."""
        rc, ms = lf_pass_times(self.ctx)
        _ok(rc, "lf_pass_times")
        return ms

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------- diagnostics, no allocation
def lf_diag_sums_noalloc(d, nx, ny, nz, walls, precision, phi_ptr, T_ptr, moments_ptr, b, kappa, c, Tc,
                         out_ptr, stream_ptr) -> int:
    """Return code of lf_diag_sums_noalloc (enqueued; no allocation)."""
    L = lib()
    if not getattr(L, "_noalloc_ready", False):
        L.lf_diag_sums_noalloc.argtypes = [C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                           C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.lf_diag_sums_noalloc.restype = C.c_int
        L._noalloc_ready = True
    return L.lf_diag_sums_noalloc(d, nx, ny, nz, walls, precision, C.c_void_p(phi_ptr), C.c_void_p(T_ptr),
                                  C.c_void_p(moments_ptr), b, kappa, c, Tc, C.c_void_p(out_ptr),
                                  C.c_void_p(stream_ptr))


# ------------------------------------------------------------- ensembles
def _ens_lib():
    L = lib()
    if not getattr(L, "_ens_ready", False):
        vp = C.c_void_p
        L.lf_ens_create.argtypes = [C.c_int, C.POINTER(lf_grid), C.POINTER(lf_walls), C.POINTER(lf_params), vp,
                                    C.POINTER(vp)]
        L.lf_ens_tune.argtypes = [vp, C.c_int]
        L.lf_ens_rows.argtypes = [vp, C.c_int]
        L.lf_ens_param.argtypes = [vp, C.c_int]
        L.lf_ens_prune.argtypes = [vp, C.POINTER(C.c_int)]
        L.lf_ens_active.argtypes = [vp, C.c_int]
        L.lf_ens_step.argtypes = [vp, C.c_int64]
        L.lf_ens_run.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.lf_ens_sync.argtypes = [vp]
        L.lf_ens_destroy.argtypes = [vp]
        L.lf_ens_destroy.restype = None
        for fn in ("lf_ens_create", "lf_ens_tune", "lf_ens_rows", "lf_ens_param", "lf_ens_prune", "lf_ens_active",
                   "lf_ens_step", "lf_ens_run", "lf_ens_sync"):
            getattr(L, fn).restype = C.c_int
        L._ens_ready = True
    return L


def lf_ens_create(grids, walls, params, stream_ptr=0):
    n = len(grids)
    G = (lf_grid * n)(*grids)
    W = (lf_walls * n)(*walls)
    P = (lf_params * n)(*params)
    ens = C.c_void_p()
    _ok(_ens_lib().lf_ens_create(n, G, W, P, C.c_void_p(stream_ptr), C.byref(ens)), "lf_ens_create")
    return ens


def lf_ens_tune(ens, reps: int = 5) -> None:
    _ok(_ens_lib().lf_ens_tune(ens, reps), "lf_ens_tune")


def lf_ens_rows(ens, run: int) -> int:
    return _ok(_ens_lib().lf_ens_rows(ens, run), "lf_ens_rows")


def lf_ens_param(ens, run: int) -> int:
    return _ok(_ens_lib().lf_ens_param(ens, run), "lf_ens_param")


def lf_ens_prune(ens) -> int:
    n = C.c_int()
    _ok(_ens_lib().lf_ens_prune(ens, C.byref(n)), "lf_ens_prune")
    return n.value


def lf_ens_active(ens, run: int) -> bool:
    return bool(_ok(_ens_lib().lf_ens_active(ens, run), "lf_ens_active"))


def lf_ens_step(ens, nsteps: int) -> None:
    _ok(_ens_lib().lf_ens_step(ens, nsteps), "lf_ens_step")


def lf_ens_run(ens, run: int):
    ctx = C.c_void_p()
    _ok(_ens_lib().lf_ens_run(ens, run, C.byref(ctx)), "lf_ens_run")
    return ctx


def lf_ens_sync(ens) -> None:
    _ok(_ens_lib().lf_ens_sync(ens), "lf_ens_sync")


def lf_ens_destroy(ens) -> None:
    _ens_lib().lf_ens_destroy(ens)


class _RunView(Lattice):
    """Field access to one run of an ensemble (no ownership)."""

    def __init__(self, ens, ctx, shape):  # noqa: D401 - no super().__init__: the context exists
        import torch
        self.torch = torch
        self.device = torch.device("cuda:0")
        self.ctx = ctx
        self.Q = 9
        self.shape = shape
        self.N = int(np.prod(shape))
        self._ens = ens

    def close(self):
        self.ctx = None

    def step(self, n: int = 1):
        raise RuntimeError("runs of an ensemble are advanced by Ensemble.step")


class Ensemble:
    """Independent 2D FP32 runs advanced together (include/lf_ens.h)."""

    def __init__(self, members, stream=None, **common):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        grids, walls, params, self.shapes = [], [], [], []
        for m in members:
            kw = dict(common)
            kw.update(m)
            grids.append(lf_grid(d=2, nx=kw["nx"], ny=kw["ny"], nz=1))
            walls.append(lf_walls(walls=kw.get("walls", 1), t_wall_mode=kw.get("t_wall_mode", 0),
                                  T_w=kw.get("T_w", 0.5)))
            params.append(lf_params(b=kw.get("b", 1.0), kappa=kw.get("kappa", -0.025), c=kw.get("c", 0.02),
                                    Gamma=kw.get("Gamma", 0.05), Tc=kw.get("Tc", 1.0), T0=kw.get("T0", 1.1),
                                    xi=kw.get("xi", 0.01), tau=kw.get("tau", 1.0), n0=kw.get("n0", 1.0),
                                    phi_amp=kw.get("phi_amp", 0.05), seed=kw.get("seed", 1), precision=LF_FP32,
                                    hydro=kw.get("hydro", 1), ideal_mode=0,
                                    stencil={"compact": LF_STENCIL_COMPACT,
                                             "isotropic": LF_STENCIL_ISOTROPIC}[kw.get("stencil", "compact")]))
            self.shapes.append((kw["ny"], kw["nx"]))
        self.ens = lf_ens_create(grids, walls, params, self.stream.cuda_stream)
        self.n = len(members)

    def step(self, n: int = 1):
        lf_ens_step(self.ens, n)

    def tune(self, reps: int = 5):
        lf_ens_tune(self.ens, reps)

    def rows(self, run: int) -> int:
        return lf_ens_rows(self.ens, run)

    def prune(self) -> int:
        """Retire the runs that went non-finite; returns the runs still stepped."""
        return lf_ens_prune(self.ens)

    def active(self, run: int) -> bool:
        return lf_ens_active(self.ens, run)

    def param(self, run: int) -> int:
        """LF_VARIANT_MARCH2 param that reproduces run `run` stepped alone."""
        return lf_ens_param(self.ens, run)

    def run(self, r: int) -> Lattice:
        return _RunView(self.ens, lf_ens_run(self.ens, r), self.shapes[r])

    def sync(self):
        lf_ens_sync(self.ens)

    def close(self):
        if getattr(self, "ens", None) is not None and self.ens.value:
            lf_ens_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- surrogate
def _sur_lib():
    L = lib()
    if not getattr(L, "_sur_ready", False):
        vp = C.c_void_p
        L.lf_sur_conv3x3.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_int, vp, vp,
                                     vp, vp, vp, vp, vp, vp, vp]
        L.lf_sur_conv3x3.restype = C.c_int
        L._sur_ready = True
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def lf_sur_conv3x3(B, NY, NX, cin, cout, inp, w, bias=None, relu=0, resid=None, mask=None, out=None, out2=None,
                   zout=None, x4=None, y4=None, err=None, stream=None):
    """One tensor-core 3x3 convolution (see include/lf_sur.h); torch tensors in."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _ok(_sur_lib().lf_sur_conv3x3(B, NY, NX, cin, cout, _p(inp), _p(w), _p(bias), relu, _p(resid), _p(mask),
                                  _p(out), _p(out2), _p(zout), _p(x4), _p(y4), _p(err), C.c_void_p(s.cuda_stream)),
        "lf_sur_conv3x3")


def pad_nhwc(h):
    """[B, NY, NX, C] torch tensor -> padded [B, NY + 2, NX + 2, C] (periodic x, zero y)."""
    import torch
    h = torch.cat([h[:, :, -1:], h, h[:, :, :1]], dim=2)
    z = torch.zeros_like(h[:, :1])
    return torch.cat([z, h, z], dim=1).contiguous()


class lf_sur_norm(C.Structure):
    _fields_ = [("scale", C.c_double * 4), ("offset", C.c_double * 4)]


class lf_sur_report(C.Structure):
    _fields_ = [("windows_done", C.c_int), ("surrogate_windows", C.c_int), ("shadow_checks", C.c_int),
                ("fallbacks", C.c_int), ("max_phi_l2_err", C.c_double), ("max_sk_err", C.c_double),
                ("last_err", C.c_double), ("t_surrogate_s", C.c_double), ("t_shadow_s", C.c_double),
                ("t_plain_s", C.c_double), ("rejected", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _sur2_lib():
    L = _sur_lib()
    if not getattr(L, "_sur2_ready", False):
        vp = C.c_void_p
        L.lf_sur_conv3x3_wgrad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_size_t, vp,
                                           vp, vp]
        L.lf_sur_wgrad_scratch_floats.argtypes = [C.c_int, C.c_int]
        L.lf_sur_wgrad_scratch_floats.restype = C.c_size_t
        L.lf_sur_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(lf_sur_norm), vp, C.POINTER(vp)]
        L.lf_sur_param_count.argtypes = []
        L.lf_sur_param_count.restype = C.c_size_t
        L.lf_sur_get_params.argtypes = [vp, vp]
        L.lf_sur_set_params.argtypes = [vp, vp]
        L.lf_sur_grads.argtypes = [vp, vp, vp, C.c_int, C.POINTER(C.c_double), vp]
        L.lf_sur_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, C.POINTER(C.c_double)]
        L.lf_sur_predict.argtypes = [vp, vp, vp, C.c_int]
        L.lf_sur_set_clip.argtypes = [vp, C.c_float]
        L.lf_sur_run.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(lf_sur_report)]
        L.lf_sur_destroy.argtypes = [vp]
        L.lf_sur_destroy.restype = None
        for fn in ("lf_sur_conv3x3_wgrad", "lf_sur_create", "lf_sur_get_params", "lf_sur_set_params",
                   "lf_sur_grads", "lf_sur_train_step", "lf_sur_predict", "lf_sur_run", "lf_sur_set_clip"):
            getattr(L, fn).restype = C.c_int
        L._sur2_ready = True
    return L


def lf_sur_conv3x3_wgrad(B, NY, NX, cin, cout, h, g, dW, err, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    n = _sur2_lib().lf_sur_wgrad_scratch_floats(cin, cout)
    part = torch.empty(n, dtype=torch.float32, device=h.device)
    _ok(_sur2_lib().lf_sur_conv3x3_wgrad(B, NY, NX, cin, cout, _p(h), _p(g), _p(part), n, _p(dW), _p(err),
                                         C.c_void_p(s.cuda_stream)), "lf_sur_conv3x3_wgrad")
    return part


class Surrogate:
    """The learned surrogate of include/lf_sur.h (marshalling only)."""

    def __init__(self, NY, NX, max_batch, scale, offset, seed=7, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nm = lf_sur_norm()
        for c in range(4):
            nm.scale[c] = float(scale[c])
            nm.offset[c] = float(offset[c])
        self.h = C.c_void_p()
        _ok(_sur2_lib().lf_sur_create(NY, NX, max_batch, seed, C.byref(nm), C.c_void_p(self.stream.cuda_stream),
                                      C.byref(self.h)), "lf_sur_create")
        self.NY, self.NX = NY, NX

    @staticmethod
    def param_count():
        return int(_sur2_lib().lf_sur_param_count())

    def get_params(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        _ok(_sur2_lib().lf_sur_get_params(self.h, out.ctypes.data), "lf_sur_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _ok(_sur2_lib().lf_sur_set_params(self.h, p.ctypes.data), "lf_sur_set_params")

    def grads(self, x, y):
        loss = C.c_double()
        g = np.empty(self.param_count(), dtype=np.float32)
        _ok(_sur2_lib().lf_sur_grads(self.h, _p(x), _p(y), x.shape[0], C.byref(loss), g.ctypes.data), "lf_sur_grads")
        return loss.value, g

    def loss(self, x, y):
        loss = C.c_double()
        _ok(_sur2_lib().lf_sur_grads(self.h, _p(x), _p(y), x.shape[0], C.byref(loss), None), "lf_sur_grads")
        return loss.value

    def train_step(self, x, y, lr):
        loss = C.c_double()
        _ok(_sur2_lib().lf_sur_train_step(self.h, _p(x), _p(y), x.shape[0], lr, C.byref(loss)), "lf_sur_train_step")
        return loss.value

    def set_clip(self, max_norm: float):
        _ok(_sur2_lib().lf_sur_set_clip(self.h, max_norm), "lf_sur_set_clip")

    def predict(self, x):
        y = self.torch.empty_like(x)
        _ok(_sur2_lib().lf_sur_predict(self.h, _p(x), _p(y), x.shape[0]), "lf_sur_predict")
        return y

    def run(self, lattice, K, nwindows, shadow_every, threshold):
        rep = lf_sur_report()
        _ok(_sur2_lib().lf_sur_run(self.h, lattice.ctx, K, nwindows, shadow_every, threshold, C.byref(rep)),
            "lf_sur_run")
        return rep.as_dict()

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _sur2_lib().lf_sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

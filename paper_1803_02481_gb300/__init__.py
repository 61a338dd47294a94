"""GB300 BoxMG: Python binding of the C ABI in include/boxmg.h.

Argument marshalling only: every step of setup and solve runs in the CUDA
library ``libboxmg.so`` (built in-tree by ``build.py``).  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is not
built, or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "BMG_OK", "BMG_EINVAL", "BMG_ENOMEM", "BMG_ECUDA", "BMG_ENOCONV", "BMG_ENAN", "BMG_ETIMEOUT",
    "BMG_FP64", "BMG_FP32_REFINE", "BoxMGError", "Options", "Info", "lib", "library_path",
    "default_options", "setup", "Hierarchy", "solve_host", "EXPORTED", "EXPORTED3", "setup3",
    "Hierarchy3", "STENCIL3_OFFSETS",
]

BMG_OK, BMG_EINVAL, BMG_ENOMEM, BMG_ECUDA, BMG_ENOCONV, BMG_ENAN, BMG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
BMG_FP64, BMG_FP32_REFINE = 0, 1
BMG_SOLVER_VCYCLE, BMG_SOLVER_PCG = 0, 1
BMG_SMOOTH_POINT, BMG_SMOOTH_XLINE, BMG_SMOOTH_YLINE, BMG_SMOOTH_ALTLINE = 0, 1, 2, 3
MAX_COARSEST = 1024


class Options(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("precision", ctypes.c_int),
                ("interp_residual_term", ctypes.c_int), ("coarse_threshold", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("log_coefficients", ctypes.c_int),
                ("solver", ctypes.c_int), ("aniso_r", ctypes.c_double),
                ("cell_aspect", ctypes.c_double), ("bc_beta", ctypes.c_double * 4),
                ("smoother", ctypes.c_int), ("coarse_ctas", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("threshold", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("coarse_ctas", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BoxMGError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().bmg_strerror(code).decode()
        detail = lib().bmg_last_error().decode()
        super().__init__(f"{where}: {msg} (code {code})" + (f" [{detail}]" if detail else ""))
        self.code = code


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_HP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); every symbol include/boxmg.h declares
EXPORTED = {
    "bmg_default_options": (None, [ctypes.POINTER(Options)]),
    "bmg_strerror": (ctypes.c_char_p, [_i]),
    "bmg_last_error": (ctypes.c_char_p, []),
    "bmg_setup": (_i, [_vp, _i, _i, ctypes.POINTER(Options), _vp, _HP]),
    "bmg_solve": (_i, [_vp, _vp, _vp, _d, ctypes.POINTER(Info), _vp]),
    "bmg_residual_history": (_i, [_vp, _vp, _i, ctypes.POINTER(_i)]),
    "bmg_set_max_cycles": (_i, [_vp, _i]),
    "bmg_solve_host": (_i, [_vp, _vp, _vp, _i, _i, ctypes.POINTER(Options), _d,
                            ctypes.POINTER(Info), _vp]),
    "bmg_destroy": (None, [_vp]),
    "bmg_num_levels": (_i, [_vp, ctypes.POINTER(_i)]),
    "bmg_level_shape": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "bmg_level_prescaled": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "bmg_level_stencil": (_i, [_vp, _i, _vp]),
    "bmg_level_interp": (_i, [_vp, _i, _vp]),
    "bmg_coarse_factor": (_i, [_vp, _vp, _i]),
    "bmg_op_relax": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp]),
    "bmg_op_residual": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "bmg_op_restrict": (_i, [_vp, _i, _vp, _vp, _vp]),
    "bmg_op_interp": (_i, [_vp, _i, _vp, _vp, _vp]),
    "bmg_assemble_backward": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "bmg_batch_setup": (_i, [_i, _vp, _vp, ctypes.POINTER(Options), _vp, _HP]),
    "bmg_batch_solve": (_i, [_vp, _vp, _vp, _d, _vp, _vp]),
    "bmg_batch_size": (_i, [_vp, ctypes.POINTER(_i)]),
    "bmg_batch_destroy": (None, [_vp]),
    "bmg_calibrate": (_i, [_vp, _vp]),
    "bmg_predict_cycle_us": (_i, [_vp, _i, ctypes.POINTER(_d)]),
    "bmg_max_coarse_ctas": (_i, [_i, ctypes.POINTER(_i)]),
    "bmg_residual_norm_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp]),
    "bmg_dd_part_create": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _HP]),
    "bmg_dd_part_destroy": (None, [_vp]),
    "bmg_dd_relax_colour": (_i, [_vp, _i, _i, _vp]),
    "bmg_dd_residual": (_i, [_vp, _i, _vp]),
    "bmg_dd_restrict": (_i, [_vp, _i, _vp]),
    "bmg_dd_interp": (_i, [_vp, _i, _vp]),
    "bmg_dd_norms": (_i, [_vp, _i, _vp, _vp]),
    "bmg_dd_copy": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "bmg_dd_block": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "bmg_op_vcycle_from": (_i, [_vp, _i, _vp, _vp, _vp]),
    "bmg_selftest_bounded_wait": (_i, [_vp]),
    "bmg_kernel_launches": (ctypes.c_longlong, []),
    "bmg_profile_set": (_i, [_i]),
    "bmg_profile_read": (_i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
}

# every symbol include/boxmg3d.h declares
EXPORTED3 = {
    "bmg3_setup": (_i, [_vp, _i, _i, _i, ctypes.POINTER(Options), _vp, _HP]),
    "bmg3_solve": (_i, [_vp, _vp, _vp, _d, ctypes.POINTER(Info), _vp]),
    "bmg3_destroy": (None, [_vp]),
    "bmg3_num_levels": (_i, [_vp, ctypes.POINTER(_i)]),
    "bmg3_level_shape": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "bmg3_level_stencil": (_i, [_vp, _i, _vp]),
    "bmg3_level_interp": (_i, [_vp, _i, _vp]),
}

PROF_CLASSES = {"fine_smooth": 1, "fine_resid": 2, "fine_interp": 3, "coarse_kernel": 4,
                "other_levels": 5, "norm": 6, "vcycle": 7, "krylov": 8}


CALIBRATION_KEYS = ("launch_us", "sync_us", "gpu_gbs", "gpu_gflops64", "gpu_gflops32", "cta_gbs",
                    "cta_gflops64", "cta_gflops32", "cluster_sync_us", "cluster_ctas")


def calibrate(stream=None) -> dict:
    """Measure the level-schedule cost-model parameters on this GPU."""
    out = (ctypes.c_double * len(CALIBRATION_KEYS))()
    _check(lib().bmg_calibrate(_stream(stream), out), "bmg_calibrate")
    return dict(zip(CALIBRATION_KEYS, list(out)))


def max_coarse_ctas(precision: int = BMG_FP64) -> int:
    """Largest thread-block cluster the coarse kernel can use on this GPU
    (1: none)."""
    out = ctypes.c_int()
    _check(lib().bmg_max_coarse_ctas(int(precision), ctypes.byref(out)), "bmg_max_coarse_ctas")
    return out.value


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().bmg_kernel_launches())


def selftest_bounded_wait(stream=None) -> int:
    """Run the sweeps' bounded mbarrier wait on a phase nothing completes;
    returns the status code (BMG_ETIMEOUT is the expected result)."""
    return int(lib().bmg_selftest_bounded_wait(_stream(stream)))


def profile_set(classes=()):
    """Start live CUDA-event timing of the named kernel classes (PROF_CLASSES)."""
    mask = 0
    for c in classes:
        mask |= 1 << PROF_CLASSES[c]
    _check(lib().bmg_profile_set(mask), "bmg_profile_set")


def profile_read(name: str):
    """(brackets, total_ms) of one class since profile_set."""
    n, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib().bmg_profile_read(PROF_CLASSES[name], ctypes.byref(n), ctypes.byref(ms)), "bmg_profile_read")
    return n.value, ms.value

_LIB = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; call paper_1803_02481_gb300.build.build()")
        cdll = ctypes.CDLL(path)
        for name, (res, args) in {**EXPORTED, **EXPORTED3}.items():
            fn = getattr(cdll, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = cdll
    return _LIB


def _check(code: int, where: str, ok=(BMG_OK,)):
    if code not in ok:
        raise BoxMGError(code, where)
    return code


def default_options(**kw) -> Options:
    o = Options()
    lib().bmg_default_options(ctypes.byref(o))
    types = dict(Options._fields_)
    for k, v in kw.items():
        if k not in types:
            raise TypeError(f"unknown option {k!r}")
        t = types[k]
        if t is ctypes.c_double:
            setattr(o, k, float(v))
        elif t is ctypes.c_int:
            setattr(o, k, int(v))
        else:   # bc_beta: west, east, south, north; None for u = 0
            setattr(o, k, t(*[-1.0 if b is None else float(b) for b in v]))
    return o


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, name, shape=None):
    """Device pointer of a contiguous float64 CUDA tensor; with `shape`, the
    tensor must have exactly that shape (the kernels index it by the sizes
    passed beside it, so a smaller tensor would be read or written past its
    end on the device)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise TypeError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Hierarchy:
    """A BoxMG hierarchy living on the GPU (wraps ``bmg_hierarchy*``)."""

    def __init__(self, handle: ctypes.c_void_p, nx: int, ny: int, options: Options):
        self._h = handle
        self.nx, self.ny = nx, ny
        self.options = options

    # -- lifetime -----------------------------------------------------------
    def destroy(self):
        if self._h:
            lib().bmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # -- solve ----------------------------------------------------------------
    def solve(self, b, x=None, tol=1e-10, stream=None, allow_noconv=False):
        """Solve A x = b (b, x: (ny, nx) float64 CUDA tensors; x is the initial
        guess, zero if None, overwritten with the solution).  Returns
        (x, Info)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        info = Info()
        ok = (BMG_OK, BMG_ENOCONV) if allow_noconv else (BMG_OK,)
        shape = (self.ny, self.nx)
        _check(lib().bmg_solve(self._h, _dev(b, "b", shape), _dev(x, "x", shape), float(tol),
                               ctypes.byref(info), _stream(stream)), "bmg_solve", ok)
        return x, info

    def set_max_cycles(self, max_cycles: int):
        _check(lib().bmg_set_max_cycles(self._h, int(max_cycles)), "bmg_set_max_cycles")
        self.options.max_cycles = int(max_cycles)

    def predict_cycle_us(self, threshold: int) -> float:
        us = ctypes.c_double()
        _check(lib().bmg_predict_cycle_us(self._h, int(threshold), ctypes.byref(us)), "bmg_predict_cycle_us")
        return us.value

    def residual_history(self) -> np.ndarray:
        """Relative residuals of the last solve (before cycle 1, after each)."""
        n = ctypes.c_int()
        out = np.zeros(4096)
        _check(lib().bmg_residual_history(self._h, out.ctypes.data_as(ctypes.c_void_p), out.size,
                                          ctypes.byref(n)), "bmg_residual_history")
        return out[:min(n.value, out.size)].copy()

    # -- introspection ----------------------------------------------------------
    @property
    def nlevels(self) -> int:
        n = ctypes.c_int()
        _check(lib().bmg_num_levels(self._h, ctypes.byref(n)), "bmg_num_levels")
        return n.value

    def level_prescaled(self, level: int) -> bool:
        out = ctypes.c_int()
        _check(lib().bmg_level_prescaled(self._h, level, ctypes.byref(out)), "bmg_level_prescaled")
        return bool(out.value)

    def level_shape(self, level: int):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        _check(lib().bmg_level_shape(self._h, level, ctypes.byref(nx), ctypes.byref(ny)), "bmg_level_shape")
        return nx.value, ny.value

    def level_stencil(self, level: int) -> dict:
        nx, ny = self.level_shape(level)
        out = np.zeros((5, ny, nx))
        _check(lib().bmg_level_stencil(self._h, level, out.ctypes.data_as(ctypes.c_void_p)),
               "bmg_level_stencil")
        return dict(zip(("C", "W", "S", "SW", "NW"), out))

    def level_interp(self, level: int) -> dict:
        ncx, ncy = self.level_shape(level - 1)
        out = np.zeros((8, ncy + 1, ncx + 1))
        _check(lib().bmg_level_interp(self._h, level, out.ctypes.data_as(ctypes.c_void_p)),
               "bmg_level_interp")
        return dict(zip(("XW", "XE", "YS", "YN", "CSW", "CSE", "CNW", "CNE"), out))

    def coarse_factor(self) -> np.ndarray:
        nx, ny = self.level_shape(0)
        n0 = nx * ny
        out = np.zeros((n0, n0))
        _check(lib().bmg_coarse_factor(self._h, out.ctypes.data_as(ctypes.c_void_p), n0),
               "bmg_coarse_factor")
        return out

    # -- single operations --------------------------------------------------------
    def _grid(self, level):
        nx, ny = self.level_shape(level)
        return ny, nx

    def op_relax(self, level, x, b, nu=1, reverse=False, stream=None):
        g = self._grid(level)
        _check(lib().bmg_op_relax(self._h, level, _dev(x, "x", g), _dev(b, "b", g), int(nu),
                                  int(bool(reverse)), _stream(stream)), "bmg_op_relax")
        return x

    def op_residual(self, level, x, b, r, stream=None):
        g = self._grid(level)
        _check(lib().bmg_op_residual(self._h, level, _dev(x, "x", g), _dev(b, "b", g), _dev(r, "r", g),
                                     _stream(stream)), "bmg_op_residual")
        return r

    def op_restrict(self, level, r, bc, stream=None):
        g, gc = self._grid(level), self._grid(level - 1)
        _check(lib().bmg_op_restrict(self._h, level, _dev(r, "r", g), _dev(bc, "bc", gc), _stream(stream)),
               "bmg_op_restrict")
        return bc

    def op_interp(self, level, xc, x, stream=None):
        g, gc = self._grid(level), self._grid(level - 1)
        _check(lib().bmg_op_interp(self._h, level, _dev(xc, "xc", gc), _dev(x, "x", g), _stream(stream)),
               "bmg_op_interp")
        return x

    def vcycle_from(self, level, b, x, stream=None):
        """x = one V-cycle on A_level x = b from x = 0 over levels 0..level
        (the agglomerated coarse cycle of Algorithm 2)."""
        g = self._grid(level)
        _check(lib().bmg_op_vcycle_from(self._h, level, _dev(b, "b", g), _dev(x, "x", g), _stream(stream)),
               "bmg_op_vcycle_from")
        return x

    def assemble_backward(self, u, lam, dtheta, stream=None):
        g = (self.ny, self.nx)
        _check(lib().bmg_assemble_backward(self._h, _dev(u, "u", g), _dev(lam, "lam", g),
                                           _dev(dtheta, "dtheta", g), _stream(stream)), "bmg_assemble_backward")
        return dtheta


def setup(k, options: Options | None = None, stream=None) -> Hierarchy:
    """BoxMG setup from cell coefficients k ((ny, nx) float64 CUDA tensor)."""
    if options is None:
        options = default_options()
    if k.dim() != 2:
        raise TypeError(f"k must be 2-D (ny, nx), got shape {tuple(k.shape)}")
    ny, nx = k.shape
    h = ctypes.c_void_p()
    _check(lib().bmg_setup(_dev(k, "k"), nx, ny, ctypes.byref(options), _stream(stream), ctypes.byref(h)),
           "bmg_setup")
    return Hierarchy(h, nx, ny, options)


class Hierarchy3:
    """A 3D BoxMG hierarchy (wraps ``bmg3_*``, include/boxmg3d.h)."""

    def __init__(self, h, nx, ny, nz):
        self._h, self.nx, self.ny, self.nz = h, nx, ny, nz

    def solve(self, b, x=None, tol=1e-10, stream=None, allow_noconv=False):
        """Solve A x = b (b, x: (nz, ny, nx) float64 CUDA tensors; x is the
        initial guess, zero if None, overwritten).  Returns (x, Info)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        info = Info()
        ok = (BMG_OK, BMG_ENOCONV) if allow_noconv else (BMG_OK,)
        shape = (self.nz, self.ny, self.nx)
        _check(lib().bmg3_solve(self._h, _dev(b, "b", shape), _dev(x, "x", shape), float(tol),
                                ctypes.byref(info), _stream(stream)), "bmg3_solve", ok)
        return x, info

    @property
    def nlevels(self) -> int:
        n = ctypes.c_int()
        _check(lib().bmg3_num_levels(self._h, ctypes.byref(n)), "bmg3_num_levels")
        return n.value

    def level_shape(self, level: int):
        nx, ny, nz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bmg3_level_shape(self._h, level, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz)),
               "bmg3_level_shape")
        return nx.value, ny.value, nz.value

    def level_stencil(self, level: int) -> np.ndarray:
        """(14, nz, ny, nx): C, then the negated couplings of the 13 negative
        offsets in the order STENCIL3_OFFSETS."""
        nx, ny, nz = self.level_shape(level)
        out = np.zeros((14, nz, ny, nx))
        _check(lib().bmg3_level_stencil(self._h, level, out.ctypes.data_as(ctypes.c_void_p)),
               "bmg3_level_stencil")
        return out

    def level_interp(self, level: int) -> np.ndarray:
        """(8, nz, ny, nx): weights of each point of level `level` to its
        parents, plane 4 cz + 2 cy + cx."""
        nx, ny, nz = self.level_shape(level)
        out = np.zeros((8, nz, ny, nx))
        _check(lib().bmg3_level_interp(self._h, level, out.ctypes.data_as(ctypes.c_void_p)),
               "bmg3_level_interp")
        return out

    def destroy(self):
        if self._h:
            lib().bmg3_destroy(self._h)
            self._h = None


# (di, dj, dk) of the 13 stored couplings of a 3D level, in storage order
STENCIL3_OFFSETS = ([(di, dj, -1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
                    + [(di, -1, 0) for di in (-1, 0, 1)] + [(-1, 0, 0)])


def setup3(k, options: Options | None = None, stream=None) -> Hierarchy3:
    """3D BoxMG setup from cell coefficients k ((nz, ny, nx) float64 CUDA
    tensor)."""
    if options is None:
        options = default_options()
    if k.dim() != 3:
        raise TypeError(f"k must be 3-D (nz, ny, nx), got shape {tuple(k.shape)}")
    nz, ny, nx = k.shape
    h = ctypes.c_void_p()
    _check(lib().bmg3_setup(_dev(k, "k"), nx, ny, nz, ctypes.byref(options), _stream(stream),
                            ctypes.byref(h)), "bmg3_setup")
    return Hierarchy3(h, nx, ny, nz)


class Batch:
    """Many independent square problems solved together (wraps ``bmg_batch*``)."""

    def __init__(self, ks, options: Options | None = None, stream=None):
        if options is None:
            options = default_options()
        self.n = [int(k.shape[0]) for k in ks]
        self._ks = ks
        kp = (ctypes.c_void_p * len(ks))(*[_dev(k, "k", (n, n)).value for k, n in zip(ks, self.n)])
        ns = (ctypes.c_int * len(ks))(*self.n)
        h = ctypes.c_void_p()
        _check(lib().bmg_batch_setup(len(ks), kp, ns, ctypes.byref(options), _stream(stream), ctypes.byref(h)),
               "bmg_batch_setup")
        self._h = h

    def solve(self, bs, xs, tol=1e-8, stream=None, allow_noconv=False):
        """Solve all problems in place (xs: initial guesses, overwritten).
        Returns the per-problem Info list."""
        m = len(self.n)
        if len(bs) != m or len(xs) != m:
            raise TypeError(f"expected {m} right-hand sides and iterates, got {len(bs)} and {len(xs)}")
        bp = (ctypes.c_void_p * m)(*[_dev(b, "b", (n, n)).value for b, n in zip(bs, self.n)])
        xp = (ctypes.c_void_p * m)(*[_dev(x, "x", (n, n)).value for x, n in zip(xs, self.n)])
        infos = (Info * m)()
        ok = (BMG_OK, BMG_ENOCONV) if allow_noconv else (BMG_OK,)
        _check(lib().bmg_batch_solve(self._h, bp, xp, float(tol), infos, _stream(stream)), "bmg_batch_solve", ok)
        return list(infos)

    def destroy(self):
        if self._h:
            lib().bmg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def residual_norm_noalloc(k, x, b, norms=None, stream=None):
    """(||b - A(k) x||_2, ||b||_2) into a 2-element float64 CUDA tensor,
    without any device allocation inside the library (see
    bmg_residual_norm_noalloc in include/boxmg.h)."""
    import torch
    if k.dim() != 2:
        raise TypeError(f"k must be 2-D (ny, nx), got shape {tuple(k.shape)}")
    ny, nx = k.shape
    if norms is None:
        norms = torch.zeros(2, dtype=torch.float64, device=k.device)
    if norms.numel() < 2:
        raise TypeError(f"norms must hold at least 2 float64 values, has {norms.numel()}")
    _check(lib().bmg_residual_norm_noalloc(_dev(k, "k"), _dev(x, "x", (ny, nx)), _dev(b, "b", (ny, nx)), nx, ny,
                                           _dev(norms, "norms"), _stream(stream)), "bmg_residual_norm_noalloc")
    return norms


def solve_host(k: np.ndarray, b: np.ndarray, x: np.ndarray, options: Options | None = None,
               tol: float = 1e-10, stream=None, allow_noconv=False) -> Info:
    """End-to-end solve from host arrays (copies, setup, solve, copy back in
    one C call).  x holds the initial guess and receives the solution."""
    for a, n in ((k, "k"), (b, "b"), (x, "x")):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError(f"{n} must be a C-contiguous float64 numpy array")
    if options is None:
        options = default_options()
    if k.ndim != 2 or b.shape != k.shape or x.shape != k.shape:
        raise TypeError(f"k, b and x must share one 2-D shape, got {k.shape}, {b.shape}, {x.shape}")
    ny, nx = k.shape
    info = Info()
    ok = (BMG_OK, BMG_ENOCONV) if allow_noconv else (BMG_OK,)
    _check(lib().bmg_solve_host(k.ctypes.data_as(_vp), b.ctypes.data_as(_vp), x.ctypes.data_as(_vp), nx, ny,
                                ctypes.byref(options), float(tol), ctypes.byref(info), _stream(stream)),
           "bmg_solve_host", ok)
    return info

"""GB300 self-gravity for gas cells and sink particles (STARFORGE methods paper, Sec. 2.2).

Thin binding over the C ABI of ``libsfg.so`` (``include/sfg.h``): argument
marshalling only -- every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current CUDA stream.  There
is no CPU fallback: if the compiled library or a GPU is missing, calls raise.

    tree = Tree(pos, mass, soft, is_sink, theta=0.5)     # sfg_build
    accel, phi = tree.accel(active)                       # sfg_accel
    d_pos, d_mass = tree.accel_vjp(active, cot_a, cot_phi)  # sfg_accel_vjp
    tree.close()                                          # sfg_free

``gravity(pos, mass, soft, is_sink, active, ...)`` wraps the three calls in a
``torch.autograd.Function`` (differentiable in ``pos`` and ``mass``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import _build

SFG_OK, SFG_EINVAL, SFG_ENOMEM, SFG_ECUDA, SFG_EOVERFLOW, SFG_ETIMEOUT = range(6)
FIELD_KEYS, FIELD_ORDER, FIELD_NODE_INT, FIELD_NODE_HQ, FIELD_NODE_F64, FIELD_FRAMES = 1, 2, 3, 4, 5, 6
FIELD_PARTICLE_F32, FIELD_NODE_F32 = 7, 8

_lock = threading.Lock()
_lib = None


class SfgError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _load().sfg_status_string(code).decode() if _lib is not None else f"status {code}"
        if _lib is not None and code == SFG_ECUDA:
            msg += f" ({_lib.sfg_last_cuda_error().decode()})"
        super().__init__(f"{what}: {msg}" if what else msg)


class Params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("theta", ctypes.c_double), ("leaf_size", ctypes.c_int),
                ("group_size", ctypes.c_int), ("list_depth", ctypes.c_int), ("quadrupole", ctypes.c_int),
                ("precision", ctypes.c_int), ("store_lists", ctypes.c_int), ("alloc", ctypes.c_void_p),
                ("free", ctypes.c_void_p), ("alloc_ctx", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("x0", ctypes.c_double * 3), ("L0", ctypes.c_double),
                ("n_groups", ctypes.c_int64), ("n_targets", ctypes.c_int64), ("n_p2p", ctypes.c_int64),
                ("n_p2m", ctypes.c_int64), ("n_overflow", ctypes.c_int64), ("n_clouds", ctypes.c_int32),
                ("n_launches", ctypes.c_int64),
                ("build_ms", ctypes.c_float), ("fwd_ms", ctypes.c_float), ("fwd_walk_ms", ctypes.c_float),
                ("vjp_ms", ctypes.c_float), ("vjp_walk_ms", ctypes.c_float), ("n_p2p_newton", ctypes.c_int64),
                ("list_walks", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["x0"] = list(self.x0)
        return d


def library_path() -> str:
    return _build.LIB


def _load():
    """Load libsfg.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.sfg_default_params.argtypes = [ctypes.POINTER(Params)]
        lib.sfg_default_params.restype = None
        lib.sfg_status_string.argtypes = [i32]
        lib.sfg_status_string.restype = ctypes.c_char_p
        lib.sfg_last_cuda_error.argtypes = []
        lib.sfg_last_cuda_error.restype = ctypes.c_char_p
        lib.sfg_build.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
        lib.sfg_build.restype = i32
        lib.sfg_build_batch.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i64), i32, ctypes.POINTER(Params), vp,
                                        ctypes.POINTER(vp)]
        lib.sfg_build_batch.restype = i32
        lib.sfg_accel.argtypes = [vp, vp, i64, vp, vp, vp]
        lib.sfg_accel.restype = i32
        lib.sfg_accel_vjp.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
        lib.sfg_accel_vjp.restype = i32
        lib.sfg_accel_tidal.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        lib.sfg_accel_tidal.restype = i32
        lib.sfg_tidal_timestep.argtypes = [vp, i64, ctypes.c_double, vp, vp]
        lib.sfg_tidal_timestep.restype = i32
        lib.sfg_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
        lib.sfg_fp32_peak.restype = i32
        lib.sfg_accel_jerk.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
        lib.sfg_accel_jerk.restype = i32
        lib.sfg_sink_timestep.argtypes = [vp, vp, vp, i64, ctypes.c_double, vp, vp]
        lib.sfg_sink_timestep.restype = i32
        lib.sfg_hermite_step.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(Params), ctypes.c_double, vp, vp, vp]
        lib.sfg_hermite_step.restype = i32
        lib.sfg_set_relative_criterion.argtypes = [vp, vp, ctypes.c_double, vp]
        lib.sfg_set_relative_criterion.restype = i32
        lib.sfg_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        lib.sfg_get_stats.restype = i32
        lib.sfg_cloud_times.argtypes = [vp, vp, vp]
        lib.sfg_cloud_times.restype = i32
        lib.sfg_set_timing.argtypes = [vp, i32]
        lib.sfg_set_timing.restype = i32
        lib.sfg_set_group_share.argtypes = [vp, i32, i32]
        lib.sfg_set_group_share.restype = i32
        lib.sfg_get_status.argtypes = [vp]
        lib.sfg_get_status.restype = i32
        lib.sfg_free.argtypes = [vp]
        lib.sfg_free.restype = None
        lib.sfg_export.argtypes = [vp, i32, vp, ctypes.c_size_t]
        lib.sfg_export.restype = i32
        lib.sfg_debug_lists.argtypes = [vp, vp, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                        vp, vp, vp, vp]
        lib.sfg_debug_lists.restype = i32
        _lib = lib
        return lib


def default_params(**kw) -> Params:
    p = Params()
    _load().sfg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if v is None:
            continue
        if k in ("quadrupole", "store_lists"):
            v = int(bool(v))
        setattr(p, k, v)
    return p


def _check(rc: int, what: str):
    if rc != SFG_OK:
        raise SfgError(rc, what)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return t.contiguous()


def _stream(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Tree:
    """A built tree over one cloud (``sfg_build``); owns its device memory."""

    def __init__(self, pos, mass, soft, is_sink=None, *, G: float = 1.0, theta: float = 0.5, leaf_size: int = 16,
                 group_size: int = 32, quadrupole: bool = True, precision: int = 0, store_lists: bool = True,
                 list_depth: int = 0, offsets=None):
        """offsets (host sequence of n_clouds + 1 ints) builds one forest over an
        ensemble of independent clouds (sfg_build_batch).  store_lists: evaluate
        from interaction lists stored by one walk (the adjoint reuses the
        forward's for the same active set) instead of walking per evaluation."""
        lib = _load()
        pos = _dev(pos, torch.float64, "pos")
        mass = _dev(mass, torch.float64, "mass")
        soft = _dev(soft, torch.float64, "soft")
        if pos.dim() != 2 or pos.shape[1] != 3:
            raise ValueError("pos must be [n, 3]")
        n = pos.shape[0]
        if mass.shape != (n,) or soft.shape != (n,):
            raise ValueError("mass and soft must be [n]")
        sink_ptr = None
        if is_sink is not None:
            is_sink = _dev(is_sink, torch.uint8, "is_sink")
            sink_ptr = is_sink.data_ptr()
        self.device = pos.device
        self.n = n
        self.params = default_params(G=G, theta=theta, leaf_size=leaf_size, group_size=group_size,
                                     quadrupole=quadrupole, precision=precision, store_lists=store_lists,
                                     list_depth=list_depth)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if offsets is None:
                rc = lib.sfg_build(pos.data_ptr(), mass.data_ptr(), soft.data_ptr(), sink_ptr, n,
                                   ctypes.byref(self.params), _stream(self.device), ctypes.byref(self._h))
            else:
                if len(offsets) < 2 or int(offsets[-1]) != n:
                    # the library only sees pointers: the total must match the arrays
                    raise SfgError(SFG_EINVAL, "sfg_build_batch: offsets[-1] must equal the number of particles")
                off = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
                rc = lib.sfg_build_batch(pos.data_ptr(), mass.data_ptr(), soft.data_ptr(), sink_ptr, off,
                                         len(offsets) - 1, ctypes.byref(self.params), _stream(self.device),
                                         ctypes.byref(self._h))
        _check(rc, "sfg_build" if offsets is None else "sfg_build_batch")

    # -- calls ------------------------------------------------------------
    def _active(self, active):
        if active is None:
            return None, self.n
        a = _dev(active, torch.int64, "active")
        return a, a.numel()

    def accel(self, active=None, out=None):
        a, na = self._active(active)
        if out is None:
            acc = torch.empty((na, 3), dtype=torch.float64, device=self.device)
            phi = torch.empty(na, dtype=torch.float64, device=self.device)
        else:
            acc, phi = out
            if not (isinstance(acc, torch.Tensor) and acc.is_cuda and acc.dtype == torch.float64
                    and acc.is_contiguous() and tuple(acc.shape) == (na, 3)):
                raise ValueError(f"out[0] must be a contiguous CUDA float64 tensor of shape [{na}, 3]")
            if phi is not None and not (isinstance(phi, torch.Tensor) and phi.is_cuda
                                        and phi.dtype == torch.float64 and phi.is_contiguous()
                                        and tuple(phi.shape) == (na,)):
                raise ValueError(f"out[1] must be None or a contiguous CUDA float64 tensor of shape [{na}]")
        with torch.cuda.device(self.device):
            rc = _load().sfg_accel(self._h, None if a is None else a.data_ptr(), na, acc.data_ptr(),
                                   phi.data_ptr() if phi is not None else None, _stream(self.device))
        _check(rc, "sfg_accel")
        return acc, phi

    def set_relative(self, g_prev=None, alpha: float = 0.0):
        """Relative opening criterion of Sec. 2.2 for the following walks:
        g_prev = |g| per particle (input order, CUDA float64), or None (off)."""
        ptr = None
        if g_prev is not None:
            g_prev = _dev(g_prev, torch.float64, "g_prev")
            ptr = g_prev.data_ptr()
        with torch.cuda.device(self.device):
            rc = _load().sfg_set_relative_criterion(self._h, ptr, float(alpha), _stream(self.device))
        _check(rc, "sfg_set_relative_criterion")

    def accel_jerk(self, vel, active=None):
        """(accel [n][3], phi [n], jerk [n][3]) at the active rows; vel [N][3] per particle."""
        a, na = self._active(active)
        vel = _dev(vel, torch.float64, "vel")
        acc = torch.empty((na, 3), dtype=torch.float64, device=self.device)
        phi = torch.empty(na, dtype=torch.float64, device=self.device)
        jerk = torch.empty((na, 3), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            rc = _load().sfg_accel_jerk(self._h, vel.data_ptr(), None if a is None else a.data_ptr(), na,
                                        acc.data_ptr(), phi.data_ptr(), jerk.data_ptr(), _stream(self.device))
        _check(rc, "sfg_accel_jerk")
        return acc, phi, jerk

    def sink_timestep(self, vel, eta: float, active=None):
        """Two-body timestep [n] of the active rows (Sec. 2.3), minima over the tree lists."""
        a, na = self._active(active)
        vel = _dev(vel, torch.float64, "vel")
        dt = torch.empty(na, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            rc = _load().sfg_sink_timestep(self._h, vel.data_ptr(), None if a is None else a.data_ptr(), na,
                                           float(eta), dt.data_ptr(), _stream(self.device))
        _check(rc, "sfg_sink_timestep")
        return dt

    def accel_tidal(self, active=None):
        """(accel [n][3], phi [n], tidal [n][6] = xx yy zz xy xz yz) at the active rows."""
        a, na = self._active(active)
        acc = torch.empty((na, 3), dtype=torch.float64, device=self.device)
        phi = torch.empty(na, dtype=torch.float64, device=self.device)
        tid = torch.empty((na, 6), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            rc = _load().sfg_accel_tidal(self._h, None if a is None else a.data_ptr(), na, acc.data_ptr(),
                                         phi.data_ptr(), tid.data_ptr(), _stream(self.device))
        _check(rc, "sfg_accel_tidal")
        return acc, phi, tid

    def accel_vjp(self, active, cot_a, cot_phi=None):
        a, na = self._active(active)
        cot_a = _dev(cot_a, torch.float64, "cot_a")
        if tuple(cot_a.shape) != (na, 3):
            raise ValueError(f"cot_a must be [{na}, 3] (one row per active index)")
        if cot_phi is not None:
            cot_phi = _dev(cot_phi, torch.float64, "cot_phi")
            if tuple(cot_phi.shape) != (na,):
                raise ValueError(f"cot_phi must be [{na}] (one entry per active index)")
        d_pos = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        d_mass = torch.empty(self.n, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            rc = _load().sfg_accel_vjp(self._h, None if a is None else a.data_ptr(), na, cot_a.data_ptr(),
                                       None if cot_phi is None else cot_phi.data_ptr(), d_pos.data_ptr(),
                                       d_mass.data_ptr(), _stream(self.device))
        _check(rc, "sfg_accel_vjp")
        return d_pos, d_mass

    def stats(self) -> dict:
        s = Stats()
        _check(_load().sfg_get_stats(self._h, ctypes.byref(s)), "sfg_get_stats")
        return s.as_dict()

    def set_group_share(self, rank: int, world: int):
        """Evaluate only share `rank` of `world` of the groups in later calls
        (sfg_set_group_share); (0, 1) evaluates everything."""
        _check(_load().sfg_set_group_share(self._h, int(rank), int(world)), "sfg_set_group_share")

    def set_timing(self, on: bool = True):
        _check(_load().sfg_set_timing(self._h, int(bool(on))), "sfg_set_timing")

    def cloud_times(self):
        """(forward, adjoint) per-cloud completion times in ms of the last walks (timing on)."""
        c = self.stats()["n_clouds"]
        f = np.zeros(c, np.float32)
        v = np.zeros(c, np.float32)
        _check(_load().sfg_cloud_times(self._h, f.ctypes.data, v.ctypes.data), "sfg_cloud_times")
        return f, v

    def status(self) -> int:
        return int(_load().sfg_get_status(self._h))

    def check(self):
        _check(self.status(), "device status")

    def export(self, field: int) -> np.ndarray:
        st = self.stats()
        n, nn = st["n"], st["n_nodes"]
        shapes = {FIELD_KEYS: ((n,), np.uint64), FIELD_ORDER: ((n,), np.int32), FIELD_NODE_INT: ((nn, 16), np.int32),
                  FIELD_NODE_HQ: ((nn,), np.uint64), FIELD_NODE_F64: ((nn, 11), np.float64),
                  FIELD_FRAMES: ((st["n_clouds"], 4), np.float64), FIELD_PARTICLE_F32: ((n, 4), np.float32),
                  FIELD_NODE_F32: ((nn, 9), np.float32)}
        shape, dt = shapes[field]
        out = np.zeros(shape, dt)
        _check(_load().sfg_export(self._h, field, out.ctypes.data, out.nbytes), "sfg_export")
        return out

    def debug_lists(self, active=None):
        """(groups [g,4] int64, p2m list, p2p list) as host numpy arrays."""
        lib = _load()
        a, na = self._active(active)
        ng, nm, npp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ap = None if a is None else a.data_ptr()
        s = _stream(self.device)
        _check(lib.sfg_debug_lists(self._h, ap, na, ctypes.byref(ng), ctypes.byref(nm), ctypes.byref(npp), None,
                                   None, None, s), "sfg_debug_lists")
        groups = np.zeros((ng.value, 4), np.int64)
        p2m = np.zeros(max(nm.value, 1), np.int32)
        p2p = np.zeros(max(npp.value, 1), np.int32)
        _check(lib.sfg_debug_lists(self._h, ap, na, ctypes.byref(ng), ctypes.byref(nm), ctypes.byref(npp),
                                   groups.ctypes.data, p2m.ctypes.data, p2p.ctypes.data, s), "sfg_debug_lists")
        return groups, p2m[:nm.value], p2p[:npp.value]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _load().sfg_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Gravity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, mass, soft, is_sink, active, kw):
        tree = Tree(pos.detach(), mass.detach(), soft.detach(), is_sink, **kw)
        acc, phi = tree.accel(active)
        tree.check()  # an out-of-range active index raises here instead of leaving rows unwritten
        ctx.tree = tree
        ctx.active = active
        return acc, phi

    @staticmethod
    def backward(ctx, g_acc, g_phi):
        # the tree lives as long as the autograd graph holds ctx, so that a
        # second backward (retain_graph=True) reuses it
        tree = ctx.tree
        g_acc = torch.zeros_like(g_acc) if g_acc is None else g_acc.contiguous()
        g_phi = None if g_phi is None else g_phi.contiguous()
        d_pos, d_mass = tree.accel_vjp(ctx.active, g_acc, g_phi)
        return d_pos, d_mass, None, None, None, None


def tidal_timestep(tidal: torch.Tensor, eta: float) -> torch.Tensor:
    """Tidal timestep sqrt(eta) (|T|_F^2 / 6)^(-1/4) of every row of tidal [n][6]."""
    tidal = _dev(tidal, torch.float64, "tidal")
    n = tidal.numel() // 6
    dt = torch.empty(n, dtype=torch.float64, device=tidal.device)
    with torch.cuda.device(tidal.device):
        rc = _load().sfg_tidal_timestep(tidal.data_ptr(), n, float(eta), dt.data_ptr(), _stream(tidal.device))
    _check(rc, "sfg_tidal_timestep")
    return dt


def hermite_step(pos, vel, mass, soft, dt: float, *, G: float = 1.0, theta: float = 0.5, leaf_size: int = 16,
                 group_size: int = 32, quadrupole: bool = True):
    """One modified Hermite step of sink particles (sfg_hermite_step, Sec. 2.3):
    returns (pos1, vel1) [n][3]; both field + jerk evaluations run in the
    library on a tree of these particles alone."""
    pos = _dev(pos, torch.float64, "pos")
    vel = _dev(vel, torch.float64, "vel")
    mass = _dev(mass, torch.float64, "mass")
    soft = _dev(soft, torch.float64, "soft")
    n = pos.shape[0]
    if pos.dim() != 2 or pos.shape[1] != 3 or tuple(vel.shape) != (n, 3):
        raise ValueError("pos and vel must be [n, 3]")
    if mass.shape != (n,) or soft.shape != (n,):
        raise ValueError("mass and soft must be [n]")
    prm = default_params(G=G, theta=theta, leaf_size=leaf_size, group_size=group_size, quadrupole=quadrupole)
    x1 = torch.empty_like(pos)
    v1 = torch.empty_like(vel)
    with torch.cuda.device(pos.device):
        rc = _load().sfg_hermite_step(pos.data_ptr(), vel.data_ptr(), mass.data_ptr(), soft.data_ptr(), n,
                                      ctypes.byref(prm), float(dt), x1.data_ptr(), v1.data_ptr(), _stream(pos.device))
    _check(rc, "sfg_hermite_step")
    return x1, v1


def fp32_peak(device=None) -> dict:
    """Measured FP32 FMA throughput of the device (sfg_fp32_peak): TFLOP/s and
    the timed launch's milliseconds."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    tf, ms = ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        rc = _load().sfg_fp32_peak(ctypes.byref(tf), ctypes.byref(ms), _stream(dev))
    _check(rc, "sfg_fp32_peak")
    return {"tflops": tf.value, "ms": ms.value}


def gravity(pos, mass, soft, is_sink=None, active=None, **kw):
    """(accel, phi) at the active particles, differentiable in pos and mass."""
    return _Gravity.apply(pos, mass, soft, is_sink, active, kw)


__all__ = ["Tree", "gravity", "hermite_step", "tidal_timestep", "fp32_peak", "Params", "Stats", "SfgError",
           "default_params", "library_path"]

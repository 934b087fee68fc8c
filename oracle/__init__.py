"""CPU FP64 oracle of the STARFORGE self-gravity path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2010_11254_gb300``) and never imports it.

The arithmetic lives in ``sfg_oracle.c`` (plain C, FP64, -ffp-contract=off);
this module compiles it with gcc into ``oracle/_lib`` and wraps it with ctypes.
Functions follow the STARFORGE methods paper, Sec. 2.2 (gravity) and
Sec. 2.2.1 (softening); see the C source for the passage each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfg_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libsfg_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        lib.sfgo_W.restype = ctypes.c_double
        lib.sfgo_W.argtypes = [ctypes.c_double]
        lib.sfgo_g.restype = ctypes.c_double
        lib.sfgo_g.argtypes = [ctypes.c_double]
        lib.sfgo_dg_over_u.restype = ctypes.c_double
        lib.sfgo_dg_over_u.argtypes = [ctypes.c_double]
        lib.sfgo_pair.restype = None
        lib.sfgo_pair.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _f64p]
        lib.sfgo_direct.restype = None
        lib.sfgo_direct.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _u8p, ctypes.c_double, ctypes.c_int64,
                                    _i64p, _f64p, _f64p]
        lib.sfgo_build.restype = _vp
        lib.sfgo_build.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _u8p, ctypes.c_int]
        lib.sfgo_free.restype = None
        lib.sfgo_free.argtypes = [_vp]
        lib.sfgo_info.restype = None
        lib.sfgo_info.argtypes = [_vp, _f64p, _i64p]
        lib.sfgo_keys.restype = None
        lib.sfgo_keys.argtypes = [_vp, _u64p, _i64p]
        lib.sfgo_nodes_int.restype = None
        lib.sfgo_nodes_int.argtypes = [_vp, _i64p]
        lib.sfgo_nodes_f64.restype = None
        lib.sfgo_nodes_f64.argtypes = [_vp, _f64p]
        lib.sfgo_walk.restype = ctypes.c_int64
        lib.sfgo_walk.argtypes = [_vp, _i64p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, _i64p, ctypes.c_int64]
        lib.sfgo_groups.restype = None
        lib.sfgo_groups.argtypes = [_vp, _i64p]
        lib.sfgo_group_targets.restype = None
        lib.sfgo_group_targets.argtypes = [_vp, _i64p]
        lib.sfgo_group_lists.restype = None
        lib.sfgo_group_lists.argtypes = [_vp, ctypes.c_int64, _i64p, _i64p]
        lib.sfgo_accel_group.restype = ctypes.c_int
        lib.sfgo_accel_group.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _i64p, ctypes.c_int64, _f64p, _f64p]
        lib.sfgo_eval_frozen.restype = ctypes.c_int
        lib.sfgo_eval_frozen.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _f64p, _f64p, _i64p, ctypes.c_int64,
                                         _f64p, _f64p]
        lib.sfgo_accel_pp.restype = None
        lib.sfgo_accel_pp.argtypes = [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _i64p, ctypes.c_int64,
                                      _f64p, _f64p, _i64p]
        lib.sfgo_vjp.restype = ctypes.c_int
        lib.sfgo_vjp.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _i64p, ctypes.c_int64, _f64p, _f64p, _f64p,
                                 _f64p]
        lib.sfgo_direct_tidal.restype = None
        lib.sfgo_direct_tidal.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _u8p, ctypes.c_double,
                                          ctypes.c_int64, _i64p, _f64p]
        lib.sfgo_tidal_group.restype = ctypes.c_int
        lib.sfgo_tidal_group.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _i64p, ctypes.c_int64, _f64p]
        lib.sfgo_tidal_dt.restype = None
        lib.sfgo_tidal_dt.argtypes = [ctypes.c_int64, _f64p, ctypes.c_double, _f64p]
        lib.sfgo_direct_jerk.restype = None
        lib.sfgo_direct_jerk.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p, _u8p, ctypes.c_double,
                                         ctypes.c_int64, _i64p, _f64p]
        lib.sfgo_jerk_group.restype = ctypes.c_int
        lib.sfgo_jerk_group.argtypes = [_vp, _f64p, ctypes.c_double, _i64p, ctypes.c_int64, _f64p]
        lib.sfgo_hermite_step.restype = None
        lib.sfgo_hermite_step.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p, ctypes.c_double, ctypes.c_double,
                                          _f64p, _f64p]
        lib.sfgo_direct_tstep.restype = None
        lib.sfgo_direct_tstep.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int64, _i64p, _f64p]
        lib.sfgo_tstep_group.restype = ctypes.c_int
        lib.sfgo_tstep_group.argtypes = [_vp, _f64p, ctypes.c_double, ctypes.c_double, _i64p, ctypes.c_int64,
                                         _f64p]
        lib.sfgo_set_relative.restype = None
        lib.sfgo_set_relative.argtypes = [_vp, _f64p, ctypes.c_double, ctypes.c_double]
        lib.sfgo_num_threads.restype = ctypes.c_int
        lib.sfgo_num_threads.argtypes = []
        _lib = lib
        return lib


def _p(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def num_threads() -> int:
    return int(_load().sfgo_num_threads())


# ---------------------------------------------------------------- kernel ----
def kernel_W(u: float) -> float:
    """Dimensionless softened potential W(u), phi = G m W(u)/h (Sec. 2.2.1, M4 spline)."""
    return float(_load().sfgo_W(float(u)))


def kernel_g(u: float) -> float:
    """Dimensionless force factor g(u), a = G m g(u)/h^3 (x_j - x_i)."""
    return float(_load().sfgo_g(float(u)))


def kernel_dg_over_u(u: float) -> float:
    return float(_load().sfgo_dg_over_u(float(u)))


def pair(r: float, hi: float, hj: float, si: int = 0, sj: int = 0):
    """(K, P, K'/r) of one pair under the pair rule of Sec. 2.2.1 (per unit G m_j)."""
    out = np.zeros(3)
    _load().sfgo_pair(float(r), float(hi), float(hj), int(si), int(sj), _p(out, _f64p))
    return float(out[0]), float(out[1]), float(out[2])


# ------------------------------------------------------------ direct sum ----
def direct(pos, mass, soft, is_sink=None, targets=None, G: float = 1.0):
    """FP64 direct sum a_i, phi_i over all j != i at the given targets."""
    pos, mass, soft = _f64(pos), _f64(mass), _f64(soft)
    n = pos.shape[0]
    tg = _i64(np.arange(n) if targets is None else targets)
    sink = _u8(np.zeros(n) if is_sink is None else is_sink)
    acc = np.zeros((tg.size, 3))
    phi = np.zeros(tg.size)
    _load().sfgo_direct(n, _p(pos, _f64p), _p(mass, _f64p), _p(soft, _f64p), _p(sink, _u8p), float(G), tg.size,
                        _p(tg, _i64p), _p(acc, _f64p), _p(phi, _f64p))
    return acc, phi


def direct_tidal(pos, mass, soft, is_sink=None, targets=None, G: float = 1.0):
    """FP64 direct-sum tidal tensor T = -grad grad Phi (Sec. 2.2) at the targets,
    as [n][6] = xx yy zz xy xz yz."""
    pos, mass, soft = _f64(pos), _f64(mass), _f64(soft)
    n = pos.shape[0]
    tg = _i64(np.arange(n) if targets is None else targets)
    sink = _u8(np.zeros(n) if is_sink is None else is_sink)
    T = np.zeros((tg.size, 6))
    _load().sfgo_direct_tidal(n, _p(pos, _f64p), _p(mass, _f64p), _p(soft, _f64p), _p(sink, _u8p), float(G),
                              tg.size, _p(tg, _i64p), _p(T, _f64p))
    return T


def direct_jerk(pos, vel, mass, soft, is_sink=None, targets=None, G: float = 1.0):
    """FP64 direct-sum jerk j = da/dt (Sec. 2.2) at the targets, [n][3]."""
    pos, vel, mass, soft = _f64(pos), _f64(vel), _f64(mass), _f64(soft)
    n = pos.shape[0]
    tg = _i64(np.arange(n) if targets is None else targets)
    sink = _u8(np.zeros(n) if is_sink is None else is_sink)
    J = np.zeros((tg.size, 3))
    _load().sfgo_direct_jerk(n, _p(pos, _f64p), _p(vel, _f64p), _p(mass, _f64p), _p(soft, _f64p), _p(sink, _u8p),
                             float(G), tg.size, _p(tg, _i64p), _p(J, _f64p))
    return J


def direct_tstep(pos, vel, mass, soft, eta: float, targets=None, G: float = 1.0):
    """Sink two-body timestep of Sec. 2.3 over all other particles (direct)."""
    pos, vel, mass, soft = _f64(pos), _f64(vel), _f64(mass), _f64(soft)
    n = pos.shape[0]
    tg = _i64(np.arange(n) if targets is None else targets)
    dt = np.zeros(tg.size)
    _load().sfgo_direct_tstep(n, _p(pos, _f64p), _p(vel, _f64p), _p(mass, _f64p), _p(soft, _f64p), float(G),
                              float(eta), tg.size, _p(tg, _i64p), _p(dt, _f64p))
    return dt


def hermite_step(pos, vel, mass, soft, dt: float, G: float = 1.0):
    """One modified Hermite step of sink particles (Sec. 2.3, predictor and
    corrector; two FP64 direct field + jerk evaluations, every particle a
    sink).  Returns (pos1, vel1), each [n][3]."""
    pos, vel, mass, soft = _f64(pos), _f64(vel), _f64(mass), _f64(soft)
    n = pos.shape[0]
    x1 = np.zeros((n, 3))
    v1 = np.zeros((n, 3))
    _load().sfgo_hermite_step(n, _p(pos, _f64p), _p(vel, _f64p), _p(mass, _f64p), _p(soft, _f64p), float(G),
                              float(dt), _p(x1, _f64p), _p(v1, _f64p))
    return x1, v1


def two_body_dt(pos, vel, mass, soft, eta: float, G: float = 1.0) -> float:
    """Smallest sink two-body timestep of Sec. 2.3 over all particles (direct)."""
    return float(direct_tstep(pos, vel, mass, soft, eta, G=G).min())


def tidal_dt(tidal, eta: float):
    """Tidal timestep sqrt(eta) (|T|_F^2 / 6)^(-1/4) of Sec. 2.3 for T given as [n][6]."""
    T = _f64(tidal).reshape(-1, 6)
    dt = np.zeros(T.shape[0])
    _load().sfgo_tidal_dt(T.shape[0], _p(T, _f64p), float(eta), _p(dt, _f64p))
    return dt


# ------------------------------------------------------------------ tree ----
class Tree:
    """Oracle oct-tree over one cloud (Sec. 2.2), built on a 2^21 grid."""

    NODE_INT_FIELDS = ["level", "first", "count", "parent", "child_first", "nchild",
                       "corner_x", "corner_y", "corner_z", "lo_x", "lo_y", "lo_z",
                       "hi_x", "hi_y", "hi_z", "cq_x", "cq_y", "cq_z", "hq"]
    GROUP_FIELDS = ["node", "tfirst", "tcount", "walked", "n_p2m", "n_p2p_leaves", "n_p2p",
                    "lo_x", "lo_y", "lo_z", "hi_x", "hi_y", "hi_z", "hq"]

    def __init__(self, pos, mass, soft, is_sink=None, leaf_size: int = 16):
        self._lib = _load()
        self.pos, self.mass, self.soft = _f64(pos), _f64(mass), _f64(soft)
        self.n = self.pos.shape[0]
        self.is_sink = _u8(np.zeros(self.n) if is_sink is None else is_sink)
        self.leaf_size = leaf_size
        self._h = self._lib.sfgo_build(self.n, _p(self.pos, _f64p), _p(self.mass, _f64p), _p(self.soft, _f64p),
                                       _p(self.is_sink, _u8p), int(leaf_size))
        if not self._h:
            raise ValueError("oracle tree build rejected its inputs")
        fr = np.zeros(4)
        nn = np.zeros(1, np.int64)
        self._lib.sfgo_info(self._h, _p(fr, _f64p), _p(nn, _i64p))
        self.x0 = fr[:3].copy()
        self.L0 = float(fr[3])
        self.n_nodes = int(nn[0])
        self.n_groups = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.sfgo_free(h)
            self._h = None

    def keys(self):
        key = np.zeros(self.n, np.uint64)
        order = np.zeros(self.n, np.int64)
        self._lib.sfgo_keys(self._h, _p(key, _u64p), _p(order, _i64p))
        return key, order

    def nodes_int(self) -> np.ndarray:
        out = np.zeros((self.n_nodes, 19), np.int64)
        self._lib.sfgo_nodes_int(self._h, _p(out, _i64p))
        return out

    def nodes_f64(self) -> np.ndarray:
        """Per node: M, com[3], Q[6] (xx yy zz xy xz yz), hmax, flo[3], fhi[3]."""
        out = np.zeros((self.n_nodes, 17))
        self._lib.sfgo_nodes_f64(self._h, _p(out, _f64p))
        return out

    def walk(self, active, group_size: int = 32, theta: float = 0.5, need=None) -> int:
        act = _i64(active)
        nd = None if need is None else _i64(need)
        self.n_groups = int(self._lib.sfgo_walk(self._h, _p(act, _i64p), act.size, int(group_size), float(theta),
                                                None if nd is None else _p(nd, _i64p),
                                                0 if nd is None else nd.size))
        return self.n_groups

    def groups(self) -> np.ndarray:
        out = np.zeros((self.n_groups, 14), np.int64)
        if self.n_groups:
            self._lib.sfgo_groups(self._h, _p(out, _i64p))
        return out

    def group_targets(self) -> np.ndarray:
        g = self.groups()
        out = np.zeros(int(g[:, 2].sum()) if len(g) else 0, np.int64)
        if out.size:
            self._lib.sfgo_group_targets(self._h, _p(out, _i64p))
        return out

    def group_lists(self, g: int, groups=None):
        groups = self.groups() if groups is None else groups
        p2m = np.zeros(int(groups[g, 4]), np.int64)
        p2p = np.zeros(int(groups[g, 5]), np.int64)
        self._lib.sfgo_group_lists(self._h, int(g), _p(p2m, _i64p), _p(p2p, _i64p))
        return p2m, p2p

    def accel_group(self, idx, G: float = 1.0, quadrupole: bool = True):
        idx = _i64(idx)
        acc = np.zeros((idx.size, 3))
        phi = np.zeros(idx.size)
        rc = self._lib.sfgo_accel_group(self._h, float(G), int(quadrupole), _p(idx, _i64p), idx.size,
                                        _p(acc, _f64p), _p(phi, _f64p))
        if rc != 0:
            raise ValueError("a requested row is not a walked target")
        return acc, phi

    def set_relative(self, g_prev=None, alpha: float = 0.0, G: float = 1.0):
        """Relative (acceleration-based) opening criterion of Sec. 2.2 for the
        next walks: |g_prev| per particle (input order) and tolerance alpha;
        None switches it off."""
        if g_prev is None:
            self._lib.sfgo_set_relative(self._h, None, 0.0, 0.0)
            return
        g = _f64(g_prev)
        self._lib.sfgo_set_relative(self._h, _p(g, _f64p), float(alpha), float(G))

    def jerk_group(self, vel, idx, G: float = 1.0):
        """Group-form jerk [n][3] on the last walk's lists (nodes by monopole)."""
        vel, idx = _f64(vel), _i64(idx)
        J = np.zeros((idx.size, 3))
        rc = self._lib.sfgo_jerk_group(self._h, _p(vel, _f64p), float(G), _p(idx, _i64p), idx.size, _p(J, _f64p))
        if rc != 0:
            raise ValueError("a requested row is not a walked target")
        return J

    def tstep_group(self, vel, eta: float, idx, G: float = 1.0):
        """Sink two-body timestep over the last walk's lists (nodes combined)."""
        vel, idx = _f64(vel), _i64(idx)
        dt = np.zeros(idx.size)
        rc = self._lib.sfgo_tstep_group(self._h, _p(vel, _f64p), float(G), float(eta), _p(idx, _i64p), idx.size,
                                        _p(dt, _f64p))
        if rc != 0:
            raise ValueError("a requested row is not a walked target")
        return dt

    def tidal_group(self, idx, G: float = 1.0, quadrupole: bool = True):
        """Group-form tidal tensor [n][6] (xx yy zz xy xz yz) on the last walk's lists."""
        idx = _i64(idx)
        T = np.zeros((idx.size, 6))
        rc = self._lib.sfgo_tidal_group(self._h, float(G), int(quadrupole), _p(idx, _i64p), idx.size,
                                        _p(T, _f64p))
        if rc != 0:
            raise ValueError("a requested row is not a walked target")
        return T

    def eval_frozen(self, pos, mass, idx, G: float = 1.0, quadrupole: bool = True):
        pos, mass, idx = _f64(pos), _f64(mass), _i64(idx)
        acc = np.zeros((idx.size, 3))
        phi = np.zeros(idx.size)
        rc = self._lib.sfgo_eval_frozen(self._h, float(G), int(quadrupole), _p(pos, _f64p), _p(mass, _f64p),
                                        _p(idx, _i64p), idx.size, _p(acc, _f64p), _p(phi, _f64p))
        if rc != 0:
            raise ValueError("a requested row is not a walked target")
        return acc, phi

    def accel_pp(self, idx, theta: float, G: float = 1.0, quadrupole: bool = True):
        idx = _i64(idx)
        acc = np.zeros((idx.size, 3))
        phi = np.zeros(idx.size)
        cnt = np.zeros((idx.size, 2), np.int64)
        self._lib.sfgo_accel_pp(self._h, float(G), float(theta), int(quadrupole), _p(idx, _i64p), idx.size,
                                _p(acc, _f64p), _p(phi, _f64p), _p(cnt, _i64p))
        return acc, phi, cnt

    def vjp(self, rows, cot_a, cot_phi, G: float = 1.0, quadrupole: bool = True):
        rows, cot_a, cot_phi = _i64(rows), _f64(cot_a), _f64(cot_phi)
        d_pos = np.zeros((self.n, 3))
        d_mass = np.zeros(self.n)
        rc = self._lib.sfgo_vjp(self._h, float(G), int(quadrupole), _p(rows, _i64p), rows.size, _p(cot_a, _f64p),
                                _p(cot_phi, _f64p), _p(d_pos, _f64p), _p(d_mass, _f64p))
        if rc != 0:
            raise ValueError("a cotangent row is not a walked target")
        return d_pos, d_mass

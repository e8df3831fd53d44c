"""Plain FP64 CPU oracle for the lattice Boltzmann schemes of Otte & Frank (arXiv:1601.08103).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package.  It shares nothing with the CUDA library in
``paper_1601_08103_gb300``: the C source ``lee_oracle.c`` builds its own velocity-set tables
from the paper's formulas, and neither side imports the other.

Python view of the C oracle: every function takes and returns numpy FP64 arrays in structure-of-
arrays layout, ``g[i, cell]`` with ``cell = x + nx * (y + ny * z)``.  The array ``g`` holds the
paper's ``g(t, .)``, the populations before collision (Sec. 6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lee_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liblee_oracle.so")

SETS = {"D1Q3": 0, "D2Q5": 1, "D2Q5_DI": 2, "D3Q7": 3, "D3Q9": 4, "D3Q13": 5, "D3Q19": 6, "D3Q7_DI": 7}
BC = {"periodic": 0, "open_zero": 1, "open_sponge": 2, "open_ghost": 3}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc (plain FP64, OpenMP over cells, no FMA contraction so that
    x86 and Arm hosts round identically).  Returns the path of the shared library."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        lib.or_set_info.argtypes = [ctypes.c_int, ip, ip, dp, ip, dp, dp]
        lib.or_equilibrium_fields.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp]
        lib.or_moments_fields.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp]
        lib.or_collide.argtypes = [ctypes.c_int, i64, ctypes.c_double, dp, dp]
        lib.or_step.argtypes = [ctypes.c_int, i64, i64, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, dp, i64, dp]
        lib.or_reduce.argtypes = [ctypes.c_int, i64, dp, dp]
        lib.or_post_state.argtypes = [ctypes.c_int, i64, i64, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, dp, dp]
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_get_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the step loop uses (default 1)."""
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


class VelSet:
    """One velocity set as the oracle builds it (Sec. 8)."""

    def __init__(self, name: str):
        lib = _load()
        D, q = ctypes.c_int(), ctypes.c_int()
        consts = np.zeros(9)
        c = (ctypes.c_int * (27 * 3))()
        f = np.zeros(27)
        beta = np.zeros(27)
        rc = lib.or_set_info(SETS[name], ctypes.byref(D), ctypes.byref(q), _p(consts), c, _p(f), _p(beta))
        if rc != 0:
            raise ValueError(name)
        self.name = name
        self.D, self.q = D.value, q.value
        (self.rho0, self.theta0, self.gamma, self.a1, self.a2, self.b, self.c1, self.c2, mono) = consts
        self.mono = bool(mono)
        self.c = np.array(list(c), dtype=np.int64).reshape(27, 3)[: self.q].copy()
        self.f = f[: self.q].copy()
        self.beta = beta[: self.q].copy()

    @property
    def cs2(self) -> float:
        """Squared speed of sound of the LEE, gamma * theta0 (Sec. 2.1)."""
        return self.gamma * self.theta0


def velset(name: str) -> VelSet:
    return VelSet(name)


def equilibrium(name: str, rho, u, theta) -> np.ndarray:
    """g = g^eq(rho', u', theta') cell by cell (the initial condition of Sec. 7)."""
    s = VelSet(name)
    rho, theta = _f64(rho).ravel(), _f64(theta).ravel()
    cells = rho.size
    u = _f64(u).reshape(s.D, cells)
    g = np.empty((s.q, cells))
    _load().or_equilibrium_fields(SETS[name], cells, _p(rho), _p(u), _p(theta), _p(g))
    return g


def moments(name: str, g):
    """(rho'[cells], u'[D, cells], theta'[cells]) of a population field (Secs. 4-5)."""
    s = VelSet(name)
    g = _f64(g)
    cells = g.shape[1]
    rho, u, theta = np.empty(cells), np.empty((s.D, cells)), np.empty(cells)
    _load().or_moments_fields(SETS[name], cells, _p(g), _p(rho), _p(u), _p(theta))
    return rho, u, theta


def collide(name: str, tau: float, g) -> np.ndarray:
    """Post-collision populations (1 - 1/tau) g + (1/tau) g^eq(g), no streaming."""
    g = _f64(g)
    out = np.empty_like(g)
    _load().or_collide(SETS[name], g.shape[1], float(tau), _p(g), _p(out))
    return out


def step(name: str, shape, tau: float, g, nsteps: int, bc: str = "periodic", sponge_w: int = 0,
         sponge_smax: float = 0.0, ghost=None) -> np.ndarray:
    """Returns g after ``nsteps`` LBE updates (Sec. 6).  ``shape`` = (nx, ny, nz)."""
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    g = _f64(g).copy()
    gp = None
    if ghost is not None:
        ghost = _f64(ghost)
        gp = _p(ghost)
    rc = _load().or_step(SETS[name], nx, ny, nz, float(tau), BC[bc], int(sponge_w), float(sponge_smax), _p(g),
                         int(nsteps), gp)
    if rc != 0:
        raise ValueError(f"or_step rejected its arguments ({rc})")
    return g


def post_state(name: str, shape, tau: float, g, bc: str = "periodic", sponge_w: int = 0,
               sponge_smax: float = 0.0) -> np.ndarray:
    """Post-collision populations of g (damped inside a sponge frame): what one step streams."""
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    g = _f64(g)
    out = np.empty_like(g)
    rc = _load().or_post_state(SETS[name], nx, ny, nz, float(tau), BC[bc], int(sponge_w), float(sponge_smax), _p(g),
                               _p(out))
    if rc != 0:
        raise ValueError(f"or_post_state rejected its arguments ({rc})")
    return out


def reduce(name: str, g) -> np.ndarray:
    """[sum rho', sum j[D], sum energy moment, sum g^2/f*, nonfinite count] (see lee_oracle.c)."""
    s = VelSet(name)
    g = _f64(g)
    out = np.empty(s.D + 4)
    _load().or_reduce(SETS[name], g.shape[1], _p(g), _p(out))
    return out

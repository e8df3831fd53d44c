"""Python binding of the GB300 lattice Boltzmann solver for the Linearized Euler Equations.

Thin ctypes layer over ``lib/liblee_lbm.so`` (C ABI in ``include/lee_lbm.h``): it marshals
arguments and raises :class:`LeeError` on a non-OK status.  Every step of the computation runs in
the CUDA kernels of the library; nothing here computes on the CPU.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); FP64 and C-contiguous as the header states.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LIB_PATH = _build.LIB

# enums of include/lee_lbm.h
SETS = {"D1Q3": 0, "D2Q5": 1, "D2Q5_DI": 2, "D3Q7": 3, "D3Q9": 4, "D3Q13": 5, "D3Q19": 6, "D3Q7_DI": 7}
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "split16": 4, "bfp16": 5}
BC = {"periodic": 0, "open_zero": 1, "open_sponge": 2, "open_learned": 3, "slab": 4}
# bytes per stored population (bfp16: a 16-bit mantissa plus an eighth of a block exponent byte)
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "bfp16": 2.125}


def state_bytes_per_cell(D: int, q: int, storage: str) -> float:
    """Bytes of one cell in one state copy: q populations, or for split16 the D + 2 FP32 moments
    and q FP16 non-equilibrium parts."""
    if storage == "split16":
        return 4 * (D + 2) + 2 * q
    return q * STORAGE_BYTES[storage]

LEE_OK = 0
LEE_ERR_INVALID_ARGUMENT = 1
LEE_ERR_UNSTABLE_TAU = 2
LEE_ERR_OUT_OF_MEMORY = 3
LEE_ERR_CUDA = 4
LEE_ERR_NONFINITE = 5
LEE_ERR_TIMEOUT = 6
LEE_ERR_UNSUPPORTED = 7
LEE_ERR_POISONED = 8


class LeeError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: status {status}"
        if _lib is not None:
            msg += f" ({_lib.lee_status_string(status).decode()})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class lee_lbm_config(ctypes.Structure):
    _fields_ = [("set", ctypes.c_int32), ("storage", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("tau", ctypes.c_double), ("bc", ctypes.c_int32),
                ("sponge_width", ctypes.c_int32), ("sponge_strength", ctypes.c_double),
                ("store_scale", ctypes.c_double), ("cuda_stream", ctypes.c_void_p)]


class lee_units(ctypes.Structure):
    _fields_ = [("rho_star", ctypes.c_double), ("theta_star", ctypes.c_double), ("u_star", ctypes.c_double),
                ("x_star", ctypes.c_double), ("t_star", ctypes.c_double), ("eps", ctypes.c_double),
                ("t_end", ctypes.c_double), ("steps", ctypes.c_int64), ("mismatch", ctypes.c_double)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_I32, _I64, _D, _P = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
_SIGS = {
    "lee_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lee_velset_info": (ctypes.c_int, [_I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32), _P, _P, _P, _P]),
    "lee_units_from_dimensional": (ctypes.c_int, [_I32, _D, _D, _D, _D, _I64, _D, ctypes.POINTER(lee_units)]),
    "lee_stability_scan": (ctypes.c_int, [_I32, _D, _I32, _D, _P, _P, _P, _P, _P]),
    "lee_lbm_create": (ctypes.c_int, [ctypes.POINTER(lee_lbm_config), ctypes.POINTER(_P)]),
    "lee_lbm_init_fields": (ctypes.c_int, [_P, _P, _P, _P, _I32]),
    "lee_lbm_step": (ctypes.c_int, [_P, _I64]),
    "lee_lbm_moments": (ctypes.c_int, [_P, _P, _P, _P, _I32]),
    "lee_lbm_reduce": (ctypes.c_int, [_P, _P, _I32]),
    "lee_lbm_check_finite": (ctypes.c_int, [_P]),
    "lee_lbm_get_populations": (ctypes.c_int, [_P, _P, _I32]),
    "lee_lbm_set_populations": (ctypes.c_int, [_P, _P, _I32]),
    "lee_lbm_set_boundary_mlp": (ctypes.c_int, [_P, _P, _I64]),
    "lee_lbm_set_boundary_mlp_for_tau": (ctypes.c_int, [_P, _P, _I64, _D, _D, ctypes.POINTER(_I32)]),
    "lee_lbm_boundary_in_use": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "lee_lbm_steps_done": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "lee_lbm_slab_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "lee_lbm_slab_buffers": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                            ctypes.POINTER(_P)]),
    "lee_lbm_slab_pack": (ctypes.c_int, [_P]),
    "lee_lbm_slab_unpack": (ctypes.c_int, [_P]),
    "lee_lbm_slab_step": (ctypes.c_int, [_P, _I32, _I64]),
    "lee_lbm_store_scale": (ctypes.c_int, [_P, ctypes.POINTER(_D)]),
    "lee_lbm_steps_per_launch": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "lee_lbm_sync": (ctypes.c_int, [_P]),
    "lee_lbm_last_error": (ctypes.c_char_p, [_P]),
    "lee_lbm_destroy": (ctypes.c_int, [_P]),
    "lee_reduce_noalloc": (ctypes.c_int, [_I32, _I32, _P, _I64, _I64, _D, _P, _P]),
    "lee_test_inject_cuda_error": (ctypes.c_int, [_I32]),
    "lee_test_inject_stage_timeout": (ctypes.c_int, [_I32, _I64]),
    "lee_probe_fp64_fma": (ctypes.c_int, [_I64, ctypes.POINTER(_D)]),
    # include/lee_batch.h
    "lee_batch_create": (ctypes.c_int, [_I32, _I32, _P, _I32, _P, ctypes.POINTER(_P)]),
    "lee_batch_init_fields": (ctypes.c_int, [_P, _I32, _P, _P, _P, _I32]),
    "lee_batch_step": (ctypes.c_int, [_P, _I64, _I32]),
    "lee_batch_moments": (ctypes.c_int, [_P, _I32, _P, _P, _P, _I32]),
    "lee_batch_reduce": (ctypes.c_int, [_P, _I32, _P, _I32]),
    "lee_batch_get_populations": (ctypes.c_int, [_P, _I32, _P, _I32]),
    "lee_batch_tune": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "lee_batch_set_tuning": (ctypes.c_int, [_P, _I32, _I32]),
    "lee_batch_tune_shape": (ctypes.c_int, [_P, _P]),
    "lee_batch_set_shape": (ctypes.c_int, [_P, _P]),
    "lee_batch_cells": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "lee_batch_sync": (ctypes.c_int, [_P]),
    "lee_batch_last_error": (ctypes.c_char_p, [_P]),
    "lee_batch_destroy": (ctypes.c_int, [_P]),
}


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIGS)


def load(path: str | None = None):
    """Loads the CUDA library (building it with nvcc first if it is not there).  Raises if it
    cannot be built or loaded: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            p = _build.build()
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, where: str, handle=None, batch=None):
    if status != LEE_OK:
        detail = ""
        if handle:
            detail = _lib.lee_lbm_last_error(handle).decode()
        if batch:
            detail = _lib.lee_batch_last_error(batch).decode()
        raise LeeError(status, where, detail)


def _addr(x):
    """(address, on_device) of a numpy array or torch tensor (None -> (None, 0))."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    raise TypeError(f"unsupported buffer type {type(x)}")


def _same_place(*bufs):
    places = {_addr(b)[1] for b in bufs if b is not None}
    if len(places) > 1:
        raise ValueError("all buffers of one call must be on the host or all on the device")
    return places.pop() if places else 0


# ------------------------------------------------------------------------------------------
# C entry points, same names
# ------------------------------------------------------------------------------------------

def lee_status_string(status: int) -> str:
    return load().lee_status_string(status).decode()


def lee_velset_info(set_name: str) -> dict:
    """Velocity set in the library's order: D, q, c[q][3], f[q], beta[q] and the Sec. 5
    coefficients (rho0, theta0, gamma, a1, a2, b, c1, c2)."""
    lib = load()
    D, q = _I32(), _I32()
    c = (_I32 * 81)()
    f = (_D * 27)()
    beta = (_D * 27)()
    consts = (_D * 8)()
    _check(lib.lee_velset_info(SETS[set_name], ctypes.byref(D), ctypes.byref(q), ctypes.cast(c, _P),
                               ctypes.cast(f, _P), ctypes.cast(beta, _P), ctypes.cast(consts, _P)), "lee_velset_info")
    n = q.value
    keys = ["rho0", "theta0", "gamma", "a1", "a2", "b", "c1", "c2"]
    out = {"D": D.value, "q": n, "c": [tuple(c[3 * i + a] for a in range(3)) for i in range(n)],
           "f": [f[i] for i in range(n)], "beta": [beta[i] for i in range(n)]}
    out.update({k: consts[j] for j, k in enumerate(keys)})
    return out


def lee_units_from_dimensional(set_name: str, rho0_dim: float, theta0_dim: float, x_star: float, length_dim: float,
                               n_cells: int, t_end_dim: float) -> dict:
    """Scales of a dimensional problem on the lattice (Sec. 2.1, Sec. 6): rho_star, theta_star,
    u_star, x_star, t_star, the lattice step eps, the non-dimensional end time t_end, the step
    count steps = round(t_end / eps) and the end-time mismatch t_end - steps * eps."""
    u = lee_units()
    _check(load().lee_units_from_dimensional(SETS[set_name], float(rho0_dim), float(theta0_dim), float(x_star),
                                             float(length_dim), int(n_cells), float(t_end_dim), ctypes.byref(u)),
           "lee_units_from_dimensional")
    return {name: getattr(u, name) for name, _ in lee_units._fields_}


def make_config(set_name: str, shape, tau: float, storage: str = "f64", bc: str = "periodic", sponge_width: int = 0,
                sponge_strength: float = 0.0, store_scale: float = 0.0, stream=None) -> lee_lbm_config:
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    cfg = lee_lbm_config()
    cfg.set = SETS[set_name]
    cfg.storage = STORAGE[storage]
    cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
    cfg.tau = float(tau)
    cfg.bc = BC[bc]
    cfg.sponge_width = int(sponge_width)
    cfg.sponge_strength = float(sponge_strength)
    cfg.store_scale = float(store_scale)
    if stream is not None:
        cfg.cuda_stream = stream if isinstance(stream, int) else int(stream.cuda_stream)
    return cfg


def lee_lbm_create(cfg: lee_lbm_config) -> int:
    lib = load()
    h = _P()
    _check(lib.lee_lbm_create(ctypes.byref(cfg), ctypes.byref(h)), "lee_lbm_create")
    return h.value


def lee_lbm_init_fields(h, rho, u, theta):
    on = _same_place(rho, u, theta)
    _check(_lib.lee_lbm_init_fields(h, _addr(rho)[0], _addr(u)[0], _addr(theta)[0], on), "lee_lbm_init_fields", h)


def lee_lbm_step(h, n: int):
    _check(_lib.lee_lbm_step(h, int(n)), "lee_lbm_step", h)


def lee_lbm_moments(h, rho=None, u=None, theta=None):
    on = _same_place(rho, u, theta)
    _check(_lib.lee_lbm_moments(h, _addr(rho)[0], _addr(u)[0], _addr(theta)[0], on), "lee_lbm_moments", h)


def lee_lbm_reduce(h, out):
    a, on = _addr(out)
    _check(_lib.lee_lbm_reduce(h, a, on), "lee_lbm_reduce", h)


def lee_lbm_check_finite(h) -> bool:
    s = _lib.lee_lbm_check_finite(h)
    if s == LEE_ERR_NONFINITE:
        return False
    _check(s, "lee_lbm_check_finite", h)
    return True


def lee_lbm_get_populations(h, g):
    a, on = _addr(g)
    _check(_lib.lee_lbm_get_populations(h, a, on), "lee_lbm_get_populations", h)


def lee_lbm_set_populations(h, g):
    a, on = _addr(g)
    _check(_lib.lee_lbm_set_populations(h, a, on), "lee_lbm_set_populations", h)


def lee_lbm_set_boundary_mlp(h, params):
    a, on = _addr(params)
    if on:
        raise ValueError("boundary network parameters are read from host memory")
    n = params.size if hasattr(params, "size") and not callable(params.size) else params.numel()
    _check(_lib.lee_lbm_set_boundary_mlp(h, a, int(n)), "lee_lbm_set_boundary_mlp", h)


def lee_lbm_slab_info(h):
    """(crossing velocities per face, cells per plane, bytes per halo message) of a slab handle."""
    c, p, b = _I32(), _I64(), _I64()
    _check(_lib.lee_lbm_slab_info(h, ctypes.byref(c), ctypes.byref(p), ctypes.byref(b)), "lee_lbm_slab_info", h)
    return c.value, p.value, b.value


def lee_lbm_slab_buffers(h):
    """Device addresses (send_lo, send_hi, recv_lo, recv_hi) of a slab handle's halo messages."""
    v = [_P() for _ in range(4)]
    _check(_lib.lee_lbm_slab_buffers(h, *[ctypes.byref(x) for x in v]), "lee_lbm_slab_buffers", h)
    return tuple(x.value for x in v)


def lee_lbm_slab_pack(h):
    _check(_lib.lee_lbm_slab_pack(h), "lee_lbm_slab_pack", h)


def lee_lbm_slab_unpack(h):
    _check(_lib.lee_lbm_slab_unpack(h), "lee_lbm_slab_unpack", h)


def lee_lbm_slab_step(solvers, n: int):
    """n steps of the slabs (Solver objects or raw handles, in order along the cut) of one
    periodic domain held in this process (see include/lee_lbm.h)."""
    hs = [x.h if hasattr(x, "h") else x for x in solvers]
    arr = (_P * len(hs))(*hs)
    _check(load().lee_lbm_slab_step(ctypes.cast(arr, _P), len(hs), int(n)), "lee_lbm_slab_step", hs[0])


def lee_lbm_set_boundary_mlp_for_tau(h, params, trained_tau: float, tau_tolerance: float = 1e-9) -> bool:
    """Installs the network if it was trained at this handle's tau (within the tolerance); returns
    whether it was installed (otherwise the learned edge runs its fallback)."""
    a, on = _addr(params)
    if on:
        raise ValueError("boundary network parameters are read from host memory")
    n = params.size if hasattr(params, "size") and not callable(params.size) else params.numel()
    v = _I32()
    _check(_lib.lee_lbm_set_boundary_mlp_for_tau(h, a, int(n), float(trained_tau), float(tau_tolerance),
                                                  ctypes.byref(v)), "lee_lbm_set_boundary_mlp_for_tau", h)
    return bool(v.value)


def lee_lbm_boundary_in_use(h) -> str:
    """Name (a key of BC) of the edge treatment the next step runs."""
    v = _I32()
    _check(_lib.lee_lbm_boundary_in_use(h, ctypes.byref(v)), "lee_lbm_boundary_in_use")
    return {k: name for name, k in BC.items()}[v.value]


def lee_lbm_steps_done(h) -> int:
    v = _I64()
    _check(_lib.lee_lbm_steps_done(h, ctypes.byref(v)), "lee_lbm_steps_done")
    return v.value


def lee_lbm_steps_per_launch(h) -> int:
    v = _I32()
    _check(_lib.lee_lbm_steps_per_launch(h, ctypes.byref(v)), "lee_lbm_steps_per_launch")
    return v.value


def lee_lbm_store_scale(h) -> float:
    v = _D()
    _check(_lib.lee_lbm_store_scale(h, ctypes.byref(v)), "lee_lbm_store_scale")
    return v.value


def lee_lbm_sync(h):
    _check(_lib.lee_lbm_sync(h), "lee_lbm_sync", h)


def lee_lbm_last_error(h) -> str:
    return load().lee_lbm_last_error(h).decode()


def lee_lbm_destroy(h):
    if h:
        _check(_lib.lee_lbm_destroy(h), "lee_lbm_destroy")


NOALLOC_DTYPES = {"f64": "float64", "f32": "float32", "f16": "float16", "bf16": "bfloat16"}


def _noalloc_check(set_name: str, storage: str, g, cells: int, pitch: int, out):
    """Host-side checks of lee_reduce_noalloc's buffers, which the C side cannot make: the dtype
    of g matches the storage, g holds (q - 1) * pitch + cells elements, out is FP64 with D + 4
    entries, and both are CUDA tensors on the current device.  Raises ValueError; launches
    nothing."""
    if storage not in NOALLOC_DTYPES:
        raise ValueError(f"lee_reduce_noalloc: storage {storage!r} is not accepted (f64, f32, f16, bf16)")
    info = lee_velset_info(set_name)
    q, D = info["q"], info["D"]
    for name, t in (("g", g), ("out", out)):
        if not (hasattr(t, "dtype") and hasattr(t, "numel") and hasattr(t, "is_cuda")):
            raise ValueError(f"lee_reduce_noalloc: {name} must be a torch tensor")
        if not t.is_contiguous():
            raise ValueError(f"lee_reduce_noalloc: {name} must be contiguous")
    if str(g.dtype).replace("torch.", "") != NOALLOC_DTYPES[storage]:
        raise ValueError(f"lee_reduce_noalloc: g is {g.dtype}, storage {storage} needs {NOALLOC_DTYPES[storage]}")
    cells, pitch = int(cells), int(pitch)
    if cells < 1 or pitch < cells:
        raise ValueError("lee_reduce_noalloc: need 1 <= cells <= pitch")
    if g.numel() < (q - 1) * pitch + cells:
        raise ValueError(f"lee_reduce_noalloc: g holds {g.numel()} elements, the layout needs {(q - 1) * pitch + cells}")
    if str(out.dtype) != "torch.float64" or out.numel() < D + 4:
        raise ValueError(f"lee_reduce_noalloc: out must be float64 with at least {D + 4} entries")
    if not (g.is_cuda and out.is_cuda):
        raise ValueError("lee_reduce_noalloc takes device buffers only")
    import torch

    cur = torch.cuda.current_device()
    if g.device.index != cur or out.device.index != cur:
        raise ValueError("lee_reduce_noalloc: g and out must be on the current CUDA device")


def lee_reduce_noalloc(set_name: str, storage: str, g, cells: int, pitch: int, out, store_scale: float = 1.0,
                       stream=None):
    """Global sums of a caller-owned device population field without any allocation (see
    include/lee_lbm.h).  g and out must be CUDA tensors on the current device; out holds D + 4
    doubles.  Runs on `stream` (a torch stream or a raw handle), by default torch's current
    stream, so it is ordered after the kernels that produced g."""
    _noalloc_check(set_name, storage, g, cells, pitch, out)
    lib = load()
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    st = stream if isinstance(stream, int) else int(stream.cuda_stream)
    _check(lib.lee_reduce_noalloc(SETS[set_name], STORAGE[storage], g.data_ptr(), int(cells), int(pitch),
                                  float(store_scale), out.data_ptr(), st), "lee_reduce_noalloc")


def lee_probe_fp64_fma(iters: int = 1 << 16) -> float:
    """The current device's measured FP64 fma rate in FLOP/s (see include/lee_lbm.h)."""
    v = _D()
    _check(load().lee_probe_fp64_fma(int(iters), ctypes.byref(v)), "lee_probe_fp64_fma")
    return v.value


def lee_test_inject_cuda_error(after: int):
    """Test hook (include/lee_lbm.h): the (after+1)-th successful CUDA call that a handle checks
    from now on is reported as failed, once; -1 disarms."""
    _check(load().lee_test_inject_cuda_error(int(after)), "lee_test_inject_cuda_error")


def lee_test_inject_stage_timeout(on: bool, wait_ns: int = 0):
    """Test hook (include/lee_lbm.h): launches of the TMA-fed 3D two-step tile announce more bytes
    than their first stage receives, so that its bounded wait (wait_ns; 0: one second) runs out and
    the handle reports LEE_ERR_TIMEOUT; on=False restores normal launches."""
    _check(load().lee_test_inject_stage_timeout(1 if on else 0, int(wait_ns)), "lee_test_inject_stage_timeout")


def lee_stability_scan(set_name: str, tau: float, m: int, rho, lam=None, kappa=None, nu=None, delta: float = 1e-6,
                       stream=None):
    """Von Neumann scan of Gamma(k) = D(k) H(tau) on the m^D grid of wave vectors (see
    include/lee_stability.h).  rho [m^D], and optionally lam [m^D][q][2], kappa [m^D], nu [m^D]:
    CUDA float64 tensors, filled on `stream` (the call waits for it)."""
    lib = load()
    bufs = [rho, lam, kappa, nu]
    for b in bufs:
        if b is not None and not _addr(b)[1]:
            raise ValueError("lee_stability_scan takes device buffers only")
    st = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    ra, la, ka, na = (_addr(b)[0] for b in bufs)
    _check(lib.lee_stability_scan(SETS[set_name], float(tau), int(m), float(delta), la, ra, ka, na, st),
           "lee_stability_scan")


class Solver:
    """Owns one handle; methods map one-to-one onto the C entry points."""

    def __init__(self, set_name: str, shape, tau: float, storage: str = "f64", bc: str = "periodic", **kw):
        load()
        self.set_name = set_name
        self.info = lee_velset_info(set_name)
        self.D, self.q = self.info["D"], self.info["q"]
        self.shape = tuple((list(shape) + [1, 1])[:3])
        self.cells = int(self.shape[0] * self.shape[1] * self.shape[2])
        self.storage = storage
        self.cfg = make_config(set_name, shape, tau, storage, bc, **kw)
        self.h = lee_lbm_create(self.cfg)

    def init_fields(self, rho, u, theta):
        lee_lbm_init_fields(self.h, rho, u, theta)

    def step(self, n: int = 1):
        lee_lbm_step(self.h, n)

    def moments(self, rho=None, u=None, theta=None):
        lee_lbm_moments(self.h, rho, u, theta)

    def reduce(self, out):
        lee_lbm_reduce(self.h, out)

    def check_finite(self) -> bool:
        return lee_lbm_check_finite(self.h)

    def get_populations(self, g):
        lee_lbm_get_populations(self.h, g)

    def set_populations(self, g):
        lee_lbm_set_populations(self.h, g)

    def set_boundary_mlp(self, params):
        lee_lbm_set_boundary_mlp(self.h, params)

    def set_boundary_mlp_for_tau(self, params, trained_tau, tau_tolerance=1e-9) -> bool:
        return lee_lbm_set_boundary_mlp_for_tau(self.h, params, trained_tau, tau_tolerance)

    @property
    def boundary_in_use(self) -> str:
        return lee_lbm_boundary_in_use(self.h)

    def slab_info(self):
        return lee_lbm_slab_info(self.h)

    def slab_buffers(self):
        return lee_lbm_slab_buffers(self.h)

    def slab_pack(self):
        lee_lbm_slab_pack(self.h)

    def slab_unpack(self):
        lee_lbm_slab_unpack(self.h)

    @property
    def steps_done(self) -> int:
        return lee_lbm_steps_done(self.h)

    @property
    def store_scale(self) -> float:
        return lee_lbm_store_scale(self.h)

    @property
    def steps_per_launch(self) -> int:
        return lee_lbm_steps_per_launch(self.h)

    def sync(self):
        lee_lbm_sync(self.h)

    def close(self):
        if self.h:
            lee_lbm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------------
# include/lee_batch.h
# ------------------------------------------------------------------------------------------
BATCH_MODE = {"graph": 0, "launch": 1, "sequential": 2}


class lee_batch_domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("tau", ctypes.c_double)]


class lee_batch_shape(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("cells_per_thread", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("tile_order", ctypes.c_int32), ("us_per_step", ctypes.c_float)]


def lee_batch_create(set_name: str, storage: str, domains, stream=None) -> int:
    """domains: sequence of (nx, ny, tau)."""
    lib = load()
    arr = (lee_batch_domain * len(domains))(*[lee_batch_domain(int(a), int(b), float(t)) for a, b, t in domains])
    st = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    h = _P()
    _check(lib.lee_batch_create(SETS[set_name], STORAGE[storage], ctypes.cast(arr, _P), len(domains), st,
                                ctypes.byref(h)), "lee_batch_create")
    return h.value


def lee_batch_init_fields(b, d, rho, u, theta):
    on = _same_place(rho, u, theta)
    _check(_lib.lee_batch_init_fields(b, int(d), _addr(rho)[0], _addr(u)[0], _addr(theta)[0], on),
           "lee_batch_init_fields", batch=b)


def lee_batch_step(b, n: int, mode: str = "graph"):
    _check(_lib.lee_batch_step(b, int(n), BATCH_MODE[mode]), "lee_batch_step", batch=b)


def lee_batch_moments(b, d, rho=None, u=None, theta=None):
    on = _same_place(rho, u, theta)
    _check(_lib.lee_batch_moments(b, int(d), _addr(rho)[0], _addr(u)[0], _addr(theta)[0], on), "lee_batch_moments",
           batch=b)


def lee_batch_reduce(b, d, out):
    a, on = _addr(out)
    _check(_lib.lee_batch_reduce(b, int(d), a, on), "lee_batch_reduce", batch=b)


def lee_batch_get_populations(b, d, g):
    a, on = _addr(g)
    _check(_lib.lee_batch_get_populations(b, int(d), a, on), "lee_batch_get_populations", batch=b)


def lee_batch_tune(b):
    t, v = _I32(), _I32()
    _check(_lib.lee_batch_tune(b, ctypes.byref(t), ctypes.byref(v)), "lee_batch_tune", batch=b)
    return t.value, v.value


def lee_batch_set_tuning(b, threads: int, cells_per_thread: int):
    _check(_lib.lee_batch_set_tuning(b, int(threads), int(cells_per_thread)), "lee_batch_set_tuning", batch=b)


def lee_batch_tune_shape(b) -> dict:
    """The launch shape in use after tuning (see include/lee_batch.h), as a dict."""
    sh = lee_batch_shape()
    _check(_lib.lee_batch_tune_shape(b, ctypes.byref(sh)), "lee_batch_tune_shape", batch=b)
    return {name: getattr(sh, name) for name, _ in lee_batch_shape._fields_}


def lee_batch_set_shape(b, threads: int, cells_per_thread: int, steps_per_launch: int, tile_rows: int = 64,
                        tile_order: int = 0):
    sh = lee_batch_shape(int(threads), int(cells_per_thread), int(steps_per_launch), int(tile_rows),
                         int(tile_order), 0.0)
    _check(_lib.lee_batch_set_shape(b, ctypes.byref(sh)), "lee_batch_set_shape", batch=b)


def lee_batch_cells(b) -> int:
    v = _I64()
    _check(_lib.lee_batch_cells(b, ctypes.byref(v)), "lee_batch_cells")
    return v.value


def lee_batch_sync(b):
    _check(_lib.lee_batch_sync(b), "lee_batch_sync", batch=b)


def lee_batch_destroy(b):
    if b:
        _check(_lib.lee_batch_destroy(b), "lee_batch_destroy")


class Batch:
    """Owns one lee_batch; methods map one-to-one onto the C entry points."""

    def __init__(self, set_name: str, storage: str, domains, stream=None):
        load()
        self.domains = [(int(a), int(b), float(t)) for a, b, t in domains]
        self.q = lee_velset_info(set_name)["q"]
        self.b = lee_batch_create(set_name, storage, self.domains, stream)

    def init_fields(self, d, rho, u, theta):
        lee_batch_init_fields(self.b, d, rho, u, theta)

    def step(self, n: int = 1, mode: str = "graph"):
        lee_batch_step(self.b, n, mode)

    def moments(self, d, rho=None, u=None, theta=None):
        lee_batch_moments(self.b, d, rho, u, theta)

    def reduce(self, d, out):
        lee_batch_reduce(self.b, d, out)

    def get_populations(self, d, g):
        lee_batch_get_populations(self.b, d, g)

    def tune(self):
        return lee_batch_tune(self.b)

    def set_tuning(self, threads, cells_per_thread):
        lee_batch_set_tuning(self.b, threads, cells_per_thread)

    def tune_shape(self) -> dict:
        return lee_batch_tune_shape(self.b)

    def set_shape(self, threads, cells_per_thread, steps_per_launch, tile_rows=64, tile_order=0):
        lee_batch_set_shape(self.b, threads, cells_per_thread, steps_per_launch, tile_rows, tile_order)

    @property
    def cells(self) -> int:
        return lee_batch_cells(self.b)

    def sync(self):
        lee_batch_sync(self.b)

    def close(self):
        if self.b:
            lee_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------------
# include/lee_mlp.h
# ------------------------------------------------------------------------------------------
MLP_NPARAM = 5313
MLP_IN = 16

_SIGS.update({
    "lee_mlp_create": (ctypes.c_int, [_P, _P, ctypes.POINTER(_P)]),
    "lee_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "lee_mlp_set_params": (ctypes.c_int, [_P, _P]),
    "lee_mlp_forward": (ctypes.c_int, [_P, _P, _I64, _P]),
    "lee_mlp_loss_grad": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P]),
    "lee_mlp_adam_step": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "lee_batch_edge_samples": (ctypes.c_int, [_P, _I64, _I64, _I64, _I64, _P, _P, _P]),
    "lee_lbm_edge_inputs": (ctypes.c_int, [_P, _P, _P]),
    "lee_mlp_destroy": (ctypes.c_int, [_P]),
})


def _dev(x):
    a, on = _addr(x)
    if x is not None and not on:
        raise ValueError("device buffer expected")
    return a


def lee_mlp_create(params=None, stream=None) -> int:
    lib = load()
    pa = None
    if params is not None:
        pa, on = _addr(params)
        if on:
            raise ValueError("parameters are read from host memory")
    st = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    h = _P()
    _check(lib.lee_mlp_create(pa, st, ctypes.byref(h)), "lee_mlp_create")
    return h.value


def lee_mlp_get_params(m, out):
    _check(_lib.lee_mlp_get_params(m, _addr(out)[0]), "lee_mlp_get_params")


def lee_mlp_set_params(m, params):
    _check(_lib.lee_mlp_set_params(m, _addr(params)[0]), "lee_mlp_set_params")


def lee_mlp_forward(m, x, rows, y):
    _check(_lib.lee_mlp_forward(m, _dev(x), int(rows), _dev(y)), "lee_mlp_forward")


def lee_mlp_loss_grad(m, x, t, rows, grad=None, loss=None):
    _check(_lib.lee_mlp_loss_grad(m, _dev(x), _dev(t), int(rows), _dev(grad), _dev(loss)), "lee_mlp_loss_grad")


def lee_mlp_adam_step(m, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(_lib.lee_mlp_adam_step(m, lr, beta1, beta2, eps), "lee_mlp_adam_step")


def lee_batch_edge_samples(b, x0, y0, nx, ny, x, t, s=None):
    _check(_lib.lee_batch_edge_samples(b, int(x0), int(y0), int(nx), int(ny), _dev(x), _dev(t), _dev(s)),
           "lee_batch_edge_samples", batch=b)


def lee_lbm_edge_inputs(h, x, s=None):
    _check(_lib.lee_lbm_edge_inputs(h, _dev(x), _dev(s)), "lee_lbm_edge_inputs", h)


def lee_mlp_destroy(m):
    if m:
        _check(_lib.lee_mlp_destroy(m), "lee_mlp_destroy")


class Mlp:
    """Owns one lee_mlp; methods map one-to-one onto the C entry points."""

    def __init__(self, params=None, stream=None):
        load()
        self.m = lee_mlp_create(params, stream)

    def get_params(self, out):
        lee_mlp_get_params(self.m, out)

    def set_params(self, params):
        lee_mlp_set_params(self.m, params)

    def forward(self, x, rows, y):
        lee_mlp_forward(self.m, x, rows, y)

    def loss_grad(self, x, t, rows, grad=None, loss=None):
        lee_mlp_loss_grad(self.m, x, t, rows, grad, loss)

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        lee_mlp_adam_step(self.m, lr, beta1, beta2, eps)

    def close(self):
        if self.m:
            lee_mlp_destroy(self.m)
            self.m = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

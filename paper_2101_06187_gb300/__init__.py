"""GB300 relativistic lattice Boltzmann (RLBM) stream-collide library.

Thin ctypes binding of the C ABI in ``include/rlbm.h`` (``librlbm.so``, built
from ``csrc/`` by ``build.py``).  Every step of the method runs in the CUDA
kernels of that library; this module only marshals arguments.  PyTorch is
used, when present, for device memory (the caching allocator) and streams.

The functions ``rlbm_create``, ``rlbm_init_fields``, ``rlbm_step``,
``rlbm_moments``, ``rlbm_energy_spectrum``, ``rlbm_destroy`` ... carry the
names of the C entry points; ``Lattice`` bundles them as methods.

There is no CPU fallback: if the CUDA library is missing or fails to load,
every call raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librlbm.so")

RLBM_OK, RLBM_ERR_ARG, RLBM_ERR_ALLOC, RLBM_ERR_CUDA, RLBM_ERR_TIMEOUT, RLBM_ERR_NAN, RLBM_ERR_STATE = range(7)
RLBM_STENCIL_SPH26_SLAB = 0
RLBM_STENCIL_RING8_2D = 1
STENCILS = {"sph26": RLBM_STENCIL_SPH26_SLAB, "ring8": RLBM_STENCIL_RING8_2D}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
ROUNDING = {"default": 0, "nearest": 1, "stochastic": 2}
LANDAU = {"fp64": 0, "fp32": 1}
KERNELS = {"auto": 0, "gather": 1, "vec": 2, "vec2": 3, "packed": 4, "tma": 5, "twopass": 6, "fused2": 7, "packed4": 8}
NCLASSES = 17

# Symbols declared in include/rlbm.h (checked by the ABI test).
EXPORTS = (
    "rlbm_opts_default", "rlbm_create", "rlbm_init_fields", "rlbm_init_fields_device", "rlbm_step", "rlbm_moments",
    "rlbm_moments_device", "rlbm_energy_spectrum", "rlbm_get_populations", "rlbm_set_populations", "rlbm_get_force",
    "rlbm_get_info", "rlbm_autotune", "rlbm_moments_static", "rlbm_synchronize", "rlbm_last_error", "rlbm_destroy",
    "rlbm_status_string", "rlbm_batch_create", "rlbm_batch_init_fields", "rlbm_batch_step", "rlbm_batch_moments",
    "rlbm_batch_energy_spectrum", "rlbm_batch_get_populations", "rlbm_batch_autotune", "rlbm_batch_get_info",
    "rlbm_batch_synchronize", "rlbm_batch_last_error", "rlbm_batch_destroy", "rlbm_filtered_velocity",
    "rlbm_spectrum_sample", "rlbm_spectrum_stats", "rlbm_spectrum_reset", "rlbm_create3d", "rlbm_init_fields3d",
    "rlbm_moments3d", "rlbm_get_force3d", "rlbm_checkpoint_size", "rlbm_checkpoint_save", "rlbm_checkpoint_load",
    "rlbm_set_launch", "rlbm_create_batch", "rlbm_set_force_frame", "rlbm_halo_pack", "rlbm_halo_unpack",
)


class RLBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class Forcing(ctypes.Structure):
    _fields_ = [("kmin", ctypes.c_int), ("kmax", ctypes.c_int), ("amp", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("redraw_period", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("landau", ctypes.c_int), ("kernel", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("eps0", ctypes.c_double), ("scale", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("cfl", ctypes.c_double), ("eta_s", ctypes.c_double),
                ("dt", ctypes.c_double), ("test_unarmed_wait", ctypes.c_int), ("rounding", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_int), ("nclasses", ctypes.c_int),
                ("dtype", ctypes.c_int), ("kernel", ctypes.c_int), ("block_x", ctypes.c_int),
                ("block_y", ctypes.c_int), ("nmodes", ctypes.c_int),
                ("step", ctypes.c_int64), ("tau", ctypes.c_double), ("eps0", ctypes.c_double),
                ("scale", ctypes.c_double), ("bytes_per_node", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t),
                ("populations", ctypes.c_void_p), ("nz", ctypes.c_int), ("launch_budget", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int)]


class RunDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double), ("forcing", Forcing)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nruns", ctypes.c_int), ("dtype", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("grid", ctypes.c_int), ("ntiles", ctypes.c_int), ("step", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("bytes_per_step", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t), ("kernel", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int)]


_lib_lock = threading.Lock()
_lib_handle = None
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib_handle
    with _lib_lock:
        if _lib_handle is not None:
            return _lib_handle
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is not built; run paper_2101_06187_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        h = ctypes.c_void_p
        lib.rlbm_opts_default.argtypes = [ctypes.POINTER(Opts)]
        lib.rlbm_opts_default.restype = None
        lib.rlbm_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Forcing),
                                    ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]
        lib.rlbm_init_fields.argtypes = [h, _dp, _dp, _dp]
        lib.rlbm_init_fields_device.argtypes = [h, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.rlbm_step.argtypes = [h, ctypes.c_int]
        lib.rlbm_moments.argtypes = [h, _dp, _dp, _dp, _dp]
        lib.rlbm_moments_device.argtypes = [h, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.rlbm_energy_spectrum.argtypes = [h, ctypes.c_int, _dp]
        lib.rlbm_get_populations.argtypes = [h, _dp]
        lib.rlbm_set_populations.argtypes = [h, _dp]
        lib.rlbm_get_force.argtypes = [h, _dp, _dp]
        lib.rlbm_get_info.argtypes = [h, ctypes.POINTER(Info)]
        lib.rlbm_synchronize.argtypes = [h]
        lib.rlbm_moments_static.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
        lib.rlbm_moments_static.restype = ctypes.c_int
        lib.rlbm_filtered_velocity.argtypes = [h, ctypes.c_double, _dp]
        lib.rlbm_spectrum_sample.argtypes = [h, ctypes.c_int]
        lib.rlbm_spectrum_stats.argtypes = [h, ctypes.c_int, _dp, _dp, ctypes.POINTER(ctypes.c_int)]
        lib.rlbm_spectrum_reset.argtypes = [h]
        for name in ("rlbm_filtered_velocity", "rlbm_spectrum_sample", "rlbm_spectrum_stats", "rlbm_spectrum_reset"):
            getattr(lib, name).restype = ctypes.c_int
        lib.rlbm_create3d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(Forcing), ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]
        lib.rlbm_init_fields3d.argtypes = [h, _dp, _dp, _dp, _dp]
        lib.rlbm_moments3d.argtypes = [h, _dp, _dp, _dp, _dp, _dp]
        lib.rlbm_get_force3d.argtypes = [h, _dp, _dp, _dp]
        for name in ("rlbm_create3d", "rlbm_init_fields3d", "rlbm_moments3d", "rlbm_get_force3d"):
            getattr(lib, name).restype = ctypes.c_int
        lib.rlbm_checkpoint_size.argtypes = [h, ctypes.POINTER(ctypes.c_size_t)]
        lib.rlbm_checkpoint_save.argtypes = [h, ctypes.c_void_p, ctypes.c_size_t]
        lib.rlbm_checkpoint_load.argtypes = [h, ctypes.c_void_p, ctypes.c_size_t]
        for name in ("rlbm_checkpoint_size", "rlbm_checkpoint_save", "rlbm_checkpoint_load"):
            getattr(lib, name).restype = ctypes.c_int
        b = ctypes.c_void_p
        ip = ctypes.POINTER(ctypes.c_int)
        lib.rlbm_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(RunDesc), ctypes.POINTER(Opts),
                                          ctypes.POINTER(ctypes.c_void_p)]
        lib.rlbm_create_batch.argtypes = lib.rlbm_batch_create.argtypes
        lib.rlbm_create_batch.restype = ctypes.c_int
        lib.rlbm_set_force_frame.argtypes = [h, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.rlbm_halo_pack.argtypes = [h, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.rlbm_halo_unpack.argtypes = [h, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        for name in ("rlbm_set_force_frame", "rlbm_halo_pack", "rlbm_halo_unpack"):
            getattr(lib, name).restype = ctypes.c_int
        lib.rlbm_batch_init_fields.argtypes = [b, ctypes.c_int, _dp, _dp, _dp]
        lib.rlbm_batch_step.argtypes = [b, ctypes.c_int]
        lib.rlbm_batch_moments.argtypes = [b, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.rlbm_batch_energy_spectrum.argtypes = [b, ctypes.c_int, ctypes.c_int, _dp]
        lib.rlbm_batch_get_populations.argtypes = [b, ctypes.c_int, _dp]
        lib.rlbm_batch_autotune.argtypes = [b, ctypes.c_int, ip, ip, ip]
        lib.rlbm_batch_get_info.argtypes = [b, ctypes.POINTER(BatchInfo)]
        lib.rlbm_batch_synchronize.argtypes = [b]
        lib.rlbm_batch_last_error.argtypes = [b, ctypes.c_char_p, ctypes.c_size_t]
        lib.rlbm_batch_destroy.argtypes = [b]
        lib.rlbm_batch_destroy.restype = None
        for name in ("rlbm_batch_create", "rlbm_batch_init_fields", "rlbm_batch_step", "rlbm_batch_moments",
                     "rlbm_batch_energy_spectrum", "rlbm_batch_get_populations", "rlbm_batch_autotune",
                     "rlbm_batch_get_info", "rlbm_batch_synchronize", "rlbm_batch_last_error"):
            getattr(lib, name).restype = ctypes.c_int
        lib.rlbm_autotune.argtypes = [h, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
        lib.rlbm_set_launch.argtypes = [h, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.rlbm_set_launch.restype = ctypes.c_int
        lib.rlbm_last_error.argtypes = [h, ctypes.c_char_p, ctypes.c_size_t]
        lib.rlbm_destroy.argtypes = [h]
        lib.rlbm_destroy.restype = None
        lib.rlbm_status_string.argtypes = [ctypes.c_int]
        lib.rlbm_status_string.restype = ctypes.c_char_p
        for name in ("rlbm_create", "rlbm_init_fields", "rlbm_init_fields_device", "rlbm_step", "rlbm_moments",
                     "rlbm_moments_device", "rlbm_energy_spectrum", "rlbm_get_populations", "rlbm_set_populations",
                     "rlbm_get_force", "rlbm_get_info", "rlbm_autotune", "rlbm_synchronize", "rlbm_last_error"):
            getattr(lib, name).restype = ctypes.c_int
        _lib_handle = lib
        return lib


def library():
    """The loaded ctypes library (raises if it is not built)."""
    return _load()


def _check(h, st: int, what: str, batch: bool = False):
    if st == RLBM_OK:
        return
    lib = _load()
    msg = lib.rlbm_status_string(st).decode()
    if h:
        buf = ctypes.create_string_buffer(512)
        (lib.rlbm_batch_last_error if batch else lib.rlbm_last_error)(h, buf, 512)
        if buf.value:
            msg += ": " + buf.value.decode()
    raise RLBMError(st, "%s failed: %s" % (what, msg))


def _f64(a, n) -> Optional[np.ndarray]:
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.size != n:
        raise ValueError("expected %d elements, got %d" % (n, a.size))
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


# ------------------------------------------------------------------ torch plumbing
class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library
    through its allocator hooks."""

    def __init__(self, device: int, stream: int):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, _ctx):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # noqa: BLE001 - reported to C as NULL
                return None

        def _free(ptr, _nbytes, _ctx):
            try:
                self.torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:  # noqa: BLE001
                pass

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


# ------------------------------------------------------------------ C-named entry points
def rlbm_opts_default() -> Opts:
    o = Opts()
    _load().rlbm_opts_default(ctypes.byref(o))
    return o


def rlbm_create(nx: int, ny: int, stencil: int, tau: float, forcing: Optional[Forcing], opts: Optional[Opts]):
    lib = _load()
    out = ctypes.c_void_p()
    st = lib.rlbm_create(int(nx), int(ny), int(stencil), float(tau), ctypes.byref(forcing) if forcing else None,
                         ctypes.byref(opts) if opts else None, ctypes.byref(out))
    _check(None, st, "rlbm_create")
    return out


def rlbm_init_fields(h, eps=None, vx=None, vy=None, n=None):
    lib = _load()
    st = lib.rlbm_init_fields(h, _p(eps), _p(vx), _p(vy))
    _check(h, st, "rlbm_init_fields")


def rlbm_init_fields_device(h, d_eps: int = 0, d_vx: int = 0, d_vy: int = 0):
    _check(h, _load().rlbm_init_fields_device(h, d_eps or None, d_vx or None, d_vy or None),
           "rlbm_init_fields_device")


def rlbm_step(h, n: int):
    _check(h, _load().rlbm_step(h, int(n)), "rlbm_step")


def rlbm_moments(h, eps, vx, vy, totals):
    st = _load().rlbm_moments(h, _p(eps), _p(vx), _p(vy), _p(totals))
    _check(h, st, "rlbm_moments")


def rlbm_moments_device(h, d_eps: int = 0, d_vx: int = 0, d_vy: int = 0, d_totals: int = 0):
    st = _load().rlbm_moments_device(h, d_eps or None, d_vx or None, d_vy or None, d_totals or None)
    _check(h, st, "rlbm_moments_device")


def rlbm_energy_spectrum(h, nshells: int, Ek):
    _check(h, _load().rlbm_energy_spectrum(h, int(nshells), _p(Ek)), "rlbm_energy_spectrum")


def rlbm_filtered_velocity(h, kf: float) -> float:
    rms = np.zeros(1)
    _check(h, _load().rlbm_filtered_velocity(h, float(kf), _p(rms)), "rlbm_filtered_velocity")
    return float(rms[0])


def rlbm_spectrum_sample(h, nshells: int):
    _check(h, _load().rlbm_spectrum_sample(h, int(nshells)), "rlbm_spectrum_sample")


def rlbm_spectrum_stats(h, nshells: int):
    mean, sem, cnt = np.empty(int(nshells)), np.empty(int(nshells)), ctypes.c_int()
    _check(h, _load().rlbm_spectrum_stats(h, int(nshells), _p(mean), _p(sem), ctypes.byref(cnt)),
           "rlbm_spectrum_stats")
    return mean, sem, cnt.value


def rlbm_spectrum_reset(h):
    _check(h, _load().rlbm_spectrum_reset(h), "rlbm_spectrum_reset")


def rlbm_get_populations(h, f):
    _check(h, _load().rlbm_get_populations(h, _p(f)), "rlbm_get_populations")


def rlbm_set_populations(h, f):
    _check(h, _load().rlbm_set_populations(h, _p(f)), "rlbm_set_populations")


def rlbm_get_force(h, Fx, Fy):
    _check(h, _load().rlbm_get_force(h, _p(Fx), _p(Fy)), "rlbm_get_force")


def rlbm_create3d(nx: int, ny: int, nz: int, tau: float, forcing: Optional[Forcing], opts: Optional[Opts]):
    lib = _load()
    out = ctypes.c_void_p()
    st = lib.rlbm_create3d(int(nx), int(ny), int(nz), float(tau), ctypes.byref(forcing) if forcing else None,
                           ctypes.byref(opts) if opts else None, ctypes.byref(out))
    _check(None, st, "rlbm_create3d")
    return out


def rlbm_init_fields3d(h, eps=None, vx=None, vy=None, vz=None):
    _check(h, _load().rlbm_init_fields3d(h, _p(eps), _p(vx), _p(vy), _p(vz)), "rlbm_init_fields3d")


def rlbm_moments3d(h, eps, vx, vy, vz, totals):
    _check(h, _load().rlbm_moments3d(h, _p(eps), _p(vx), _p(vy), _p(vz), _p(totals)), "rlbm_moments3d")


def rlbm_checkpoint_size(h) -> int:
    n = ctypes.c_size_t()
    _check(h, _load().rlbm_checkpoint_size(h, ctypes.byref(n)), "rlbm_checkpoint_size")
    return int(n.value)


def rlbm_checkpoint_save(h, buf: np.ndarray):
    _check(h, _load().rlbm_checkpoint_save(h, buf.ctypes.data, buf.nbytes), "rlbm_checkpoint_save")


def rlbm_checkpoint_load(h, buf: np.ndarray):
    _check(h, _load().rlbm_checkpoint_load(h, buf.ctypes.data, buf.nbytes), "rlbm_checkpoint_load")


def rlbm_get_force3d(h, Fx, Fy, Fz):
    _check(h, _load().rlbm_get_force3d(h, _p(Fx), _p(Fy), _p(Fz)), "rlbm_get_force3d")


def rlbm_get_info(h) -> Info:
    info = Info()
    _check(h, _load().rlbm_get_info(h, ctypes.byref(info)), "rlbm_get_info")
    return info


def rlbm_autotune(h, reps: int = 20):
    k, bx, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(h, _load().rlbm_autotune(h, int(reps), ctypes.byref(k), ctypes.byref(bx), ctypes.byref(by)),
           "rlbm_autotune")
    return k.value, bx.value, by.value


def rlbm_set_launch(h, kernel: int, block_x: int, block_y: int, launch_budget: int):
    _check(h, _load().rlbm_set_launch(h, int(kernel), int(block_x), int(block_y), int(launch_budget)),
           "rlbm_set_launch")


def rlbm_moments_static(stencil: int, dtype: int, d_q: int, nx: int, ny: int, pitch: int, eps0: float, scale: float,
                        cfl: float = 1.0, d_eps: int = 0, d_vx: int = 0, d_vy: int = 0, d_totals: int = 0,
                        d_bad: int = 0, stream: int = 0):
    """Allocation-free moments from a caller-owned device population array
    (see include/rlbm.h); all pointers are device addresses as ints."""
    st = _load().rlbm_moments_static(int(stencil), int(dtype), d_q or None, int(nx), int(ny), int(pitch), float(eps0),
                                     float(scale), float(cfl), d_eps or None, d_vx or None, d_vy or None,
                                     d_totals or None, d_bad or None, stream or None)
    _check(None, st, "rlbm_moments_static")


def rlbm_set_force_frame(h, nx_global: int, ny_global: int, x0: int, y0: int):
    _check(h, _load().rlbm_set_force_frame(h, int(nx_global), int(ny_global), int(x0), int(y0)),
           "rlbm_set_force_frame")


def rlbm_halo_pack(h, row: int, nrows: int, d_buf: int):
    _check(h, _load().rlbm_halo_pack(h, int(row), int(nrows), d_buf), "rlbm_halo_pack")


def rlbm_halo_unpack(h, row: int, nrows: int, d_buf: int):
    _check(h, _load().rlbm_halo_unpack(h, int(row), int(nrows), d_buf), "rlbm_halo_unpack")


def rlbm_synchronize(h):
    _check(h, _load().rlbm_synchronize(h), "rlbm_synchronize")


def rlbm_last_error(h) -> str:
    buf = ctypes.create_string_buffer(512)
    _load().rlbm_last_error(h, buf, 512)
    return buf.value.decode()


def rlbm_status_string(status: int) -> str:
    return _load().rlbm_status_string(int(status)).decode()


def rlbm_batch_create(runs, opts: Optional[Opts]):
    arr = (RunDesc * len(runs))(*runs)
    out = ctypes.c_void_p()
    st = _load().rlbm_batch_create(len(runs), arr, ctypes.byref(opts) if opts else None, ctypes.byref(out))
    _check(None, st, "rlbm_batch_create")
    return out


def rlbm_create_batch(runs, opts: Optional[Opts]):
    """rlbm_batch_create under its other name."""
    arr = (RunDesc * len(runs))(*runs)
    out = ctypes.c_void_p()
    st = _load().rlbm_create_batch(len(runs), arr, ctypes.byref(opts) if opts else None, ctypes.byref(out))
    _check(None, st, "rlbm_create_batch")
    return out


def rlbm_batch_init_fields(b, run: int, eps=None, vx=None, vy=None):
    _check(b, _load().rlbm_batch_init_fields(b, int(run), _p(eps), _p(vx), _p(vy)), "rlbm_batch_init_fields", True)


def rlbm_batch_step(b, n: int):
    _check(b, _load().rlbm_batch_step(b, int(n)), "rlbm_batch_step", True)


def rlbm_batch_moments(b, run: int, eps, vx, vy, totals):
    _check(b, _load().rlbm_batch_moments(b, int(run), _p(eps), _p(vx), _p(vy), _p(totals)), "rlbm_batch_moments",
           True)


def rlbm_batch_energy_spectrum(b, run: int, nshells: int, Ek):
    _check(b, _load().rlbm_batch_energy_spectrum(b, int(run), int(nshells), _p(Ek)), "rlbm_batch_energy_spectrum",
           True)


def rlbm_batch_get_populations(b, run: int, f):
    _check(b, _load().rlbm_batch_get_populations(b, int(run), _p(f)), "rlbm_batch_get_populations", True)


def rlbm_batch_autotune(b, reps: int = 10):
    bx, by, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(b, _load().rlbm_batch_autotune(b, int(reps), ctypes.byref(bx), ctypes.byref(by), ctypes.byref(g)),
           "rlbm_batch_autotune", True)
    return bx.value, by.value, g.value


def rlbm_batch_get_info(b) -> BatchInfo:
    info = BatchInfo()
    _check(b, _load().rlbm_batch_get_info(b, ctypes.byref(info)), "rlbm_batch_get_info", True)
    return info


def rlbm_batch_synchronize(b):
    _check(b, _load().rlbm_batch_synchronize(b), "rlbm_batch_synchronize", True)


def rlbm_batch_last_error(b) -> str:
    buf = ctypes.create_string_buffer(512)
    _load().rlbm_batch_last_error(b, buf, 512)
    return buf.value.decode()


def rlbm_batch_destroy(b):
    if b:
        _load().rlbm_batch_destroy(b)


def rlbm_destroy(h):
    if h:
        _load().rlbm_destroy(h)


# ------------------------------------------------------------------ convenience class
class Lattice:
    """One periodic nx x ny RLBM lattice on a GPU.

    dtype: "f64" | "f32" | "bf16" | "f16" (storage form); landau: "fp64" |
    "fp32" (precision of the Landau solve in the 32/16-bit forms); forcing:
    None or dict(kmin, kmax, amp, seed, redraw_period); allocator: "torch"
    (PyTorch caching allocator) or "cuda" (cudaMalloc inside the library);
    stream: a torch.cuda.Stream, an int cudaStream_t, or None (a new torch
    stream for this lattice); stencil: "sph26" (the paper's 26-direction
    node, 17 stored classes) or "ring8" (the 2D massless gas on an
    8-direction ring, P = eps/2; gather kernel, cfl 1, fixed tau).
    """

    def __init__(self, nx: int, ny: int, tau: float, *, dtype: str = "f32", landau: str = "fp32",
                 forcing: Optional[dict] = None, eps0: float = 1.0, scale: float = 0.0, kernel: str = "auto",
                 use_graphs: bool = True, allocator: str = "torch", stream=None, device: Optional[int] = None,
                 cfl: float = 1.0, eta_s: float = 0.0, dt: float = 1.0, stencil: str = "sph26",
                 test_unarmed_wait: bool = False, rounding: str = "default"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the RLBM library runs on the GPU only")
        self.nx, self.ny, self.tau = int(nx), int(ny), float(tau)
        self._h = None
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        if stream is None:
            self._torch_stream = torch.cuda.Stream(device=dev)
            s = self._torch_stream.cuda_stream
        elif isinstance(stream, int):
            self._torch_stream = None
            s = stream
        else:
            self._torch_stream = stream
            s = stream.cuda_stream
        self.stream_handle = s
        o = rlbm_opts_default()
        o.dtype = DTYPES[dtype]
        o.landau = LANDAU[landau]
        o.kernel = KERNELS[kernel]
        o.use_graphs = 1 if use_graphs else 0
        o.eps0 = float(eps0)
        o.scale = float(scale)
        o.stream = s
        o.device = dev
        o.cfl = float(cfl)
        o.eta_s = float(eta_s)
        o.dt = float(dt)
        o.test_unarmed_wait = 1 if test_unarmed_wait else 0
        o.rounding = ROUNDING[rounding]
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(dev, s)
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        f = None
        if forcing:
            f = Forcing(int(forcing.get("kmin", 0)), int(forcing.get("kmax", 0)), float(forcing.get("amp", 0.0)),
                        int(forcing.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF, int(forcing.get("redraw_period", 100)))
        self.dtype = dtype
        self.stencil = stencil
        self._h = self._create(f, o)
        self.nclasses = self.info()["nclasses"]

    def _create(self, forcing, opts):
        return rlbm_create(self.nx, self.ny, STENCILS[self.stencil], self.tau, forcing, opts)

    # -- life cycle
    def close(self):
        if self._h:
            rlbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("lattice is closed")
        return self._h

    # -- calls
    def init_fields(self, eps=None, vx=None, vy=None):
        n = self.nx * self.ny
        rlbm_init_fields(self.handle, _f64(eps, n), _f64(vx, n), _f64(vy, n))

    def init_fields_device(self, eps=None, vx=None, vy=None):
        ptr = lambda t: 0 if t is None else int(t.data_ptr())
        rlbm_init_fields_device(self.handle, ptr(eps), ptr(vx), ptr(vy))

    def step(self, n: int = 1):
        rlbm_step(self.handle, n)

    def moments(self, out=None):
        """(eps, vx, vy, totals): (ny, nx) FP64 fields and totals[3].  out:
        optional (eps, vx, vy, totals) C-contiguous FP64 arrays to fill (for
        example views of pinned host memory), returned as given."""
        if out is None:
            out = (np.empty((self.ny, self.nx)), np.empty((self.ny, self.nx)), np.empty((self.ny, self.nx)),
                   np.empty(3))
        eps, vx, vy, tot = out
        for a, n in ((eps, self.nx * self.ny), (vx, self.nx * self.ny), (vy, self.nx * self.ny), (tot, 3)):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
                raise ValueError("moments(out=...) needs C-contiguous FP64 arrays of the lattice's size")
        rlbm_moments(self.handle, eps, vx, vy, tot)
        return eps, vx, vy, tot

    def set_force_frame(self, nx_global: int, ny_global: int, x0: int, y0: int):
        """Draw the stirring force in the frame of a larger lattice (a slab of
        a decomposed lattice; see slab.py)."""
        rlbm_set_force_frame(self.handle, nx_global, ny_global, x0, y0)

    def halo_pack(self, row: int, nrows: int, d_buf: int):
        rlbm_halo_pack(self.handle, row, nrows, d_buf)

    def halo_unpack(self, row: int, nrows: int, d_buf: int):
        rlbm_halo_unpack(self.handle, row, nrows, d_buf)

    def moments_device(self, eps=None, vx=None, vy=None, totals=None):
        ptr = lambda t: 0 if t is None else int(t.data_ptr())
        rlbm_moments_device(self.handle, ptr(eps), ptr(vx), ptr(vy), ptr(totals))

    def energy_spectrum(self, nshells: int) -> np.ndarray:
        E = np.empty(int(nshells))
        rlbm_energy_spectrum(self.handle, nshells, E)
        return E

    def filtered_velocity(self, kf: float) -> float:
        """RMS velocity with the modes |k| >= kf removed (Sec. 5)."""
        return rlbm_filtered_velocity(self.handle, kf)

    def spectrum_sample(self, nshells: int):
        rlbm_spectrum_sample(self.handle, nshells)

    def spectrum_stats(self, nshells: int):
        """(mean E(k), standard error of the mean, sample count)."""
        return rlbm_spectrum_stats(self.handle, nshells)

    def spectrum_reset(self):
        rlbm_spectrum_reset(self.handle)

    def populations(self) -> np.ndarray:
        f = np.empty((self.nclasses, self.ny, self.nx))
        rlbm_get_populations(self.handle, f)
        return f

    def set_populations(self, f):
        rlbm_set_populations(self.handle, _f64(f, self.nclasses * self.nx * self.ny))

    def checkpoint(self) -> np.ndarray:
        """The state and step counter as a byte array (rlbm_checkpoint_save)."""
        buf = np.empty(rlbm_checkpoint_size(self.handle), dtype=np.uint8)
        rlbm_checkpoint_save(self.handle, buf)
        return buf

    def restore(self, buf):
        """Resume from a checkpoint of a lattice created with the same arguments."""
        rlbm_checkpoint_load(self.handle, np.ascontiguousarray(np.asarray(buf, dtype=np.uint8)))

    def save(self, path: str):
        self.checkpoint().tofile(path)

    def load(self, path: str):
        self.restore(np.fromfile(path, dtype=np.uint8))

    def force(self):
        Fx = np.empty((self.ny, self.nx))
        Fy = np.empty((self.ny, self.nx))
        rlbm_get_force(self.handle, Fx, Fy)
        return Fx, Fy

    def info(self) -> dict:
        i = rlbm_get_info(self.handle)
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def autotune(self, reps: int = 20):
        """Pick the fastest launch configuration of the fused step (state unchanged)."""
        return rlbm_autotune(self.handle, reps)

    def set_launch(self, kernel: str, block_x: int, block_y: int, launch_budget: int):
        """Pin the fused step to one of the autotuner's launch configurations."""
        rlbm_set_launch(self.handle, KERNELS[kernel], block_x, block_y, launch_budget)

    def synchronize(self):
        rlbm_synchronize(self.handle)


class Lattice3D(Lattice):
    """A three-dimensional periodic lattice of the paper's node (26 stored
    directions, trilinear streaming, 3D stirring on a shell).  Same options
    as Lattice (kernel "auto" or "gather", cfl 1); fields are (nz, ny, nx)
    arrays, populations (26, nz, ny, nx)."""

    def __init__(self, nx: int, ny: int, nz: int, tau: float, **kw):
        self.nz = int(nz)
        super().__init__(nx, ny, tau, **kw)

    def _create(self, forcing, opts):
        return rlbm_create3d(self.nx, self.ny, self.nz, self.tau, forcing, opts)

    def _shape(self):
        return (self.nz, self.ny, self.nx)

    def init_fields(self, eps=None, vx=None, vy=None, vz=None):
        n = self.nx * self.ny * self.nz
        rlbm_init_fields3d(self.handle, _f64(eps, n), _f64(vx, n), _f64(vy, n), _f64(vz, n))

    def moments(self):
        """(eps, vx, vy, vz, totals): (nz, ny, nx) FP64 fields and totals[4]."""
        out = [np.empty(self._shape()) for _ in range(4)]
        tot = np.empty(4)
        rlbm_moments3d(self.handle, *out, tot)
        return (*out, tot)

    def populations(self) -> np.ndarray:
        f = np.empty((self.nclasses,) + self._shape())
        rlbm_get_populations(self.handle, f)
        return f

    def set_populations(self, f):
        rlbm_set_populations(self.handle, _f64(f, self.nclasses * self.nx * self.ny * self.nz))

    def force(self):
        F = [np.empty(self._shape()) for _ in range(3)]
        rlbm_get_force3d(self.handle, *F)
        return tuple(F)


class Ensemble:
    """Independent lattices advanced together by one launch per step (per two
    steps with the two-step body the autotuner may pick).

    runs: list of dicts with nx, ny, tau and optional forcing (as for
    Lattice).  dtype / landau / allocator / stream as for Lattice.
    """

    def __init__(self, runs, *, dtype: str = "f32", landau: str = "fp32", use_graphs: bool = True,
                 allocator: str = "torch", stream=None, device: Optional[int] = None, kernel: str = "auto",
                 rounding: str = "default"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the RLBM library runs on the GPU only")
        self._b = None
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        if stream is None:
            self._torch_stream = torch.cuda.Stream(device=dev)
            s = self._torch_stream.cuda_stream
        elif isinstance(stream, int):
            self._torch_stream = None
            s = stream
        else:
            self._torch_stream = stream
            s = stream.cuda_stream
        o = rlbm_opts_default()
        o.dtype = DTYPES[dtype]
        o.landau = LANDAU[landau]
        o.kernel = KERNELS[kernel]
        o.use_graphs = 1 if use_graphs else 0
        o.rounding = ROUNDING[rounding]
        o.stream = s
        o.device = dev
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(dev, s)
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        descs = []
        self.shapes = []
        for r in runs:
            fz = r.get("forcing") or {}
            f = Forcing(int(fz.get("kmin", 0)), int(fz.get("kmax", 0)), float(fz.get("amp", 0.0)),
                        int(fz.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF, int(fz.get("redraw_period", 100)))
            descs.append(RunDesc(int(r["nx"]), int(r["ny"]), float(r["tau"]), f))
            self.shapes.append((int(r["ny"]), int(r["nx"])))
        self._b = rlbm_batch_create(descs, o)

    def close(self):
        if self._b:
            rlbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    @property
    def handle(self):
        if not self._b:
            raise RuntimeError("ensemble is closed")
        return self._b

    def init_fields(self, run: int, eps=None, vx=None, vy=None):
        ny, nx = self.shapes[run]
        n = nx * ny
        rlbm_batch_init_fields(self.handle, run, _f64(eps, n), _f64(vx, n), _f64(vy, n))

    def step(self, n: int = 1):
        rlbm_batch_step(self.handle, n)

    def moments(self, run: int):
        ny, nx = self.shapes[run]
        eps, vx, vy, tot = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx)), np.empty(3)
        rlbm_batch_moments(self.handle, run, eps, vx, vy, tot)
        return eps, vx, vy, tot

    def energy_spectrum(self, run: int, nshells: int) -> np.ndarray:
        E = np.empty(int(nshells))
        rlbm_batch_energy_spectrum(self.handle, run, nshells, E)
        return E

    def populations(self, run: int) -> np.ndarray:
        ny, nx = self.shapes[run]
        f = np.empty((NCLASSES, ny, nx))
        rlbm_batch_get_populations(self.handle, run, f)
        return f

    def autotune(self, reps: int = 10):
        return rlbm_batch_autotune(self.handle, reps)

    def info(self) -> dict:
        i = rlbm_batch_get_info(self.handle)
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def synchronize(self):
        rlbm_batch_synchronize(self.handle)

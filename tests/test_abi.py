"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point include/rlbm.h declares, and rejects
invalid arguments before touching the device."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rlbm.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2101_06187_gb300 as rl
    return rl.library()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RLBM_API[^;(]*?\b(rlbm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rlbm_create", "rlbm_step", "rlbm_moments", "rlbm_energy_spectrum", "rlbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rlbm_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_names_match_header():
    import paper_2101_06187_gb300 as rl
    assert sorted(rl.EXPORTS) == _declared()
    for name in rl.EXPORTS:
        assert callable(getattr(rl, name)), name


def test_create_rejects_invalid_arguments_without_touching_the_device(lib):
    import paper_2101_06187_gb300 as rl
    out = ctypes.c_void_p()
    F = rl.Forcing

    def create(nx, ny, tau, forcing=None, opts=None, st=0):
        return lib.rlbm_create(nx, ny, st, tau, ctypes.byref(forcing) if forcing else None,
                               ctypes.byref(opts) if opts else None, ctypes.byref(out))

    assert create(3, 16, 0.8) == rl.RLBM_ERR_ARG          # nx < 4
    assert create(16, 2, 0.8) == rl.RLBM_ERR_ARG          # ny < 4
    assert create(16, 65536, 0.8) == rl.RLBM_ERR_ARG      # ny beyond the launch grid's y dimension
    assert create(16, 16, 0.5) == rl.RLBM_ERR_ARG         # tau must exceed 1/2
    assert create(16, 16, float("nan")) == rl.RLBM_ERR_ARG
    assert create(16, 16, 0.8, st=2) == rl.RLBM_ERR_ARG   # unknown stencil
    assert create(16, 16, 0.8, F(2, 8, 1e-3, 1, 100)) == rl.RLBM_ERR_ARG   # kmax >= n/2
    assert create(16, 16, 0.8, F(0, 3, 1e-3, 1, 100)) == rl.RLBM_ERR_ARG   # kmin < 1
    assert create(16, 16, 0.8, F(3, 2, 1e-3, 1, 100)) == rl.RLBM_ERR_ARG   # kmin > kmax
    assert create(16, 16, 0.8, F(1, 3, -1.0, 1, 100)) == rl.RLBM_ERR_ARG   # amp < 0
    assert create(16, 16, 0.8, F(1, 3, 1e-3, 1, 0)) == rl.RLBM_ERR_ARG     # redraw period
    o = rl.rlbm_opts_default()
    o.dtype = 9
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG
    o = rl.rlbm_opts_default()
    o.scale = -1.0
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG
    o = rl.rlbm_opts_default()
    o.scale = 2.0   # FP32 and FP64 storage keep the deviation unscaled
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG
    o.dtype = rl.DTYPES["f64"]
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG
    o = rl.rlbm_opts_default()
    o.kernel = rl.KERNELS["vec"]
    assert create(37, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG   # vector kernel needs nx % 4 == 0
    o = rl.rlbm_opts_default()
    o.cfl = 2.0
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG   # displacement of two cells or more (halo 2)
    o.cfl = 0.5
    o.kernel = rl.KERNELS["vec"]
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG   # vector kernels stream at CFL 1 only
    o = rl.rlbm_opts_default()
    o.eta_s = -0.01
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG
    # two steps per launch: packed FP32 lanes (nx even) at cfl <= 1, one-layer lattice only; the FP64 Landau
    # solve on them (the frame refined on the FP32 lanes) at cfl 1 only
    for field, value, nx in (("dtype", rl.DTYPES["f64"], 16), (None, None, 17), ("cfl", 1.25, 16)):
        o = rl.rlbm_opts_default()
        o.kernel = rl.KERNELS["fused2"]
        if field:
            setattr(o, field, value)
        assert create(nx, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG, (field, value, nx)
    for kernel in ("fused2", "packed", "twopass"):
        o = rl.rlbm_opts_default()
        o.kernel = rl.KERNELS[kernel]
        o.landau = rl.LANDAU["fp64"]
        o.cfl = 0.5 if kernel != "twopass" else 1.0
        assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG, kernel
    # stochastic rounding of 16-bit stores: the packed kernels only; unknown rounding modes refused
    for kernel, rounding in (("gather", 2), ("vec", 2), ("auto", 3), ("auto", -1)):
        o = rl.rlbm_opts_default()
        o.dtype = rl.DTYPES["bf16"]
        o.kernel = rl.KERNELS[kernel]
        o.rounding = rounding
        assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG, (kernel, rounding)
    o = rl.rlbm_opts_default()
    o.kernel = rl.KERNELS["fused2"]
    o.dtype = rl.DTYPES["f64"]
    assert create(16, 16, 0.8, opts=o, st=rl.RLBM_STENCIL_RING8_2D) == rl.RLBM_ERR_ARG   # ring: FP32 lanes
    o.dtype = rl.DTYPES["f32"]
    assert lib.rlbm_create3d(16, 16, 16, ctypes.c_double(0.8), None, ctypes.byref(o),
                             ctypes.byref(out)) == rl.RLBM_ERR_ARG   # not on the 3D lattice
    o.kernel = 9
    assert create(16, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG   # no kernel 9
    # four nodes per thread: aligned runs of four, CFL 1, FP32 / 16-bit storage, the one-layer lattice
    for field, value, nx in (("dtype", rl.DTYPES["f32"], 18), ("dtype", rl.DTYPES["f64"], 16),
                             ("cfl", 0.625, 16), ("cfl", 1.25, 16)):
        o = rl.rlbm_opts_default()
        o.kernel = rl.KERNELS["packed4"]
        setattr(o, field, value)
        assert create(nx, 16, 0.8, opts=o) == rl.RLBM_ERR_ARG, (field, value, nx)
    o = rl.rlbm_opts_default()
    o.kernel = rl.KERNELS["packed4"]
    assert create(16, 16, 0.8, opts=o, st=rl.RLBM_STENCIL_RING8_2D) == rl.RLBM_ERR_ARG
    assert lib.rlbm_create3d(16, 16, 16, ctypes.c_double(0.8), None, ctypes.byref(o),
                             ctypes.byref(out)) == rl.RLBM_ERR_ARG
    ring = rl.RLBM_STENCIL_RING8_2D   # the ring runs the gather kernel at CFL 1 with a fixed tau
    for field, value in (("kernel", rl.KERNELS["vec"]), ("kernel", rl.KERNELS["tma"]), ("cfl", 0.5),
                         ("eta_s", 0.1)):
        o = rl.rlbm_opts_default()
        setattr(o, field, value)
        assert create(16, 16, 0.8, opts=o, st=ring) == rl.RLBM_ERR_ARG
    assert create(3, 16, 0.8, st=ring) == rl.RLBM_ERR_ARG
    assert out.value is None
    assert lib.rlbm_create(16, 16, 0, 0.8, None, None, None) == rl.RLBM_ERR_ARG


def test_batch_create_rejects_invalid_members(lib):
    import paper_2101_06187_gb300 as rl
    out = ctypes.c_void_p()
    good = rl.RunDesc(64, 64, 0.7, rl.Forcing(0, 0, 0.0, 0, 100))
    odd = rl.RunDesc(66, 64, 0.7, rl.Forcing(0, 0, 0.0, 0, 100))  # nx % 4 != 0
    arr = (rl.RunDesc * 2)(good, odd)
    assert lib.rlbm_batch_create(2, arr, None, ctypes.byref(out)) == rl.RLBM_ERR_ARG
    assert lib.rlbm_batch_create(0, arr, None, ctypes.byref(out)) == rl.RLBM_ERR_ARG
    assert lib.rlbm_batch_create(1, None, None, ctypes.byref(out)) == rl.RLBM_ERR_ARG
    assert lib.rlbm_create_batch(2, arr, None, ctypes.byref(out)) == rl.RLBM_ERR_ARG  # the same call, other name
    # decomposition calls refuse a missing handle
    assert lib.rlbm_set_force_frame(None, 64, 64, 0, 0) == rl.RLBM_ERR_ARG
    assert lib.rlbm_halo_pack(None, 0, 1, None) == rl.RLBM_ERR_ARG
    assert lib.rlbm_halo_unpack(None, 0, 1, None) == rl.RLBM_ERR_ARG
    # ensemble bodies: vector, packed or two-step; the lane bodies need FP32 compute, FP32 Landau, nx even
    for field, value, kernel in ((None, None, "tma"), (None, None, "gather"), ("dtype", rl.DTYPES["f64"], "fused2"),
                                 ("landau", rl.LANDAU["fp64"], "packed"), ("cfl", 0.5, "fused2")):
        o = rl.rlbm_opts_default()
        o.kernel = rl.KERNELS[kernel]
        if field:
            setattr(o, field, value)
        assert lib.rlbm_batch_create(1, arr, ctypes.byref(o), ctypes.byref(out)) == rl.RLBM_ERR_ARG, (field, kernel)
    o = rl.rlbm_opts_default()
    o.kernel = rl.KERNELS["fused2"]
    odd2 = (rl.RunDesc * 1)(rl.RunDesc(63, 64, 0.7, rl.Forcing(0, 0, 0.0, 0, 100)))  # nx odd
    assert lib.rlbm_batch_create(1, odd2, ctypes.byref(o), ctypes.byref(out)) == rl.RLBM_ERR_ARG
    assert out.value is None
    lib.rlbm_batch_destroy(None)


def test_null_handle_calls_are_rejected(lib):
    import paper_2101_06187_gb300 as rl
    assert lib.rlbm_step(None, 1) == rl.RLBM_ERR_ARG
    assert lib.rlbm_moments(None, None, None, None, None) == rl.RLBM_ERR_ARG
    assert lib.rlbm_energy_spectrum(None, 4, None) == rl.RLBM_ERR_ARG
    lib.rlbm_destroy(None)
    assert lib.rlbm_status_string(rl.RLBM_ERR_NAN) == b"non-finite or non-physical state"


def test_opts_defaults(lib):
    import paper_2101_06187_gb300 as rl
    o = rl.rlbm_opts_default()
    assert o.dtype == rl.DTYPES["f32"] and o.landau == rl.LANDAU["fp32"] and o.use_graphs == 1 and o.eps0 == 1.0 and o.device == -1
    assert o.cfl == 1.0 and o.eta_s == 0.0 and o.dt == 1.0


def test_binding_fails_loudly_without_the_library(tmp_path):
    code = ("import paper_2101_06187_gb300 as rl; rl.LIB_PATH = %r\n"
            "try:\n    rl.library()\nexcept RuntimeError as e:\n    print('raised', e)\n") % str(tmp_path / "none.so")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "raised" in r.stdout

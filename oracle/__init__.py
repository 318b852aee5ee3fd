"""Plain FP64 CPU oracle of the RLBM stream-collide step (arXiv:2101.06187).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
(``paper_2101_06187_gb300``) never does, and the two share no code.

The arithmetic lives in ``rlbm_oracle.c`` (see its header for the equations
followed, by section and equation of the paper).  This module compiles it
with gcc (``-O2 -ffp-contract=off -fopenmp``), loads it with ctypes and wraps
it with numpy arrays.  Populations are ``float64`` arrays of shape
``(26, ny, nx)``.

Function status (pins live in ``tests/test_oracle_*.py``):
  stencil, moments, ideal_T, feq, landau, force_term, collide, stream,
  forcing field, totals, spectrum: pinned (closed forms, invariants,
  library eigen-solver, linear-mode analysis).
  philox4x32_10: pinned word for word against Triton's Philox4x32
  (CPU interpreter, tests/test_oracle_philox.py) and cuRAND's
  Philox4x32-10 (GPU, tests/test_gpu_philox.py) on the forcing's counters
  and seeded random words; its statistics are pinned too.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NDIR = 26

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)


_SRCS = (_SRC, os.path.join(_HERE, "ring2d_oracle.c"), os.path.join(_HERE, "lattice3d_oracle.c"))


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    if not force and os.path.exists(_LIB_PATH) and all(
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src) for src in _SRCS):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_ndirs.restype = ctypes.c_int
        lib.oracle_stencil.argtypes = [_dp, _dp]
        lib.oracle_moments_node.argtypes = [_dp, _dp]
        lib.oracle_landau.argtypes = [_dp, _dp, _dp]
        lib.oracle_landau.restype = ctypes.c_int
        lib.oracle_ideal_T.argtypes = [ctypes.c_double, _dp, _dp]
        lib.oracle_feq.argtypes = [ctypes.c_double, _dp, _dp]
        lib.oracle_force_term.argtypes = [_dp, _dp, _dp]
        lib.oracle_collide_node.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp]
        lib.oracle_collide_node.restype = ctypes.c_int
        lib.oracle_stream.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.oracle_forcing_modes.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, ctypes.c_int]
        lib.oracle_forcing_modes.restype = ctypes.c_int
        lib.oracle_forcing_draw.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                            ctypes.c_uint64, _dp, _dp, _dp]
        lib.oracle_force_field.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint64, _dp, _dp]
        lib.oracle_force_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _ip, _ip, _dp, _dp]
        lib.oracle_init.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.oracle_init.restype = ctypes.c_int
        lib.oracle_step.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
        lib.oracle_step.restype = ctypes.c_int
        lib.oracle_fields.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.oracle_fields.restype = ctypes.c_int
        lib.oracle_run.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_long,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_int]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_totals.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
        lib.oracle_tau_of.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_tau_of.restype = ctypes.c_double
        lib.oracle_collide_node_ex.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
        lib.oracle_collide_node_ex.restype = ctypes.c_int
        lib.oracle_stream_cfl.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.oracle_fields_ex.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_fields_ex.restype = ctypes.c_int
        lib.oracle_run_ex.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_long,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_run_ex.restype = ctypes.c_int
        lib.ring_stencil.argtypes = [_dp, _dp]
        lib.ring_moments_node.argtypes = [_dp, _dp]
        lib.ring_landau.argtypes = [_dp, _dp, _dp]
        lib.ring_landau.restype = ctypes.c_int
        lib.ring_ideal_T.argtypes = [ctypes.c_double, _dp, _dp]
        lib.ring_feq.argtypes = [ctypes.c_double, _dp, _dp]
        lib.ring_force_term.argtypes = [_dp, _dp, _dp]
        lib.ring_collide_node.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp]
        lib.ring_collide_node.restype = ctypes.c_int
        lib.ring_stream.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int]
        lib.ring_init.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.ring_init.restype = ctypes.c_int
        lib.ring_run.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_long,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                 ctypes.c_int]
        lib.ring_run.restype = ctypes.c_int
        lib.ring_fields.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.ring_fields.restype = ctypes.c_int
        lib.ring_totals.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
        i3 = [ctypes.c_int] * 3
        lib.oracle3d_stream.argtypes = [_dp, _dp, *i3]
        lib.oracle3d_init.argtypes = [_dp, *i3, _dp, _dp, _dp, _dp]
        lib.oracle3d_init.restype = ctypes.c_int
        lib.oracle3d_forcing_modes.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip, ctypes.c_int]
        lib.oracle3d_forcing_modes.restype = ctypes.c_int
        lib.oracle3d_forcing_draw.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                              ctypes.c_uint64, _dp, _dp, _dp]
        lib.oracle3d_force_field.argtypes = [*i3, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                             ctypes.c_uint64, _dp, _dp, _dp]
        lib.oracle3d_step.argtypes = [_dp, _dp, *i3, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle3d_step.restype = ctypes.c_int
        lib.oracle3d_fields.argtypes = [_dp, _dp, *i3, _dp, _dp, _dp, _dp]
        lib.oracle3d_fields.restype = ctypes.c_int
        lib.oracle3d_run.argtypes = [_dp, _dp, _dp, _dp, _dp, *i3, ctypes.c_double, ctypes.c_long, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
        lib.oracle3d_run.restype = ctypes.c_int
        lib.oracle3d_totals.argtypes = [_dp, *i3, _dp]
        _lib = lib
        return lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    """Set the OpenMP thread count used by the oracle's lattice loops."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(ctypes.c_int(int(n)))
    except OSError:
        pass


def stencil():
    """Return (v, w): the 26 unit directions (26, 3) and weights (26,)."""
    lib = _load()
    v = np.zeros((NDIR, 3))
    w = np.zeros(NDIR)
    lib.oracle_stencil(_p(v), _p(w))
    return v, w


def moments(f_node) -> np.ndarray:
    """T^{mu nu} (4x4) of one node's 26 populations."""
    lib = _load()
    f = _f64(f_node)
    T = np.zeros((4, 4))
    lib.oracle_moments_node(_p(f), _p(T))
    return T


def landau(T):
    """(eps, u^mu, passes) solving T^{mu nu} u_nu = -eps u^mu; passes < 0 on failure."""
    lib = _load()
    T = _f64(T)
    eps = np.zeros(1)
    u = np.zeros(4)
    it = lib.oracle_landau(_p(T), _p(eps), _p(u))
    return float(eps[0]), u, int(it)


def ideal_T(eps: float, u) -> np.ndarray:
    lib = _load()
    T = np.zeros((4, 4))
    lib.oracle_ideal_T(float(eps), _p(_f64(u)), _p(T))
    return T


def feq(eps: float, u) -> np.ndarray:
    lib = _load()
    out = np.zeros(NDIR)
    lib.oracle_feq(float(eps), _p(_f64(u)), _p(out))
    return out


def force_term(f_node, F) -> np.ndarray:
    lib = _load()
    G = np.zeros(NDIR)
    lib.oracle_force_term(_p(_f64(f_node)), _p(_f64(F)), _p(G))
    return G


def tau_of(eps: float, tau: float, eta_s: float = 0.0, dt: float = 1.0) -> float:
    """Relaxation time in steps: tau, or 5 (eta/s) / (T dt) with eps = 3 T^4 / pi^2."""
    return float(_load().oracle_tau_of(float(eps), float(tau), float(eta_s), float(dt)))


def collide(f_node, F, tau: float, eta_s: float = 0.0, dt: float = 1.0):
    """Collide one node; returns (f_new, eps, u^mu)."""
    lib = _load()
    f = _f64(f_node).copy()
    eps = np.zeros(1)
    u = np.zeros(4)
    rc = lib.oracle_collide_node_ex(_p(f), _p(_f64(F)) if F is not None else None, float(tau), float(eta_s),
                                    float(dt), _p(eps), _p(u))
    if rc != 0:
        raise FloatingPointError("Landau solve failed")
    return f, float(eps[0]), u


def stream(f, cfl: float = 1.0) -> np.ndarray:
    lib = _load()
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    lib.oracle_stream_cfl(_p(f), _p(out), nx, ny, float(cfl))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p), o.ctypes.data_as(_u32p))
    return o


def forcing_modes(kmin: int, kmax: int) -> np.ndarray:
    """Half-plane integer wavevectors of the driven shell, shape (m, 2) as (kx, ky)."""
    lib = _load()
    m = lib.oracle_forcing_modes(kmin, kmax, None, None, 0)
    kx = np.zeros(max(m, 1), dtype=np.int32)
    ky = np.zeros(max(m, 1), dtype=np.int32)
    lib.oracle_forcing_modes(kmin, kmax, kx.ctypes.data_as(_ip), ky.ctypes.data_as(_ip), m)
    return np.stack([kx[:m], ky[:m]], axis=1)


def forcing_draw(kmin, kmax, amp, seed, epoch):
    lib = _load()
    m = len(forcing_modes(kmin, kmax))
    mag, ph, th = np.zeros(max(m, 1)), np.zeros(max(m, 1)), np.zeros(max(m, 1))
    lib.oracle_forcing_draw(kmin, kmax, float(amp), int(seed), int(epoch), _p(mag), _p(ph), _p(th))
    return mag[:m], ph[:m], th[:m]


def force_field(nx, ny, kmin, kmax, amp, seed, epoch):
    lib = _load()
    Fx = np.zeros((ny, nx))
    Fy = np.zeros((ny, nx))
    lib.oracle_force_field(nx, ny, kmin, kmax, float(amp), int(seed), int(epoch), _p(Fx), _p(Fy))
    return Fx, Fy


def force_points(nx, ny, kmin, kmax, amp, seed, epoch, xs, ys):
    """The stirring force at the nodes (xs[k], ys[k]) only."""
    lib = _load()
    xs = np.ascontiguousarray(np.asarray(xs, dtype=np.int32))
    ys = np.ascontiguousarray(np.asarray(ys, dtype=np.int32))
    Fx = np.zeros(len(xs))
    Fy = np.zeros(len(xs))
    lib.oracle_force_points(nx, ny, kmin, kmax, float(amp), int(seed), int(epoch), len(xs), xs.ctypes.data_as(_ip),
                            ys.ctypes.data_as(_ip), _p(Fx), _p(Fy))
    return Fx, Fy


def init(nx, ny, eps=None, vx=None, vy=None) -> np.ndarray:
    lib = _load()
    f = np.zeros((NDIR, ny, nx))
    e = None if eps is None else _f64(eps).reshape(ny, nx)
    a = None if vx is None else _f64(vx).reshape(ny, nx)
    b = None if vy is None else _f64(vy).reshape(ny, nx)
    rc = lib.oracle_init(_p(f), nx, ny, _p(e), _p(a), _p(b))
    if rc != 0:
        raise ValueError("invalid initial fields (eps <= 0 or |v| >= 1)")
    return f


def step(f, tau, Fx=None, Fy=None) -> np.ndarray:
    """One step in place on f (26, ny, nx); returns f."""
    lib = _load()
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _, ny, nx = f.shape
    tmp = np.empty_like(f)
    bad = lib.oracle_step(_p(f), _p(tmp), nx, ny, float(tau), _p(None if Fx is None else _f64(Fx)),
                          _p(None if Fy is None else _f64(Fy)))
    if bad:
        raise FloatingPointError("Landau solve failed at %d nodes" % bad)
    return f


def fields(f, cfl: float = 1.0):
    """(eps, vx, vy) seen by the next collision (post-stream Landau frame)."""
    lib = _load()
    f = _f64(f)
    _, ny, nx = f.shape
    tmp = np.empty_like(f)
    eps, vx, vy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
    lib.oracle_fields_ex(_p(f), _p(tmp), nx, ny, float(cfl), _p(eps), _p(vx), _p(vy))
    return eps, vx, vy


def run(f, tau, nsteps, step0=0, kmin=0, kmax=0, amp=0.0, seed=0, redraw=100, cfl=1.0, eta_s=0.0,
        dt=1.0) -> np.ndarray:
    """nsteps steps in place on f with the epoch-redrawn stirring force
    (cfl: streaming displacement per step in cells; eta_s > 0: per-node
    relaxation time 5 (eta/s) / (T dt))."""
    lib = _load()
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _, ny, nx = f.shape
    tmp = np.empty_like(f)
    Fx = np.zeros((ny, nx))
    Fy = np.zeros((ny, nx))
    bad = lib.oracle_run_ex(_p(f), _p(tmp), _p(Fx), _p(Fy), nx, ny, float(tau), int(step0), int(nsteps), int(kmin),
                            int(kmax), float(amp), int(seed), int(redraw), float(cfl), float(eta_s), float(dt))
    if bad:
        raise FloatingPointError("Landau solve failed %d times" % bad)
    return f


def totals(f) -> np.ndarray:
    """Sum over nodes of T^{0 mu}, mu = 0..3."""
    lib = _load()
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.zeros(4)
    lib.oracle_totals(_p(f), nx, ny, _p(out))
    return out


def energy_spectrum(vx, vy, nshells: int) -> np.ndarray:
    """E(n), n = 0..nshells-1, of the 3-velocity field (Sec. 4).

    v_hat(k) = (1/(nx ny)) sum_x v(x) exp(-2 pi i k.x / N) (numpy FFT as the
    transform); shell n collects |k| in [n - 1/2, n + 1/2) with signed
    integer wavenumbers; E(n) = 1/2 sum_shell |v_hat_x|^2 + |v_hat_y|^2.
    """
    vx = np.asarray(vx, dtype=np.float64)
    vy = np.asarray(vy, dtype=np.float64)
    ny, nx = vx.shape
    ax = np.fft.fft2(vx) / (nx * ny)
    ay = np.fft.fft2(vy) / (nx * ny)
    p = 0.5 * (np.abs(ax) ** 2 + np.abs(ay) ** 2)
    kx = np.fft.fftfreq(nx, d=1.0 / nx)
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    K = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    shell = np.floor(K + 0.5).astype(np.int64)
    E = np.zeros(nshells)
    for n in range(nshells):
        E[n] = p[shell == n].sum()
    return E


def filtered_velocity_rms(vx, vy, kf: float) -> float:
    """RMS of the 3-velocity after removing the driven band (Sec. 5): keep
    the Fourier modes with |k| < kf (signed integer wavenumbers), transform
    back, and take sqrt(mean |v|^2) over the lattice."""
    vx = np.asarray(vx, dtype=np.float64)
    vy = np.asarray(vy, dtype=np.float64)
    ny, nx = vx.shape
    kx = np.fft.fftfreq(nx, d=1.0 / nx)
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    keep = (kx[None, :] ** 2 + ky[:, None] ** 2) < kf * kf
    fx = np.real(np.fft.ifft2(np.fft.fft2(vx) * keep))
    fy = np.real(np.fft.ifft2(np.fft.fft2(vy) * keep))
    return float(np.sqrt(np.mean(fx * fx + fy * fy)))


def merge_classes(f) -> np.ndarray:
    """Sum the z-mirror pairs of the 26 directions into the 17 in-plane classes.

    Class order: rest (0,0); (1,0),(-1,0),(0,1),(0,-1); (a,0),(-a,0),(0,a),
    (0,-a) with a = 1/sqrt2; (a,a),(-a,a),(a,-a),(-a,-a); (b,b),(-b,b),(b,-b),
    (-b,-b) with b = 1/sqrt3.  Used by tests to compare raw populations.
    """
    v, _ = stencil()
    f = np.asarray(f)
    a = 1.0 / np.sqrt(2.0)
    b = 1.0 / np.sqrt(3.0)
    targets = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (a, 0), (-a, 0), (0, a), (0, -a), (a, a), (-a, a), (a, -a),
               (-a, -a), (b, b), (-b, b), (b, -b), (-b, -b)]
    out = np.zeros((17,) + f.shape[1:])
    for c, (tx, ty) in enumerate(targets):
        for i in range(NDIR):
            if abs(v[i, 0] - tx) < 1e-12 and abs(v[i, 1] - ty) < 1e-12:
                out[c] += f[i]
    return out


# --------------------------------------------------------------------------- 2D ring model
RING = 8


class ring:
    """The genuinely 2D massless variant (8-direction ring, P = eps/2); see
    ring2d_oracle.c.  Populations are (8, ny, nx) FP64 arrays."""

    @staticmethod
    def stencil():
        lib = _load()
        v = np.zeros((RING, 2))
        w = np.zeros(RING)
        lib.ring_stencil(_p(v), _p(w))
        return v, w

    @staticmethod
    def moments(f_node):
        T = np.zeros((3, 3))
        _load().ring_moments_node(_p(_f64(f_node)), _p(T))
        return T

    @staticmethod
    def landau(T):
        eps, u = np.zeros(1), np.zeros(3)
        it = _load().ring_landau(_p(_f64(T)), _p(eps), _p(u))
        return float(eps[0]), u, int(it)

    @staticmethod
    def ideal_T(eps, u):
        T = np.zeros((3, 3))
        _load().ring_ideal_T(float(eps), _p(_f64(u)), _p(T))
        return T

    @staticmethod
    def feq(eps, u):
        out = np.zeros(RING)
        _load().ring_feq(float(eps), _p(_f64(u)), _p(out))
        return out

    @staticmethod
    def force_term(f_node, F):
        G = np.zeros(RING)
        _load().ring_force_term(_p(_f64(f_node)), _p(_f64(F)), _p(G))
        return G

    @staticmethod
    def collide(f_node, F, tau):
        f = _f64(f_node).copy()
        eps, u = np.zeros(1), np.zeros(3)
        rc = _load().ring_collide_node(_p(f), _p(_f64(F)) if F is not None else None, float(tau), _p(eps), _p(u))
        if rc != 0:
            raise FloatingPointError("Landau solve failed")
        return f, float(eps[0]), u

    @staticmethod
    def stream(f):
        f = _f64(f)
        _, ny, nx = f.shape
        out = np.empty_like(f)
        _load().ring_stream(_p(f), _p(out), nx, ny)
        return out

    @staticmethod
    def init(nx, ny, eps=None, vx=None, vy=None):
        f = np.zeros((RING, ny, nx))
        conv = lambda a: None if a is None else _f64(a).reshape(ny, nx)
        rc = _load().ring_init(_p(f), nx, ny, _p(conv(eps)), _p(conv(vx)), _p(conv(vy)))
        if rc != 0:
            raise ValueError("invalid initial fields")
        return f

    @staticmethod
    def run(f, tau, nsteps, step0=0, kmin=0, kmax=0, amp=0.0, seed=0, redraw=100):
        assert f.dtype == np.float64 and f.flags.c_contiguous
        _, ny, nx = f.shape
        tmp = np.empty_like(f)
        Fx, Fy = np.zeros((ny, nx)), np.zeros((ny, nx))
        bad = _load().ring_run(_p(f), _p(tmp), _p(Fx), _p(Fy), nx, ny, float(tau), int(step0), int(nsteps), int(kmin),
                               int(kmax), float(amp), int(seed), int(redraw))
        if bad:
            raise FloatingPointError("Landau solve failed %d times" % bad)
        return f

    @staticmethod
    def fields(f):
        f = _f64(f)
        _, ny, nx = f.shape
        tmp = np.empty_like(f)
        eps, vx, vy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
        _load().ring_fields(_p(f), _p(tmp), nx, ny, _p(eps), _p(vx), _p(vy))
        return eps, vx, vy

    @staticmethod
    def totals(f):
        f = _f64(f)
        _, ny, nx = f.shape
        out = np.zeros(3)
        _load().ring_totals(_p(f), nx, ny, _p(out))
        return out


# --------------------------------------------------------------------------- 3D lattice
class lattice3d:
    """The three-dimensional periodic lattice of the paper's node (see
    lattice3d_oracle.c).  Populations are (26, nz, ny, nx) FP64 arrays;
    fields are (nz, ny, nx)."""

    @staticmethod
    def stream(f):
        f = _f64(f)
        _, nz, ny, nx = f.shape
        out = np.empty_like(f)
        _load().oracle3d_stream(_p(f), _p(out), nx, ny, nz)
        return out

    @staticmethod
    def init(nx, ny, nz, eps=None, vx=None, vy=None, vz=None):
        f = np.zeros((NDIR, nz, ny, nx))
        conv = lambda a: None if a is None else _f64(a).reshape(nz, ny, nx)
        rc = _load().oracle3d_init(_p(f), nx, ny, nz, _p(conv(eps)), _p(conv(vx)), _p(conv(vy)), _p(conv(vz)))
        if rc != 0:
            raise ValueError("invalid initial fields")
        return f

    @staticmethod
    def forcing_modes(kmin, kmax):
        lib = _load()
        n = lib.oracle3d_forcing_modes(kmin, kmax, None, None, None, 0)
        kx, ky, kz = (np.zeros(max(n, 1), dtype=np.int32) for _ in range(3))
        lib.oracle3d_forcing_modes(kmin, kmax, kx.ctypes.data_as(_ip), ky.ctypes.data_as(_ip), kz.ctypes.data_as(_ip), n)
        return kx[:n], ky[:n], kz[:n]

    @staticmethod
    def forcing_draw(kmin, kmax, amp, seed, epoch):
        n = len(lattice3d.forcing_modes(kmin, kmax)[0])
        mag, ph, d = np.zeros(n), np.zeros(n), np.zeros((n, 3))
        _load().oracle3d_forcing_draw(kmin, kmax, float(amp), int(seed) & 0xFFFFFFFFFFFFFFFF, int(epoch), _p(mag),
                                      _p(ph), _p(d))
        return mag, ph, d

    @staticmethod
    def force_field(nx, ny, nz, kmin, kmax, amp, seed, epoch):
        F = [np.zeros((nz, ny, nx)) for _ in range(3)]
        _load().oracle3d_force_field(nx, ny, nz, kmin, kmax, float(amp), int(seed) & 0xFFFFFFFFFFFFFFFF, int(epoch),
                                     *(_p(a) for a in F))
        return tuple(F)

    @staticmethod
    def run(f, tau, nsteps, step0=0, kmin=0, kmax=0, amp=0.0, seed=0, redraw=100):
        assert f.dtype == np.float64 and f.flags.c_contiguous
        _, nz, ny, nx = f.shape
        tmp = np.empty_like(f)
        F = [np.zeros((nz, ny, nx)) for _ in range(3)]
        bad = _load().oracle3d_run(_p(f), _p(tmp), *(_p(a) for a in F), nx, ny, nz, float(tau), int(step0),
                                   int(nsteps), int(kmin), int(kmax), float(amp), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                   int(redraw))
        if bad:
            raise FloatingPointError("Landau solve failed %d times" % bad)
        return f

    @staticmethod
    def fields(f):
        f = _f64(f)
        _, nz, ny, nx = f.shape
        tmp = np.empty_like(f)
        out = [np.empty((nz, ny, nx)) for _ in range(4)]
        _load().oracle3d_fields(_p(f), _p(tmp), nx, ny, nz, *(_p(a) for a in out))
        return tuple(out)

    @staticmethod
    def totals(f):
        f = _f64(f)
        _, nz, ny, nx = f.shape
        out = np.zeros(4)
        _load().oracle3d_totals(_p(f), nx, ny, nz, _p(out))
        return out

    @staticmethod
    def energy_spectrum(vx, vy, vz, nshells: int) -> np.ndarray:
        """E(n) of a 3D velocity field: v_hat = (1/N) sum v exp(-2 pi i k.x/N)
        (numpy FFT as the transform), shell n collects |k| in [n - 1/2,
        n + 1/2), E(n) = 1/2 sum_shell |v_hat|^2 over the three components."""
        comps = [np.asarray(a, dtype=np.float64) for a in (vx, vy, vz)]
        nz, ny, nx = comps[0].shape
        p = sum(np.abs(np.fft.fftn(a) / (nx * ny * nz)) ** 2 for a in comps) * 0.5
        kx = np.fft.fftfreq(nx, d=1.0 / nx)
        ky = np.fft.fftfreq(ny, d=1.0 / ny)
        kz = np.fft.fftfreq(nz, d=1.0 / nz)
        K = np.sqrt(kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + kz[:, None, None] ** 2)
        shell = np.floor(K + 0.5).astype(np.int64)
        return np.array([p[shell == n].sum() for n in range(nshells)])

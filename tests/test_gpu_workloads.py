"""The benchmark workloads at their full sizes, through the C ABI, in the
launch configuration the benchmark uses (autotuned).

* 128^2 shear wave, FP64 form, tau = 0.8: parity with the oracle over 100
  steps; decay over 2000 steps against the linear-mode analysis; totals
  conserved; rest state fixed.
* 1024^2 stirred run (tau = 0.52, shell 4..6, amplitude 1e-5): 100 steps
  against the oracle at full size, FP32 and FP64 forms, each kernel
  variant, and the bench's variants at that size (the paper's time step
  cfl 0.625 with eta/s; the 2D ring).
* 4096^2 (16-bit forms) and 8192^2 (FP32): too large for the oracle, so
  (a) a lattice started from a field periodic with period 64 must stay an
  exact tiling of the oracle's 64^2 run (a property that holds at any size),
  and (b) the force field at sampled nodes must equal the oracle's force at
  those nodes.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from linear_modes import _predict_velocity_mode

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2101_06187_gb300 as rl  # noqa: E402

oracle.set_threads(os.cpu_count() or 4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _errs(ref, got):
    e_r, vx_r, vy_r = ref
    e_g, vx_g, vy_g = got[:3]
    err_e = np.max(np.abs(e_g - e_r)) / np.max(np.abs(e_r))
    vn = max(np.max(np.abs(vx_r)), np.max(np.abs(vy_r)))
    err_v = max(np.max(np.abs(vx_g - vx_r)), np.max(np.abs(vy_g - vy_r))) / vn
    return err_e, err_v


def _forcing(w):
    return dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw)


# --------------------------------------------------------------------------- 128^2 shear wave
def test_shear_wave_128_parity_decay_conservation():
    w = workloads.SHEAR_128
    n = w.nx
    eps, vx, vy = workloads.shear_wave(n, n, w.extra["u0"])
    lat = rl.Lattice(n, n, w.tau, dtype="f64")
    lat.autotune(5)
    lat.init_fields(eps, vx, vy)
    t0 = lat.moments()[3]
    lat.step(100)
    got = lat.moments()
    f = oracle.init(n, n, eps, vx, vy)
    oracle.run(f, w.tau, 100)
    err_e, err_v = _errs(oracle.fields(f), got)
    assert err_e < 1e-12 and err_v < 1e-12, (err_e, err_v)
    lat.step(w.steps - 100)
    e, vxg, vyg, t1 = lat.moments()
    # the whole 2000-step run against the oracle (round-off accumulates over 20x the steps)
    oracle.run(f, w.tau, w.steps - 100, step0=100)
    err_e, err_v = _errs(oracle.fields(f), (e, vxg, vyg))
    assert err_e < 1e-11 and err_v < 1e-11, (err_e, err_v)
    # decay of the shear mode against the linearised step (independent of both codes)
    v, wt = oracle.stencil()
    c0 = np.fft.fft(vx[:, 0])[1] / n
    _, pred, _ = _predict_velocity_mode(v, wt, (0.0, 2 * np.pi / n), w.tau, w.steps, c0, 0.0)
    sim = np.fft.fft(vxg[:, 0])[1] / n
    assert abs(sim - pred) < 1e-4 * abs(pred), (sim, pred)
    # v_y stays at the second-order level (the shear wave drives y-motion only through O(u0^2) terms)
    assert np.max(np.abs(vyg)) < w.extra["u0"] ** 2
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]
    np.testing.assert_allclose(t1[1:], t0[1:], rtol=0, atol=1e-13 * t0[0])
    lat.close()


# --------------------------------------------------------------------------- 1024^2 stirred
@pytest.fixture(scope="module")
def stirred_1024_oracle():
    w = workloads.STIRRED_1024
    f = oracle.init(w.nx, w.ny)
    oracle.run(f, w.tau, 100, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
    return oracle.fields(f)


@pytest.mark.parametrize("dtype,tol,kernel", [("f32", 1e-5, "auto"), ("f64", 1e-12, "auto"), ("f32", 1e-5, "tma"),
                                             ("f32", 1e-5, "packed"), ("f32", 1e-5, "twopass"),
                                             ("f32", 1e-5, "fused2")])
def test_stirred_1024_full_size_matches_oracle(stirred_1024_oracle, dtype, tol, kernel):
    w = workloads.STIRRED_1024
    lat = rl.Lattice(w.nx, w.ny, w.tau, dtype=dtype, forcing=_forcing(w), kernel=kernel)
    if kernel == "auto":
        lat.autotune(5)
    lat.init_fields()
    lat.step(100)
    err_e, err_v = _errs(stirred_1024_oracle, lat.moments())
    assert err_e < tol and err_v < tol, (err_e, err_v)
    lat.close()


def test_paper_time_step_full_size_matches_oracle():
    """The paper's own time step on the 1024^2 workload (cfl 0.625, eta/s =
    0.01, dt = 0.05: the bench's variant), autotuned as the bench runs it
    (two steps per launch with runtime weights), 100 steps against the
    oracle at full size."""
    w = workloads.STIRRED_1024
    kw = dict(cfl=0.625, eta_s=0.01, dt=0.05)
    lat = rl.Lattice(w.nx, w.ny, w.tau, dtype="f32", forcing=_forcing(w), **kw)
    lat.autotune(5)
    lat.init_fields()
    lat.step(100)
    got = lat.moments()
    lat.close()
    f = oracle.init(w.nx, w.ny)
    oracle.run(f, w.tau, 100, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw, **kw)
    err_e, err_v = _errs(oracle.fields(f, kw["cfl"]), got)
    assert err_e < 1e-5 and err_v < 1e-5, (err_e, err_v)


def test_ring_full_size_matches_oracle():
    """The 2D ring at the bench's variant size (1024^2, stirred), autotuned
    as the bench runs it (two steps per launch), 100 steps against the ring
    oracle at full size."""
    w = workloads.STIRRED_1024
    lat = rl.Lattice(w.nx, w.ny, w.tau, dtype="f32", forcing=_forcing(w), stencil="ring8")
    lat.autotune(5)
    lat.init_fields()
    lat.step(100)
    got = lat.moments()
    lat.close()
    f = oracle.ring.init(w.nx, w.ny)
    oracle.ring.run(f, w.tau, 100, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
    err_e, err_v = _errs(oracle.ring.fields(f), got)
    assert err_e < 1e-5 and err_v < 1e-5, (err_e, err_v)


# --------------------------------------------------------------------------- 4096^2 / 8192^2
TILED_TOL = {"f32": 1e-5, "bf16": 5e-3, "f16": 5e-4}


@pytest.fixture(scope="module")
def tiled_reference():
    period, tau, nsteps = 64, 0.51, 20
    e, a, b = workloads.random_smooth(period, period, seed=77, deps=0.02, vmax=0.02)
    f = oracle.init(period, period, e, a, b)
    oracle.run(f, tau, nsteps)
    return period, tau, nsteps, oracle.fields(f)


@pytest.mark.parametrize("n,dtype,kernel", [(4096, "bf16", "auto"), (4096, "f16", "auto"), (4096, "f32", "auto"),
                                           (8192, "f32", "auto"), (8192, "f32", "tma"), (8192, "f32", "fused2"),
                                           (4096, "bf16", "fused2")])
def test_full_size_lattice_stays_an_exact_tiling(tiled_reference, n, dtype, kernel):
    period, tau, nsteps, ref = tiled_reference
    e, a, b = workloads.random_tiled(n, n, period, seed=77, deps=0.02, vmax=0.02)
    # nearest rounding: every period of the tiling then evolves identically (stochastic rounding draws
    # per node)
    lat = rl.Lattice(n, n, tau, dtype=dtype, kernel=kernel, rounding="nearest")
    if kernel == "auto":
        lat.autotune(3)
    lat.init_fields(e, a, b)
    lat.step(nsteps)
    e_g, vx_g, vy_g, _ = lat.moments()
    lat.close()
    rep = n // period
    tiled = tuple(np.tile(r, (rep, rep)) for r in ref)
    err_e, err_v = _errs(tiled, (e_g, vx_g, vy_g))
    assert err_e < TILED_TOL[dtype] and err_v < TILED_TOL[dtype], (err_e, err_v)


@pytest.mark.parametrize("w,dtype", [(workloads.PRECISION_4096, "bf16"), (workloads.LARGE_8192, "f32")])
def test_full_size_force_at_sampled_nodes(w, dtype):
    lat = rl.Lattice(w.nx, w.ny, w.tau, dtype=dtype, forcing=_forcing(w))
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.integers(0, w.nx, 200), [0, w.nx - 1]])
    ys = np.concatenate([rng.integers(0, w.ny, 200), [w.ny - 1, 0]])
    for epoch in (0, 2):
        lat.init_fields()
        if epoch:
            lat.step(epoch * w.redraw)
        Fx, Fy = lat.force()
        ox, oy = oracle.force_points(w.nx, w.ny, w.kmin, w.kmax, w.amp, w.seed, epoch, xs, ys)
        scale = max(np.max(np.abs(ox)), np.max(np.abs(oy)))
        assert np.max(np.abs(Fx[ys, xs] - ox)) < 2e-6 * scale
        assert np.max(np.abs(Fy[ys, xs] - oy)) < 2e-6 * scale
    lat.close()


def test_full_size_8192_spectrum_of_two_modes():
    """E(k) at the 8192^2 workload's size (the radix-2 transform at its
    largest side): fields set on the device to a shear mode v_x = a sin(2 pi
    y/N) and a mode v_y = b cos(2 pi 37 x/N) put their energies a^2/4 and
    b^2/4 in shells 1 and 37 and nothing elsewhere (Parseval, a single mode
    lands in its shell), read back through the FP32 populations.  The
    diagnostic reports the state the next collision sees (after one pull
    stream), whose bilinear interpolation damps a mode by O((k dx)^2):
    2e-7 at k = 1, 8e-4 at k = 37 -- hence the looser bound there."""
    w = workloads.LARGE_8192
    n, k1, a, b = w.nx, 37, 1e-3, 2e-3
    lat = rl.Lattice(n, n, w.tau, dtype="f32")
    c = torch.arange(n, dtype=torch.float64, device="cuda")
    vx = (a * torch.sin(2 * np.pi * c / n)).unsqueeze(1).expand(n, n).contiguous()
    vy = (b * torch.cos(2 * np.pi * k1 * c / n)).unsqueeze(0).expand(n, n).contiguous()
    eps = torch.ones((n, n), dtype=torch.float64, device="cuda")
    lat.init_fields_device(eps, vx, vy)
    E = lat.energy_spectrum(64)
    lat.close()
    del eps, vx, vy
    assert abs(E[1] - a * a / 4) < 1e-5 * a * a / 4, E[1]
    assert abs(E[k1] - b * b / 4) < 1e-3 * b * b / 4, E[k1]
    others = np.delete(E, [1, k1])
    assert np.max(others) < 1e-9 * E[k1], np.max(others)


@pytest.mark.parametrize("dtype,kernel", [("f32", "packed"), ("f32", "fused2"), ("f32", "packed4"),
                                          ("bf16", "packed4")])
def test_lattice_beyond_32bit_offsets_stays_an_exact_tiling(tiled_reference, dtype, kernel):
    """12032^2 (145 M nodes, 17 planes = 2.5 G elements: the 64-bit offset
    path of the packed, four-node and two-step kernels), started on the
    device from the tiled fields; sampled rows of the moments against the
    oracle's 64^2 tile (16-bit stores rounded to nearest, so every period of
    the tiling evolves identically)."""
    period, tau, nsteps, ref = tiled_reference
    n = 12032
    rep = n // period
    e, a, b = workloads.random_smooth(period, period, seed=77, deps=0.02, vmax=0.02)
    dev = lambda g: torch.as_tensor(g, dtype=torch.float64, device="cuda").repeat(rep, rep).contiguous()
    lat = rl.Lattice(n, n, tau, dtype=dtype, kernel=kernel, rounding="nearest")
    fe, fa, fb = dev(e), dev(a), dev(b)
    lat.init_fields_device(fe, fa, fb)
    lat.step(nsteps)
    out = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(3)]
    lat.moments_device(*out)
    lat.synchronize()
    rows = [0, 1, 4095, 4096, 9000, n - 1]
    got = [o[rows].cpu().numpy() for o in out]
    lat.close()
    del fe, fa, fb, out
    want = [np.tile(r, (1, rep))[[y % period for y in rows]] for r in ref]
    err_e, err_v = _errs(want, got)
    assert err_e < TILED_TOL[dtype] and err_v < TILED_TOL[dtype], (err_e, err_v)

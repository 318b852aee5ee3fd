"""Pins of the oracle's lattice-level functions.

Streaming is checked against a library interpolator (scipy's periodic linear
interpolation), the whole step against an independent linear-mode analysis
(the linearised update built from the paper's equations and
eigen-decomposed with numpy), and the forcing field and spectrum against
FFT identities.
"""
import numpy as np
import pytest

import oracle
import workloads
from linear_modes import _linear_step, _predict_velocity_mode

scipy_ndimage = pytest.importorskip("scipy.ndimage")


# --------------------------------------------------------------------------- streaming
def test_stream_matches_library_linear_interpolation():
    rng = np.random.default_rng(1)
    nx, ny = 7, 5
    f = rng.uniform(0.5, 1.5, size=(26, ny, nx))
    out = oracle.stream(f)
    v, _ = oracle.stencil()
    yy, xx = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    for i in range(26):
        ref = scipy_ndimage.map_coordinates(f[i], [yy - v[i, 1], xx - v[i, 0]], order=1, mode="grid-wrap")
        np.testing.assert_allclose(out[i], ref, rtol=0, atol=1e-14)


def test_stream_axis_directions_are_exact_shifts_and_sums_preserved():
    rng = np.random.default_rng(2)
    f = rng.uniform(size=(26, 6, 9))
    out = oracle.stream(f)
    v, _ = oracle.stencil()
    for i in range(26):
        if abs(v[i, 0]) == 1.0 or abs(v[i, 1]) == 1.0:
            np.testing.assert_array_equal(out[i], np.roll(f[i], shift=(int(v[i, 1]), int(v[i, 0])), axis=(0, 1)))
        if v[i, 0] == 0.0 and v[i, 1] == 0.0:
            np.testing.assert_array_equal(out[i], f[i])
        assert abs(out[i].sum() - f[i].sum()) < 1e-13


# --------------------------------------------------------------------------- invariants of the full step
@pytest.mark.parametrize("vel", [(0.0, 0.0), (0.3, -0.2)])
def test_uniform_state_is_fixed_point(vel):
    nx = ny = 8
    eps = np.full((ny, nx), 1.3)
    f = oracle.init(nx, ny, eps, np.full((ny, nx), vel[0]), np.full((ny, nx), vel[1]))
    f0 = f.copy()
    oracle.run(f, 0.8, 50)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-14)
    e, vx, vy = oracle.fields(f)
    np.testing.assert_allclose(e, 1.3, rtol=1e-14)
    np.testing.assert_allclose(vx, vel[0], rtol=0, atol=1e-14)


def test_unforced_run_conserves_total_energy_momentum():
    nx = ny = 16
    e, a, b = workloads.random_smooth(nx, ny, seed=5, deps=0.1, vmax=0.1)
    f = oracle.init(nx, ny, e, a, b)
    t0 = oracle.totals(f)
    oracle.run(f, 0.6, 200)
    t1 = oracle.totals(f)
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]
    np.testing.assert_allclose(t1[1:], t0[1:], rtol=0, atol=1e-13 * t0[0])


def test_forced_step_injects_FM_and_FE():
    nx = ny = 16
    e, a, b = workloads.random_smooth(nx, ny, seed=6, deps=0.05, vmax=0.05)
    f = oracle.init(nx, ny, e, a, b)
    Fx, Fy = oracle.force_field(nx, ny, 2, 3, 1e-3, seed=99, epoch=0)
    t0 = oracle.totals(f)
    streamed = oracle.stream(f)
    v, _ = oracle.stencil()
    E = streamed.sum(axis=0)
    Mx = np.einsum("i,iyx->yx", v[:, 0], streamed)
    My = np.einsum("i,iyx->yx", v[:, 1], streamed)
    oracle.step(f, 0.7, Fx, Fy)
    t1 = oracle.totals(f)
    tol = 1e-13 * t0[0]  # round-off of the two lattice sums
    assert abs((t1[0] - t0[0]) - np.sum(Fx * Mx + Fy * My)) < tol
    assert abs((t1[1] - t0[1]) - np.sum(Fx * E)) < tol
    assert abs((t1[2] - t0[2]) - np.sum(Fy * E)) < tol


# --------------------------------------------------------------------------- linear-mode analysis
@pytest.mark.parametrize("tau", [0.8, 0.6])
def test_shear_wave_matches_linear_mode_analysis(tau):
    N, nst = 32, 200
    e, a, b = workloads.shear_wave(N, N, 0.01)
    f = oracle.init(N, N, e, a, b)
    oracle.run(f, tau, nst)
    _, vx, _ = oracle.fields(f)
    sim = np.fft.fft(vx[:, 0])[1] / N
    c0 = np.fft.fft(a[:, 0])[1] / N
    v, w = oracle.stencil()
    _, pred, _ = _predict_velocity_mode(v, w, (0.0, 2 * np.pi / N), tau, nst, c0, 0.0)
    assert abs(sim - pred) < 2e-5 * abs(pred)


def test_viscosity_follows_tau_over_five():
    """eta = tau (eps + P)/5: the simulated shear-decay rate changes by
    Delta tau / 5 per unit k^2 between two relaxation times (the absolute
    value carries the interpolation's numerical viscosity)."""
    N = 32
    k2 = (2 * np.pi / N) ** 2
    nu = []
    for tau in (0.8, 0.6):
        e, a, b = workloads.shear_wave(N, N, 0.01)
        f = oracle.init(N, N, e, a, b)
        oracle.run(f, tau, 40)
        amp1 = abs(np.fft.fft(oracle.fields(f)[1][:, 0])[1])
        oracle.run(f, tau, 120, step0=40)
        amp2 = abs(np.fft.fft(oracle.fields(f)[1][:, 0])[1])
        nu.append(-np.log(amp2 / amp1) / 120 / k2)
    assert abs((nu[0] - nu[1]) - 0.2 * 0.2) < 0.005 * 0.04


def test_sound_speed_is_one_over_sqrt3():
    """Phase speed of the acoustic eigenmodes at small k is c_s = 1/sqrt(3)
    (P = eps/3, Sec. 3.1), and the oracle follows that mode."""
    v, w = oracle.stencil()
    N = 256
    k = 2 * np.pi / N
    lam = np.linalg.eigvals(_linear_step(v, w, (k, 0.0), 0.8))
    speeds = sorted(abs(np.angle(l)) / k for l in lam if abs(l) > 0.99 and abs(np.angle(l)) > 1e-8)
    assert abs(speeds[0] - 1 / np.sqrt(3)) < 1e-4
    # acoustic standing wave in the oracle vs the linear prediction
    N, nst, tau = 32, 60, 0.8
    x = np.arange(N)
    eps = np.tile(1.0 + 1e-3 * np.cos(2 * np.pi * x / N), (N, 1))
    f = oracle.init(N, N, eps, np.zeros((N, N)), np.zeros((N, N)))
    oracle.run(f, tau, nst)
    e, vx, _ = oracle.fields(f)
    sim_e = np.fft.fft(e[0, :])[1] / N
    sim_v = np.fft.fft(vx[0, :])[1] / N
    pe, pvx, _ = _predict_velocity_mode(v, w, (2 * np.pi / N, 0.0), tau, nst, 0.0, 0.0, deps=0.5e-3)
    assert abs(sim_e - pe) < 1e-3 * 0.5e-3
    assert abs(sim_v - pvx) < 1e-3 * 0.5e-3


# --------------------------------------------------------------------------- forcing field
def test_forcing_modes_shell_and_half_plane():
    for kmin, kmax, count in ((4, 6, 34), (8, 10, 62), (16, 18, 108)):
        m = oracle.forcing_modes(kmin, kmax)
        assert len(m) == count
        k2 = (m ** 2).sum(axis=1)
        assert np.all((k2 >= kmin ** 2) & (k2 <= kmax ** 2))
        assert np.all((m[:, 1] > 0) | ((m[:, 1] == 0) & (m[:, 0] > 0)))
        assert len({tuple(r) for r in m}) == len(m)


def test_force_field_spectrum_is_the_drawn_modes():
    nx, ny = 48, 40
    kmin, kmax, amp, seed, epoch = 3, 5, 2e-3, 12345, 7
    Fx, Fy = oracle.force_field(nx, ny, kmin, kmax, amp, seed, epoch)
    mag, ph, th = oracle.forcing_draw(kmin, kmax, amp, seed, epoch)
    modes = oracle.forcing_modes(kmin, kmax)
    assert abs(Fx.mean()) < 1e-17 and abs(Fy.mean()) < 1e-17
    hx = np.fft.fft2(Fx) / (nx * ny)
    hy = np.fft.fft2(Fy) / (nx * ny)
    expect_x = np.zeros_like(hx)
    expect_y = np.zeros_like(hy)
    for (kx, ky), r, p, t in zip(modes, mag, ph, th):
        c = r * np.exp(1j * p)
        expect_x[ky % ny, kx % nx] += c * np.cos(t)
        expect_y[ky % ny, kx % nx] += c * np.sin(t)
        expect_x[-ky % ny, -kx % nx] += np.conj(c) * np.cos(t)
        expect_y[-ky % ny, -kx % nx] += np.conj(c) * np.sin(t)
    np.testing.assert_allclose(hx, expect_x, rtol=0, atol=1e-16)
    np.testing.assert_allclose(hy, expect_y, rtol=0, atol=1e-16)
    assert np.all((mag >= 0) & (mag < amp))
    assert np.all((ph >= 0) & (ph < 2 * np.pi)) and np.all((th >= 0) & (th < 2 * np.pi))


def test_force_points_equal_the_field():
    nx, ny = 40, 36
    Fx, Fy = oracle.force_field(nx, ny, 2, 5, 1e-3, 321, 4)
    rng = np.random.default_rng(0)
    xs, ys = rng.integers(0, nx, 50), rng.integers(0, ny, 50)
    px, py = oracle.force_points(nx, ny, 2, 5, 1e-3, 321, 4, xs, ys)
    np.testing.assert_array_equal(px, Fx[ys, xs])
    np.testing.assert_array_equal(py, Fy[ys, xs])


def test_force_redraw_changes_with_epoch_and_seed():
    a = oracle.forcing_draw(4, 6, 1.0, 1, 0)
    b = oracle.forcing_draw(4, 6, 1.0, 1, 1)
    c = oracle.forcing_draw(4, 6, 1.0, 2, 0)
    assert not np.allclose(a[0], b[0]) and not np.allclose(a[0], c[0])
    np.testing.assert_array_equal(a[0], oracle.forcing_draw(4, 6, 1.0, 1, 0)[0])


def test_philox_output_statistics():
    """Statistical sanity of the counter-based generator (its bit pattern is
    pinned in tests/test_oracle_philox.py): uniform words, uncorrelated
    counters."""
    words = np.array([oracle.philox4x32_10([e, m, s, 0], [0xDEADBEEF, 0x12345678])
                      for e in range(40) for m in range(50) for s in range(2)], dtype=np.uint64)
    u = words.astype(np.float64) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.005
    hist = np.bincount((words & 0xFF).ravel().astype(np.int64), minlength=256)
    expected = words.size / 256
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 340  # 255 dof, p ~ 0.0003
    # consecutive counters decorrelated
    c = np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]
    assert abs(c) < 0.05
    # a single-bit change of key or counter flips about half the output bits
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for ctr, key in (([1, 2, 3, 5], [5, 6]), ([1, 2, 3, 4], [5, 7])):
        diff = np.bitwise_xor(base, oracle.philox4x32_10(ctr, key))
        flipped = sum(bin(int(d)).count("1") for d in diff)
        assert 40 < flipped < 88


# --------------------------------------------------------------------------- energy spectrum
def test_spectrum_single_mode_lands_in_its_shell():
    N = 64
    x = np.arange(N)
    a = 0.02
    vx = np.tile(a * np.sin(2 * np.pi * 5 * x / N), (N, 1))
    E = oracle.energy_spectrum(vx, np.zeros((N, N)), 20)
    assert abs(E[5] - a * a / 4) < 1e-18
    assert np.all(np.abs(np.delete(E, 5)) < 1e-20)


def test_spectrum_parseval():
    N = 32
    e, a, b = workloads.random_smooth(N, N, seed=9, vmax=0.1)
    E = oracle.energy_spectrum(a, b, 30)
    assert abs(E.sum() - 0.5 * np.mean(a * a + b * b)) < 1e-15


def test_filtered_velocity_keeps_only_modes_below_kf():
    N = 64
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    low = 0.01 * np.sin(2 * np.pi * 3 * x / N)
    high = 0.02 * np.cos(2 * np.pi * (6 * x + 4 * y) / N)  # |k| = 7.2
    assert abs(oracle.filtered_velocity_rms(low, np.zeros((N, N)), 6) - 0.01 / np.sqrt(2)) < 1e-15
    assert oracle.filtered_velocity_rms(high, np.zeros((N, N)), 6) < 1e-15
    both = oracle.filtered_velocity_rms(low + high, high, 6)
    assert abs(both - 0.01 / np.sqrt(2)) < 1e-15

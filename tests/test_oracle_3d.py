"""Pins of the three-dimensional lattice oracle (lattice3d_oracle.c): the
paper's node on an nx x ny x nz periodic lattice, trilinear streaming, and
the stirring force carried to a 3D shell.  Each pin comes from outside the
oracle: scipy's interpolation, the (already pinned) two-dimensional oracle
through exact symmetries, the linearised step, conservation laws and the
Fourier transform of the force."""
import numpy as np
import pytest

import oracle
import workloads
from linear_modes import linear_step3, _symbols3

L = oracle.lattice3d
scipy_ndimage = pytest.importorskip("scipy.ndimage")


def test_stream_matches_library_trilinear_interpolation():
    rng = np.random.default_rng(1)
    nz, ny, nx = 5, 6, 7
    f = rng.standard_normal((26, nz, ny, nx))
    out = L.stream(f)
    v, _ = oracle.stencil()
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for i in range(26):
        ref = scipy_ndimage.map_coordinates(f[i], [zz - v[i, 2], yy - v[i, 1], xx - v[i, 0]], order=1,
                                            mode="grid-wrap")
        np.testing.assert_allclose(out[i], ref, rtol=0, atol=1e-13)


def test_z_uniform_run_is_the_two_dimensional_run():
    """Fields independent of z stay so, and every layer follows the one-layer
    lattice of the paper (the 2D oracle), forced by a z-independent force."""
    nx, ny, nz = 12, 10, 3
    e, a, b = workloads.random_smooth(nx, ny, seed=4, deps=0.05, vmax=0.05)
    tile = lambda g: np.repeat(g[None], nz, axis=0)
    f3 = L.init(nx, ny, nz, tile(e), tile(a), tile(b), None)
    L.run(f3, 0.7, 25)
    f2 = oracle.init(nx, ny, e, a, b)
    oracle.run(f2, 0.7, 25)
    e3, vx3, vy3, vz3 = L.fields(f3)
    e2, vx2, vy2 = oracle.fields(f2)
    for z in range(nz):
        np.testing.assert_allclose(e3[z], e2, rtol=0, atol=1e-13)
        np.testing.assert_allclose(vx3[z], vx2, rtol=0, atol=1e-14)
        np.testing.assert_allclose(vy3[z], vy2, rtol=0, atol=1e-14)
    assert np.max(np.abs(vz3)) < 1e-15


def test_axis_exchange_symmetry():
    """The 26 directions are invariant under exchanging x and z, so a wave
    along z with velocity along z is the 2D lattice's wave along x with
    velocity along x (pins the z-streaming and the z-components of moments,
    frame and equilibrium against the pinned 2D oracle)."""
    n, m = 16, 4
    x = np.arange(n)
    eps1 = 1.0 + 0.03 * np.cos(2 * np.pi * x / n)
    v1 = 0.04 * np.sin(2 * np.pi * x / n + 0.3)
    # 2D lattice (ny = m, nx = n): fields vary along x
    e2d = np.tile(eps1, (m, 1))
    vx2d = np.tile(v1, (m, 1))
    f2 = oracle.init(n, m, e2d, vx2d, np.zeros((m, n)))
    oracle.run(f2, 0.65, 30)
    E2, VX2, VY2 = oracle.fields(f2)
    # 3D lattice (nz = n, ny = nx = m): fields vary along z, velocity along z
    e3d = np.broadcast_to(eps1[:, None, None], (n, m, m)).copy()
    vz3d = np.broadcast_to(v1[:, None, None], (n, m, m)).copy()
    f3 = L.init(m, m, n, e3d, None, None, vz3d)
    L.run(f3, 0.65, 30)
    E3, VX3, VY3, VZ3 = L.fields(f3)
    np.testing.assert_allclose(E3[:, 0, 0], E2[0, :], rtol=0, atol=1e-13)
    np.testing.assert_allclose(VZ3[:, 0, 0], VX2[0, :], rtol=0, atol=1e-14)
    assert np.max(np.abs(VX3)) < 1e-15 and np.max(np.abs(VY3)) < 1e-15


def _predict_mode(v, w, k, tau, nsteps, df):
    fn = np.linalg.matrix_power(linear_step3(v, w, k, tau), nsteps) @ df
    return _symbols3(v, k) * fn


def test_diagonal_shear_wave_follows_linear_analysis():
    """A shear wave with k along (0, 1, 1) and velocity along x: a fully 3D
    stream symbol; amplitude after 60 steps vs the linearised step."""
    n, tau, u0, nst = 16, 0.8, 1e-3, 60
    z, y = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ph = 2 * np.pi * (y + z) / n
    vx = np.broadcast_to((u0 * np.sin(ph))[:, :, None], (n, n, 4)).copy()
    f = L.init(4, n, n, None, vx, None, None)
    L.run(f, tau, nst)
    _, VX, _, _ = L.fields(f)
    sim = np.fft.fftn(VX[:, :, 0])[1, 1] / (n * n)
    v, w = oracle.stencil()
    k = (0.0, 2 * np.pi / n, 2 * np.pi / n)
    c0 = np.fft.fftn(vx[:, :, 0])[1, 1] / (n * n)
    df = w * 3.0 * (4.0 / 3.0) * v[:, 0] * c0
    post = _predict_mode(v, w, k, tau, nst, df)
    pred = 0.75 * (v[:, 0] @ post)
    assert abs(sim - pred) < 2e-3 * abs(pred), (sim, pred)


def test_sound_speed_is_isotropic():
    """c_s = 1/sqrt(3) along an axis, a face diagonal and the body diagonal
    (linearised 3D step, small k)."""
    v, w = oracle.stencil()
    for d in ((1, 0, 0), (1, 1, 0), (1, 1, 1)):
        d = np.asarray(d, float) / np.linalg.norm(d)
        kk = 2 * np.pi / 512
        lam = np.linalg.eigvals(linear_step3(v, w, kk * d, 0.8))
        speeds = sorted(abs(np.angle(l)) / kk for l in lam if abs(l) > 0.99 and abs(np.angle(l)) > 1e-9)
        assert abs(speeds[0] - 1 / np.sqrt(3)) < 1e-3, (d, speeds[:3])


def test_unforced_totals_conserved_and_forced_injection():
    n = 6
    rng = np.random.default_rng(9)
    e = 1 + 0.05 * rng.standard_normal((n, n, n)) ** 2
    vs = [0.03 * np.sin(2 * np.pi * (np.arange(n)[:, None, None] + k) / n) * np.ones((n, n, n)) for k in range(3)]
    f = L.init(n, n, n, e, *vs)
    t0 = L.totals(f)
    L.run(f, 0.7, 50)
    np.testing.assert_allclose(L.totals(f), t0, rtol=0, atol=1e-13 * t0[0])
    # one forced step injects sum_x (F.M, F E) of the post-stream state
    kw = dict(kmin=1, kmax=2, amp=1e-3, seed=11, redraw=100)
    g = f.copy()
    s = L.stream(g)
    Fx, Fy, Fz = L.force_field(n, n, n, 1, 2, 1e-3, 11, 0)
    v, _ = oracle.stencil()
    E = s.sum(axis=0)
    M = np.einsum("izyx,ia->azyx", s, v)
    want = np.array([(Fx * M[0] + Fy * M[1] + Fz * M[2]).sum(), (Fx * E).sum(), (Fy * E).sum(), (Fz * E).sum()])
    before = L.totals(g)
    L.run(g, 0.7, 1, **kw)
    np.testing.assert_allclose(L.totals(g) - before, want, rtol=1e-9, atol=1e-14 * before[0])


def test_force_field_holds_the_drawn_modes():
    nx, ny, nz, kmin, kmax, amp, seed = 12, 10, 8, 2, 3, 1e-3, 77
    Fx, Fy, Fz = L.force_field(nx, ny, nz, kmin, kmax, amp, seed, 5)
    kx, ky, kz = L.forcing_modes(kmin, kmax)
    mag, ph, d = L.forcing_draw(kmin, kmax, amp, seed, 5)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=1e-14)
    for comp, F in enumerate((Fx, Fy, Fz)):
        assert abs(F.mean()) < 1e-15
        Fh = np.fft.fftn(F) / F.size
        want = np.zeros_like(Fh)
        for m in range(len(kx)):
            c = mag[m] * d[m, comp] * np.exp(1j * ph[m])
            want[kz[m] % nz, ky[m] % ny, kx[m] % nx] += c
            want[-kz[m] % nz, -ky[m] % ny, -kx[m] % nx] += np.conj(c)
        np.testing.assert_allclose(Fh, want, rtol=0, atol=1e-15)
    # the kz = 0 modes come first, in the 2D order, with the 2D magnitudes, phases and azimuths
    m2 = oracle.forcing_modes(kmin, kmax)
    mag2, ph2, th2 = oracle.forcing_draw(kmin, kmax, amp, seed, 5)
    k2 = len(m2)
    np.testing.assert_array_equal(np.stack([kx[:k2], ky[:k2]], axis=1), m2)
    assert np.all(kz[:k2] == 0) and np.all(kz[k2:] > 0)
    np.testing.assert_allclose(mag[:k2], mag2, rtol=0, atol=0)
    np.testing.assert_allclose(ph[:k2], ph2, rtol=0, atol=0)
    np.testing.assert_allclose(np.arctan2(d[:k2, 1], d[:k2, 0]) % (2 * np.pi), th2 % (2 * np.pi), rtol=0,
                               atol=1e-12)


def test_spectrum_single_mode_and_parseval():
    n = 8
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vx = 0.01 * np.cos(2 * np.pi * (2 * x + y + 2 * z) / n)  # |k| = 3
    E = L.energy_spectrum(vx, np.zeros_like(vx), np.zeros_like(vx), 8)
    assert abs(E[3] - 0.5 * 0.01 ** 2 / 2) < 1e-18 and abs(E.sum() - E[3]) < 1e-18
    rng = np.random.default_rng(3)
    vs = [rng.standard_normal((n, n, n)) for _ in range(3)]
    E = L.energy_spectrum(*vs, 12)
    assert abs(E.sum() - 0.5 * sum((a ** 2).mean() for a in vs)) < 1e-12


def test_body_diagonal_density_wave_follows_linear_analysis():
    """A density wave with k along (1, 1, 1) in the oracle against the
    linearised 3D step (its second-order remainder is far below 1e-5 of the
    amplitude at A = 1e-4)."""
    n, tau, A = 32, 0.8, 1e-4
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    f = L.init(n, n, n, 1.0 + A * np.cos(2 * np.pi * (x + y + z) / n))
    v, w = oracle.stencil()
    k = np.full(3, 2 * np.pi / n)
    Lk = linear_step3(v, w, k, tau)
    S = _symbols3(v, k)
    fn = w * (A / 2)
    done = 0
    for nst in (10, 25):
        L.run(f, tau, nst - done, step0=done)
        fn = np.linalg.matrix_power(Lk, nst - done) @ fn
        done = nst
        e = L.fields(f)[0]
        sim = np.fft.fftn(e)[1, 1, 1] / e.size
        assert abs(sim - (S * fn).sum()) < 1e-5 * (A / 2)

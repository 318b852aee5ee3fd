"""Pins of the oracle's CFL number and eta/s relaxation (the paper's own
parameters: lattice spacing Delta x with Delta t = 0.05, eta/s = 0.01)."""
import os

import numpy as np
import pytest

import oracle
import workloads
from linear_modes import _linear_step, _predict_velocity_mode

scipy_ndimage = pytest.importorskip("scipy.ndimage")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    vals = {}
    for line in open(os.path.join(GOLDEN, "sec5_relaxation_time.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, val = line.split()[:2]
        vals[name] = float(eval(val.replace("^", "**"), {"pi": np.pi}))
    return vals


@pytest.mark.parametrize("cfl", [0.5, 0.15625, 1.0, 1.25, 1.75])
def test_stream_at_cfl_matches_library_interpolation(cfl):
    rng = np.random.default_rng(3)
    nx, ny = 9, 7
    f = rng.uniform(0.5, 1.5, size=(26, ny, nx))
    out = oracle.stream(f, cfl)
    v, _ = oracle.stencil()
    yy, xx = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    for i in range(26):
        ref = scipy_ndimage.map_coordinates(f[i], [yy - cfl * v[i, 1], xx - cfl * v[i, 0]], order=1,
                                            mode="grid-wrap")
        np.testing.assert_allclose(out[i], ref, rtol=0, atol=1e-14)


def test_relaxation_time_from_eta_over_s_golden():
    g = _golden()
    assert abs(oracle.tau_of(g["eps_T1"], 0.8, g["eta_over_s"], g["dt"]) - g["tau_steps"]) < 1e-15
    # eps = 16 * 3/pi^2 -> T = 2 -> tau halves
    assert abs(oracle.tau_of(16 * g["eps_T1"], 0.8, g["eta_over_s"], g["dt"]) - 0.5 * g["tau_steps"]) < 1e-15
    assert oracle.tau_of(1.0, 0.8, 0.0, 0.05) == 0.8   # eta/s off: the constant tau


def test_eta_over_s_collision_relaxes_at_the_local_rate():
    """At rest a non-conserved perturbation relaxes by (1 - 1/tau(eps))."""
    g = _golden()
    v, w = oracle.stencil()
    rng = np.random.default_rng(5)
    A = np.vstack([np.ones(26), v.T])
    for eps in (g["eps_T1"], 0.7, 2.0):
        d = rng.normal(size=26) * w
        d -= A.T @ np.linalg.lstsq(A.T, d, rcond=None)[0]
        fe = oracle.feq(eps, [1, 0, 0, 0])
        f = fe + 1e-4 * d
        f2, e2, _ = oracle.collide(f, None, 0.8, g["eta_over_s"], g["dt"])
        tau = 5 * g["eta_over_s"] / (np.pi ** 2 * eps / 3) ** 0.25 / g["dt"]
        np.testing.assert_allclose(f2 - fe, (1 - 1 / tau) * (f - fe), rtol=0, atol=1e-15 * np.max(fe))


@pytest.mark.parametrize("cfl", [0.5, 0.25, 1.25])
def test_shear_wave_at_cfl_matches_linear_mode_analysis(cfl):
    N, nst, tau = 32, 200, 0.8
    e, a, b = workloads.shear_wave(N, N, 0.01)
    f = oracle.init(N, N, e, a, b)
    oracle.run(f, tau, nst, cfl=cfl)
    _, vx, _ = oracle.fields(f, cfl)
    sim = np.fft.fft(vx[:, 0])[1] / N
    c0 = np.fft.fft(a[:, 0])[1] / N
    v, w = oracle.stencil()
    _, pred, _ = _predict_velocity_mode(v, w, (0.0, 2 * np.pi / N), tau, nst, c0, 0.0, cfl=cfl)
    assert abs(sim - pred) < 2e-5 * abs(pred)


@pytest.mark.parametrize("cfl", [0.5, 0.25, 1.25])
def test_sound_speed_and_viscosity_scale_with_cfl(cfl):
    """In cells per step the light cone shrinks by the CFL number: c_s =
    cfl/sqrt(3), and the tau-dependent part of the shear viscosity is
    cfl^2 (tau - 1/2)/5 + const, i.e. d nu / d tau = cfl^2/5."""
    v, w = oracle.stencil()
    N = 512
    k = 2 * np.pi / N
    lam = np.linalg.eigvals(_linear_step(v, w, (k, 0.0), 0.8, cfl))
    speeds = sorted(abs(np.angle(l)) / k for l in lam if abs(l) > 0.99 and abs(np.angle(l)) > 1e-9)
    assert abs(speeds[0] - cfl / np.sqrt(3)) < 2e-4 * cfl

    def nu(tau):
        kk = (0.0, 2 * np.pi / 64)
        lam, V = np.linalg.eig(_linear_step(v, w, kk, tau, cfl))
        idx = np.argmax(np.abs(v[:, 0] @ V) * (np.abs(lam) > 0.9))
        return -np.log(abs(lam[idx])) / kk[1] ** 2

    assert abs((nu(0.8) - nu(0.6)) - cfl ** 2 * 0.2 / 5) < 0.01 * cfl ** 2 * 0.2 / 5

"""Pins of the 2D ring oracle (the genuinely two-dimensional massless
variant: 8-direction ring, P = eps/2, sound speed c_s^2 = 1/2)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from linear_modes import _linear_step, _symbols

R = oracle.ring
G3 = np.diag([-1.0, 1.0, 1.0])


def _u(v):
    v = np.asarray(v, dtype=float)
    g = 1 / np.sqrt(1 - v @ v)
    return np.concatenate([[g], g * v])


def _boost(u):
    g, b = u[0], u[1:] / u[0]
    L = np.eye(3)
    L[0, 0] = g
    L[0, 1:] = L[1:, 0] = g * b
    if b @ b > 0:
        L[1:, 1:] += (g - 1) * np.outer(b, b) / (b @ b)
    return L


def _circle_moment(a, b):
    """<cos^a sin^b> over the circle, a and b even: (a-1)!!(b-1)!!/(a+b)!!"""
    def df(n):
        r = 1
        while n > 1:
            r *= n
            n -= 2
        return r
    return Fraction(df(a - 1) * df(b - 1), df(a + b))


@pytest.mark.parametrize("p", [(0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (1, 0), (3, 2), (1, 1), (5, 0)])
def test_ring_quadrature_exact_to_degree_7(p):
    v, w = R.stencil()
    q = np.sum(w * v[:, 0] ** p[0] * v[:, 1] ** p[1])
    exact = float(_circle_moment(*p)) if p[0] % 2 == 0 and p[1] % 2 == 0 else 0.0
    assert abs(q - exact) < 1e-15


def test_ring_feq_reproduces_ideal_tensor_and_is_traceless():
    rng = np.random.default_rng(1)
    for _ in range(100):
        e = rng.uniform(0.5, 2)
        vv = rng.uniform(-0.4, 0.4, 2)
        u = _u(vv)
        L = _boost(u)
        T_exp = L @ np.diag([e, e / 2, e / 2]) @ L.T
        np.testing.assert_allclose(R.ideal_T(e, u), T_exp, rtol=0, atol=1e-13 * e * u[0] ** 2)
        assert abs(np.trace(G3 @ R.ideal_T(e, u))) < 1e-13 * e * u[0] ** 2
        np.testing.assert_allclose(R.moments(R.feq(e, u)), T_exp, rtol=0, atol=2e-14 * e * u[0] ** 2)


def test_ring_landau_matches_library_eigensolver():
    rng = np.random.default_rng(2)
    for _ in range(100):
        e = rng.uniform(0.5, 2)
        f = R.feq(e, _u(rng.uniform(-0.4, 0.4, 2))) * rng.uniform(0.7, 1.3, 8)
        T = R.moments(f)
        e_o, u_o, it = R.landau(T)
        lam, V = np.linalg.eig(T @ G3)
        sel = [k for k in range(3) if abs(lam[k].imag) < 1e-12 and np.real(V[:, k]) @ G3 @ np.real(V[:, k]) < 0]
        k = sel[0]
        uu = np.real(V[:, k])
        uu = uu / np.sqrt(-(uu @ G3 @ uu))
        uu = uu if uu[0] > 0 else -uu
        assert it > 0 and abs(e_o + np.real(lam[k])) < 1e-12 * e_o
        np.testing.assert_allclose(u_o, uu, rtol=0, atol=1e-12 * uu[0])


def test_ring_force_term_carries_the_kinetic_moments():
    """sum G = F.M, sum G v = F E, sum G v v = F M + M F - F.Q."""
    rng = np.random.default_rng(3)
    v, _ = R.stencil()
    for _ in range(40):
        f = R.feq(1.0, _u(rng.uniform(-0.3, 0.3, 2))) * rng.uniform(0.8, 1.2, 8)
        F = rng.normal(size=2) * 1e-3
        G = R.force_term(f, F)
        E, M = f.sum(), f @ v
        Q = np.einsum("i,ia,ib,ic->abc", f, v, v, v)
        assert abs(G.sum() - F @ M) < 1e-18
        np.testing.assert_allclose(G @ v, F * E, rtol=0, atol=1e-18)
        X = np.outer(F, M) + np.outer(M, F) - np.einsum("a,ade->de", F, Q)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", G, v, v), X, rtol=0, atol=1e-18)


def test_ring_collision_conserves_and_fixes_equilibrium():
    rng = np.random.default_rng(4)
    v, _ = R.stencil()
    for _ in range(30):
        fe = R.feq(rng.uniform(0.5, 2), _u(rng.uniform(-0.4, 0.4, 2)))
        f2, _, _ = R.collide(fe, None, 0.7)
        np.testing.assert_allclose(f2, fe, rtol=0, atol=1e-14)
        f = fe * rng.uniform(0.7, 1.3, 8)
        f2, _, _ = R.collide(f, None, 0.6)
        assert abs(f2.sum() - f.sum()) < 1e-14 * f.sum()
        np.testing.assert_allclose(f2 @ v, f @ v, rtol=0, atol=1e-14 * f.sum())


def _ring_linear_step(k, tau):
    v, w = R.stencil()
    return _linear_step(v, w, k, tau, a=2.0), _symbols(v, k)


def test_ring_sound_speed_squared_is_one_half():
    """P = eps/2 gives c_s^2 = dP/deps = 1/2: the acoustic eigenmodes of the
    linearised ring step travel at 1/sqrt(2), and a density wave in the
    oracle follows the linear prediction."""
    N = 512
    k = 2 * np.pi / N
    L, _ = _ring_linear_step((k, 0.0), 0.8)
    lam = np.linalg.eigvals(L)
    speeds = sorted(abs(np.angle(l)) / k for l in lam if abs(l) > 0.99 and abs(np.angle(l)) > 1e-9)
    assert abs(speeds[0] ** 2 - 0.5) < 2e-4
    # acoustic standing wave in the oracle vs the linear prediction
    N, nst, tau = 32, 60, 0.8
    x = np.arange(N)
    eps = np.tile(1.0 + 1e-3 * np.cos(2 * np.pi * x / N), (N, 1))
    f = R.init(N, N, eps, np.zeros((N, N)), np.zeros((N, N)))
    R.run(f, tau, nst)
    e, vx, _ = R.fields(f)
    sim_e = np.fft.fft(e[0, :])[1] / N
    v, w = R.stencil()
    kk = (2 * np.pi / N, 0.0)
    L, S = _ring_linear_step(kk, tau)
    df = w * 0.5e-3
    fn = np.linalg.matrix_power(L, nst) @ df
    pred_e = (S * fn).sum()
    assert abs(sim_e - pred_e) < 1e-3 * 0.5e-3


def test_ring_unforced_run_conserves_totals():
    n = 16
    e, a, b = workloads.random_smooth(n, n, seed=8, deps=0.05, vmax=0.05)
    f = R.init(n, n, e, a, b)
    t0 = R.totals(f)
    R.run(f, 0.6, 100)
    np.testing.assert_allclose(R.totals(f), t0, rtol=0, atol=1e-13 * t0[0])

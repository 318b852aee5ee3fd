"""Linear-mode analysis of the RLBM step about rest (eps = 1, u = 0), built
from the paper's equations independently of both the oracle and the CUDA
path: pull-streaming with bilinear interpolation (Sec. 3.2) as a per-k
Fourier symbol, BGK relaxation towards the linearised truncated equilibrium
(Eqs. rel_pdf_exp, rel_pdf_exp_coef), eigen-decomposed with numpy.  Used to
pin shear decay, sound speed and the viscosity-tau relation."""
import numpy as np


def _symbols(v, k, cfl=1.0):
    """Fourier symbol of pull-streaming with bilinear interpolation from
    x - cfl v_i, per direction."""
    S = np.zeros(len(v), dtype=complex)
    for i in range(len(v)):
        sx, sy = -cfl * v[i, 0], -cfl * v[i, 1]
        ox, oy = np.floor(sx), np.floor(sy)
        tx, ty = sx - ox, sy - oy
        e = lambda dx, dy: np.exp(1j * (k[0] * dx + k[1] * dy))
        S[i] = ((1 - tx) * (1 - ty) * e(ox, oy) + tx * (1 - ty) * e(ox + 1, oy) + (1 - tx) * ty * e(ox, oy + 1)
                + tx * ty * e(ox + 1, oy + 1))
    return S


def _symbols3(v, k):
    """Fourier symbol of pull-streaming with trilinear interpolation from
    x - v_i on a 3D lattice, per direction (k a 3-vector)."""
    S = np.zeros(len(v), dtype=complex)
    for i in range(len(v)):
        s = -np.asarray(v[i], dtype=float)
        o = np.floor(s)
        t = s - o
        acc = 0.0
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    wgt = (t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2])
                    acc = acc + wgt * np.exp(1j * (k[0] * (o[0] + dx) + k[1] * (o[1] + dy) + k[2] * (o[2] + dz)))
        S[i] = acc
    return S


def linear_step3(v, w, k, tau):
    """The 3D linearised step about rest: trilinear streaming, then BGK
    towards delta f_eq,i = w_i (delta E + 3 v_i . delta M)."""
    A = w[:, None] * (1.0 + 3.0 * v @ v.T)
    C = np.eye(len(w)) - (np.eye(len(w)) - A) / tau
    return C @ np.diag(_symbols3(v, k))


def ring_directions():
    """The 2D ring: 8 unit momenta at 45 degree steps, weight 1/8."""
    ang = np.arange(8) * np.pi / 4
    return np.stack([np.cos(ang), np.sin(ang)], axis=1), np.full(8, 1.0 / 8.0)


def _linear_step(v, w, k, tau, cfl=1.0, a=3.0):
    """Linearised step about eps = 1, u = 0: stream, then BGK towards the
    linearised equilibrium delta f_eq,i = w_i (delta E + a v_i . delta M),
    a = 1 / <v_x^2> over the stencil: 3 for the sphere, 2 for the ring."""
    A = w[:, None] * (1.0 + a * v @ v.T)
    C = np.eye(len(w)) - (np.eye(len(w)) - A) / tau
    return C @ np.diag(_symbols(v, k, cfl))


def _predict_velocity_mode(v, w, k, tau, nsteps, dv_x, dv_y, deps=0.0, cfl=1.0):
    """Linear prediction of the Fourier amplitude of (eps, v) seen by the
    next collision after nsteps, for an initial f_eq mode of amplitude
    (deps, dv) (M = 4/3 v and v = 3/4 M at linear order, eps = 1)."""
    df = w * (deps + 3.0 * (4.0 / 3.0) * (v[:, 0] * dv_x + v[:, 1] * dv_y))
    fn = np.linalg.matrix_power(_linear_step(v, w, k, tau, cfl), nsteps) @ df
    post = _symbols(v, k, cfl) * fn
    return post.sum(), 0.75 * (v[:, 0] @ post), 0.75 * (v[:, 1] @ post)



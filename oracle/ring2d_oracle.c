/*
 * ring2d_oracle.c -- plain FP64 CPU oracle of the genuinely two-dimensional
 * massless RLBM variant: momenta confined to the plane, an 8-direction ring
 * node, ideal-gas pressure P = eps/2 (massless in 2+1 dimensions).
 *
 * TEST INFRASTRUCTURE ONLY (see rlbm_oracle.c).  This is not the paper's
 * scheme -- the paper evolves the 3D spherical node on a one-layer lattice,
 * with P = eps/3 -- but its two-dimensional counterpart, built the same way
 * (Sec. 3.1-3.3 with the angular polynomials of App. A taken on the circle):
 *   stencil:  v_k = (cos 2 pi k/8, sin 2 pi k/8), w_k = 1/8 (exact for
 *             trigonometric polynomials up to degree 7);
 *   moments:  T^{mu nu} = sum_k f_k v_k^mu v_k^nu, v_k^mu = (1, v_k), 3x3;
 *   Landau:   T^{mu nu} u_nu = -eps u^mu;
 *   f_eq:     projection of T_eq = (eps + P) u u + P g, P = eps/2, on
 *             P^(0) = 1, P^(1) = v, P^(2) = v v - I/2 with the circle norms
 *             1, 2, 4: f_eq,k = w_k [a0 + 2 a1.v_k + 4 a2 : P^(2)(v_k)];
 *   relax:    Anderson-Witting, rate (u^0 - v_k.u)/tau;
 *   force:    the driving term projected on the same polynomials with the
 *             kinetic moments of F . d/dp f: sum G = F.M, sum G v = F E,
 *             sum G v v = F M + M F - F.Q (the moments the 3D term of App. B
 *             carries), i.e. G_k = w_k [F.M + 2 E (F.v_k) + 4 C : P^(2)(v_k)]
 *             with C the traceless part of F M + M F - F.Q.
 * Layout f[k][y][x], FP64; signature (-,+,+); Delta x = Delta t = 1, CFL 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define RDIR 8

static const double R_PI = 3.14159265358979323846264338327950288;

static double r_v[RDIR][2];
static int r_ready = 0;

static void ring_build(void)
{
    if (r_ready) return;
    for (int k = 0; k < RDIR; ++k) {
        double a = 2.0 * R_PI * k / RDIR;
        r_v[k][0] = cos(a);
        r_v[k][1] = sin(a);
    }
    /* exact zeros and unit components for the axis directions */
    r_v[2][0] = r_v[6][0] = 0.0;
    r_v[0][1] = r_v[4][1] = 0.0;
    r_ready = 1;
}

void ring_stencil(double *v, double *w)
{
    ring_build();
    for (int k = 0; k < RDIR; ++k) {
        v[2 * k] = r_v[k][0];
        v[2 * k + 1] = r_v[k][1];
        w[k] = 1.0 / RDIR;
    }
}

void ring_moments_node(const double *f, double *T)
{
    ring_build();
    for (int m = 0; m < 9; ++m) T[m] = 0.0;
    for (int k = 0; k < RDIR; ++k) {
        double p[3] = {1.0, r_v[k][0], r_v[k][1]};
        for (int mu = 0; mu < 3; ++mu)
            for (int nu = 0; nu < 3; ++nu) T[3 * mu + nu] += f[k] * p[mu] * p[nu];
    }
}

/* Landau frame by the fixed-point pair eps = T^00 - T^0j v_j,
 * (T^ij + eps delta^ij) v_j = T^0i (2x2 solve by Cramer's rule). */
int ring_landau(const double *T, double *eps_out, double *u_out)
{
    double v[2] = {0.0, 0.0}, eps = T[0];
    int it;
    for (it = 1; it <= 200; ++it) {
        double e = T[0] - (T[1] * v[0] + T[2] * v[1]);
        double a = T[4] + e, b = T[5], c = T[7], d = T[8] + e;
        double det = a * d - b * c;
        if (det == 0.0) return -1;
        double vx = (d * T[1] - b * T[2]) / det;
        double vy = (a * T[2] - c * T[1]) / det;
        double de = fabs(e - eps), dv = fabs(vx - v[0]) + fabs(vy - v[1]);
        eps = e;
        v[0] = vx;
        v[1] = vy;
        if (de <= 1e-15 * fabs(eps) && dv <= 1e-15) break;
    }
    if (it > 200) return -1;
    double v2 = v[0] * v[0] + v[1] * v[1];
    if (!(v2 < 1.0) || !(eps > 0.0)) return -1;
    double u0 = 1.0 / sqrt(1.0 - v2);
    *eps_out = eps;
    u_out[0] = u0;
    u_out[1] = u0 * v[0];
    u_out[2] = u0 * v[1];
    return it;
}

/* T_eq = (eps + P) u u + P g, P = eps/2, g = diag(-1, 1, 1). */
void ring_ideal_T(double eps, const double *u, double *T)
{
    double P = eps / 2.0;
    for (int mu = 0; mu < 3; ++mu)
        for (int nu = 0; nu < 3; ++nu) {
            double g = (mu == nu) ? (mu == 0 ? -1.0 : 1.0) : 0.0;
            T[3 * mu + nu] = (eps + P) * u[mu] * u[nu] + P * g;
        }
}

void ring_feq(double eps, const double *u, double *feq)
{
    ring_build();
    double T[9];
    ring_ideal_T(eps, u, T);
    double a0 = T[0], a1[2] = {T[1], T[2]}, a2[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) a2[j][k] = T[3 * (j + 1) + (k + 1)] - (j == k ? a0 / 2.0 : 0.0);
    for (int i = 0; i < RDIR; ++i) {
        double p1 = a1[0] * r_v[i][0] + a1[1] * r_v[i][1], p2 = 0.0;
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) p2 += a2[j][k] * (r_v[i][j] * r_v[i][k] - (j == k ? 0.5 : 0.0));
        feq[i] = (1.0 / RDIR) * (a0 + 2.0 * p1 + 4.0 * p2);
    }
}

void ring_force_term(const double *f, const double *F, double *G)
{
    ring_build();
    double E = 0.0, M[2] = {0.0, 0.0}, Q[2][2][2] = {{{0}}};
    for (int i = 0; i < RDIR; ++i) {
        E += f[i];
        for (int a = 0; a < 2; ++a) M[a] += f[i] * r_v[i][a];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) Q[a][b][c] += f[i] * r_v[i][a] * r_v[i][b] * r_v[i][c];
    }
    double FM = F[0] * M[0] + F[1] * M[1];
    double X[2][2];
    for (int d = 0; d < 2; ++d)
        for (int e = 0; e < 2; ++e) {
            double FQ = 0.0;
            for (int a = 0; a < 2; ++a) FQ += F[a] * Q[a][d][e];
            X[d][e] = F[d] * M[e] + M[d] * F[e] - FQ;
        }
    double trX = X[0][0] + X[1][1];
    for (int i = 0; i < RDIR; ++i) {
        double Fv = F[0] * r_v[i][0] + F[1] * r_v[i][1];
        double CP = 0.0;
        for (int d = 0; d < 2; ++d)
            for (int e = 0; e < 2; ++e) {
                double C = X[d][e] - (d == e ? trX / 2.0 : 0.0);
                CP += C * (r_v[i][d] * r_v[i][e] - (d == e ? 0.5 : 0.0));
            }
        G[i] = (1.0 / RDIR) * (FM + 2.0 * E * Fv + 4.0 * CP);
    }
}

int ring_collide_node(double *f, const double *F, double tau, double *eps_out, double *u_out)
{
    ring_build();
    double T[9], eps, u[3], feq[RDIR], G[RDIR];
    ring_moments_node(f, T);
    if (ring_landau(T, &eps, u) < 0) return -1;
    ring_feq(eps, u, feq);
    int forced = F && (F[0] != 0.0 || F[1] != 0.0);
    if (forced) ring_force_term(f, F, G);
    for (int i = 0; i < RDIR; ++i) {
        double vu = r_v[i][0] * u[1] + r_v[i][1] * u[2];
        f[i] = f[i] - (u[0] - vu) / tau * (f[i] - feq[i]) + (forced ? G[i] : 0.0);
    }
    if (eps_out) *eps_out = eps;
    if (u_out)
        for (int m = 0; m < 3; ++m) u_out[m] = u[m];
    return 0;
}

static long rwrap(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* Pull with bilinear interpolation from x - v_k, periodic. */
void ring_stream(const double *fin, double *fout, int nx, int ny)
{
    ring_build();
    size_t plane = (size_t)nx * ny;
    for (int k = 0; k < RDIR; ++k) {
        double sx = -r_v[k][0], sy = -r_v[k][1];
        double flx = floor(sx), fly = floor(sy), tx = sx - flx, ty = sy - fly;
        long ox = (long)flx, oy = (long)fly;
        const double *src = fin + (size_t)k * plane;
        double *dst = fout + (size_t)k * plane;
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            long y0 = rwrap(y + oy, ny), y1 = rwrap(y + oy + 1, ny);
            for (int x = 0; x < nx; ++x) {
                long x0 = rwrap(x + ox, nx), x1 = rwrap(x + ox + 1, nx);
                dst[(size_t)y * nx + x] =
                    (1.0 - tx) * (1.0 - ty) * src[(size_t)y0 * nx + x0] + tx * (1.0 - ty) * src[(size_t)y0 * nx + x1] +
                    (1.0 - tx) * ty * src[(size_t)y1 * nx + x0] + tx * ty * src[(size_t)y1 * nx + x1];
            }
        }
    }
}

int ring_init(double *f, int nx, int ny, const double *eps, const double *vx, const double *vy)
{
    size_t plane = (size_t)nx * ny;
    int bad = 0;
    for (size_t n = 0; n < plane; ++n) {
        double e = eps ? eps[n] : 1.0, a = vx ? vx[n] : 0.0, b = vy ? vy[n] : 0.0;
        double v2 = a * a + b * b;
        if (!(v2 < 1.0) || !(e > 0.0)) {
            bad = 1;
            continue;
        }
        double u0 = 1.0 / sqrt(1.0 - v2), u[3] = {u0, u0 * a, u0 * b}, feq[RDIR];
        ring_feq(e, u, feq);
        for (int k = 0; k < RDIR; ++k) f[(size_t)k * plane + n] = feq[k];
    }
    return bad ? -1 : 0;
}

void oracle_force_field(int nx, int ny, int kmin, int kmax, double amp, uint64_t seed, uint64_t epoch, double *Fx,
                        double *Fy);

int ring_run(double *f, double *tmp, double *Fx, double *Fy, int nx, int ny, double tau, long step0, int nsteps,
             int kmin, int kmax, double amp, uint64_t seed, int redraw)
{
    size_t plane = (size_t)nx * ny;
    int forced = (amp > 0.0 && kmax > 0);
    long cur = -1;
    int bad = 0;
    for (int s = 0; s < nsteps; ++s) {
        long step = step0 + s;
        if (forced) {
            long e = redraw > 0 ? step / redraw : 0;
            if (e != cur) {
                oracle_force_field(nx, ny, kmin, kmax, amp, seed, (uint64_t)e, Fx, Fy);
                cur = e;
            }
        }
        ring_stream(f, tmp, nx, ny);
#pragma omp parallel for schedule(static) reduction(+ : bad)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t n = (size_t)y * nx + x;
                double node[RDIR], F[2] = {forced ? Fx[n] : 0.0, forced ? Fy[n] : 0.0};
                for (int k = 0; k < RDIR; ++k) node[k] = tmp[(size_t)k * plane + n];
                if (ring_collide_node(node, forced ? F : NULL, tau, NULL, NULL) != 0) bad += 1;
                for (int k = 0; k < RDIR; ++k) f[(size_t)k * plane + n] = node[k];
            }
    }
    return bad;
}

int ring_fields(const double *f, double *tmp, int nx, int ny, double *eps, double *vx, double *vy)
{
    size_t plane = (size_t)nx * ny;
    ring_stream(f, tmp, nx, ny);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double node[RDIR], T[9], e, u[3];
            for (int k = 0; k < RDIR; ++k) node[k] = tmp[(size_t)k * plane + n];
            ring_moments_node(node, T);
            if (ring_landau(T, &e, u) < 0) {
                bad += 1;
                e = NAN;
                u[0] = 1.0;
                u[1] = u[2] = NAN;
            }
            if (eps) eps[n] = e;
            if (vx) vx[n] = u[1] / u[0];
            if (vy) vy[n] = u[2] / u[0];
        }
    return bad;
}

void ring_totals(const double *f, int nx, int ny, double *out)
{
    ring_build();
    size_t plane = (size_t)nx * ny;
    double a = 0.0, b = 0.0, c = 0.0;
    for (size_t n = 0; n < plane; ++n)
        for (int k = 0; k < RDIR; ++k) {
            double fk = f[(size_t)k * plane + n];
            a += fk;
            b += fk * r_v[k][0];
            c += fk * r_v[k][1];
        }
    out[0] = a;
    out[1] = b;
    out[2] = c;
}

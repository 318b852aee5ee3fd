/*
 * rlbm_oracle.c -- plain FP64 CPU oracle of one relativistic lattice Boltzmann
 * (RLBM) step for a massless fluid on a periodic 2D lattice (Watson,
 * arXiv:2101.06187).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, loads or calls it, and it shares no code,
 * table or header with the CUDA path.
 *
 * Layout: populations f[i][y][x], i = 0..25 the 26 moving momentum
 * directions of the spherical "D3Q27" node (Sec. 5: one lattice node in z, so
 * the 3D stencil lives on a 2D lattice), y = 0..ny-1, x = 0..nx-1, row-major,
 * FP64.  f_i is the energy-weighted angular population: T^{mu nu} =
 * sum_i f_i v_i^mu v_i^nu with v_i^mu = (1, v_i), |v_i| = 1 (Eq.
 * energyMomentumIntegral discretised; the radial integral with alpha = 3 is a
 * constant absorbed into f_i, Sec. 3.2).  The 27th ("rest") slot of D3Q27
 * carries zero weight for a massless particle and is omitted.
 *
 * One step follows the loop of Sec. 3.3 ((b) stream, (c) moments, (d)
 * equilibrium, (e) collision + driving term):
 *   stream:  pull with linear (bilinear in x,y) interpolation from x - v_i
 *            (Sec. 3.2, the off-lattice stencil "overcome ... using a linear
 *            interpolation scheme"), periodic boundaries, Delta x = Delta t = 1.
 *   moments: T^{mu nu} = sum_i f_i v_i^mu v_i^nu            (Eq. energyMomentumIntegral)
 *   Landau:  T^{mu nu} u_nu = -eps u^mu, u.u = -1           (Sec. 3.2, Landau-Lifshitz)
 *   f_eq:    truncated expansion, coefficients from T_eq   (Eqs. rel_pdf_exp, rel_pdf_exp_coef,
 *            stressEnergyT with P = eps/3, App. A)
 *   relax:   f - (1/tau)(u^0 - v_i.u)(f - f_eq)            (Eq. boltzmanneq_rel, Anderson-Witting)
 *   force:   + G_i, the projected driving term             (Eq. forceTerm, App. B)
 *   store.
 *
 * Signature (-,+,+,+).  Everything is FP64, fixed loop order; compile with
 * -ffp-contract=off so results do not depend on FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NDIR 26

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------------------
 * Stencil (Sec. 3.2 / Sec. 5 "spherical D3Q27"; App. A orthogonality).
 * The 26 directions are the normalised non-zero vectors of {-1,0,1}^3: faces
 * (1 nonzero), edges (2 nonzero, /sqrt 2), corners (3 nonzero, /sqrt 3).
 * Weights are the degree-7 spherical rule on that point set:
 * faces 1/21, edges 4/105, corners 9/280 (sum 1).  Reading: the paper names
 * the node "spherical D3Q27" but does not print the set; this one reproduces
 * the angular integrals of App. A exactly up to degree 7.
 * ------------------------------------------------------------------------- */
static double g_v[NDIR][3];
static double g_w[NDIR];
static int g_stencil_ready = 0;

static void build_stencil(void)
{
    if (g_stencil_ready) return;
    int n = 0;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
                int nz = (a != 0) + (b != 0) + (c != 0);
                if (nz == 0) continue;
                double norm = sqrt((double)nz);
                g_v[n][0] = a / norm;
                g_v[n][1] = b / norm;
                g_v[n][2] = c / norm;
                g_w[n] = (nz == 1) ? 1.0 / 21.0 : (nz == 2) ? 4.0 / 105.0 : 9.0 / 280.0;
                ++n;
            }
    g_stencil_ready = 1;
}

int oracle_ndirs(void) { return NDIR; }

void oracle_stencil(double *v, double *w)
{
    build_stencil();
    for (int i = 0; i < NDIR; ++i) {
        for (int a = 0; a < 3; ++a) v[3 * i + a] = g_v[i][a];
        w[i] = g_w[i];
    }
}

/* ---------------------------------------------------------------------------
 * Moments: T^{mu nu} = sum_i f_i v_i^mu v_i^nu, v_i^0 = 1
 * (Eq. energyMomentumIntegral, discretised).  T is 4x4, row-major.
 * ------------------------------------------------------------------------- */
void oracle_moments_node(const double *f, double *T)
{
    build_stencil();
    for (int m = 0; m < 16; ++m) T[m] = 0.0;
    for (int i = 0; i < NDIR; ++i) {
        double p[4] = {1.0, g_v[i][0], g_v[i][1], g_v[i][2]};
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu)
                T[4 * mu + nu] += f[i] * p[mu] * p[nu];
    }
}

/* Third angular moment Q^{abc} = sum_i f_i v_i^a v_i^b v_i^c, used by the
 * driving term (Eq. forceTerm: the integral of f v^i v^j v^k). */
static void third_moment(const double *f, double Q[3][3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) Q[a][b][c] = 0.0;
    for (int i = 0; i < NDIR; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c)
                    Q[a][b][c] += f[i] * g_v[i][a] * g_v[i][b] * g_v[i][c];
}

/* Solve the 3x3 system A x = b by Gaussian elimination with partial pivoting.
 * Returns 0 on success, -1 if singular. */
static int solve3(double A_in[3][3], const double b_in[3], double x[3])
{
    double A[3][4];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) A[r][c] = A_in[r][c];
        A[r][3] = b_in[r];
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 4; ++c) {
                double t = A[col][c];
                A[col][c] = A[piv][c];
                A[piv][c] = t;
            }
        for (int r = col + 1; r < 3; ++r) {
            double m = A[r][col] / A[col][col];
            for (int c = col; c < 4; ++c) A[r][c] -= m * A[col][c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = A[r][3];
        for (int c = r + 1; c < 3; ++c) s -= A[r][c] * x[c];
        x[r] = s / A[r][r];
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Landau-Lifshitz frame (Sec. 3.1 and the eigenvalue problem closing Sec.
 * 3.2): find eps > 0 and the timelike u^mu (u.u = -1, u^0 > 0) with
 *     T^{mu nu} u_nu = -eps u^mu          (signature -,+,+,+)
 * Written with the 3-velocity v = u/u^0 this reads, for mu = 0 and mu = i,
 *     eps = T^{00} - T^{0j} v_j ,   (T^{ij} + eps delta^{ij}) v_j = T^{0i}.
 * The oracle iterates these two relations from v = 0 (each pass a 3x3 linear
 * solve) until eps and v stop changing to 1e-15, at most 200 passes.
 * Returns the number of passes, or -1 if it did not converge / |v| >= 1.
 * ------------------------------------------------------------------------- */
int oracle_landau(const double *T, double *eps_out, double *u_out)
{
    double v[3] = {0.0, 0.0, 0.0};
    double eps = T[0];
    int it;
    for (it = 1; it <= 200; ++it) {
        double eps_new = T[0] - (T[1] * v[0] + T[2] * v[1] + T[3] * v[2]);
        double A[3][3], b[3], vn[3];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) A[i][j] = T[4 * (i + 1) + (j + 1)];
            A[i][i] += eps_new;
            b[i] = T[4 * 0 + (i + 1)];
        }
        if (solve3(A, b, vn) != 0) return -1;
        double de = fabs(eps_new - eps);
        double dv = fabs(vn[0] - v[0]) + fabs(vn[1] - v[1]) + fabs(vn[2] - v[2]);
        eps = eps_new;
        v[0] = vn[0];
        v[1] = vn[1];
        v[2] = vn[2];
        if (de <= 1e-15 * fabs(eps) && dv <= 1e-15) break;
    }
    if (it > 200) return -1;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (!(v2 < 1.0) || !(eps > 0.0)) return -1;
    double u0 = 1.0 / sqrt(1.0 - v2);
    *eps_out = eps;
    u_out[0] = u0;
    u_out[1] = u0 * v[0];
    u_out[2] = u0 * v[1];
    u_out[3] = u0 * v[2];
    return it;
}

/* Ideal-fluid tensor T_eq^{mu nu} = (eps + P) u^mu u^nu + P g^{mu nu},
 * P = eps/3, g = diag(-1,1,1,1)  (Eq. stressEnergyT, Sec. 3.1 EOS). */
void oracle_ideal_T(double eps, const double *u, double *T)
{
    double P = eps / 3.0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
            double g = (mu == nu) ? (mu == 0 ? -1.0 : 1.0) : 0.0;
            T[4 * mu + nu] = (eps + P) * u[mu] * u[nu] + P * g;
        }
}

/* ---------------------------------------------------------------------------
 * Equilibrium (Eqs. rel_pdf_exp and rel_pdf_exp_coef, App. A): the Juttner
 * distribution projected on the angular polynomials P^(0) = 1, P^(1)_i = v_i,
 * P^(2)_ij = v_i v_j - delta_ij/3, truncated after n = 2.  Its coefficients
 * are the projections of T_eq (the matrix relating T^{mu nu} to a^(0),
 * a^(1)_i, a^(2)_ij closing Sec. 3.2, with the radial constant absorbed):
 *   a0 = T^{00},  a1_i = T^{0i},  a2_ij = T^{ij} - delta_ij T^{00}/3.
 * The discrete population is the quadrature weight times the expansion, with
 * the orthogonality normalisations 1, 3, 15/2 (App. A):
 *   f_i^eq = w_i [ a0 P^(0) + 3 a1_j P^(1)_j(v_i) + (15/2) a2_jk P^(2)_jk(v_i) ].
 * ------------------------------------------------------------------------- */
void oracle_feq(double eps, const double *u, double *feq)
{
    build_stencil();
    double T[16];
    oracle_ideal_T(eps, u, T);
    double a0 = T[0];
    double a1[3] = {T[1], T[2], T[3]};
    double a2[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            a2[j][k] = T[4 * (j + 1) + (k + 1)] - (j == k ? a0 / 3.0 : 0.0);
    for (int i = 0; i < NDIR; ++i) {
        double p1 = 0.0, p2 = 0.0;
        for (int j = 0; j < 3; ++j) p1 += a1[j] * g_v[i][j];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                p2 += a2[j][k] * (g_v[i][j] * g_v[i][k] - (j == k ? 1.0 / 3.0 : 0.0));
        feq[i] = g_w[i] * (a0 + 3.0 * p1 + 7.5 * p2);
    }
}

/* ---------------------------------------------------------------------------
 * Driving term (Eq. forceTerm, App. B), F^mu = (0, F^a):
 *   G_i = C w_i [ (3/12) F_a M^a - (1/2)(F.v_i) E
 *                 + (5/4) F_a v_i^b v_i^c Q^{abc} - (5/2)(F.v_i)(v_i.M) ]
 * with E = sum f, M^a = sum f v^a, Q^{abc} = sum f v^a v^b v^c taken from the
 * (post-stream) populations.  Reading: the prefactor -1/T_0 of App. B with
 * the radial constants is folded into F and fixed by C = -6, which makes the
 * driving term inject energy F.M and momentum F E per unit time:
 *   sum_i G_i = F.M,  sum_i G_i v_i = F E.
 * ------------------------------------------------------------------------- */
void oracle_force_term(const double *f, const double *F, double *G)
{
    build_stencil();
    double E = 0.0, M[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NDIR; ++i) {
        E += f[i];
        for (int a = 0; a < 3; ++a) M[a] += f[i] * g_v[i][a];
    }
    double Q[3][3][3];
    third_moment(f, Q);
    double FM = F[0] * M[0] + F[1] * M[1] + F[2] * M[2];
    for (int i = 0; i < NDIR; ++i) {
        double Fv = F[0] * g_v[i][0] + F[1] * g_v[i][1] + F[2] * g_v[i][2];
        double vM = g_v[i][0] * M[0] + g_v[i][1] * M[1] + g_v[i][2] * M[2];
        double FQvv = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) FQvv += F[a] * g_v[i][b] * g_v[i][c] * Q[a][b][c];
        double bracket = (3.0 / 12.0) * FM - 0.5 * Fv * E + 1.25 * FQvv - 2.5 * Fv * vM;
        G[i] = -6.0 * g_w[i] * bracket;
    }
}

/* ---------------------------------------------------------------------------
 * Collision of one node (steps (c)-(e) of Sec. 3.3): moments, Landau frame,
 * equilibrium, Anderson-Witting relaxation (Eq. boltzmanneq_rel: the rate is
 * proportional to -p^mu u_mu / tau_R = |p| (u^0 - v_i.u)/tau_R, relaxing
 * towards f_eq; Delta t = 1), plus the driving term computed from the same
 * pre-collision populations (f* = f + Delta t C + F^mu nabla_mu f).
 * tau is the relaxation time in units of Delta t.  F is the 3-vector (F_z =
 * 0 for the 2D stirring).  Returns 0, or -1 if the Landau solve failed.
 * On success eps_out / u_out (may be NULL) receive the Landau frame.
 * ------------------------------------------------------------------------- */
/* Relaxation time of a node in units of Delta t.  eta_s <= 0: the constant
 * tau.  eta_s > 0 (viscosity-to-entropy ratio): tau_R = 5 (eta/s) / T with
 * the temperature from eps = 3 T^4 / pi^2 (Sec. 3.1, Sec. 3.2), divided by
 * the time step dt. */
double oracle_tau_of(double eps, double tau, double eta_s, double dt)
{
    if (!(eta_s > 0.0)) return tau;
    double T = pow(ORACLE_PI * ORACLE_PI * eps / 3.0, 0.25);
    return 5.0 * eta_s / T / dt;
}

int oracle_collide_node_ex(double *f, const double *F, double tau, double eta_s, double dt, double *eps_out,
                           double *u_out)
{
    build_stencil();
    double T[16], eps, u[4], feq[NDIR], G[NDIR];
    oracle_moments_node(f, T);
    if (oracle_landau(T, &eps, u) < 0) return -1;
    tau = oracle_tau_of(eps, tau, eta_s, dt);
    oracle_feq(eps, u, feq);
    int have_force = F && (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0);
    if (have_force) oracle_force_term(f, F, G);
    for (int i = 0; i < NDIR; ++i) {
        double vu = g_v[i][0] * u[1] + g_v[i][1] * u[2] + g_v[i][2] * u[3];
        double relax = (u[0] - vu) / tau * (f[i] - feq[i]);
        f[i] = f[i] - relax + (have_force ? G[i] : 0.0);
    }
    if (eps_out) *eps_out = eps;
    if (u_out)
        for (int m = 0; m < 4; ++m) u_out[m] = u[m];
    return 0;
}

int oracle_collide_node(double *f, const double *F, double tau, double *eps_out, double *u_out)
{
    return oracle_collide_node_ex(f, F, tau, 0.0, 1.0, eps_out, u_out);
}

/* ---------------------------------------------------------------------------
 * Streaming (step (b)): pull with bilinear interpolation.  Population i at
 * node (x, y) takes the value of the post-collision field of direction i at
 * the off-lattice point (x - l v_i^x, y - l v_i^y), l = Delta t / Delta x the
 * CFL number (0 < l <= 1: at most one cell), interpolated linearly
 * in x and y between the four surrounding nodes; periodic wrap.  With one
 * node in z, z-streaming is the identity.  The interpolation offset and
 * weights depend only on the displacement:  source = x + floor(-c) + frac,
 * frac = -c - floor(-c).
 * ------------------------------------------------------------------------- */
static inline long wrap(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

void oracle_stream_cfl(const double *fin, double *fout, int nx, int ny, double cfl)
{
    build_stencil();
    size_t plane = (size_t)nx * (size_t)ny;
    for (int i = 0; i < NDIR; ++i) {
        double sx = -cfl * g_v[i][0], sy = -cfl * g_v[i][1];
        double flx = floor(sx), fly = floor(sy);
        double tx = sx - flx, ty = sy - fly; /* fractional parts in [0,1) */
        long ox = (long)flx, oy = (long)fly;
        const double *src = fin + (size_t)i * plane;
        double *dst = fout + (size_t)i * plane;
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            long y0 = wrap(y + oy, ny), y1 = wrap(y + oy + 1, ny);
            for (int x = 0; x < nx; ++x) {
                long x0 = wrap(x + ox, nx), x1 = wrap(x + ox + 1, nx);
                double v00 = src[(size_t)y0 * nx + x0];
                double v10 = src[(size_t)y0 * nx + x1];
                double v01 = src[(size_t)y1 * nx + x0];
                double v11 = src[(size_t)y1 * nx + x1];
                dst[(size_t)y * nx + x] = (1.0 - tx) * (1.0 - ty) * v00 + tx * (1.0 - ty) * v10 +
                                          (1.0 - tx) * ty * v01 + tx * ty * v11;
            }
        }
    }
}

void oracle_stream(const double *fin, double *fout, int nx, int ny) { oracle_stream_cfl(fin, fout, nx, ny, 1.0); }

/* ---------------------------------------------------------------------------
 * Philox4x32-10 counter-based generator, written from its published
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplications by
 * 0xD2511F53 and 0xCD9E8D57, the S-box/P-box word exchange, and a key
 * schedule bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85.
 * Pinned word for word against two implementations it shares nothing
 * with (Triton's Philox4x32 on the CPU, cuRAND's Philox4x32-10 on the
 * GPU), and statistically.
 * ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* 53-bit uniform double in [0,1) from two 32-bit words. */
static double u01_from_words(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
    return (double)m * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------------------
 * Stirring force (Sec. 5): modes on the wavenumber shell kmin <= |k| <= kmax
 * (integer k = (kx, ky), k = 0 excluded so the force averages to zero), each
 * with a random magnitude up to `amp`, a random phase and a random in-plane
 * direction, transformed to configuration space.  Reading: one Hermitian
 * pair per half-plane mode (ky > 0, or ky = 0 and kx > 0), enumerated in
 * the order ky = 0..kmax, kx = -kmax..kmax; mode m of epoch e draws
 *   Philox(ctr = {e, m, 0, 0}, key = {seed_lo, seed_hi}) -> r, phi
 *   Philox(ctr = {e, m, 1, 0}, key)                      -> theta
 * with magnitude r*amp, phase 2 pi * u, direction 2 pi * u, and
 *   F(x) = sum_m 2 r_m amp (cos th_m, sin th_m) cos(2 pi (kx x/nx + ky y/ny) + phi_m).
 * ------------------------------------------------------------------------- */
int oracle_forcing_modes(int kmin, int kmax, int *kx_out, int *ky_out, int cap)
{
    int m = 0;
    for (int ky = 0; ky <= kmax; ++ky)
        for (int kx = -kmax; kx <= kmax; ++kx) {
            if (ky == 0 && kx <= 0) continue;
            int k2 = kx * kx + ky * ky;
            if (k2 < kmin * kmin || k2 > kmax * kmax) continue;
            if (m < cap && kx_out) {
                kx_out[m] = kx;
                ky_out[m] = ky;
            }
            ++m;
        }
    return m;
}

void oracle_forcing_draw(int kmin, int kmax, double amp, uint64_t seed, uint64_t epoch, double *mag,
                         double *phase, double *theta)
{
    int nm = oracle_forcing_modes(kmin, kmax, NULL, NULL, 0);
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int m = 0; m < nm; ++m) {
        uint32_t c0[4] = {(uint32_t)epoch, (uint32_t)m, 0u, 0u}, o0[4];
        uint32_t c1[4] = {(uint32_t)epoch, (uint32_t)m, 1u, 0u}, o1[4];
        oracle_philox4x32_10(c0, key, o0);
        oracle_philox4x32_10(c1, key, o1);
        mag[m] = amp * u01_from_words(o0[0], o0[1]);
        phase[m] = 2.0 * ORACLE_PI * u01_from_words(o0[2], o0[3]);
        theta[m] = 2.0 * ORACLE_PI * u01_from_words(o1[0], o1[1]);
    }
}

void oracle_force_field(int nx, int ny, int kmin, int kmax, double amp, uint64_t seed, uint64_t epoch,
                        double *Fx, double *Fy)
{
    int nm = oracle_forcing_modes(kmin, kmax, NULL, NULL, 0);
    int *kx = (int *)malloc(sizeof(int) * (nm > 0 ? nm : 1));
    int *ky = (int *)malloc(sizeof(int) * (nm > 0 ? nm : 1));
    double *mag = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    double *ph = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    double *th = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    oracle_forcing_modes(kmin, kmax, kx, ky, nm);
    oracle_forcing_draw(kmin, kmax, amp, seed, epoch, mag, ph, th);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double fx = 0.0, fy = 0.0;
            for (int m = 0; m < nm; ++m) {
                double arg = 2.0 * ORACLE_PI *
                                 ((double)wrap((long)kx[m] * x, nx) / nx + (double)wrap((long)ky[m] * y, ny) / ny) +
                             ph[m];
                double c = cos(arg);
                fx += 2.0 * mag[m] * cos(th[m]) * c;
                fy += 2.0 * mag[m] * sin(th[m]) * c;
            }
            Fx[(size_t)y * nx + x] = fx;
            Fy[(size_t)y * nx + x] = fy;
        }
    free(kx);
    free(ky);
    free(mag);
    free(ph);
    free(th);
}

/* The same force evaluated only at the npts nodes (xs[k], ys[k]) of an nx x
 * ny lattice (for checking large lattices point by point). */
void oracle_force_points(int nx, int ny, int kmin, int kmax, double amp, uint64_t seed, uint64_t epoch, int npts,
                         const int *xs, const int *ys, double *Fx, double *Fy)
{
    int nm = oracle_forcing_modes(kmin, kmax, NULL, NULL, 0);
    int *kx = (int *)malloc(sizeof(int) * (nm > 0 ? nm : 1));
    int *ky = (int *)malloc(sizeof(int) * (nm > 0 ? nm : 1));
    double *mag = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    double *ph = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    double *th = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    oracle_forcing_modes(kmin, kmax, kx, ky, nm);
    oracle_forcing_draw(kmin, kmax, amp, seed, epoch, mag, ph, th);
    for (int k = 0; k < npts; ++k) {
        double fx = 0.0, fy = 0.0;
        for (int m = 0; m < nm; ++m) {
            double arg = 2.0 * ORACLE_PI *
                             ((double)wrap((long)kx[m] * xs[k], nx) / nx + (double)wrap((long)ky[m] * ys[k], ny) / ny) +
                         ph[m];
            double c = cos(arg);
            fx += 2.0 * mag[m] * cos(th[m]) * c;
            fy += 2.0 * mag[m] * sin(th[m]) * c;
        }
        Fx[k] = fx;
        Fy[k] = fy;
    }
    free(kx);
    free(ky);
    free(mag);
    free(ph);
    free(th);
}

/* ---------------------------------------------------------------------------
 * Initialisation (step (a)): f* = f_eq(eps, u) of the initial fields.  eps,
 * vx, vy are nx*ny arrays (vx, vy the 3-velocity); NULL means eps = 1, v = 0.
 * ------------------------------------------------------------------------- */
int oracle_init(double *f, int nx, int ny, const double *eps, const double *vx, const double *vy)
{
    build_stencil();
    size_t plane = (size_t)nx * (size_t)ny;
    int bad = 0;
    for (size_t n = 0; n < plane; ++n) {
        double e = eps ? eps[n] : 1.0;
        double a = vx ? vx[n] : 0.0, b = vy ? vy[n] : 0.0;
        double v2 = a * a + b * b;
        if (!(v2 < 1.0) || !(e > 0.0)) {
            bad = 1;
            continue;
        }
        double u0 = 1.0 / sqrt(1.0 - v2);
        double u[4] = {u0, u0 * a, u0 * b, 0.0};
        double feq[NDIR];
        oracle_feq(e, u, feq);
        for (int i = 0; i < NDIR; ++i) f[(size_t)i * plane + n] = feq[i];
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * One full step: stream f (post-collision, in) into tmp, collide every node
 * of tmp with the force field (Fx, Fy may be NULL: no force), write the new
 * post-collision state back into f.  Returns 0 or the number of nodes whose
 * Landau solve failed.
 * ------------------------------------------------------------------------- */
int oracle_step_ex(double *f, double *tmp, int nx, int ny, double tau, const double *Fx, const double *Fy,
                   double cfl, double eta_s, double dt)
{
    build_stencil();
    size_t plane = (size_t)nx * (size_t)ny;
    oracle_stream_cfl(f, tmp, nx, ny, cfl);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double node[NDIR];
            for (int i = 0; i < NDIR; ++i) node[i] = tmp[(size_t)i * plane + n];
            double F[3] = {Fx ? Fx[n] : 0.0, Fy ? Fy[n] : 0.0, 0.0};
            if (oracle_collide_node_ex(node, F, tau, eta_s, dt, NULL, NULL) != 0) bad += 1;
            for (int i = 0; i < NDIR; ++i) f[(size_t)i * plane + n] = node[i];
        }
    return bad;
}

int oracle_step(double *f, double *tmp, int nx, int ny, double tau, const double *Fx, const double *Fy)
{
    return oracle_step_ex(f, tmp, nx, ny, tau, Fx, Fy, 1.0, 0.0, 1.0);
}

/* ---------------------------------------------------------------------------
 * Macroscopic fields seen by the next collision: stream the stored state into
 * tmp, then per node the moments and the Landau frame.  Outputs eps and the
 * 3-velocity v = u^i / u^0 (vx, vy).  Any output pointer may be NULL.
 * ------------------------------------------------------------------------- */
int oracle_fields_ex(const double *f, double *tmp, int nx, int ny, double cfl, double *eps, double *vx, double *vy)
{
    build_stencil();
    size_t plane = (size_t)nx * (size_t)ny;
    oracle_stream_cfl(f, tmp, nx, ny, cfl);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double node[NDIR], T[16], e, u[4];
            for (int i = 0; i < NDIR; ++i) node[i] = tmp[(size_t)i * plane + n];
            oracle_moments_node(node, T);
            if (oracle_landau(T, &e, u) < 0) {
                bad += 1;
                e = NAN;
                u[0] = 1.0;
                u[1] = u[2] = u[3] = NAN;
            }
            if (eps) eps[n] = e;
            if (vx) vx[n] = u[1] / u[0];
            if (vy) vy[n] = u[2] / u[0];
        }
    return bad;
}

int oracle_fields(const double *f, double *tmp, int nx, int ny, double *eps, double *vx, double *vy)
{
    return oracle_fields_ex(f, tmp, nx, ny, 1.0, eps, vx, vy);
}

/* ---------------------------------------------------------------------------
 * A run of nsteps steps starting at global step index step0, with the
 * stirring force redrawn every `redraw` steps (epoch = step / redraw); amp =
 * 0 (or kmax <= 0) means no force.  f holds the post-collision state; tmp,
 * Fx, Fy are caller scratch of 26*nx*ny, nx*ny, nx*ny doubles.
 * ------------------------------------------------------------------------- */
int oracle_run_ex(double *f, double *tmp, double *Fx, double *Fy, int nx, int ny, double tau, long step0,
                  int nsteps, int kmin, int kmax, double amp, uint64_t seed, int redraw, double cfl, double eta_s,
                  double dt)
{
    int forced = (amp > 0.0 && kmax > 0);
    long cur_epoch = -1;
    int bad = 0;
    for (int s = 0; s < nsteps; ++s) {
        long step = step0 + s;
        if (forced) {
            long e = redraw > 0 ? step / redraw : 0;
            if (e != cur_epoch) {
                oracle_force_field(nx, ny, kmin, kmax, amp, seed, (uint64_t)e, Fx, Fy);
                cur_epoch = e;
            }
        }
        bad += oracle_step_ex(f, tmp, nx, ny, tau, forced ? Fx : NULL, forced ? Fy : NULL, cfl, eta_s, dt);
    }
    return bad;
}

int oracle_run(double *f, double *tmp, double *Fx, double *Fy, int nx, int ny, double tau, long step0, int nsteps,
               int kmin, int kmax, double amp, uint64_t seed, int redraw)
{
    return oracle_run_ex(f, tmp, Fx, Fy, nx, ny, tau, step0, nsteps, kmin, kmax, amp, seed, redraw, 1.0, 0.0, 1.0);
}

/* Total energy-momentum of a population field: sum over nodes of T^{0 mu}
 * (mu = 0..3), summed node by node in FP64 in row-major order. */
void oracle_totals(const double *f, int nx, int ny, double *out)
{
    build_stencil();
    size_t plane = (size_t)nx * (size_t)ny;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t n = 0; n < plane; ++n)
        for (int i = 0; i < NDIR; ++i) {
            double fi = f[(size_t)i * plane + n];
            acc[0] += fi;
            acc[1] += fi * g_v[i][0];
            acc[2] += fi * g_v[i][1];
            acc[3] += fi * g_v[i][2];
        }
    for (int m = 0; m < 4; ++m) out[m] = acc[m];
}

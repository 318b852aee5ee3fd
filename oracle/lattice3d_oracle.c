/* lattice3d_oracle.c -- TEST INFRASTRUCTURE ONLY: the plain FP64 reference
 * of the three-dimensional lattice (the paper's conclusion, Sec. 6, names a
 * three-dimensional model as the next test).  The node is the paper's own
 * (rlbm_oracle.c: 26 directions, Landau frame, equilibrium, relaxation,
 * driving term); only the lattice around it is new:
 *
 *  - populations f[26][nz][ny][nx], periodic in x, y and z;
 *  - pull-streaming with trilinear interpolation from x - v_i (Sec. 3.2's
 *    linear interpolation in three dimensions, CFL 1);
 *  - the stirring force of Sec. 5 carried to three dimensions: modes on the
 *    shell kmin <= |k| <= kmax of integer k = (kx, ky, kz), one per
 *    half-space pair, each with a random magnitude, phase and a direction
 *    uniform on the sphere.
 *
 * Only tests, the smoke check and the benchmark's CPU baseline use it; the
 * library never does.  Everything here is FP64, compiled with
 * -ffp-contract=off, with fixed loop orders.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define N3DIR 26
#define PI3D 3.14159265358979323846

/* The node functions of rlbm_oracle.c. */
void oracle_stencil(double *v, double *w);
void oracle_moments_node(const double *f, double *T);
int oracle_landau(const double *T, double *eps_out, double *u_out);
void oracle_feq(double eps, const double *u, double *feq);
int oracle_collide_node(double *f, const double *F, double tau, double *eps_out, double *u_out);
void oracle_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out);

static double s_v[N3DIR][3], s_w[N3DIR];
static int s_built = 0;

static void build3(void)
{
    if (s_built) return;
    double v[3 * N3DIR], w[N3DIR];
    oracle_stencil(v, w);
    for (int i = 0; i < N3DIR; ++i) {
        for (int a = 0; a < 3; ++a) s_v[i][a] = v[3 * i + a];
        s_w[i] = w[i];
    }
    s_built = 1;
}

static long wrap3(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* Pull with trilinear interpolation from x - v_i, periodic in all axes. */
void oracle3d_stream(const double *fin, double *fout, int nx, int ny, int nz)
{
    build3();
    size_t vol = (size_t)nx * ny * nz;
    for (int i = 0; i < N3DIR; ++i) {
        double s[3], t[3];
        long o[3];
        for (int a = 0; a < 3; ++a) {
            s[a] = -s_v[i][a];
            double fl = floor(s[a]);
            o[a] = (long)fl;
            t[a] = s[a] - fl;
        }
        const double *src = fin + (size_t)i * vol;
        double *dst = fout + (size_t)i * vol;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double acc = 0.0;
                    for (int dz = 0; dz < 2; ++dz)
                        for (int dy = 0; dy < 2; ++dy)
                            for (int dx = 0; dx < 2; ++dx) {
                                double wgt = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) *
                                             (dz ? t[2] : 1.0 - t[2]);
                                if (wgt == 0.0) continue;
                                long xx = wrap3(x + o[0] + dx, nx), yy = wrap3(y + o[1] + dy, ny),
                                     zz = wrap3(z + o[2] + dz, nz);
                                acc += wgt * src[((size_t)zz * ny + yy) * nx + xx];
                            }
                    dst[((size_t)z * ny + y) * nx + x] = acc;
                }
    }
}

/* f = f_eq(eps, v) of the initial fields (nx*ny*nz each, [z][y][x]; NULL:
 * eps = 1, v = 0).  Returns -1 if a node has eps <= 0 or |v| >= 1. */
int oracle3d_init(double *f, int nx, int ny, int nz, const double *eps, const double *vx, const double *vy,
                  const double *vz)
{
    build3();
    size_t vol = (size_t)nx * ny * nz;
    int bad = 0;
    for (size_t n = 0; n < vol; ++n) {
        double e = eps ? eps[n] : 1.0;
        double a = vx ? vx[n] : 0.0, b = vy ? vy[n] : 0.0, c = vz ? vz[n] : 0.0;
        double v2 = a * a + b * b + c * c;
        if (!(v2 < 1.0) || !(e > 0.0)) {
            bad = 1;
            continue;
        }
        double u0 = 1.0 / sqrt(1.0 - v2);
        double u[4] = {u0, u0 * a, u0 * b, u0 * c};
        double feq[N3DIR];
        oracle_feq(e, u, feq);
        for (int i = 0; i < N3DIR; ++i) f[(size_t)i * vol + n] = feq[i];
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Three-dimensional stirring (Sec. 5's force on a 3D shell).  Modes: integer
 * k with kmin <= |k| <= kmax, one per pair +-k, the representative in the
 * half-space kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and kx > 0,
 * enumerated kz = 0..kmax, ky = -kmax..kmax, kx = -kmax..kmax (the kz = 0
 * modes come first, in the order of the two-dimensional list).  Mode m of
 * epoch e draws
 *   Philox(ctr = {e, m, 0, 0}, key = {seed_lo, seed_hi}) -> r, phi
 *   Philox(ctr = {e, m, 1, 0}, key)                      -> az, mu
 * magnitude r*amp, phase 2 pi u, direction (sqrt(1 - mu^2) cos az,
 * sqrt(1 - mu^2) sin az, mu) with az = 2 pi u and mu = 2u - 1 (uniform on
 * the sphere; the two-dimensional draw is the same with mu taken as 0), and
 *   F(x) = sum_m 2 r_m amp d_m cos(2 pi (kx x/nx + ky y/ny + kz z/nz) + phi_m).
 * ------------------------------------------------------------------------- */
static double u01_words(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
    return (double)m * (1.0 / 9007199254740992.0);
}

int oracle3d_forcing_modes(int kmin, int kmax, int *kx_out, int *ky_out, int *kz_out, int cap)
{
    int m = 0;
    for (int kz = 0; kz <= kmax; ++kz)
        for (int ky = -kmax; ky <= kmax; ++ky)
            for (int kx = -kmax; kx <= kmax; ++kx) {
                if (kz == 0 && (ky < 0 || (ky == 0 && kx <= 0))) continue;
                int k2 = kx * kx + ky * ky + kz * kz;
                if (k2 < kmin * kmin || k2 > kmax * kmax) continue;
                if (m < cap) {
                    if (kx_out) kx_out[m] = kx;
                    if (ky_out) ky_out[m] = ky;
                    if (kz_out) kz_out[m] = kz;
                }
                ++m;
            }
    return m;
}

void oracle3d_forcing_draw(int kmin, int kmax, double amp, uint64_t seed, uint64_t epoch, double *mag,
                           double *phase, double *dir)
{
    int nm = oracle3d_forcing_modes(kmin, kmax, NULL, NULL, NULL, 0);
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int m = 0; m < nm; ++m) {
        uint32_t c0[4] = {(uint32_t)epoch, (uint32_t)m, 0u, 0u}, o0[4];
        uint32_t c1[4] = {(uint32_t)epoch, (uint32_t)m, 1u, 0u}, o1[4];
        oracle_philox4x32_10(c0, key, o0);
        oracle_philox4x32_10(c1, key, o1);
        mag[m] = amp * u01_words(o0[0], o0[1]);
        phase[m] = 2.0 * PI3D * u01_words(o0[2], o0[3]);
        double az = 2.0 * PI3D * u01_words(o1[0], o1[1]);
        double mu = 2.0 * u01_words(o1[2], o1[3]) - 1.0;
        double sn = sqrt(1.0 - mu * mu);
        dir[3 * m + 0] = sn * cos(az);
        dir[3 * m + 1] = sn * sin(az);
        dir[3 * m + 2] = mu;
    }
}

void oracle3d_force_field(int nx, int ny, int nz, int kmin, int kmax, double amp, uint64_t seed, uint64_t epoch,
                          double *Fx, double *Fy, double *Fz)
{
    int nm = oracle3d_forcing_modes(kmin, kmax, NULL, NULL, NULL, 0);
    int cap = nm > 0 ? nm : 1;
    int *kx = (int *)malloc(sizeof(int) * cap), *ky = (int *)malloc(sizeof(int) * cap),
        *kz = (int *)malloc(sizeof(int) * cap);
    double *mag = (double *)malloc(sizeof(double) * cap), *ph = (double *)malloc(sizeof(double) * cap),
           *dir = (double *)malloc(sizeof(double) * 3 * cap);
    oracle3d_forcing_modes(kmin, kmax, kx, ky, kz, nm);
    oracle3d_forcing_draw(kmin, kmax, amp, seed, epoch, mag, ph, dir);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double f[3] = {0.0, 0.0, 0.0};
                for (int m = 0; m < nm; ++m) {
                    double arg = 2.0 * PI3D *
                                     ((double)wrap3((long)kx[m] * x, nx) / nx + (double)wrap3((long)ky[m] * y, ny) / ny +
                                      (double)wrap3((long)kz[m] * z, nz) / nz) +
                                 ph[m];
                    double c = 2.0 * mag[m] * cos(arg);
                    for (int a = 0; a < 3; ++a) f[a] += c * dir[3 * m + a];
                }
                size_t n = ((size_t)z * ny + y) * nx + x;
                Fx[n] = f[0];
                Fy[n] = f[1];
                Fz[n] = f[2];
            }
    free(kx);
    free(ky);
    free(kz);
    free(mag);
    free(ph);
    free(dir);
}

/* One step: stream f into tmp, collide every node of tmp (force may be
 * NULL), store the post-collision state in f.  Returns the number of nodes
 * whose Landau solve failed. */
int oracle3d_step(double *f, double *tmp, int nx, int ny, int nz, double tau, const double *Fx, const double *Fy,
                  const double *Fz)
{
    build3();
    size_t vol = (size_t)nx * ny * nz;
    oracle3d_stream(f, tmp, nx, ny, nz);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long n = 0; n < (long)vol; ++n) {
        double node[N3DIR];
        for (int i = 0; i < N3DIR; ++i) node[i] = tmp[(size_t)i * vol + n];
        double F[3] = {Fx ? Fx[n] : 0.0, Fy ? Fy[n] : 0.0, Fz ? Fz[n] : 0.0};
        if (oracle_collide_node(node, F, tau, NULL, NULL) != 0) bad += 1;
        for (int i = 0; i < N3DIR; ++i) f[(size_t)i * vol + n] = node[i];
    }
    return bad;
}

/* Fields the next collision sees: stream into tmp, then per node the moments
 * and the Landau frame; eps and v = u^i/u^0.  Outputs may be NULL. */
int oracle3d_fields(const double *f, double *tmp, int nx, int ny, int nz, double *eps, double *vx, double *vy,
                    double *vz)
{
    build3();
    size_t vol = (size_t)nx * ny * nz;
    oracle3d_stream(f, tmp, nx, ny, nz);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long n = 0; n < (long)vol; ++n) {
        double node[N3DIR], T[16], e, u[4];
        for (int i = 0; i < N3DIR; ++i) node[i] = tmp[(size_t)i * vol + n];
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
        if (vz) vz[n] = u[3] / u[0];
    }
    return bad;
}

/* nsteps steps from global step step0, the force redrawn every `redraw`
 * steps (amp = 0 or kmax <= 0: unforced).  tmp: 26*vol, Fx/Fy/Fz: vol each. */
int oracle3d_run(double *f, double *tmp, double *Fx, double *Fy, double *Fz, int nx, int ny, int nz, double tau,
                 long step0, int nsteps, int kmin, int kmax, double amp, uint64_t seed, int redraw)
{
    int forced = (amp > 0.0 && kmax > 0);
    long cur_epoch = -1;
    int bad = 0;
    for (int s = 0; s < nsteps; ++s) {
        long step = step0 + s;
        if (forced) {
            long e = redraw > 0 ? step / redraw : 0;
            if (e != cur_epoch) {
                oracle3d_force_field(nx, ny, nz, kmin, kmax, amp, seed, (uint64_t)e, Fx, Fy, Fz);
                cur_epoch = e;
            }
        }
        bad += oracle3d_step(f, tmp, nx, ny, nz, tau, forced ? Fx : NULL, forced ? Fy : NULL, forced ? Fz : NULL);
    }
    return bad;
}

/* Sum over nodes of T^{0 mu}, mu = 0..3 (node order [z][y][x]). */
void oracle3d_totals(const double *f, int nx, int ny, int nz, double *out)
{
    build3();
    size_t vol = (size_t)nx * ny * nz;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t n = 0; n < vol; ++n)
        for (int i = 0; i < N3DIR; ++i) {
            double fi = f[(size_t)i * vol + n];
            acc[0] += fi;
            acc[1] += fi * s_v[i][0];
            acc[2] += fi * s_v[i][1];
            acc[3] += fi * s_v[i][2];
        }
    for (int m = 0; m < 4; ++m) out[m] = acc[m];
}

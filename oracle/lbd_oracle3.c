/*
 * lbd_oracle3.c -- plain FP64 CPU oracle of the coupled lattice-Boltzmann /
 * finite-difference step of arXiv 1711.10984 (Section 2) extended to three
 * dimensions, the extension the paper's conclusions call desirable.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests and the CPU leg of the
 * benchmark, never by the product path; it shares no code with the CUDA
 * sources.  Same style and compiler flags as lbd_oracle.c (per-site loops,
 * one pass per operator, -O2 -ffp-contract=off).
 *
 * Readings (the paper is two-dimensional; this is the same scheme on the
 * D3Q19 lattice, every 2D reading kept):
 *   - D3Q19 velocities: rest; the 6 axis links (weight 1/18); the 12 edge
 *     diagonals (+-1, +-1, 0) etc. (weight 1/36); rest weight 1/3; c_s^2 = 1/3.
 *   - Eq. (12) with the same second-order expansion, Guo forcing as in 2D.
 *   - Isotropic stencils with the D3Q19 weights:
 *       d_a g = 3 sum_i w_i e_ia g(x + e_i),  lap g = 6 sum_i w_i (g(x + e_i) - g(x)),
 *     and the surfactant divergence in the same link form as in 2D.
 *   - Conservative donor-cell advection over the 6 faces of the cell.
 *   - Source disks become balls (x, y, z, R), inclusive, periodic minimum image.
 *   - Body force and frozen velocity carry a z component (fz, uz0).
 * With fields independent of z and u_z = 0 the D3Q19 weights summed over e_z
 * are the D2Q9 weights, and this step reduces to the 2D one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC3_FROZEN_U 1u
#define ORC3_BODY_FORCE 2u

typedef struct {
    int32_t nx, ny, nz;
    double a, b, B0, B1, M, D, tau, gamma, c0, A0, A_max;
    int64_t t_on;
    int32_t n_src, flags;
    const double *src; /* n_src quadruples (x, y, z, R) */
    double fx, fy, fz, ux0, uy0, uz0;
} orc3_params;

enum { Q = 19 };
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W[Q] = {1.0 / 3, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
static size_t nsites(const orc3_params *p) { return (size_t)p->nx * p->ny * p->nz; }
static size_t site(const orc3_params *p, int x, int y, int z) {
    return ((size_t)wrap(z, p->nz) * p->ny + wrap(y, p->ny)) * p->nx + wrap(x, p->nx);
}
static double *alloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

void orc3_grad(const orc3_params *p, const double *g, double *gx, double *gy, double *gz) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double sx = 0, sy = 0, sz = 0;
                for (int i = 1; i < Q; ++i) {
                    double v = g[site(p, x + EX[i], y + EY[i], z + EZ[i])];
                    sx += W[i] * EX[i] * v;
                    sy += W[i] * EY[i] * v;
                    sz += W[i] * EZ[i] * v;
                }
                size_t s = site(p, x, y, z);
                gx[s] = 3.0 * sx;
                gy[s] = 3.0 * sy;
                gz[s] = 3.0 * sz;
            }
}

void orc3_lap(const orc3_params *p, const double *g, double *out) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                double s0 = 0;
                for (int i = 1; i < Q; ++i)
                    s0 += W[i] * (g[site(p, x + EX[i], y + EY[i], z + EZ[i])] - g[s]);
                out[s] = 6.0 * s0;
            }
}

/* mu_phi (Eq. 3) with the cubic from phi3src, and m = (B1/2)|grad phi|^2 (Eq. 5). */
static void chem(const orc3_params *p, const double *phi, const double *phi3src, const double *c,
                 double *mu, double *m) {
    size_t n = nsites(p);
    double *px = alloc(n), *py = alloc(n), *pz = alloc(n), *lp = alloc(n);
    double *cx = alloc(n), *cy = alloc(n), *cz = alloc(n);
    orc3_grad(p, phi, px, py, pz);
    orc3_lap(p, phi, lp);
    orc3_grad(p, c, cx, cy, cz);
    for (size_t s = 0; s < n; ++s) {
        double B = p->B0 + p->B1 * c[s];
        double f3 = phi3src[s] * phi3src[s] * phi3src[s];
        mu[s] = p->a * phi[s] + p->b * f3 - B * lp[s] -
                p->B1 * (px[s] * cx[s] + py[s] * cy[s] + pz[s] * cz[s]);
        m[s] = 0.5 * p->B1 * (px[s] * px[s] + py[s] * py[s] + pz[s] * pz[s]);
    }
    free(px); free(py); free(pz); free(lp); free(cx); free(cy); free(cz);
}

/* Eq. (14): F = -phi grad mu_phi - (grad c + c grad m), plus the body force. */
void orc3_force(const orc3_params *p, const double *phi, const double *c, double *F /* 3n */) {
    size_t n = nsites(p);
    double *mu = alloc(n), *m = alloc(n);
    double *mx = alloc(n), *my = alloc(n), *mz = alloc(n);
    double *nx_ = alloc(n), *ny_ = alloc(n), *nz_ = alloc(n);
    double *cx = alloc(n), *cy = alloc(n), *cz = alloc(n);
    chem(p, phi, phi, c, mu, m);
    orc3_grad(p, mu, mx, my, mz);
    orc3_grad(p, m, nx_, ny_, nz_);
    orc3_grad(p, c, cx, cy, cz);
    int body = (p->flags & ORC3_BODY_FORCE) != 0;
    for (size_t s = 0; s < n; ++s) {
        F[s] = -phi[s] * mx[s] - (cx[s] + c[s] * nx_[s]) + (body ? p->fx : 0.0);
        F[n + s] = -phi[s] * my[s] - (cy[s] + c[s] * ny_[s]) + (body ? p->fy : 0.0);
        F[2 * n + s] = -phi[s] * mz[s] - (cz[s] + c[s] * nz_[s]) + (body ? p->fz : 0.0);
    }
    free(mu); free(m); free(mx); free(my); free(mz); free(nx_); free(ny_); free(nz_);
    free(cx); free(cy); free(cz);
}

/* Eq. (12) on D3Q19. */
void orc3_equilibrium(double n, double ux, double uy, double uz, double feq[Q]) {
    double usq = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < Q; ++i) {
        double eu = EX[i] * ux + EY[i] * uy + EZ[i] * uz;
        feq[i] = W[i] * n * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
    }
}

/* Guo forcing term of Eq. (10) on D3Q19. */
void orc3_guo(double tau, double ux, double uy, double uz, double Fx, double Fy, double Fz,
              double Fi[Q]) {
    for (int i = 0; i < Q; ++i) {
        double eu = EX[i] * ux + EY[i] * uy + EZ[i] * uz;
        double t = 3.0 * ((EX[i] - ux) * Fx + (EY[i] - uy) * Fy + (EZ[i] - uz) * Fz) +
                   9.0 * eu * (EX[i] * Fx + EY[i] * Fy + EZ[i] * Fz);
        Fi[i] = (1.0 - 0.5 / tau) * W[i] * t;
    }
}

/* Eq. (11): n and u = (sum f e + F/2) / n. */
static void moments(const orc3_params *p, const double *f, const double *F, double *n,
                    double *u /* 3N */) {
    size_t N = nsites(p);
    for (size_t s = 0; s < N; ++s) {
        double r = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < Q; ++i) {
            double fi = f[(size_t)i * N + s];
            r += fi; jx += fi * EX[i]; jy += fi * EY[i]; jz += fi * EZ[i];
        }
        n[s] = r;
        u[s] = (jx + 0.5 * F[s]) / r;
        u[N + s] = (jy + 0.5 * F[N + s]) / r;
        u[2 * N + s] = (jz + 0.5 * F[2 * N + s]) / r;
    }
}

static void collide_stream(const orc3_params *p, double *f, const double *F, const double *n,
                           const double *u) {
    size_t N = nsites(p);
    double *fn = alloc((size_t)Q * N);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                double feq[Q], Fi[Q];
                orc3_equilibrium(n[s], u[s], u[N + s], u[2 * N + s], feq);
                orc3_guo(p->tau, u[s], u[N + s], u[2 * N + s], F[s], F[N + s], F[2 * N + s], Fi);
                for (int i = 0; i < Q; ++i) {
                    double fi = f[(size_t)i * N + s];
                    fn[(size_t)i * N + site(p, x + EX[i], y + EY[i], z + EZ[i])] =
                        fi - (fi - feq[i]) / p->tau + Fi[i];
                }
            }
    memcpy(f, fn, (size_t)Q * N * sizeof(double));
    free(fn);
}

/* Eqs. (16)-(17): g* = g - div(g u), donor-cell fluxes on the 6 faces. */
static void advect(const orc3_params *p, const double *g, const double *u, double *out) {
    size_t N = nsites(p);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                double net = 0;
                for (int a = 0; a < 3; ++a) {
                    int dx = a == 0, dy = a == 1, dz = a == 2;
                    size_t up = site(p, x + dx, y + dy, z + dz), dn = site(p, x - dx, y - dy, z - dz);
                    const double *ua = u + (size_t)a * N;
                    double fp = 0.5 * (ua[s] + ua[up]), fm = 0.5 * (ua[dn] + ua[s]);
                    double out_f = fp * (fp > 0 ? g[s] : g[up]);
                    double in_f = fm * (fm > 0 ? g[dn] : g[s]);
                    net += out_f - in_f;
                }
                out[s] = g[s] - net;
            }
}

static int in_source(const orc3_params *p, int x, int y, int z) {
    for (int k = 0; k < p->n_src; ++k) {
        const double *q = p->src + 4 * k;
        double d[3] = {x - q[0], y - q[1], z - q[2]};
        int L[3] = {p->nx, p->ny, p->nz};
        for (int a = 0; a < 3; ++a) {
            while (d[a] > 0.5 * L[a]) d[a] -= L[a];
            while (d[a] < -0.5 * L[a]) d[a] += L[a];
        }
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= q[3] * q[3]) return 1;
    }
    return 0;
}

void orc3_activity(const orc3_params *p, int64_t t, double *A, double *gamma) {
    if (t < p->t_on) { *A = 0.0; *gamma = 0.0; return; }
    double a = p->A0 * (double)(t - p->t_on);
    *A = a < p->A_max ? a : p->A_max;
    *gamma = p->gamma;
}

void orc3_step(const orc3_params *p, double *f, double *phi, double *c, int64_t t) {
    size_t N = nsites(p);
    double *F = alloc(3 * N), *n = alloc(N), *u = alloc(3 * N);
    double *phs = alloc(N), *cs = alloc(N), *mu = alloc(N), *m = alloc(N), *lmu = alloc(N);
    double A, gamma;
    orc3_activity(p, t, &A, &gamma);
    orc3_force(p, phi, c, F);
    moments(p, f, F, n, u);
    collide_stream(p, f, F, n, u);
    if (p->flags & ORC3_FROZEN_U)
        for (size_t s = 0; s < N; ++s) { u[s] = p->ux0; u[N + s] = p->uy0; u[2 * N + s] = p->uz0; }
    advect(p, phi, u, phs);
    advect(p, c, u, cs);
    /* Eq. (19) + source and sink, link form of the divergence */
    chem(p, phs, phs, cs, mu, m);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                double div = 0;
                for (int i = 1; i < Q; ++i) {
                    size_t j = site(p, x + EX[i], y + EY[i], z + EZ[i]);
                    div += 6.0 * W[i] * ((cs[j] - cs[s]) + 0.5 * (cs[s] + cs[j]) * (m[j] - m[s]));
                }
                double src = in_source(p, x, y, z) ? A : 0.0;
                c[s] = cs[s] + (p->D * div - gamma * (cs[s] - p->c0) + src);
            }
    /* Eq. (18), cubic from phi^n */
    chem(p, phs, phi, cs, mu, m);
    orc3_lap(p, mu, lmu);
    for (size_t s = 0; s < N; ++s) phi[s] = phs[s] + p->M * lmu[s];
    free(F); free(n); free(u); free(phs); free(cs); free(mu); free(m); free(lmu);
}

void orc3_run(const orc3_params *p, double *f, double *phi, double *c, int64_t t0, int64_t nsteps) {
    for (int64_t k = 0; k < nsteps; ++k) orc3_step(p, f, phi, c, t0 + k);
}

void orc3_init_equilibrium(const orc3_params *p, const double *rho, const double *ux,
                           const double *uy, const double *uz, double *f) {
    size_t N = nsites(p);
    for (size_t s = 0; s < N; ++s) {
        double feq[Q];
        orc3_equilibrium(rho[s], ux[s], uy[s], uz[s], feq);
        for (int i = 0; i < Q; ++i) f[(size_t)i * N + s] = feq[i];
    }
}

/* rho, u (Eq. 11 with the force of the current phi, c) */
void orc3_fields(const orc3_params *p, const double *f, const double *phi, const double *c,
                 double *rho, double *u /* 3N */) {
    size_t N = nsites(p);
    double *F = alloc(3 * N);
    orc3_force(p, phi, c, F);
    moments(p, f, F, rho, u);
    free(F);
}

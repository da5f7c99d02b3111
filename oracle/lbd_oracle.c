/*
 * lbd_oracle.c -- plain FP64 CPU oracle of the coupled hybrid lattice-Boltzmann /
 * finite-difference time step of Fadda, Gonnella, Lamura & Tiribocchi,
 * "Lattice Boltzmann study of chemically-driven self-propelled droplets"
 * (arXiv 1711.10984), Section 2.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library against
 * the paper.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never calls it.  It shares no code,
 * header, table or helper with the CUDA sources.
 *
 * Style: per-site loops over a periodic nx*ny lattice, site (x,y) at y*nx+x,
 * every operator a separate pass with its own temporary arrays, in the order the
 * paper states the scheme.  Compiled with -O2 -ffp-contract=off so that the
 * arithmetic is the plain IEEE sequence written here.  OpenMP only splits the
 * row loops; every site's arithmetic is independent of the thread count.
 *
 * Readings of the paper that this file takes (the paper is silent or garbled):
 *   - Eq. (12): the quadratic term carries the usual factor 1/2, i.e.
 *     uu:(ee - cs^2 I)/(2 cs^4); without it the second moment is wrong.
 *   - Eqs. (2), (18): a phi mobility M multiplies the Laplacian of mu_phi
 *     (the paper's runs use M = 1).
 *   - Eqs. (16)-(17): the advection half step is taken in conservative
 *     donor-cell flux form over the four axis faces, with the face velocity
 *     the mean of the two site velocities (ORC_LITERAL_ADVECTION keeps the
 *     printed product-rule form: centred grad u, upwind grad phi).
 *   - Eqs. (5), (14), (19): the log term of mu_c enters only through
 *     c grad(ln c) = grad c, so c grad mu_c = grad c + c grad m and
 *     Dc grad mu_c = D grad c + D c grad m, with m = (B1/2)|grad phi|^2
 *     (ORC_LITERAL_LOG evaluates ln c + 1 + m and differentiates it).
 *   - "Centred scheme": the isotropic D2Q9 stencils
 *     d_a g = 3 sum_i w_i e_ia g(x+e_i),  lap g = 6 sum_i w_i (g(x+e_i)-g(x)),
 *     and div(k grad g) = 6 sum_i w_i k_ij (g_j - g_x), k_ij = (k_x+k_j)/2.
 *   - Order within one step: force from phi^n, c^n; LB moments and collision
 *     with that force (giving u^n); advection with u^n; then the diffusion
 *     steps, both reading phi*, c* (and phi^n for the cubic, as printed).
 *   - Source Theta(R - |r - r_P|) is inclusive and uses the periodic minimum
 *     image; several source disks combine as a union.
 *   - Activity schedule: for t < t_on, A = gamma = 0; afterwards gamma is on
 *     and A(t) = min(A0 (t - t_on), A_max)  (Section 4: A = A0 t, then held).
 *   - Walls (ORC_WALLS; Section 2.2 refers them to another paper, Section 2.3
 *     asks for n.grad mu_phi = n.grad mu_c = 0): two resting plates at
 *     y = -1/2 and y = ny - 1/2, x stays periodic.  LB: halfway bounce-back, a
 *     population that would stream through a plate returns to its own site
 *     reversed, f_i(x, t+1) = f*_{-i}(x, t).  FD: every stencil sees the fields
 *     mirrored across each plate (row -1-k is row k, row ny+k is row ny-1-k),
 *     so mu_phi, mu_c (and phi, c) have zero normal derivative there; the
 *     advective flux through a plate face is zero.  Source disks do not wrap
 *     through the plates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FROZEN_U          1u   /* advection uses the uniform velocity (ux0, uy0) */
#define ORC_BODY_FORCE        2u   /* add the constant body force (fx, fy) to F      */
#define ORC_LITERAL_ADVECTION 4u   /* product-rule advection exactly as printed      */
#define ORC_LITERAL_LOG       8u   /* differentiate ln c + 1 + m numerically         */
#define ORC_WALLS            16u   /* plates at y = -1/2 and y = ny - 1/2            */

typedef struct {
    int32_t nx, ny;
    double a, b, B0, B1;      /* f_GL = a/2 phi^2 + b/4 phi^4;  B(c) = B0 + B1 c     */
    double M, D, tau;         /* phi mobility, surfactant diffusion L(c)=Dc, BGK tau */
    double gamma, c0;         /* sink -gamma (c - c0)                               */
    double A0, A_max;         /* source strength schedule                           */
    int64_t t_on;             /* activation time of source and sink                 */
    int32_t n_src;            /* number of source disks                             */
    int32_t flags;
    const double *src;        /* n_src triples (x, y, R)                            */
    double fx, fy;            /* body force (ORC_BODY_FORCE)                        */
    double ux0, uy0;          /* frozen advection velocity (ORC_FROZEN_U)           */
} orc_params;

/* D2Q9 lattice of Section 2.2: rest, four axis links, four diagonal links. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = e^2/3 with e = 1 */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6}; /* e_OPP[i] = -e_i */

/* periodic index for v in [-n, 2n): every stencil offset here is -1, 0 or +1 */
static int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
/* row seen by a stencil: periodic, or mirrored across the plates with walls */
static int row(const orc_params *p, int y) {
    if (!(p->flags & ORC_WALLS)) return wrap(y, p->ny);
    return y < 0 ? -1 - y : (y >= p->ny ? 2 * p->ny - 1 - y : y);
}
static size_t site(const orc_params *p, int x, int y) {
    return (size_t)row(p, y) * (size_t)p->nx + (size_t)wrap(x, p->nx);
}
static size_t nsites(const orc_params *p) { return (size_t)p->nx * (size_t)p->ny; }
static double *alloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* ---- isotropic finite-difference stencils ("centred scheme", Section 2.3) ---- */

void orc_grad(const orc_params *p, const double *g, double *gx, double *gy) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double sx = 0, sy = 0;
            for (int i = 1; i < 9; ++i) {
                double v = g[site(p, x + EX[i], y + EY[i])];
                sx += W[i] * EX[i] * v;
                sy += W[i] * EY[i] * v;
            }
            gx[site(p, x, y)] = 3.0 * sx;
            gy[site(p, x, y)] = 3.0 * sy;
        }
}

void orc_lap(const orc_params *p, const double *g, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double g0 = g[site(p, x, y)], s = 0;
            for (int i = 1; i < 9; ++i) s += W[i] * (g[site(p, x + EX[i], y + EY[i])] - g0);
            out[site(p, x, y)] = 6.0 * s;
        }
}

/* ---- thermodynamics, Section 2.1 ---- */

/* Eq. (3): mu_phi = a phi + b phi^3 - B(c) lap phi - B1 grad phi . grad c, with the
 * cubic taken from phi3src (phi itself at time n; phi^n in the second FD step).
 * m = (B1/2)|grad phi|^2 is the gradient part of mu_c, Eq. (5). */
static void chem_potentials(const orc_params *p, const double *phi, const double *phi3src,
                            const double *c, double *mu, double *m) {
    size_t n = nsites(p);
    double *px = alloc(n), *py = alloc(n), *lp = alloc(n), *cx = alloc(n), *cy = alloc(n);
    orc_grad(p, phi, px, py);
    orc_lap(p, phi, lp);
    orc_grad(p, c, cx, cy);
    for (size_t s = 0; s < n; ++s) {
        double B = p->B0 + p->B1 * c[s];
        double f3 = phi3src[s] * phi3src[s] * phi3src[s];
        mu[s] = p->a * phi[s] + p->b * f3 - B * lp[s] - p->B1 * (px[s] * cx[s] + py[s] * cy[s]);
        m[s] = 0.5 * p->B1 * (px[s] * px[s] + py[s] * py[s]);
    }
    free(px); free(py); free(lp); free(cx); free(cy);
}

/* Eq. (14): F = -phi grad mu_phi - c grad mu_c at time n. */
void orc_force(const orc_params *p, const double *phi, const double *c, double *Fx, double *Fy) {
    size_t n = nsites(p);
    double *mu = alloc(n), *m = alloc(n);
    double *gmx = alloc(n), *gmy = alloc(n), *gcx = alloc(n), *gcy = alloc(n);
    chem_potentials(p, phi, phi, c, mu, m);
    orc_grad(p, mu, gmx, gmy);
    for (size_t s = 0; s < n; ++s) { Fx[s] = -phi[s] * gmx[s]; Fy[s] = -phi[s] * gmy[s]; }
    if (p->flags & ORC_LITERAL_LOG) {
        double *muc = alloc(n);
        for (size_t s = 0; s < n; ++s) muc[s] = log(c[s]) + 1.0 + m[s];
        orc_grad(p, muc, gcx, gcy);
        for (size_t s = 0; s < n; ++s) { Fx[s] -= c[s] * gcx[s]; Fy[s] -= c[s] * gcy[s]; }
        free(muc);
    } else {
        double *gnx = alloc(n), *gny = alloc(n);
        orc_grad(p, c, gcx, gcy);
        orc_grad(p, m, gnx, gny);
        for (size_t s = 0; s < n; ++s) {
            Fx[s] -= gcx[s] + c[s] * gnx[s];
            Fy[s] -= gcy[s] + c[s] * gny[s];
        }
        free(gnx); free(gny);
    }
    if (p->flags & ORC_BODY_FORCE)
        for (size_t s = 0; s < n; ++s) { Fx[s] += p->fx; Fy[s] += p->fy; }
    free(mu); free(m); free(gmx); free(gmy); free(gcx); free(gcy);
}

/* ---- lattice Boltzmann, Section 2.2 ---- */

/* Eq. (12), second-order Maxwell-Boltzmann expansion (with the factor 1/2). */
void orc_equilibrium(double n, double ux, double uy, double feq[9]) {
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double uu = ux * ux + uy * uy;
        double quad = (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2);
        feq[i] = W[i] * n * (1.0 + eu / CS2 + quad);
    }
}

/* Eq. (13), Guo forcing with Delta t = 1. */
void orc_guo(double tau, double ux, double uy, double Fx, double Fy, double Fi[9]) {
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double vx = (EX[i] - ux) / CS2 + eu * EX[i] / (CS2 * CS2);
        double vy = (EY[i] - uy) / CS2 + eu * EY[i] / (CS2 * CS2);
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * W[i] * (vx * Fx + vy * Fy);
    }
}

/* Eq. (11): n = sum f, n u = sum f e + F/2. */
void orc_moments(const orc_params *p, const double *f, const double *Fx, const double *Fy,
                 double *n, double *ux, double *uy) {
    size_t N = nsites(p);
    for (size_t s = 0; s < N; ++s) {
        double rho = 0, jx = 0, jy = 0;
        for (int i = 0; i < 9; ++i) {
            double fi = f[(size_t)i * N + s];
            rho += fi; jx += fi * EX[i]; jy += fi * EY[i];
        }
        n[s] = rho;
        ux[s] = (jx + 0.5 * Fx[s]) / rho;
        uy[s] = (jy + 0.5 * Fy[s]) / rho;
    }
}

/* Eq. (10): BGK collision with forcing, then streaming f_i(r + e_i, t + 1). */
static void lb_collide_stream(const orc_params *p, double *f, const double *Fx, const double *Fy,
                              const double *ux, const double *uy, const double *n) {
    size_t N = nsites(p);
    double *fnew = alloc(9 * N);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t s = site(p, x, y);
            double feq[9], Fi[9];
            orc_equilibrium(n[s], ux[s], uy[s], feq);
            orc_guo(p->tau, ux[s], uy[s], Fx[s], Fy[s], Fi);
            for (int i = 0; i < 9; ++i) {
                double fi = f[(size_t)i * N + s];
                double post = fi - (fi - feq[i]) / p->tau + Fi[i];
                int yd = y + EY[i];
                if ((p->flags & ORC_WALLS) && (yd < 0 || yd >= p->ny))
                    fnew[(size_t)OPP[i] * N + s] = post;   /* bounce-back at a plate */
                else
                    fnew[(size_t)i * N + site(p, x + EX[i], yd)] = post;
            }
        }
    memcpy(f, fnew, 9 * N * sizeof(double));
    free(fnew);
}

/* ---- finite differences, Section 2.3 ---- */

/* First FD step, Eqs. (16)-(17): g* = g - div(g u), conservative donor-cell
 * fluxes through the four axis faces (reading listed at the top of the file). */
static void advect(const orc_params *p, const double *g, const double *ux, const double *uy,
                   double *out) {
    if (p->flags & ORC_LITERAL_ADVECTION) {
        size_t n = nsites(p);
        double *dxux = alloc(n), *tmp = alloc(n), *dyuy = alloc(n);
        orc_grad(p, ux, dxux, tmp);
        orc_grad(p, uy, tmp, dyuy);
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y);
                double u = ux[s], v = uy[s];
                double gxu = u > 0 ? g[s] - g[site(p, x - 1, y)] : g[site(p, x + 1, y)] - g[s];
                double gyu = v > 0 ? g[s] - g[site(p, x, y - 1)] : g[site(p, x, y + 1)] - g[s];
                out[s] = g[s] - (g[s] * (dxux[s] + dyuy[s]) + u * gxu + v * gyu);
            }
        free(dxux); free(tmp); free(dyuy);
        return;
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t s = site(p, x, y);
            /* face between sites l (left/below) and r: flux = u_f * g_upwind */
            double flux[4];
            int lx[4] = {x, x - 1, x, x}, ly[4] = {y, y, y, y - 1};
            int rx[4] = {x + 1, x, x, x}, ry[4] = {y, y, y + 1, y};
            for (int k = 0; k < 4; ++k) {
                size_t l = site(p, lx[k], ly[k]), r = site(p, rx[k], ry[k]);
                double uf = (k < 2) ? 0.5 * (ux[l] + ux[r]) : 0.5 * (uy[l] + uy[r]);
                flux[k] = uf * (uf > 0 ? g[l] : g[r]);
                /* no flux through a plate: north face of the top row, south of row 0 */
                if ((p->flags & ORC_WALLS) && ((k == 2 && y == p->ny - 1) || (k == 3 && y == 0)))
                    flux[k] = 0.0;
            }
            /* east - west + north - south */
            out[s] = g[s] - ((flux[0] - flux[1]) + (flux[2] - flux[3]));
        }
}

static int in_source(const orc_params *p, int x, int y) {
    for (int k = 0; k < p->n_src; ++k) {
        double dx = x - p->src[3 * k], dy = y - p->src[3 * k + 1], R = p->src[3 * k + 2];
        while (dx > 0.5 * p->nx) dx -= p->nx;
        while (dx < -0.5 * p->nx) dx += p->nx;
        if (!(p->flags & ORC_WALLS)) {
            while (dy > 0.5 * p->ny) dy -= p->ny;
            while (dy < -0.5 * p->ny) dy += p->ny;
        }
        if (dx * dx + dy * dy <= R * R) return 1;
    }
    return 0;
}

/* Source strength and sink rate in force at step t (Section 4 schedule). */
void orc_activity(const orc_params *p, int64_t t, double *A, double *gamma) {
    if (t < p->t_on) { *A = 0.0; *gamma = 0.0; return; }
    double a = p->A0 * (double)(t - p->t_on);
    *A = a < p->A_max ? a : p->A_max;
    *gamma = p->gamma;
}

/* Second FD step for phi, Eq. (18) with mobility M. */
static void phi_diffuse(const orc_params *p, const double *phs, const double *cs,
                        const double *phin, double *out) {
    size_t n = nsites(p);
    double *mu = alloc(n), *m = alloc(n), *lmu = alloc(n);
    chem_potentials(p, phs, phin, cs, mu, m);
    orc_lap(p, mu, lmu);
    for (size_t s = 0; s < n; ++s) out[s] = phs[s] + p->M * lmu[s];
    free(mu); free(m); free(lmu);
}

/* Second FD step for c, Eq. (19) plus the source and sink of Section 2.1. */
static void c_diffuse(const orc_params *p, const double *phs, const double *cs, double A,
                      double gamma, double *out) {
    size_t n = nsites(p);
    double *mu = alloc(n), *m = alloc(n);
    chem_potentials(p, phs, phs, cs, mu, m);
    if (p->flags & ORC_LITERAL_LOG)
        for (size_t s = 0; s < n; ++s) m[s] = log(cs[s]) + 1.0 + m[s];
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t s = site(p, x, y);
            double div = 0;
            for (int i = 1; i < 9; ++i) {
                size_t j = site(p, x + EX[i], y + EY[i]);
                double kf = 0.5 * (cs[s] + cs[j]);
                double term = (p->flags & ORC_LITERAL_LOG)
                                  ? kf * (m[j] - m[s])
                                  : (cs[j] - cs[s]) + kf * (m[j] - m[s]);
                div += 6.0 * W[i] * term;
            }
            double src = in_source(p, x, y) ? A : 0.0;
            out[s] = cs[s] + (p->D * div - gamma * (cs[s] - p->c0) + src);
        }
    free(mu); free(m);
}

/* One coupled time step n -> n+1.  f holds the pre-collision populations
 * f_i(r, t^n) (9 planes of nx*ny); phi, c are phi^n, c^n; all updated in place. */
void orc_step(const orc_params *p, double *f, double *phi, double *c, int64_t t) {
    size_t n = nsites(p);
    double *Fx = alloc(n), *Fy = alloc(n), *rho = alloc(n), *ux = alloc(n), *uy = alloc(n);
    double *phs = alloc(n), *cs = alloc(n);
    double A, gamma;
    orc_activity(p, t, &A, &gamma);

    orc_force(p, phi, c, Fx, Fy);                    /* Eq. (14) at time n     */
    orc_moments(p, f, Fx, Fy, rho, ux, uy);          /* Eq. (11)               */
    lb_collide_stream(p, f, Fx, Fy, ux, uy, rho);    /* Eqs. (10), (12), (13)  */

    if (p->flags & ORC_FROZEN_U)
        for (size_t s = 0; s < n; ++s) { ux[s] = p->ux0; uy[s] = p->uy0; }
    advect(p, phi, ux, uy, phs);                     /* Eq. (16)               */
    advect(p, c, ux, uy, cs);                        /* Eq. (17)               */
    c_diffuse(p, phs, cs, A, gamma, c);              /* Eq. (19) + activity    */
    phi_diffuse(p, phs, cs, phi, phi);               /* Eq. (18)  (reads phi^n for the cubic first) */

    free(Fx); free(Fy); free(rho); free(ux); free(uy); free(phs); free(cs);
}

void orc_run(const orc_params *p, double *f, double *phi, double *c, int64_t t0, int64_t nsteps) {
    for (int64_t k = 0; k < nsteps; ++k) orc_step(p, f, phi, c, t0 + k);
}

/* Fields at time n: n, u from Eq. (11) with the force of Eq. (14). */
void orc_fields(const orc_params *p, const double *f, const double *phi, const double *c,
                double *rho, double *ux, double *uy) {
    size_t n = nsites(p);
    double *Fx = alloc(n), *Fy = alloc(n);
    orc_force(p, phi, c, Fx, Fy);
    orc_moments(p, f, Fx, Fy, rho, ux, uy);
    free(Fx); free(Fy);
}

/* f_i = f_i^eq(n, u) at every site. */
void orc_init_equilibrium(const orc_params *p, const double *rho, const double *ux,
                          const double *uy, double *f) {
    size_t N = nsites(p);
    for (size_t s = 0; s < N; ++s) {
        double feq[9];
        orc_equilibrium(rho[s], ux[s], uy[s], feq);
        for (int i = 0; i < 9; ++i) f[(size_t)i * N + s] = feq[i];
    }
}

/* Eq. (9): scalar part p0 of the pressure tensor, with p^i = n T and T = c_s^2. */
void orc_pressure(const orc_params *p, const double *rho, const double *phi, const double *c,
                  double *p0) {
    size_t n = nsites(p);
    double *px = alloc(n), *py = alloc(n), *lp = alloc(n), *cx = alloc(n), *cy = alloc(n);
    orc_grad(p, phi, px, py);
    orc_lap(p, phi, lp);
    orc_grad(p, c, cx, cy);
    for (size_t s = 0; s < n; ++s) {
        double ph = phi[s], B = p->B0 + p->B1 * c[s];
        p0[s] = rho[s] * CS2 + 0.5 * p->a * ph * ph + 0.75 * p->b * ph * ph * ph * ph
              - B * ph * lp[s] - p->B1 * ph * (cx[s] * px[s] + cy[s] * py[s]) + c[s]
              - 0.5 * p->B0 * (px[s] * px[s] + py[s] * py[s]);
    }
    free(px); free(py); free(lp); free(cx); free(cy);
}

/* Eq. (1) without the n T ln n term: f_GL + B(c)/2 |grad phi|^2 + c ln c. */
void orc_free_energy(const orc_params *p, const double *phi, const double *c, double *fe) {
    size_t n = nsites(p);
    double *px = alloc(n), *py = alloc(n);
    orc_grad(p, phi, px, py);
    for (size_t s = 0; s < n; ++s) {
        double ph = phi[s], B = p->B0 + p->B1 * c[s];
        fe[s] = 0.5 * p->a * ph * ph + 0.25 * p->b * ph * ph * ph * ph
              + 0.5 * B * (px[s] * px[s] + py[s] * py[s]) + c[s] * log(c[s]);
    }
    free(px); free(py);
}

/* Neumaier-compensated sum. */
static void nsum(double *s, double *comp, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *comp += (*s - t) + v; else *comp += (v - t) + *s;
    *s = t;
}

/* Diagnostics: out[0..2] = sum n, sum phi, sum c; out[3..4] = centre of mass of the
 * phi >= 0 region (Section 4: sum phi r / sum phi over phi >= 0), each site taken at
 * its minimum image relative to (refx, refy); out[5] = min B(c); out[6] = min c;
 * out[7] = number of non-finite values among n, phi, c; out[8] = sum of phi over phi>=0. */
void orc_diagnostics(const orc_params *p, const double *f, const double *phi, const double *c,
                     double refx, double refy, double *out) {
    size_t N = nsites(p);
    double sn = 0, cn = 0, sp = 0, cp = 0, sc = 0, cc = 0;
    double wx = 0, cwx = 0, wy = 0, cwy = 0, w = 0, cw = 0;
    double minB = INFINITY, minc = INFINITY, bad = 0;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t s = (size_t)y * p->nx + x;
            double rho = 0;
            for (int i = 0; i < 9; ++i) rho += f[(size_t)i * N + s];
            if (!isfinite(rho) || !isfinite(phi[s]) || !isfinite(c[s])) bad += 1;
            nsum(&sn, &cn, rho);
            nsum(&sp, &cp, phi[s]);
            nsum(&sc, &cc, c[s]);
            double B = p->B0 + p->B1 * c[s];
            if (B < minB) minB = B;
            if (c[s] < minc) minc = c[s];
            if (phi[s] >= 0) {
                double dx = x - refx, dy = y - refy;
                while (dx >= 0.5 * p->nx) dx -= p->nx;
                while (dx < -0.5 * p->nx) dx += p->nx;
                while (dy >= 0.5 * p->ny) dy -= p->ny;
                while (dy < -0.5 * p->ny) dy += p->ny;
                nsum(&wx, &cwx, phi[s] * dx);
                nsum(&wy, &cwy, phi[s] * dy);
                nsum(&w, &cw, phi[s]);
            }
        }
    double W0 = w + cw;
    out[0] = sn + cn; out[1] = sp + cp; out[2] = sc + cc;
    out[3] = W0 > 0 ? refx + (wx + cwx) / W0 : NAN;
    out[4] = W0 > 0 ? refy + (wy + cwy) / W0 : NAN;
    out[5] = minB; out[6] = minc; out[7] = bad; out[8] = W0;
}

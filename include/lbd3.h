/* lbd3.h -- C ABI of the three-dimensional coupled step: the scheme of
 * arXiv 1711.10984, Section 2 (Eqs. 3, 5, 10-14, 16-19), on the D3Q19 lattice,
 * the extension the paper's conclusions call desirable.
 *
 * The scheme is the 2D one with D3Q19 in place of D2Q9: velocities rest (weight
 * 1/3), the 6 axis links (1/18) and the 12 edge diagonals (1/36) in the order
 *   0 (0,0,0); 1,2 (+-1,0,0); 3,4 (0,+-1,0); 5,6 (0,0,+-1);
 *   7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
 *   13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1);
 * the same equilibrium (second-order expansion) and Guo forcing; isotropic
 * finite differences with the D3Q19 weights (d_a g = 3 sum_i w_i e_ia g(x+e_i),
 * lap g = 6 sum_i w_i (g(x+e_i) - g(x))); conservative donor-cell advection
 * over the 6 faces; the surfactant divergence in link form; source balls.  The
 * lattice is periodic in x, y and z.  With fields independent of z and no z
 * velocity the step reduces exactly to the 2D one.
 *
 * Arrays passed in or out are host arrays of nz*ny*nx doubles, site (x, y, z)
 * at (z*ny + y)*nx + x; populations are 19 such planes.  Error codes and
 * precision constants are those of lbd.h; errors of CUDA calls are sticky.
 */
#ifndef LBD3_H
#define LBD3_H

#include <stdint.h>

#include "lbd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbd3_ctx lbd3_ctx;

typedef struct {
    int32_t nx, ny, nz; /* each in [1, 4096]; 19 * nz * ny * (nx rounded up to 128
                           bytes) < 2^32 elements (512^3 in FP32 and FP64) */
} lbd3_grid;

typedef struct {
    double x, y, z, R; /* source ball Theta(R - |r - r_P|), inclusive, periodic */
} lbd3_source;

typedef struct {
    lbd_params base;   /* model parameters, flags (LBD_FROZEN_U, LBD_BODY_FORCE)
                          and precision as in 2D; base.n_src, base.src ignored */
    double fz, uz0;    /* z components of the body force and the frozen velocity */
    int32_t n_src;     /* number of source balls, [0, LBD_MAX_SOURCES] */
    int32_t reserved;
    lbd3_source src[LBD_MAX_SOURCES];
} lbd3_params;

typedef struct {
    double sum_rho, sum_phi, sum_psi; /* totals over the lattice                 */
    double cm_x, cm_y, cm_z;          /* centre of mass of the phi >= 0 region,
                                         minimum image about the reference      */
    double mass_pos;                  /* sum of phi over phi >= 0                */
    int64_t nonfinite;                /* non-finite values among rho, phi, psi   */
} lbd3_diag;

/* Create a context on the calling thread's current device with the rest state
 * (f = w_i, phi = psi = 0); stream may be NULL (legacy default stream).
 * LBD_EINVAL for bad parameters (including LBD_WALLS, which 3D does not
 * support), LBD_ENOMEM when device memory runs out. */
int lbd3_create(const lbd3_grid *grid, const lbd3_params *params, void *stream, lbd3_ctx **out);
const char *lbd3_last_error(const lbd3_ctx *ctx);
/* Replace the parameters (same precision). */
int lbd3_set_params(lbd3_ctx *ctx, const lbd3_params *params);
/* phi, psi required; rho (default 1) and u (default 0) may be NULL; the
 * populations become f^eq(rho, u) (Eq. 12).  LBD_ENONFINITE for NaN/Inf,
 * LBD_EUNSTABLE for B(psi) <= 0 or psi <= 0, LBD_EINVAL for rho <= 0, for the
 * first such site in index order (nothing is changed then), as in 2D; the
 * arrays are uploaded and checked on the device.  Synchronises. */
int lbd3_set_fields(lbd3_ctx *ctx, const double *rho, const double *ux, const double *uy,
                    const double *uz, const double *phi, const double *psi);
/* Advance by n coupled steps (asynchronous). */
int lbd3_step(lbd3_ctx *ctx, int64_t n);
/* rho, u (Eq. 11 with the force of the current fields), phi, psi; any pointer
 * may be NULL.  Synchronises. */
int lbd3_get_fields(lbd3_ctx *ctx, double *rho, double *ux, double *uy, double *uz,
                    double *phi, double *psi);
/* Pre-collision populations, 19 planes of nz*ny*nx doubles.  Synchronises. */
int lbd3_get_populations(lbd3_ctx *ctx, double *f);
/* Totals and the centre of mass about (ref_x, ref_y, ref_z), which must lie
 * inside the lattice.  Synchronises. */
int lbd3_diagnostics(lbd3_ctx *ctx, double ref_x, double ref_y, double ref_z, lbd3_diag *out);
int lbd3_synchronize(lbd3_ctx *ctx);
int lbd3_get_time(const lbd3_ctx *ctx, int64_t *t);
/* Launch shape of the step: each CTA walks a run of `planes` z planes of a
 * 32 x 8 tile of the xy plane; 0 restores the automatic choice (about sixteen
 * CTAs per SM over the lattice, runs of at least four planes).  Results do not
 * depend on it.  LBD_EINVAL unless 0 <= planes <= nz. */
int lbd3_set_zrun(lbd3_ctx *ctx, int32_t planes);
int lbd3_get_zrun(const lbd3_ctx *ctx, int32_t *planes);
void lbd3_destroy(lbd3_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBD3_H */

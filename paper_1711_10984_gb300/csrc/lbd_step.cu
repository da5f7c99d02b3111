// lbd_step.cu -- fused coupled time step of the hybrid LB/FD droplet model
// (arXiv 1711.10984, Sections 2.1-2.3) for sm_103a.
//
// One CTA owns a BX x BY tile of output sites and recomputes everything the
// tile needs from phi^n, psi^n on a halo of 5 and from the populations on a
// halo of 4, so that one launch is one whole step and each field is read from
// HBM about once (halo re-reads of neighbouring tiles hit L2):
//
//   stage 0  phi^n, psi^n            on R5 (tile + 5)  global -> smem
//   stage A  mu_phi (Eq. 3), m       on R4             m = (B1/2)|grad phi|^2
//   stage B  F (Eq. 14), u (Eq. 11)  on R3             pull f_i(x - e_i);
//            interior sites also collide (Eqs. 10, 12, 13) and store g_i
//   stage C  phi*, psi* (Eqs. 16-17) on R2             donor-cell face fluxes
//   stage D  mu*, m*                 on R1             (phi^n)^3 as printed
//   stage E  phi^{n+1} (Eq. 18), psi^{n+1} (Eq. 19 + source/sink) on the tile
//
// The path is bound by HBM bandwidth (no contraction, so no tensor cores).
#include <cstdint>

#include "lbd_internal.h"

namespace lbd {
namespace {

struct SourceList {
    lbd_source s[LBD_MAX_SOURCES];
};

constexpr int NT = 256;   // threads per CTA
constexpr int HALO = 5;   // phi/psi halo: u on R3 needs F on R3, which needs R5

__device__ __forceinline__ int pmod(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Isotropic D2Q9 stencils on a row-major smem array with row stride S, centred
// on pointer c:  d/dx = (1/3)(E - W) + (1/12)(NE - NW + SE - SW), and
// lap = (2/3)(E + W + N + S - 4 c) + (1/6)(NE + NW + SE + SW - 4 c).
template <typename T, int S>
struct Stencil {
    __device__ __forceinline__ static T dx(const T *c) {
        return (c[1] - c[-1]) * T(1.0 / 3.0) +
               ((c[S + 1] - c[S - 1]) + (c[-S + 1] - c[-S - 1])) * T(1.0 / 12.0);
    }
    __device__ __forceinline__ static T dy(const T *c) {
        return (c[S] - c[-S]) * T(1.0 / 3.0) +
               ((c[S + 1] - c[-S + 1]) + (c[S - 1] - c[-S - 1])) * T(1.0 / 12.0);
    }
    __device__ __forceinline__ static T lap(const T *c) {
        T c0 = c[0];
        T ax = (c[1] - c0) + (c[-1] - c0) + (c[S] - c0) + (c[-S] - c0);
        T dg = (c[S + 1] - c0) + (c[S - 1] - c0) + (c[-S + 1] - c0) + (c[-S - 1] - c0);
        return ax * T(2.0 / 3.0) + dg * T(1.0 / 6.0);
    }
};

// Source indicator Theta(R - |r - r_P|), Section 2.1: inclusive, periodic minimum
// image (in x only when plates bound the lattice in y), union of the disks.  Evaluated once per parameter set (in double, with
// no contraction into FMAs so that the boundary test is the plain IEEE one);
// the step kernel reads one bit per site.
__global__ void theta_mask_kernel(int nx, int ny, int n_src, SourceList src, int wrap_y,
                                  uint32_t *mask) {
    const int words = (nx + 31) / 32;
    const long long total = (long long)words * ny;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(w / words), x0 = (int)(w - (long long)y * words) * 32;
        uint32_t bits = 0;
        for (int b = 0; b < 32 && x0 + b < nx; ++b) {
            for (int k = 0; k < n_src; ++k) {
                double dx = (double)(x0 + b) - src.s[k].x, dy = (double)y - src.s[k].y;
                if (dx > 0.5 * nx) dx -= nx; else if (dx < -0.5 * nx) dx += nx;
                if (wrap_y) {
                    if (dy > 0.5 * ny) dy -= ny; else if (dy < -0.5 * ny) dy += ny;
                }
                if (__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <=
                    __dmul_rn(src.s[k].R, src.s[k].R)) {
                    bits |= 1u << b;
                    break;
                }
            }
        }
        mask[w] = bits;
    }
}

template <typename T, int BX, int BY, int MODE>
__global__ void __launch_bounds__(NT) step_kernel(const StepArgs<T> p) {
    constexpr int W5 = BX + 10, H5 = BY + 10;
    constexpr int W4 = BX + 8, H4 = BY + 8;
    constexpr int W3 = BX + 6, H3 = BY + 6;
    constexpr int W2 = BX + 4, H2 = BY + 4;
    constexpr int W1 = BX + 2, H1 = BY + 2;
    static_assert(BX % 32 == 0, "tile width must be a multiple of the warp");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_phi = reinterpret_cast<T *>(smem_raw);
    T *s_psi = s_phi + W5 * H5;
    T *s_mu = s_psi + W5 * H5;  // R4 in stage A/B, then mu* on R1
    T *s_m = s_mu + W4 * H4;    // R4 in stage A/B, then m* on R1
    T *s_ux = s_m + W4 * H4;    // R3
    T *s_uy = s_ux + W3 * H3;
    T *s_phs = s_uy + W3 * H3;  // R2
    T *s_pss = s_phs + W2 * H2;
    int *s_gx = reinterpret_cast<int *>(s_pss + W2 * H2);  // wrapped x of R5 columns
    int *s_gy = s_gx + W5;                                 // wrapped y of R5 rows

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int nx = p.nx, ny = p.ny;
    const long long pitch = p.pitch;

    for (int k = tid; k < W5; k += NT) s_gx[k] = pmod(x0 - HALO + k, nx);
    // rows beyond a plate are read mirrored (walls: y = -1/2 and ny - 1/2)
    const bool walls = (p.flags & LBD_WALLS) != 0;
    for (int k = tid; k < H5; k += NT) {
        const int y = y0 - HALO + k;
        // (rows past the last tile's halo are never used; clamped to stay in bounds)
        s_gy[k] = !walls ? pmod(y, ny)
                         : min(max(y < 0 ? -1 - y : (y >= ny ? 2 * ny - 1 - y : y), 0), ny - 1);
    }
    __syncthreads();

    // ---- stage 0: phi^n, psi^n on R5 -------------------------------------
    for (int k = tid; k < W5 * H5; k += NT) {
        const int ly = k / W5, lx = k - ly * W5;
        const long long idx = (long long)s_gy[ly] * pitch + s_gx[lx];
        s_phi[k] = p.phi_in[idx];
        s_psi[k] = p.psi_in[idx];
    }
    __syncthreads();

    // ---- stage A: mu_phi (Eq. 3) and m = (B1/2)|grad phi|^2 on R4 --------
    for (int k = tid; k < W4 * H4; k += NT) {
        const int ly = k / W4, lx = k - ly * W4;
        const int c5 = (ly + 1) * W5 + (lx + 1);
        const T *P = s_phi + c5, *C = s_psi + c5;
        const T phx = Stencil<T, W5>::dx(P), phy = Stencil<T, W5>::dy(P);
        const T lph = Stencil<T, W5>::lap(P);
        const T cx = Stencil<T, W5>::dx(C), cy = Stencil<T, W5>::dy(C);
        const T ph = P[0];
        const T B = p.B0 + p.B1 * C[0];
        s_mu[k] = p.a * ph + p.b * (ph * ph * ph) - B * lph - p.B1 * (phx * cx + phy * cy);
        s_m[k] = T(0.5) * p.B1 * (phx * phx + phy * phy);
    }
    __syncthreads();

    // ---- stage B: force, moments, collision --------------------------------
    // Site (lx3, ly3) of R3: smem R4 centre (ly3+1, lx3+1), R5 centre (ly3+2, lx3+2).
    auto site_state = [&](int lx3, int ly3, T g[9], T &Fx, T &Fy, T &dn, T &ux, T &uy) {
        const int c4 = (ly3 + 1) * W4 + (lx3 + 1);
        const int c5 = (ly3 + 2) * W5 + (lx3 + 2);
        const T *MU = s_mu + c4, *Mm = s_m + c4, *C = s_psi + c5;
        const T ph = s_phi[c5], c = C[0];
        // Eq. (14) with psi grad mu_psi = grad psi + psi grad m.
        Fx = -ph * Stencil<T, W4>::dx(MU) - (Stencil<T, W5>::dx(C) + c * Stencil<T, W4>::dx(Mm));
        Fy = -ph * Stencil<T, W4>::dy(MU) - (Stencil<T, W5>::dy(C) + c * Stencil<T, W4>::dy(Mm));
        if (p.flags & LBD_BODY_FORCE) {
            Fx += p.fx;
            Fy += p.fy;
        }
        // Pull f_i(x, n) = buffer_i(x - e_i).
        const int xc = lx3 + 2, yc = ly3 + 2;
        const int gxm = s_gx[xc - 1], gx0 = s_gx[xc], gxp = s_gx[xc + 1];
        const long long rym = (long long)s_gy[yc - 1] * pitch, ry0 = (long long)s_gy[yc] * pitch,
                        ryp = (long long)s_gy[yc + 1] * pitch;
        const T *G = p.g_in;
        const long long P_ = p.plane;
        g[0] = G[ry0 + gx0];
        g[1] = G[P_ + ry0 + gxm];           // e = ( 1, 0) comes from x - 1
        g[2] = G[2 * P_ + rym + gx0];       // e = ( 0, 1) from y - 1
        g[3] = G[3 * P_ + ry0 + gxp];       // e = (-1, 0) from x + 1
        g[4] = G[4 * P_ + ryp + gx0];       // e = ( 0,-1) from y + 1
        g[5] = G[5 * P_ + rym + gxm];       // e = ( 1, 1)
        g[6] = G[6 * P_ + rym + gxp];       // e = (-1, 1)
        g[7] = G[7 * P_ + ryp + gxp];       // e = (-1,-1)
        g[8] = G[8 * P_ + ryp + gxm];       // e = ( 1,-1)
        if (walls) {  // halfway bounce-back: what would come through a plate is
                      // the site's own reversed post-collision population
            const int yr = y0 - HALO + yc;
            if (yr == 0) {
                g[2] = G[4 * P_ + ry0 + gx0];
                g[5] = G[7 * P_ + ry0 + gx0];
                g[6] = G[8 * P_ + ry0 + gx0];
            }
            if (yr == ny - 1) {
                g[4] = G[2 * P_ + ry0 + gx0];
                g[7] = G[5 * P_ + ry0 + gx0];
                g[8] = G[6 * P_ + ry0 + gx0];
            }
        }
        // Eq. (11) on the deviations: n = 1 + sum g, sum f e = sum g e.
        dn = g[0] + ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
        const T jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
        const T jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
        const T n = T(1) + dn;
        ux = (jx + T(0.5) * Fx) / n;
        uy = (jy + T(0.5) * Fy) / n;
    };

    // halo ring of R3 (u only)
    {
        constexpr int TOP = 3 * W3, SIDE = 6 * BY;
        for (int k = tid; k < 2 * TOP + SIDE; k += NT) {
            int lx, ly;
            if (k < TOP) {
                ly = k / W3;
                lx = k - ly * W3;
            } else if (k < 2 * TOP) {
                const int kk = k - TOP;
                ly = H3 - 3 + kk / W3;
                lx = kk % W3;
            } else {
                const int kk = k - 2 * TOP;
                ly = 3 + kk / 6;
                const int c = kk % 6;
                lx = c < 3 ? c : W3 - 6 + c;
            }
            T g[9], Fx, Fy, dn, ux, uy;
            site_state(lx, ly, g, Fx, Fy, dn, ux, uy);
            if (p.flags & LBD_FROZEN_U) {
                ux = p.ux0;
                uy = p.uy0;
            }
            s_ux[ly * W3 + lx] = ux;
            s_uy[ly * W3 + lx] = uy;
        }
    }
    // interior of R3 = the output tile: u, and collide
    for (int k = tid; k < BX * BY; k += NT) {
        const int ty = k / BX, tx = k - ty * BX;
        const int lx = tx + 3, ly = ty + 3;
        T g[9], Fx, Fy, dn, ux, uy;
        site_state(lx, ly, g, Fx, Fy, dn, ux, uy);
        const bool inside = (x0 + tx < nx) && (y0 + ty < ny);
        const long long o = (long long)s_gy[ty + HALO] * pitch + s_gx[tx + HALO];
        if (MODE == MODE_FIELDS) {
            if (inside) {
                const long long d = (long long)(y0 + ty) * nx + (x0 + tx);
                p.rho_f[d] = 1.0 + (double)dn;
                p.ux_f[d] = (double)ux;
                p.uy_f[d] = (double)uy;
                p.phi_f[d] = (double)s_phi[(ty + HALO) * W5 + tx + HALO];
                p.psi_f[d] = (double)s_psi[(ty + HALO) * W5 + tx + HALO];
            }
        } else {
            if (inside) {
                // BGK collision with Guo forcing, Eqs. (10), (12), (13), on g = f - w.
                const T n = T(1) + dn;
                const T usq = ux * ux + uy * uy;
                const T uF = ux * Fx + uy * Fy;
                const T om = p.omega, gk = p.guo;
                T *Go = p.g_out + o;
                const long long P_ = p.plane;
#define LBD_COLLIDE(I, W, EX, EY)                                                        \
    {                                                                                   \
        const T eu = T(EX) * ux + T(EY) * uy;                                           \
        const T eF = T(EX) * Fx + T(EY) * Fy;                                           \
        const T geq = T(W) * (dn + n * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * usq));  \
        const T Fi = gk * T(W) * (T(3) * (eF - uF) + T(9) * eu * eF);                   \
        Go[(I) * P_] = g[I] - om * (g[I] - geq) + Fi;                                   \
    }
                LBD_COLLIDE(0, 4.0 / 9.0, 0, 0)
                LBD_COLLIDE(1, 1.0 / 9.0, 1, 0)
                LBD_COLLIDE(2, 1.0 / 9.0, 0, 1)
                LBD_COLLIDE(3, 1.0 / 9.0, -1, 0)
                LBD_COLLIDE(4, 1.0 / 9.0, 0, -1)
                LBD_COLLIDE(5, 1.0 / 36.0, 1, 1)
                LBD_COLLIDE(6, 1.0 / 36.0, -1, 1)
                LBD_COLLIDE(7, 1.0 / 36.0, -1, -1)
                LBD_COLLIDE(8, 1.0 / 36.0, 1, -1)
#undef LBD_COLLIDE
            }
            if (p.flags & LBD_FROZEN_U) {
                ux = p.ux0;
                uy = p.uy0;
            }
            s_ux[ly * W3 + lx] = ux;
            s_uy[ly * W3 + lx] = uy;
        }
    }
    if (MODE == MODE_FIELDS) return;
    __syncthreads();

    // ---- stage C: advection half step on R2 (Eqs. 16-17, donor-cell fluxes) ----
    for (int k = tid; k < W2 * H2; k += NT) {
        const int ly = k / W2, lx = k - ly * W2;
        const int c3 = (ly + 1) * W3 + (lx + 1);
        const int c5 = (ly + 3) * W5 + (lx + 3);
        const T *UX = s_ux + c3, *UY = s_uy + c3;
        const T *P = s_phi + c5, *C = s_psi + c5;
        // face velocities: mean of the two sites; flux = u_f * upwind value
        const T ue = T(0.5) * (UX[0] + UX[1]), uw = T(0.5) * (UX[-1] + UX[0]);
        const T un = T(0.5) * (UY[0] + UY[W3]), us = T(0.5) * (UY[-W3] + UY[0]);
        const T pe = ue * (ue > T(0) ? P[0] : P[1]), pw = uw * (uw > T(0) ? P[-1] : P[0]);
        T pn = un * (un > T(0) ? P[0] : P[W5]), ps = us * (us > T(0) ? P[-W5] : P[0]);
        const T ce = ue * (ue > T(0) ? C[0] : C[1]), cw = uw * (uw > T(0) ? C[-1] : C[0]);
        T cn = un * (un > T(0) ? C[0] : C[W5]), cs = us * (us > T(0) ? C[-W5] : C[0]);
        if (walls) {  // no advective flux through a plate face
            const int yr = y0 - 2 + ly;
            if (yr == 0) {
                ps = T(0);
                cs = T(0);
            }
            if (yr == ny - 1) {
                pn = T(0);
                cn = T(0);
            }
        }
        s_phs[k] = P[0] - ((pe - pw) + (pn - ps));
        s_pss[k] = C[0] - ((ce - cw) + (cn - cs));
    }
    __syncthreads();
    // With plates, phi* and psi* on the two rows beyond a plate are the mirror
    // of the two rows inside (row -1 - k is row k); every output row reads no
    // further, and the mirrored rows lie in the same R2 region.
    if (walls && (y0 - 2 < 0 || y0 + BY + 2 > ny)) {
        for (int k = tid; k < W2 * H2; k += NT) {
            const int ly = k / W2, lx = k - ly * W2;
            const int yr = y0 - 2 + ly;
            if (yr == -2 || yr == -1 || yr == ny || yr == ny + 1) {
                const int ym = yr < 0 ? -1 - yr : 2 * ny - 1 - yr;
                const int m = (ym - (y0 - 2)) * W2 + lx;
                s_phs[k] = s_phs[m];
                s_pss[k] = s_pss[m];
            }
        }
        __syncthreads();
    }

    // ---- stage D: mu* and m* on R1 (into the R4 buffers, R1 stride) --------
    for (int k = tid; k < W1 * H1; k += NT) {
        const int ly = k / W1, lx = k - ly * W1;
        const int c2 = (ly + 1) * W2 + (lx + 1);
        const T *P = s_phs + c2, *C = s_pss + c2;
        const T phx = Stencil<T, W2>::dx(P), phy = Stencil<T, W2>::dy(P);
        const T lph = Stencil<T, W2>::lap(P);
        const T cx = Stencil<T, W2>::dx(C), cy = Stencil<T, W2>::dy(C);
        const T pn = s_phi[(ly + 4) * W5 + (lx + 4)];  // phi^n for the cubic (Eq. 18)
        const T B = p.B0 + p.B1 * C[0];
        s_mu[k] = p.a * P[0] + p.b * (pn * pn * pn) - B * lph - p.B1 * (phx * cx + phy * cy);
        s_m[k] = T(0.5) * p.B1 * (phx * phx + phy * phy);
    }
    __syncthreads();

    // ---- stage E: phi^{n+1}, psi^{n+1} on the tile ----------------------------
    for (int k = tid; k < BX * BY; k += NT) {
        const int ty = k / BX, tx = k - ty * BX;
        if (x0 + tx >= nx || y0 + ty >= ny) continue;
        const T *MU = s_mu + (ty + 1) * W1 + (tx + 1);
        const T *Mm = s_m + (ty + 1) * W1 + (tx + 1);
        const T *C = s_pss + (ty + 2) * W2 + (tx + 2);
        const T ph = s_phs[(ty + 2) * W2 + (tx + 2)];
        // Eq. (18): phi* + M lap mu*
        const T phi_new = ph + p.M * Stencil<T, W1>::lap(MU);
        // Eq. (19) with D psi grad mu_psi = D (grad psi + psi grad m), link form
        const T c0 = C[0], m0 = Mm[0];
#define LBD_LINK(OFF2, OFF1) ((C[OFF2] - c0) + T(0.5) * (c0 + C[OFF2]) * (Mm[OFF1] - m0))
        const T ax = LBD_LINK(1, 1) + LBD_LINK(-1, -1) + LBD_LINK(W2, W1) + LBD_LINK(-W2, -W1);
        const T dg = LBD_LINK(W2 + 1, W1 + 1) + LBD_LINK(W2 - 1, W1 - 1) +
                     LBD_LINK(-W2 + 1, -W1 + 1) + LBD_LINK(-W2 - 1, -W1 - 1);
#undef LBD_LINK
        const T div = ax * T(2.0 / 3.0) + dg * T(1.0 / 6.0);
        T src = T(0);
        if (p.theta) {
            const int gx = x0 + tx;
            const uint32_t w = p.theta[(long long)(y0 + ty) * p.theta_words + (gx >> 5)];
            if ((w >> (gx & 31)) & 1u) src = p.A;
        }
        const T psi_new = c0 + (p.D * div - p.gamma * (c0 - p.c0) + src);
        const long long o = (long long)(y0 + ty) * pitch + (x0 + tx);
        p.phi_out[o] = phi_new;
        p.psi_out[o] = psi_new;
    }
}

template <typename T, int BX, int BY>
constexpr size_t smem_for() {
    return sizeof(T) * (size_t)(2 * (BX + 10) * (BY + 10) + 2 * (BX + 8) * (BY + 8) +
                                2 * (BX + 6) * (BY + 6) + 2 * (BX + 4) * (BY + 4)) +
           sizeof(int) * (size_t)((BX + 10) + (BY + 10));
}

template <typename T, int BX, int BY>
cudaError_t launch_tile(const StepArgs<T> &a, int mode, cudaStream_t s) {
    constexpr size_t smem = smem_for<T, BX, BY>();
    // The shared-memory opt-in is a per-device attribute of each instantiation.
    static unsigned long long configured = 0;
    int dev = 0;
    cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) return ge;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        cudaError_t e;
        e = cudaFuncSetAttribute(step_kernel<T, BX, BY, MODE_STEP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(step_kernel<T, BX, BY, MODE_FIELDS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY);
    if (mode == MODE_STEP)
        step_kernel<T, BX, BY, MODE_STEP><<<grid, NT, smem, s>>>(a);
    else
        step_kernel<T, BX, BY, MODE_FIELDS><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

constexpr Tile kTiles[] = {{32, 8},   {32, 16},  {64, 8},    {32, 32},  {64, 16},
                           {118, 16}, {118, 32}, {118, 64}, {118, 128}, {246, 32},
                           {246, 64}, {116, 32},  {116, 64}, {116, 96},  {116, 128}};

}  // namespace

cudaError_t launch_theta_mask(int nx, int ny, int n_src, const lbd_source *src, bool wrap_y,
                              uint32_t *mask, cudaStream_t s) {
    SourceList l;
    for (int k = 0; k < n_src; ++k) l.s[k] = src[k];
    const long long words = (long long)((nx + 31) / 32) * ny;
    const int nb = (int)((words + 255) / 256 < 4096 ? (words + 255) / 256 : 4096);
    theta_mask_kernel<<<nb, 256, 0, s>>>(nx, ny, n_src, l, wrap_y ? 1 : 0, mask);
    return cudaGetLastError();
}

int n_tiles() { return (int)(sizeof(kTiles) / sizeof(kTiles[0])); }
Tile tile_at(int k) { return kTiles[k]; }

template <typename T>
size_t step_smem_bytes(Tile t) {
    if (t.bx >= 118) return stripe_smem_bytes<T>(t.bx + 10);
    if (t.bx == 32 && t.by == 8) return smem_for<T, 32, 8>();
    if (t.bx == 32 && t.by == 16) return smem_for<T, 32, 16>();
    if (t.bx == 64 && t.by == 8) return smem_for<T, 64, 8>();
    if (t.bx == 32 && t.by == 32) return smem_for<T, 32, 32>();
    if (t.bx == 64 && t.by == 16) return smem_for<T, 64, 16>();
    return 0;
}

bool tile_valid(Tile t, bool fp32, int nx, long long plane) {
    bool known = false;
    for (const Tile &k : kTiles) known |= (k.bx == t.bx && k.by == t.by);
    if (!known) return false;
    if (t.bx >= 118 && 9.0 * (double)plane * (fp32 ? 4.0 : 8.0) >= 4294967295.0) return false;
    if (t.bx == 116) return fp32 && vstripe_supported(nx, plane);
    return true;
}

template <typename T>
cudaError_t launch_vstripe_if_float(const StepArgs<T> &, int, cudaStream_t) {
    return cudaErrorInvalidValue;
}
template <>
cudaError_t launch_vstripe_if_float<float>(const StepArgs<float> &a, int seg, cudaStream_t s) {
    return launch_vstripe(a, seg, s);
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, int mode, Tile t, cudaStream_t s) {
    if (t.bx == 116) {
        if (mode == MODE_STEP) return launch_vstripe_if_float<T>(a, t.by, s);
        t = Tile{32, 16};  // the fields evaluation always uses the tiled kernel
    }
    if (t.bx >= 118) {
        if (mode == MODE_STEP) {
            return launch_stripe<T>(a, t.bx + 10, t.by, s);
        }
        t = Tile{32, 16};  // the fields evaluation always uses the tiled kernel
    }
    if (t.bx == 32 && t.by == 8) return launch_tile<T, 32, 8>(a, mode, s);
    if (t.bx == 32 && t.by == 16) return launch_tile<T, 32, 16>(a, mode, s);
    if (t.bx == 64 && t.by == 8) return launch_tile<T, 64, 8>(a, mode, s);
    if (t.bx == 32 && t.by == 32) return launch_tile<T, 32, 32>(a, mode, s);
    if (t.bx == 64 && t.by == 16) return launch_tile<T, 64, 16>(a, mode, s);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_step<float>(const StepArgs<float> &, int, Tile, cudaStream_t);
template cudaError_t launch_step<double>(const StepArgs<double> &, int, Tile, cudaStream_t);
template size_t step_smem_bytes<float>(Tile);
template size_t step_smem_bytes<double>(Tile);

}  // namespace lbd

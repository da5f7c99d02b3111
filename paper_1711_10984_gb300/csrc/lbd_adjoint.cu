// lbd_adjoint.cu -- hand-written adjoint (reverse mode) of the coupled step of
// arXiv 1711.10984, Sections 2.1-2.3, for the loss
//     L = X_cm(t0 + T) - X_cm(t0),
// X_cm the x centre of mass of the phi >= 0 region (Section 4), with respect to
// the initial surfactant field psi(t0) and the coupling B1 of B(psi) = B0 + B1 psi.
//
// Forward: the step kernel advances the state, with a checkpoint every K steps.
// Reverse: for each segment (last first) the checkpoint is restored, the K
// states of the segment are recomputed and kept, and the step is reversed one
// at a time.  Reversing a step recomputes its intermediates (gradients,
// Laplacians, chemical potentials, force, pulled populations, moments,
// advected fields) in the step's precision (float for the FP32 form, double for
// FP64) and applies the transposed operators:
//   psi update  (Eq. 19, link form)          -> lambda psi*, lambda m*
//   phi update  (Eq. 18)                     -> lambda mu*, lambda phi*
//   mu*, m*     (Eq. 3 on phi*, psi*)        -> lambda phi*, lambda psi*, lambda phi^n
//   advection   (donor cell, Eqs. 16-17)     -> lambda phi, lambda psi, lambda u
//   collision   (Eqs. 10-13) and u (Eq. 11)  -> lambda f_i, lambda F
//   streaming   (pull)                       -> lambda buffer (push)
//   force       (Eq. 14)                     -> lambda phi, lambda psi, lambda mu, lambda m
//   mu, m       (Eqs. 3, 5)                  -> lambda phi, lambda psi
// with dL/dB1 accumulated per site in double.  The transposes use that the isotropic
// gradient stencil is antisymmetric (G^T = -G) and the Laplacian symmetric.
// A reversed step is five kernels, one thread per site.  Where a stage
// differentiates the output of the stage before it, the two share a kernel: the
// first is evaluated on the block's tile and a one-site halo into shared
// memory.  Pointwise products that feed a transposed stencil are formed once per
// halo-tile site there (or, where their factors come from the previous kernel,
// at each neighbour) instead of being stored in global memory, and the reverse
// of the collision runs in the kernel that produces its lambda u.
// The upwind choices and the phi >= 0 mask of the centroid are taken from the
// forward state (they are piecewise constant).
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "lbd_internal.h"

namespace lbd {
namespace {

// The 3 x 3 neighbourhood of a site as indices into some array; slot k of
// operator[] is C, E, W, N, S, NE, NW, SE, SW (N: y + 1, E: x + 1).
enum { C_, E_, W_, N_, S_, NE_, NW_, SE_, SW_ };
struct Nbr {
    long long c, e, w, n, s, ne, nw, se, sw;
    __device__ __forceinline__ long long operator[](int k) const {
        return k == C_ ? c : k == E_ ? e : k == W_ ? w : k == N_ ? n : k == S_ ? s
             : k == NE_ ? ne : k == NW_ ? nw : k == SE_ ? se : sw;
    }
};

// periodic neighbourhood of (x, y) in a row-major array with rows of `row` elements
__device__ __forceinline__ Nbr nbr(int x, int y, int nx, int ny, long long row) {
    const int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
    const int ym = y ? y - 1 : ny - 1, yp = y + 1 < ny ? y + 1 : 0;
    const long long r0 = (long long)y * row, rm = (long long)ym * row, rp = (long long)yp * row;
    return Nbr{r0 + x, r0 + xp, r0 + xm, rp + x, rm + x, rp + xp, rp + xm, rm + xp, rm + xm};
}

// isotropic D2Q9 stencils of a function A(k) of the neighbourhood slot (an array
// read, a value in shared memory, or a product formed at the neighbour)
template <class F>
__device__ __forceinline__ auto Gx(const F &A) {
    using R = decltype(A(C_));
    return (A(E_) - A(W_)) / R(3.0) + ((A(NE_) - A(NW_)) + (A(SE_) - A(SW_))) / R(12.0);
}
template <class F>
__device__ __forceinline__ auto Gy(const F &A) {
    using R = decltype(A(C_));
    return (A(N_) - A(S_)) / R(3.0) + ((A(NE_) - A(SE_)) + (A(NW_) - A(SW_))) / R(12.0);
}
template <class F>
__device__ __forceinline__ auto Lap(const F &A) {
    using R = decltype(A(C_));
    const R c = A(C_);
    return (R(2.0) / R(3.0)) * ((A(E_) - c) + (A(W_) - c) + (A(N_) - c) + (A(S_) - c)) +
           (R(1.0) / R(6.0)) * ((A(NE_) - c) + (A(NW_) - c) + (A(SE_) - c) + (A(SW_) - c));
}
// sum_alpha G_alpha(V_alpha)
template <class F, class G>
__device__ __forceinline__ auto Div(const F &Vx, const G &Vy) {
    return Gx(Vx) + Gy(Vy);
}
// array A over the neighbourhood q
template <typename R>
struct At {
    const R *a;
    Nbr q;
    __device__ __forceinline__ R operator()(int k) const { return a[q[k]]; }
};
template <typename R>
__device__ __forceinline__ At<R> at(const R *a, const Nbr &q) {
    return At<R>{a, q};
}

// One thread per site on a 2D grid of TBX x TBY blocks: (x, y) and the dense index s.
constexpr int TBX = 32, TBY = 8;
#define LBD_SITE(p)                                                                       \
    const int x = blockIdx.x * TBX + threadIdx.x, y = blockIdx.y * TBY + threadIdx.y;     \
    if (x >= (p).nx || y >= (p).ny) return;                                               \
    const long long s = (long long)y * (p).nx + x;

// Two-stage kernels: the first stage is evaluated on the block's tile and a
// one-site halo (THN sites, periodic) into shared memory, then the second stage
// differentiates it on the tile.  f(e, x, y) evaluates halo-tile site e.
constexpr int THX = TBX + 2, THN = THX * (TBY + 2);
template <class F>
__device__ __forceinline__ void over_halo_tile(int nx, int ny, F f) {
    const int x0 = blockIdx.x * TBX - 1, y0 = blockIdx.y * TBY - 1;
    for (int e = threadIdx.y * TBX + threadIdx.x; e < THN; e += TBX * TBY) {
        int x = (x0 + e % THX) % nx, y = (y0 + e / THX) % ny;
        x += x < 0 ? nx : 0;
        y += y < 0 ? ny : 0;
        f(e, x, y);
    }
}
// the neighbourhood of the thread's own site in a halo tile
__device__ __forceinline__ Nbr tile_nbr() {
    const long long c = (threadIdx.y + 1) * THX + threadIdx.x + 1;
    return Nbr{c, c + 1, c - 1, c + THX, c - THX, c + THX + 1, c + THX - 1, c - THX + 1,
               c - THX - 1};
}

#define LBD_SITES(N)                                                                   \
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < (N);       \
         s += (long long)gridDim.x * blockDim.x)

// D2Q9 velocity components of direction i (order (0,0) (1,0) (0,1) (-1,0) (0,-1)
// (1,1) (-1,1) (-1,-1) (1,-1))
__device__ __forceinline__ int EX(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ int EY(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
template <typename R>
__device__ __forceinline__ R wgt(int i) {
    return i == 0 ? R(4.0) / R(9.0) : (i < 5 ? R(1.0) / R(9.0) : R(1.0) / R(36.0));
}

// Scalars of one step.
template <typename R>
struct AdjPar {
    int nx, ny;
    long long N, pitch, plane;
    R a, b, B0, B1, M, D, omega, guo, gamma, c0, fx, fy;
    int body;
};

// Dense work arrays of one reversed step (R: the step's precision).
template <typename R>
struct Work {
    // forward intermediates
    R *PH, *PS, *GPx, *GPy, *LP, *GSx, *GSy;
    R *GMx, *GMy, *GNx, *GNy, *Fx, *Fy, *RHO, *UX, *UY;
    R *PSS, *GQx, *GQy, *LQ, *GRx, *GRy, *MS;
    // adjoints
    R *Lphi, *Lpsi, *Lbuf;       // of the step output (9 planes for Lbuf)
    R *Lphi0, *Lpsi0, *Lbuf0;    // of the step input
    R *LPHS, *LPSS, *LFX, *LFY;
    double *dB1;                           // per-site accumulator of dL/dB1 (double)
};

// ---- forward intermediates ----------------------------------------------------
// On the tile and its halo: gradients and Laplacian of phi^n, psi^n and mu, m
// (Eqs. 3, 5), kept for the tile's own sites; on the tile: F (Eq. 14), the
// pulled populations, n and u (Eq. 11).
template <typename R>
__global__ void fwd123(AdjPar<R> p, const R *phi, const R *psi, const R *g, Work<R> w) {
    __shared__ R sMU[THN], sMM[THN];
    over_halo_tile(p.nx, p.ny, [&](int e, int x, int y) {
        const Nbr q = nbr(x, y, p.nx, p.ny, p.pitch);  // into the pitched state
        const R px = Gx(at(phi, q)), py = Gy(at(phi, q)), lp = Lap(at(phi, q));
        const R cx = Gx(at(psi, q)), cy = Gy(at(psi, q));
        const R ph = phi[q.c], c = psi[q.c];
        sMU[e] = p.a * ph + p.b * ph * ph * ph - (p.B0 + p.B1 * c) * lp - p.B1 * (px * cx + py * cy);
        sMM[e] = R(0.5) * p.B1 * (px * px + py * py);
        const int ex = e % THX, ey = e / THX;  // the tile's own sites keep the rest
        if (ex >= 1 && ex <= TBX && ey >= 1 && ey <= TBY &&
            (int)blockIdx.x * TBX + ex - 1 < p.nx && (int)blockIdx.y * TBY + ey - 1 < p.ny) {
            const long long s = (long long)y * p.nx + x;
            w.PH[s] = ph; w.PS[s] = c;
            w.GPx[s] = px; w.GPy[s] = py; w.LP[s] = lp; w.GSx[s] = cx; w.GSy[s] = cy;
        }
    });
    __syncthreads();
    LBD_SITE(p)
    const Nbr t = tile_nbr();
    const R gmx = Gx(at((const R *)sMU, t)), gmy = Gy(at((const R *)sMU, t));
    const R gnx = Gx(at((const R *)sMM, t)), gny = Gy(at((const R *)sMM, t));
    w.GMx[s] = gmx; w.GMy[s] = gmy; w.GNx[s] = gnx; w.GNy[s] = gny;
    const long long o = (long long)y * p.pitch + x;
    const R ph = phi[o], c = psi[o];
    R Fx = -ph * gmx - (w.GSx[s] + c * gnx);
    R Fy = -ph * gmy - (w.GSy[s] + c * gny);
    if (p.body) { Fx += p.fx; Fy += p.fy; }
    w.Fx[s] = Fx; w.Fy[s] = Fy;
    R n = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int xs = x - EX(i), ys = y - EY(i);
        xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
        ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
        const R f = wgt<R>(i) + g[i * p.plane + (long long)ys * p.pitch + xs];
        n += f; jx += f * EX(i); jy += f * EY(i);
    }
    w.RHO[s] = n;
    w.UX[s] = (jx + R(0.5) * Fx) / n;
    w.UY[s] = (jy + R(0.5) * Fy) / n;
}

template <typename R>
__device__ __forceinline__ R up(R u, R a, R b) { return u > R(0.0) ? a : b; }

// phi*, psi* by donor-cell advection (Eqs. 16-17) on the tile and its halo, then
// their gradients, the Laplacian of phi* and m* on the tile
template <typename R>
__global__ void fwd45(AdjPar<R> p, Work<R> w) {
    __shared__ R sP[THN], sC[THN];
    over_halo_tile(p.nx, p.ny, [&](int e, int x, int y) {
        const Nbr q = nbr(x, y, p.nx, p.ny, p.nx);
        const long long s = q.c;
        const R *UX = w.UX, *UY = w.UY;
        const R ue = R(0.5) * (UX[s] + UX[q.e]), uw = R(0.5) * (UX[q.w] + UX[s]);
        const R un = R(0.5) * (UY[s] + UY[q.n]), us = R(0.5) * (UY[q.s] + UY[s]);
        const R *P = w.PH, *C = w.PS;
        const R fe = ue * up(ue, P[s], P[q.e]), fw = uw * up(uw, P[q.w], P[s]);
        const R fn = un * up(un, P[s], P[q.n]), fs = us * up(us, P[q.s], P[s]);
        const R ge = ue * up(ue, C[s], C[q.e]), gw = uw * up(uw, C[q.w], C[s]);
        const R gn = un * up(un, C[s], C[q.n]), gs = us * up(us, C[q.s], C[s]);
        sP[e] = P[s] - ((fe - fw) + (fn - fs));
        sC[e] = C[s] - ((ge - gw) + (gn - gs));
    });
    __syncthreads();
    LBD_SITE(p)
    const Nbr t = tile_nbr();
    const R px = Gx(at((const R *)sP, t)), py = Gy(at((const R *)sP, t));
    w.PSS[s] = sC[t.c];
    w.GQx[s] = px; w.GQy[s] = py; w.LQ[s] = Lap(at((const R *)sP, t));
    w.GRx[s] = Gx(at((const R *)sC, t)); w.GRy[s] = Gy(at((const R *)sC, t));
    w.MS[s] = R(0.5) * p.B1 * (px * px + py * py);
}

// ---- reverse of the phi and psi updates (Eqs. 18, 19) on the tile and its halo,
// with the products that the transposed stencils of mu*, m* need formed there;
// then the reverse of mu*, m* (Eq. 3 on phi*, psi*) on the tile: the local
// terms, dB1, and the transposed stencils ------------------------------------------
template <typename R>
__global__ void adj_ed(AdjPar<R> p, const R *gam, int jstep, Work<R> w) {
    __shared__ R sMU[THN], sM[THN], sPSS[THN];  // lambda mu*, lambda m*, lambda psi* (partial)
    __shared__ R sT[7][THN];                     // products at each halo-tile site
    const R gamma = gam[jstep];  // sink rate of the reversed step (j-th of its segment)
    const R B0 = p.B0, B1 = p.B1;
    over_halo_tile(p.nx, p.ny, [&](int e, int x, int y) {
        const Nbr q = nbr(x, y, p.nx, p.ny, p.nx);
        const long long s = q.c;
        const R lmus = p.M * Lap(at(w.Lphi, q));
        const long long nb[8] = {q.e, q.w, q.n, q.s, q.ne, q.nw, q.se, q.sw};
        const R *Lp = w.Lpsi, *m = w.MS, *c = w.PSS;
        R lpss = Lp[s] * (R(1.0) - gamma), lms = R(0.0);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const R lam = k < 4 ? R(2.0) / R(3.0) : R(1.0) / R(6.0);
            const long long j = nb[k];
            // psi'_s's own link to j, and psi'_j's link back to s
            lpss += p.D * lam * (Lp[s] * (-R(1.0) + R(0.5) * (m[j] - m[s])) +
                                 Lp[j] * (R(1.0) + R(0.5) * (m[s] - m[j])));
            lms += p.D * lam * R(0.5) * (c[s] + c[j]) * (Lp[j] - Lp[s]);
        }
        sMU[e] = lmus;
        sM[e] = lms;
        sPSS[e] = lpss;
        const R gqx = w.GQx[s], gqy = w.GQy[s];
        sT[0][e] = (B0 + B1 * c[s]) * lmus;  // for -L(.)
        sT[1][e] = lmus * w.GRx[s];         // B1 div(lambda mu* grad psi*) -> phi*
        sT[2][e] = lmus * w.GRy[s];
        sT[3][e] = lmus * gqx;              // B1 div(lambda mu* grad phi*) -> psi*
        sT[4][e] = lmus * gqy;
        sT[5][e] = lms * gqx;               // -B1 div(lambda m* grad phi*) -> phi*
        sT[6][e] = lms * gqy;
    });
    __syncthreads();
    LBD_SITE(p)
    const Nbr t = tile_nbr();
    auto T = [&](int i) { return At<R>{sT[i], t}; };
    const R lmu = sMU[t.c], lm = sM[t.c];
    const R qx = w.GQx[s], qy = w.GQy[s], rx = w.GRx[s], ry = w.GRy[s];
    const R ph = w.PH[s];
    w.Lphi0[s] = R(3.0) * p.b * ph * ph * lmu;  // cubic term uses phi^n
    w.dB1[s] += (double)(lmu * (-w.PSS[s] * w.LQ[s] - (qx * rx + qy * ry)) +
                         lm * R(0.5) * (qx * qx + qy * qy));
    w.LPHS[s] = w.Lphi[s] + p.a * lmu - Lap(T(0)) + B1 * Div(T(1), T(2)) - B1 * Div(T(5), T(6));
    w.LPSS[s] = (sPSS[t.c] + -B1 * w.LQ[s] * lmu) + B1 * Div(T(3), T(4));
}

// ---- reverse of the donor-cell advection (Eqs. 16-17), then of the collision
// (Eqs. 10-13), moments (Eq. 11) and streaming at the same site ------------------
// lambda F of site (x, y) (dense index s) into lFx, lFy; with own, the site's
// other results too: lambda phi^n, psi^n (added to, set) and the streamed
// lambda of the populations.
template <typename R>
__device__ __forceinline__ void adj_cb_site(const AdjPar<R> &p, const Work<R> &w, int x, int y,
                                            long long s, bool own, R &lFx, R &lFy) {
    const Nbr q = nbr(x, y, p.nx, p.ny, p.nx);
    const R *UX = w.UX, *UY = w.UY, *P = w.PH, *C = w.PS;
    const R *LP = w.LPHS, *LC = w.LPSS;
    const R ue = R(0.5) * (UX[s] + UX[q.e]), uw = R(0.5) * (UX[q.w] + UX[s]);
    const R un = R(0.5) * (UY[s] + UY[q.n]), us = R(0.5) * (UY[q.s] + UY[s]);
    // adjoint of each face flux: (lambda at the right/upper site) - (left/lower)
    const R lpe = LP[q.e] - LP[s], lpw = LP[s] - LP[q.w];
    const R lpn = LP[q.n] - LP[s], lps = LP[s] - LP[q.s];
    const R lce = LC[q.e] - LC[s], lcw = LC[s] - LC[q.w];
    const R lcn = LC[q.n] - LC[s], lcs = LC[s] - LC[q.s];
    R lphi = LP[s], lpsi = LC[s];
    // this site is upwind of the east / north face when u_f > 0, of west / south when u_f <= 0
    if (ue > 0) { lphi += lpe * ue; lpsi += lce * ue; }
    if (!(uw > 0)) { lphi += lpw * uw; lpsi += lcw * uw; }
    if (un > 0) { lphi += lpn * un; lpsi += lcn * un; }
    if (!(us > 0)) { lphi += lps * us; lpsi += lcs * us; }
    if (own) {
        w.Lphi0[s] += lphi;
        w.Lpsi0[s] = lpsi;
    }
    R lux = R(0.5) * (lpe * up(ue, P[s], P[q.e]) + lce * up(ue, C[s], C[q.e]) +
                      lpw * up(uw, P[q.w], P[s]) + lcw * up(uw, C[q.w], C[s]));
    R luy = R(0.5) * (lpn * up(un, P[s], P[q.n]) + lcn * up(un, C[s], C[q.n]) +
                      lps * up(us, P[q.s], P[s]) + lcs * up(us, C[q.s], C[s]));
    // collision, moments and streaming
    const R n = w.RHO[s], ux = UX[s], uy = UY[s], Fx = w.Fx[s], Fy = w.Fy[s];
    const R om = p.omega, gk = p.guo, usq = ux * ux + uy * uy;
    R ln = 0;
    lFx = 0;
    lFy = 0;
    R lpost[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R lp = w.Lbuf[i * p.N + s];
        lpost[i] = lp;
        const R ex = EX(i), ey = EY(i), wi = wgt<R>(i);
        const R eu = ex * ux + ey * uy, eF = ex * Fx + ey * Fy;
        ln += lp * om * wi * (R(1.0) + R(3.0) * eu + R(4.5) * eu * eu - R(1.5) * usq);
        // d feq/du and d F_i/du
        lux += lp * (om * wi * n * (R(3.0) * ex + R(9.0) * eu * ex - R(3.0) * ux) +
                     gk * wi * (-R(3.0) * Fx + R(9.0) * eF * ex));
        luy += lp * (om * wi * n * (R(3.0) * ey + R(9.0) * eu * ey - R(3.0) * uy) +
                     gk * wi * (-R(3.0) * Fy + R(9.0) * eF * ey));
        lFx += lp * gk * wi * (R(3.0) * (ex - ux) + R(9.0) * eu * ex);
        lFy += lp * gk * wi * (R(3.0) * (ey - uy) + R(9.0) * eu * ey);
    }
    // u = (j + F/2) / n
    const R ljx = lux / n, ljy = luy / n;
    lFx += R(0.5) * lux / n;
    lFy += R(0.5) * luy / n;
    ln += -(lux * ux + luy * uy) / n;
    if (!own) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R lf = (R(1.0) - om) * lpost[i] + ln + ljx * EX(i) + ljy * EY(i);
        // f_i(x) was pulled from buffer_i(x - e_i)
        int xs = x - EX(i), ys = y - EY(i);
        xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
        ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
        w.Lbuf0[i * p.N + (long long)ys * p.nx + xs] = lf;
    }
}

// ---- reverse of the advection, collision and streaming, then of the force
// (Eq. 14) and of mu, m (Eqs. 3, 5).  Three stages, two barriers:
//  1. lambda F (adj_cb_site) on the tile and a two-site halo into shared
//     memory; the tile's own sites also write lambda phi^n, psi^n and the
//     streamed lambda of the populations;
//  2. on the tile and a one-site halo: lambda mu = div(phi lambda F), lambda m =
//     div(psi lambda F), and there the products that the transposed stencils of
//     mu, m need;
//  3. on the tile: the force's local terms and grad psi term, and the reverse of
//     mu, m.
constexpr int T2X = TBX + 4, T2N = T2X * (TBY + 4);
template <typename R>
__global__ void adj_cba(AdjPar<R> p, Work<R> w) {
    __shared__ R sFX[T2N], sFY[T2N];  // lambda F on the tile and a two-site halo
    __shared__ R sMU[THN], sM[THN];   // lambda mu, lambda m on the tile and a one-site halo
    __shared__ R sT[7][THN];          // products at each halo-tile site
    const int bx0 = blockIdx.x * TBX, by0 = blockIdx.y * TBY;
    for (int e = threadIdx.y * TBX + threadIdx.x; e < T2N; e += TBX * TBY) {
        const int ex = e % T2X, ey = e / T2X;
        int x = (bx0 - 2 + ex) % p.nx, y = (by0 - 2 + ey) % p.ny;
        x += x < 0 ? p.nx : 0;
        y += y < 0 ? p.ny : 0;
        // the tile's own sites (one writer per lattice site)
        const bool own = ex >= 2 && ex < 2 + TBX && ey >= 2 && ey < 2 + TBY &&
                         bx0 + ex - 2 < p.nx && by0 + ey - 2 < p.ny;
        R lFx, lFy;
        adj_cb_site(p, w, x, y, (long long)y * p.nx + x, own, lFx, lFy);
        sFX[e] = lFx;
        sFY[e] = lFy;
    }
    __syncthreads();
    // neighbourhood of the two-site-halo index c
    auto nb2 = [](int c) {
        return Nbr{c, c + 1, c - 1, c + T2X, c - T2X, c + T2X + 1, c + T2X - 1, c - T2X + 1,
                   c - T2X - 1};
    };
    const R *PH = w.PH, *PS = w.PS;
    const R B0 = p.B0, B1 = p.B1;
    over_halo_tile(p.nx, p.ny, [&](int e, int x, int y) {
        const Nbr q = nbr(x, y, p.nx, p.ny, p.nx);
        const Nbr u = nb2((e / THX + 1) * T2X + e % THX + 1);
        auto T1 = [&](int k) { return PH[q[k]] * sFX[u[k]]; };  // -> lambda mu
        auto T2 = [&](int k) { return PH[q[k]] * sFY[u[k]]; };
        auto T3 = [&](int k) { return PS[q[k]] * sFX[u[k]]; };  // -> lambda m
        auto T4 = [&](int k) { return PS[q[k]] * sFY[u[k]]; };
        const R lmu = Div(T1, T2), lm = Div(T3, T4);
        sMU[e] = lmu;
        sM[e] = lm;
        const long long s = q.c;
        const R gpx = w.GPx[s], gpy = w.GPy[s];
        sT[0][e] = (B0 + B1 * PS[s]) * lmu;
        sT[1][e] = lmu * w.GSx[s];
        sT[2][e] = lmu * w.GSy[s];
        sT[3][e] = lmu * gpx;
        sT[4][e] = lmu * gpy;
        sT[5][e] = lm * gpx;
        sT[6][e] = lm * gpy;
    });
    __syncthreads();
    LBD_SITE(p)
    const Nbr t = tile_nbr();
    const Nbr u = nb2((threadIdx.y + 2) * T2X + threadIdx.x + 2);
    auto T = [&](int i) { return At<R>{sT[i], t}; };
    const R lfx = sFX[u.c], lfy = sFY[u.c];
    const R lphi = w.Lphi0[s] + -(lfx * w.GMx[s] + lfy * w.GMy[s]);
    const R lpsi = (w.Lpsi0[s] + -(lfx * w.GNx[s] + lfy * w.GNy[s])) +
                   Div(At<R>{sFX, u}, At<R>{sFY, u});
    const R lmu = sMU[t.c], lm = sM[t.c];
    const R px = w.GPx[s], py = w.GPy[s], cx = w.GSx[s], cy = w.GSy[s];
    const R ph = PH[s];
    w.dB1[s] += (double)(lmu * (-PS[s] * w.LP[s] - (px * cx + py * cy)) +
                         lm * R(0.5) * (px * px + py * py));
    w.Lphi0[s] = (lphi + (p.a + R(3.0) * p.b * ph * ph) * lmu) +
                 (-Lap(T(0)) + B1 * Div(T(1), T(2)) - B1 * Div(T(5), T(6)));
    w.Lpsi0[s] = (lpsi + -B1 * w.LP[s] * lmu) + B1 * Div(T(3), T(4));
}

// ---- loss: centroid x of the phi >= 0 region and its gradient ---------------------
template <typename T>
__global__ void centroid_partial(int nx, int ny, long long pitch, const T *phi, double refx,
                                 double *partial) {
    __shared__ double sa[256], sb[256];
    double wx = 0, w0 = 0;
    for (int y = blockIdx.x; y < ny; y += gridDim.x)
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const double ph = (double)phi[(long long)y * pitch + x];
            if (ph >= 0.0) {
                double dx = x - refx;
                if (dx >= 0.5 * nx) dx -= nx; else if (dx < -0.5 * nx) dx += nx;
                wx += ph * dx;
                w0 += ph;
            }
        }
    sa[threadIdx.x] = wx;
    sb[threadIdx.x] = w0;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            sa[threadIdx.x] += sa[threadIdx.x + k];
            sb[threadIdx.x] += sb[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sa[0];
        partial[2 * blockIdx.x + 1] = sb[0];
    }
}

template <typename T>
__global__ void centroid_seed(int nx, int ny, long long pitch, const T *phi, double refx,
                              double X, double W, T *Lphi) {
    const long long N = (long long)nx * ny;
    LBD_SITES(N) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        const double ph = (double)phi[(long long)y * pitch + x];
        double dx = x - refx;
        if (dx >= 0.5 * nx) dx -= nx; else if (dx < -0.5 * nx) dx += nx;
        Lphi[s] = (T)(ph >= 0.0 ? (dx - (X - refx)) / W : 0.0);
    }
}

__global__ void sum_kernel(long long n, const double *a, double *partial) {
    __shared__ double sa[256];
    double v = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        v += a[s];
    sa[threadIdx.x] = v;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sa[threadIdx.x] += sa[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sa[0];
}

constexpr int RB = 256;  // reduction blocks

}  // namespace

// ------------------------------------------------------------------- host driver

template <typename T>
int adjoint_run(const AdjointJob<T> &job) {
    const int nx = job.nx, ny = job.ny;
    const long long N = (long long)nx * ny;
    const long long plane = job.plane, pitch = job.pitch;
    const size_t state_elems = (size_t)11 * plane;  // 9 populations + phi + psi
    // the reverse sweep is captured as CUDA graphs, which the legacy default
    // stream does not allow: a context on it lends the call a private stream,
    // ordered after the work already queued (the call synchronises at the end)
    cudaStream_t st = job.stream, own = nullptr;
    if (!st) {
        if (cudaStreamSynchronize(nullptr) != cudaSuccess ||
            cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return LBD_ECUDA;
        }
        st = own;
    }
    const int nb = (int)((N + 255) / 256 < 2048 ? (N + 255) / 256 : 2048);
    const dim3 b2(TBX, TBY), g2((unsigned)((nx + TBX - 1) / TBX), (unsigned)((ny + TBY - 1) / TBY));
    const int64_t nsteps = job.nsteps, K = job.ckpt_every;
    const int64_t nseg = (nsteps + K - 1) / K;

    // device allocations (released before returning)
    std::vector<void *> allocs;
    auto dalloc = [&](size_t bytes) -> void * {
        void *ptr = nullptr;
        if (lbd::dev_malloc((void **)&ptr, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        allocs.push_back(ptr);
        return ptr;
    };
    // reverse sweep of a segment, per segment buffer set and adjoint buffer parity
    cudaGraphExec_t graphs[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    // The recompute of segment s - 1 runs on a second stream while segment s is
    // reversed: the two use the two segment buffer sets in turn, ordered by events.
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fwd = nullptr, rec_done[2] = {nullptr, nullptr}, rev_done[2] = {nullptr, nullptr};
    // Within a reverse sweep the forward intermediates of step k (fwd123, fwd45)
    // need only state k, so they run on a third stream, into the set of the
    // step's parity, while the adjoint kernels of step k + 1 run.
    cudaStream_t sf = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_f[2] = {nullptr, nullptr},
                ev_a[2] = {nullptr, nullptr};
    auto release = [&]() {
        if (st2) {
            cudaStreamSynchronize(st2);
            cudaStreamDestroy(st2);
            st2 = nullptr;
        }
        if (sf) {
            cudaStreamSynchronize(sf);
            cudaStreamDestroy(sf);
            sf = nullptr;
        }
        for (cudaEvent_t *e : {&ev_fwd, &rec_done[0], &rec_done[1], &rev_done[0], &rev_done[1],
                               &ev_fork, &ev_join, &ev_f[0], &ev_f[1], &ev_a[0], &ev_a[1]})
            if (*e) {
                cudaEventDestroy(*e);
                *e = nullptr;
            }
        for (auto &gp : graphs)
            for (auto &g : gp)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
        for (void *ptr : allocs) cudaFree(ptr);
        allocs.clear();
        if (own) {
            cudaStreamSynchronize(own);
            cudaStreamDestroy(own);
            own = nullptr;
        }
    };
    T *ckpt = (T *)dalloc(sizeof(T) * state_elems * (size_t)(nseg + 1));
    T *seg = (T *)dalloc(sizeof(T) * state_elems * (size_t)(K + 1) * 2);
    T *const segs[2] = {seg, seg ? seg + state_elems * (size_t)(K + 1) : nullptr};
    const int n_dense = 72;  // dense arrays of the step's precision carved out below,
                             // after the per-site dL/dB1 accumulator in double: 49, and a
                             // second set of the 23 forward intermediates
    void *dense_raw = dalloc(sizeof(double) * (size_t)N + sizeof(T) * (size_t)N * n_dense);
    double *part = (double *)dalloc(sizeof(double) * 2 * RB);
    T *gam = (T *)dalloc(sizeof(T) * (size_t)K);  // sink rate of each step of a segment
    if (!ckpt || !seg || !dense_raw || !part || !gam) {
        release();
        return LBD_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_fwd, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&rec_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&rec_done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&rev_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&rev_done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sf, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_f[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_f[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_a[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_a[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release();
        return LBD_ECUDA;
    }
    Work<T> w, wf;  // wf: the second set of forward intermediates (the rest unused)
    {
        w.dB1 = reinterpret_cast<double *>(dense_raw);
        T *const dense = reinterpret_cast<T *>(w.dB1 + N);
        T *d = dense;
        auto take = [&](int k) { T *r = d; d += (size_t)k * N; return r; };
        w.PH = take(1); w.PS = take(1); w.GPx = take(1); w.GPy = take(1); w.LP = take(1);
        w.GSx = take(1); w.GSy = take(1);
        w.GMx = take(1); w.GMy = take(1); w.GNx = take(1); w.GNy = take(1);
        w.Fx = take(1); w.Fy = take(1); w.RHO = take(1); w.UX = take(1);
        w.UY = take(1); w.PSS = take(1); w.GQx = take(1); w.GQy = take(1);
        w.LQ = take(1); w.GRx = take(1); w.GRy = take(1); w.MS = take(1);
        w.Lphi = take(1); w.Lpsi = take(1); w.Lbuf = take(9);
        w.Lphi0 = take(1); w.Lpsi0 = take(1); w.Lbuf0 = take(9);
        w.LPHS = take(1); w.LPSS = take(1); w.LFX = take(1); w.LFY = take(1);
        wf = w;
        wf.PH = take(1); wf.PS = take(1); wf.GPx = take(1); wf.GPy = take(1); wf.LP = take(1);
        wf.GSx = take(1); wf.GSy = take(1);
        wf.GMx = take(1); wf.GMy = take(1); wf.GNx = take(1); wf.GNy = take(1);
        wf.Fx = take(1); wf.Fy = take(1); wf.RHO = take(1); wf.UX = take(1);
        wf.UY = take(1); wf.PSS = take(1); wf.GQx = take(1); wf.GQy = take(1);
        wf.LQ = take(1); wf.GRx = take(1); wf.GRy = take(1); wf.MS = take(1);
        if (d - dense != (ptrdiff_t)n_dense * N) {  // carve-out must match the allocation
            release();
            return LBD_EINVAL;
        }
    }
#define ACK(call)                                     \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            release();                                \
            return LBD_ECUDA;                         \
        }                                             \
    } while (0)
    auto slot = [&](T *base, int64_t k) { return base + (size_t)k * state_elems; };
    auto copy_state = [&](T *dst, const T *g, const T *phi, const T *psi,
                          cudaStream_t s) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, g, sizeof(T) * 9 * plane, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst + 9 * plane, phi, sizeof(T) * plane, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst + 10 * plane, psi, sizeof(T) * plane, cudaMemcpyDeviceToDevice, s);
        return e;
    };
    auto step_between = [&](const T *in, T *out, int64_t t, cudaStream_t s) -> cudaError_t {
        StepArgs<T> a = job.args;
        a.g_in = in; a.phi_in = in + 9 * plane; a.psi_in = in + 10 * plane;
        a.g_out = out; a.phi_out = out + 9 * plane; a.psi_out = out + 10 * plane;
        double A, gm;
        activity_at(*job.params, t, &A, &gm);
        a.A = (T)A;
        a.gamma = (T)gm;
        return launch_step<T>(a, MODE_STEP, job.tile, s);
    };
    auto centroid = [&](const T *phi, double *X, double *W) -> cudaError_t {
        centroid_partial<T><<<RB, 256, 0, st>>>(nx, ny, pitch, phi, job.refx, part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        std::vector<double> h(2 * RB);
        e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * RB, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        double a = 0, b = 0;
        for (int k = 0; k < RB; ++k) { a += h[2 * k]; b += h[2 * k + 1]; }
        *X = job.refx + a / b;
        *W = b;
        return e;
    };

    // ---- forward with checkpoints ----
    ACK(copy_state(slot(ckpt, 0), job.g0, job.phi0, job.psi0, st));
    double X0, W0;
    ACK(centroid(job.phi0, &X0, &W0));
    for (int64_t sgi = 0; sgi < nseg; ++sgi) {
        const int64_t k0 = sgi * K, k1 = k0 + K < nsteps ? k0 + K : nsteps;
        // the last segment keeps all its states (buffer set (nseg - 1) & 1): the
        // reverse sweep starts on them without a recompute; the others alternate
        // between two slots
        const bool keep = sgi == nseg - 1;
        T *const sb = keep ? segs[sgi & 1] : seg;
        auto at = [&](int64_t j) { return slot(sb, keep ? j : j % 2); };
        ACK(copy_state(at(0), slot(ckpt, sgi), slot(ckpt, sgi) + 9 * plane,
                       slot(ckpt, sgi) + 10 * plane, st));
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t j = k - k0;
            ACK(step_between(at(j), at(j + 1), job.t0 + k, st));
        }
        const T *endp = at(k1 - k0);
        ACK(copy_state(slot(ckpt, sgi + 1), endp, endp + 9 * plane, endp + 10 * plane, st));
    }
    const T *fin = slot(ckpt, nseg);
    double XT, WT;
    ACK(centroid(fin + 9 * plane, &XT, &WT));
    *job.loss = XT - X0;
    // final state back into the context
    ACK(cudaMemcpyAsync(job.g_final, fin, sizeof(T) * 9 * plane, cudaMemcpyDeviceToDevice, st));
    ACK(cudaMemcpyAsync(job.phi_final, fin + 9 * plane, sizeof(T) * plane, cudaMemcpyDeviceToDevice, st));
    ACK(cudaMemcpyAsync(job.psi_final, fin + 10 * plane, sizeof(T) * plane, cudaMemcpyDeviceToDevice, st));

    // ---- seed: lambda phi = dX/dphi at T, lambda psi = lambda populations = 0 ----
    centroid_seed<T><<<nb, 256, 0, st>>>(nx, ny, pitch, fin + 9 * plane, job.refx, XT, WT, w.Lphi);
    ACK(cudaGetLastError());
    ACK(cudaMemsetAsync(w.Lpsi, 0, sizeof(T) * N, st));
    ACK(cudaMemsetAsync(w.Lbuf, 0, sizeof(T) * 9 * N, st));
    ACK(cudaMemsetAsync(w.dB1, 0, sizeof(double) * N, st));

    AdjPar<T> ap;
    ap.nx = nx; ap.ny = ny; ap.N = N; ap.pitch = pitch; ap.plane = plane;
    ap.a = (T)job.a; ap.b = (T)job.b; ap.B0 = (T)job.B0; ap.B1 = (T)job.B1; ap.M = (T)job.M;
    ap.D = (T)job.D; ap.omega = (T)(1.0 / job.tau); ap.guo = (T)(1.0 - 0.5 / job.tau);
    ap.gamma = 0; ap.c0 = (T)job.c0; ap.fx = (T)job.fx; ap.fy = (T)job.fy; ap.body = job.body;

    // ---- reverse, segment by segment ----
    // The reversed steps of a full segment (K of them) are captured once as a
    // CUDA graph and replayed for the other full segments: their launches and
    // arguments are the same (the recomputed states sit in the same slots; the
    // sink rate is read from gam[j]), except for the alternation of the adjoint
    // buffers, so a graph is kept per buffer parity at the segment start.
    std::vector<T> gam_h((size_t)nsteps);
    for (int64_t k = 0; k < nsteps; ++k) {
        double A, gm;
        activity_at(*job.params, job.t0 + k, &A, &gm);
        gam_h[(size_t)k] = (T)gm;
    }
    // Step j = k - k0 of a sweep uses forward set j & 1.  fwd(k) on sf waits
    // for the adjoint kernels of step k + 2 (the last readers of its set); the
    // adjoint kernels of step k on st wait for fwd(k).  Both orders are events,
    // so that a captured sweep keeps them as graph edges.
    auto reverse_steps = [&](const T *sb, int64_t k0, int64_t k1) -> cudaError_t {
        cudaError_t e = cudaEventRecord(ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sf, ev_fork, 0);
        for (int64_t k = k1 - 1; k >= k0 && e == cudaSuccess; --k) {
            const T *in = sb + (size_t)(k - k0) * state_elems;
            const int q = (int)((k - k0) & 1);
            Work<T> wk = w;
            if (q) {
                wk.PH = wf.PH; wk.PS = wf.PS; wk.GPx = wf.GPx; wk.GPy = wf.GPy; wk.LP = wf.LP;
                wk.GSx = wf.GSx; wk.GSy = wf.GSy; wk.GMx = wf.GMx; wk.GMy = wf.GMy;
                wk.GNx = wf.GNx; wk.GNy = wf.GNy; wk.Fx = wf.Fx; wk.Fy = wf.Fy; wk.RHO = wf.RHO;
                wk.UX = wf.UX; wk.UY = wf.UY; wk.PSS = wf.PSS; wk.GQx = wf.GQx; wk.GQy = wf.GQy;
                wk.LQ = wf.LQ; wk.GRx = wf.GRx; wk.GRy = wf.GRy; wk.MS = wf.MS;
            }
            if (k + 2 < k1) e = cudaStreamWaitEvent(sf, ev_a[q], 0);
            if (e != cudaSuccess) break;
            fwd123<T><<<g2, b2, 0, sf>>>(ap, in + 9 * plane, in + 10 * plane, in, wk);
            fwd45<T><<<g2, b2, 0, sf>>>(ap, wk);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ev_f[q], sf);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_f[q], 0);
            if (e != cudaSuccess) break;
            adj_ed<T><<<g2, b2, 0, st>>>(ap, gam, (int)(k - k0), wk);
            adj_cba<T><<<g2, b2, 0, st>>>(ap, wk);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ev_a[q], st);
            if (e != cudaSuccess) break;
            // the input adjoints become the output adjoints of the previous step
            T *tp;
            tp = w.Lphi; w.Lphi = w.Lphi0; w.Lphi0 = tp;
            tp = w.Lpsi; w.Lpsi = w.Lpsi0; w.Lpsi0 = tp;
            tp = w.Lbuf; w.Lbuf = w.Lbuf0; w.Lbuf0 = tp;
        }
        // join: the sweep ends when both streams have
        if (e == cudaSuccess) e = cudaEventRecord(ev_join, sf);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_join, 0);
        return e;
    };
    // the states of segment sgi, recomputed from its checkpoint into buffer set
    // sgi & 1 on the second stream
    auto recompute = [&](int64_t sgi) -> cudaError_t {
        T *const sb = segs[sgi & 1];
        const int64_t k0 = sgi * K, k1 = k0 + K < nsteps ? k0 + K : nsteps;
        cudaError_t e = copy_state(slot(sb, 0), slot(ckpt, sgi), slot(ckpt, sgi) + 9 * plane,
                                   slot(ckpt, sgi) + 10 * plane, st2);
        for (int64_t k = k0; k < k1 - 1 && e == cudaSuccess; ++k)
            e = step_between(slot(sb, k - k0), slot(sb, k - k0 + 1), job.t0 + k, st2);
        if (e == cudaSuccess) e = cudaEventRecord(rec_done[sgi & 1], st2);
        return e;
    };
    // every recompute follows the forward pass, which used buffer set 0 and left
    // the last segment's states in its set
    ACK(cudaEventRecord(ev_fwd, st));
    ACK(cudaStreamWaitEvent(st2, ev_fwd, 0));
    ACK(cudaEventRecord(rec_done[(nseg - 1) & 1], st));
    int parity = 0;  // adjoint buffer alternation at the current segment start
    for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
        const int64_t k0 = sgi * K, k1 = k0 + K < nsteps ? k0 + K : nsteps;
        const int set = (int)(sgi & 1);
        // the next segment's recompute overlaps this segment's reverse sweep; its
        // buffer set was last read by the reverse sweep of segment sgi + 1
        if (sgi >= 1) {
            if (sgi + 1 <= nseg - 1) ACK(cudaStreamWaitEvent(st2, rev_done[(sgi + 1) & 1], 0));
            ACK(recompute(sgi - 1));
        }
        ACK(cudaStreamWaitEvent(st, rec_done[set], 0));
        // stream-ordered after the previous segment's reads of gam
        ACK(cudaMemcpyAsync(gam, gam_h.data() + k0, sizeof(T) * (size_t)(k1 - k0),
                            cudaMemcpyHostToDevice, st));
        if (k1 - k0 == K && K > 1) {
            cudaGraphExec_t &ge = graphs[set][parity];
            if (!ge) {
                cudaGraph_t g = nullptr;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    release();
                    return LBD_ECUDA;
                }
                const cudaError_t e1 = reverse_steps(segs[set], k0, k1);
                const cudaError_t e2 = cudaStreamEndCapture(st, &g);
                cudaError_t e3 = cudaErrorUnknown;
                if (e1 == cudaSuccess && e2 == cudaSuccess)
                    e3 = cudaGraphInstantiate(&ge, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e3 != cudaSuccess) {
                    cudaGetLastError();
                    ge = nullptr;
                    release();
                    return LBD_ECUDA;
                }
            } else {
                // replay: the host-side buffer alternation advances as in the capture
                for (int64_t k = 0; k < K; ++k) {
                    T *tp;
                    tp = w.Lphi; w.Lphi = w.Lphi0; w.Lphi0 = tp;
                    tp = w.Lpsi; w.Lpsi = w.Lpsi0; w.Lpsi0 = tp;
                    tp = w.Lbuf; w.Lbuf = w.Lbuf0; w.Lbuf0 = tp;
                }
            }
            if (cudaGraphLaunch(ge, st) != cudaSuccess) {
                cudaGetLastError();
                release();
                return LBD_ECUDA;
            }
        } else {
            const cudaError_t e = reverse_steps(segs[set], k0, k1);
            if (e != cudaSuccess) {
                release();
                return LBD_ECUDA;
            }
        }
        ACK(cudaEventRecord(rev_done[set], st));
        parity ^= (int)((k1 - k0) & 1);
    }
    // dL/dpsi(t0) = lambda psi; dL/dB1 = sum of the per-site accumulator
    std::vector<T> dpsi_t;
    if (job.dpsi_host) {
        dpsi_t.resize((size_t)N);
        ACK(cudaMemcpyAsync(dpsi_t.data(), w.Lpsi, sizeof(T) * N, cudaMemcpyDeviceToHost, st));
    }
    sum_kernel<<<RB, 256, 0, st>>>(N, w.dB1, part);
    ACK(cudaGetLastError());
    std::vector<double> h(RB);
    ACK(cudaMemcpyAsync(h.data(), part, sizeof(double) * RB, cudaMemcpyDeviceToHost, st));
    ACK(cudaStreamSynchronize(st));
    double sb = 0;
    for (int k = 0; k < RB; ++k) sb += h[k];
    *job.dB1 = sb;
    for (size_t k = 0; k < dpsi_t.size(); ++k) job.dpsi_host[k] = (double)dpsi_t[k];
#undef ACK
    release();
    return LBD_OK;
}

template int adjoint_run<float>(const AdjointJob<float> &);
template int adjoint_run<double>(const AdjointJob<double> &);

}  // namespace lbd

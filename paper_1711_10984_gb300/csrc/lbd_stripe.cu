// lbd_stripe.cu -- the coupled time step (arXiv 1711.10984, Sections 2.1-2.3) as
// a stripe-marching kernel for sm_103a.
//
// A CTA of NT threads owns a stripe of NT - 10 output columns and a segment of
// `seg` rows.  Thread c owns lattice column x0 - 5 + c (periodic) for the whole
// launch and marches down the rows; the x-halo (5 columns each side) is the only
// redundant work, the y-halo is paid once per segment.  Per row, five stages run
// as a software pipeline with one barrier per iteration; stage k works two rows
// behind stage k-1 so that it only reads rows finished in earlier iterations:
//
//   loader  phi^n, psi^n row            cp.async, 2 iterations ahead
//   A       mu_phi (Eq. 3), m, grad psi  row l - 2
//   B       F (Eq. 14), pull f_i (cp.async, 2 ahead), u (Eq. 11), BGK + Guo
//           collision (Eqs. 10, 12, 13) on the owned rows            row l - 4
//   C       phi*, psi* donor-cell advection (Eqs. 16-17)            row l - 6
//   D       mu*, m* and p* = psi* m* (Eq. 18 operands)              row l - 8
//   E       phi^{n+1} (Eq. 18), psi^{n+1} (Eq. 19 + source, sink)   row l - 10
//
// x-neighbours come from small row rings in shared memory; each thread keeps
// its own column's stencil history in registers (Win*), in the well-conditioned
// form T = L + R - 2C (x second difference), D = R - L, and the centre values:
//   d/dx = (4 D_r + D_{r-1} + D_{r+1}) / 12
//   d/dy = (C_{r+1} - C_{r-1}) / 2 + (T_{r+1} - T_{r-1}) / 12
//   lap  = (2/3) T_r + (T_{r-1} + T_{r+1}) / 6 + (C_{r+1} - 2 C_r + C_{r-1})
// which are the isotropic D2Q9 stencils (1/3, 1/12 gradient weights; 2/3, 1/6
// Laplacian link weights).  The surfactant divergence of Eq. (19),
// sum_j (2/3 or 1/6)[(psi_j - psi) + (psi + psi_j)(m_j - m)/2], is evaluated
// through the identity  lap psi + (psi lap m + lap(psi m) - m lap psi) / 2.
#include <cstdint>

#include "lbd_internal.h"

namespace lbd {
namespace {

constexpr int LD = 16;  // rows in the phi^n / psi^n ring
constexpr int RD = 4;   // rows in the mu, m, u, mu*, m*, p* rings
constexpr int CD = 8;   // rows in the phi* / psi* ring
constexpr int PS = 3;   // population staging depth (rows in flight)

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

template <typename T>
__device__ __forceinline__ void cp_async(T *dst_smem, const T *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Stencil history of one column: rows r-1 and r are kept; push(r+1) yields the
// derivatives at row r and then advances.
template <typename T>
struct WinLap {
    T cm, c0, tm, t0;
    __device__ __forceinline__ void reset() { cm = c0 = tm = t0 = T(0); }
    // returns lap at the middle row
    __device__ __forceinline__ T push(T c, T l, T r) {
        const T t = (l + r) - T(2) * c;
        const T lap = T(2.0 / 3.0) * t0 + T(1.0 / 6.0) * (tm + t) + ((c - c0) - (c0 - cm));
        cm = c0; c0 = c; tm = t0; t0 = t;
        return lap;
    }
};

template <typename T>
struct WinFull {
    T cm, c0, tm, t0, dm, d0;
    __device__ __forceinline__ void reset() { cm = c0 = tm = t0 = dm = d0 = T(0); }
    // gradient and Laplacian at the middle row; `mid` receives its centre value
    __device__ __forceinline__ void push(T c, T l, T r, T &gx, T &gy, T &lap, T &mid) {
        const T t = (l + r) - T(2) * c;
        const T d = r - l;
        gx = (T(4) * d0 + (dm + d)) * T(1.0 / 12.0);
        gy = T(0.5) * (c - cm) + T(1.0 / 12.0) * (t - tm);
        lap = T(2.0 / 3.0) * t0 + T(1.0 / 6.0) * (tm + t) + ((c - c0) - (c0 - cm));
        mid = c0;
        cm = c0; c0 = c; tm = t0; t0 = t; dm = d0; d0 = d;
    }
    __device__ __forceinline__ void push_grad(T c, T l, T r, T &gx, T &gy, T &mid) {
        const T t = (l + r) - T(2) * c;
        const T d = r - l;
        gx = (T(4) * d0 + (dm + d)) * T(1.0 / 12.0);
        gy = T(0.5) * (c - cm) + T(1.0 / 12.0) * (t - tm);
        mid = c0;
        cm = c0; c0 = c; tm = t0; t0 = t; dm = d0; d0 = d;
    }
};

template <typename T>
struct StripeSmem {
    static constexpr size_t floats(int nt) {
        return (size_t)nt * (2 * LD + 6 * RD + 2 * CD + PS * 9);
    }
};

// Resident CTAs per SM the register allocation is held to: 4 (FP32) or 2 (FP64)
// CTAs of 128 threads, i.e. at most 128 / 255 registers per thread.
template <typename T, int NT>
struct StripeOcc {
    static constexpr int value = (sizeof(T) == 4 ? 512 : 256) / NT;
};

template <typename T, int NT>
__device__ __forceinline__ void stripe_body(const StepArgs<T> &p, const int x0, const int y0,
                                            const int seg, const T A_t, const T gamma_t,
                                            unsigned char *smem_raw) {
    T *s_phi = reinterpret_cast<T *>(smem_raw);  // [LD][NT]
    T *s_psi = s_phi + LD * NT;                   // [LD][NT]
    T *s_mu = s_psi + LD * NT;                    // [RD][NT]  mu_phi      (A -> B)
    T *s_m = s_mu + RD * NT;                      // [RD][NT]  m           (A -> B)
    T *s_ux = s_m + RD * NT;                      // [RD][NT]  u_x         (B -> C)
    T *s_mus = s_ux + RD * NT;                    // [RD][NT]  mu*         (D -> E)
    T *s_ms = s_mus + RD * NT;                    // [RD][NT]  m*          (D -> E)
    T *s_ps = s_ms + RD * NT;                     // [RD][NT]  psi* m*     (D -> E)
    T *s_phs = s_ps + RD * NT;                    // [CD][NT]  phi*        (C -> D, E)
    T *s_pss = s_phs + CD * NT;                   // [CD][NT]  psi*        (C -> D, E)
    T *s_pop = s_pss + CD * NT;                   // [PS][9][NT] pulled populations

    const int c = threadIdx.x;
    const int nx = p.nx, ny = p.ny;
    const long long pitch = p.pitch, plane = p.plane;
    const int xg = wrapi(x0 - 5 + c, nx);
    const int xm = xg == 0 ? nx - 1 : xg - 1;
    const int xp = xg == nx - 1 ? 0 : xg + 1;
    const int cl = c > 0 ? c - 1 : 0, cr = c < NT - 1 ? c + 1 : NT - 1;
    const bool inA = c >= 1 && c < NT - 1;
    const bool inB = c >= 2 && c < NT - 2;
    const bool inC = c >= 3 && c < NT - 3;
    const bool inD = c >= 4 && c < NT - 4;
    const bool inE = c >= 5 && c < NT - 5 && (x0 + c - 5) < nx;
    const int yend = min(y0 + seg, ny);  // owned rows [y0, yend)

    // Wrapped lattice rows of the asynchronous loads, advanced by one per
    // iteration (no integer division in the loop): loader row y0 - 5 + k and the
    // rows rb - 1, rb, rb + 1 around stage-B row rb = y0 - 9 + k.
    int yl = wrapi(y0 - 5, ny);
    int ybm = wrapi(y0 - 10, ny), yb0 = wrapi(y0 - 9, ny), ybp = wrapi(y0 - 8, ny);
    auto adv = [&](int &y) { y = (y + 1 == ny) ? 0 : y + 1; };
    const T *gcm = p.g_in + xm, *gc0 = p.g_in + xg, *gcp = p.g_in + xp;

    // Issue the asynchronous loads of iteration k: phi^n, psi^n of loader row
    // y0 - 5 + k, and the pulled populations of stage-B row y0 - 9 + k.
    auto issue = [&](int k) {
        const int rl = y0 - 5 + k;
        if (rl < yend + 5) {
            const long long o = (long long)yl * pitch + xg;
            const int so = (rl & (LD - 1)) * NT + c;
            cp_async(s_phi + so, p.phi_in + o);
            cp_async(s_psi + so, p.psi_in + o);
        }
        const int rb = y0 - 9 + k;
        if (inB && rb >= y0 - 3 && rb < yend + 3) {
            const long long om = (long long)ybm * pitch, o0 = (long long)yb0 * pitch,
                            op = (long long)ybp * pitch;
            T *dst = s_pop + (k % PS) * 9 * NT + c;
            // plane i of the pull source f_i(x - e_i): walk the planes
            const T *q0 = gc0 + o0, *qm = gcm + o0, *qp = gcp + o0;
            const T *q0m = gc0 + om, *qmm = gcm + om, *qpm = gcp + om;
            const T *q0p = gc0 + op, *qmp = gcm + op, *qpp = gcp + op;
            cp_async(dst + 0 * NT, q0);                // e = ( 0, 0)
            cp_async(dst + 1 * NT, qm + plane);        // e = ( 1, 0) from x - 1
            cp_async(dst + 2 * NT, q0m + 2 * plane);   // e = ( 0, 1) from y - 1
            cp_async(dst + 3 * NT, qp + 3 * plane);    // e = (-1, 0) from x + 1
            cp_async(dst + 4 * NT, q0p + 4 * plane);   // e = ( 0,-1) from y + 1
            cp_async(dst + 5 * NT, qmm + 5 * plane);   // e = ( 1, 1)
            cp_async(dst + 6 * NT, qpm + 6 * plane);   // e = (-1, 1)
            cp_async(dst + 7 * NT, qpp + 7 * plane);   // e = (-1,-1)
            cp_async(dst + 8 * NT, qmp + 8 * plane);   // e = ( 1,-1)
        }
        cp_commit();
        adv(yl);
        adv(ybm);
        adv(yb0);
        adv(ybp);
    };

    WinFull<T> wPhiA, wPsiA, wMuB, wMB, wPhsD, wPssD;
    WinLap<T> wMusE, wMsE, wPssE, wPsE;
    wPhiA.reset(); wPsiA.reset(); wMuB.reset(); wMB.reset(); wPhsD.reset(); wPssD.reset();
    wMusE.reset(); wMsE.reset(); wPssE.reset(); wPsE.reset();
    T gpx1 = 0, gpy1 = 0, gpx2 = 0, gpy2 = 0;  // grad psi from A, 1 and 2 iterations old
    T ux1 = 0, ux2 = 0, uy1 = 0, uy2 = 0, uy3 = 0;  // own u from B, 1..3 iterations old

    const T a = p.a, b = p.b, B0 = p.B0, B1 = p.B1;
    issue(0);
    issue(1);
    const int iters = (yend - y0) + 15;
    for (int i = 0; i < iters; ++i) {
        cp_wait1();
        __syncthreads();
        issue(i + 2);

        // ---- E: phi^{n+1}, psi^{n+1} at row y0 - 15 + i --------------------------
        {
            const int r = y0 - 15 + i;   // output row; pushes row r + 1
            if (i >= 13 && inE) {
                const int s1 = ((r + 1) & (RD - 1)) * NT, s1c = ((r + 1) & (CD - 1)) * NT;
                const T lmu = wMusE.push(s_mus[s1 + c], s_mus[s1 + cl], s_mus[s1 + cr]);
                const T mc = wMsE.c0;
                const T lm = wMsE.push(s_ms[s1 + c], s_ms[s1 + cl], s_ms[s1 + cr]);
                const T psc = wPssE.c0;
                const T lps = wPssE.push(s_pss[s1c + c], s_pss[s1c + cl], s_pss[s1c + cr]);
                const T lp = wPsE.push(s_ps[s1 + c], s_ps[s1 + cl], s_ps[s1 + cr]);
                if (r >= y0) {
                    const T phs = s_phs[(r & (CD - 1)) * NT + c];
                    // Eq. (18): phi* + M lap mu*
                    const T phi_new = phs + p.M * lmu;
                    // Eq. (19): div(D psi grad mu_psi) in the log-free form
                    const T div = lps + T(0.5) * ((psc * lm + lp) - mc * lps);
                    T src = T(0);
                    if (p.theta) {
                        const int gx = x0 + c - 5;
                        const uint32_t w = p.theta[(long long)r * p.theta_words + (gx >> 5)];
                        if ((w >> (gx & 31)) & 1u) src = A_t;
                    }
                    const T psi_new = psc + (p.D * div - gamma_t * (psc - p.c0) + src);
                    const long long o = (long long)r * pitch + (x0 + c - 5);
                    p.phi_out[o] = phi_new;
                    p.psi_out[o] = psi_new;
                }
            }
        }
        // ---- D: mu*, m*, p* at row y0 - 13 + i -----------------------------------
        {
            const int r = y0 - 13 + i;
            if (i >= 10 && inD && r < yend + 1) {
                const int s1 = ((r + 1) & (CD - 1)) * NT;
                T px, py, plap, ph, cx, cy, cs;
                wPhsD.push(s_phs[s1 + c], s_phs[s1 + cl], s_phs[s1 + cr], px, py, plap, ph);
                wPssD.push_grad(s_pss[s1 + c], s_pss[s1 + cl], s_pss[s1 + cr], cx, cy, cs);
                if (i >= 12) {
                    const T pn = s_phi[(r & (LD - 1)) * NT + c];  // phi^n for the cubic
                    const T mus = a * ph + b * (pn * pn * pn) - (B0 + B1 * cs) * plap -
                                  B1 * (px * cx + py * cy);
                    const T ms = T(0.5) * B1 * (px * px + py * py);
                    const int so = (r & (RD - 1)) * NT + c;
                    s_mus[so] = mus;
                    s_ms[so] = ms;
                    s_ps[so] = cs * ms;
                }
            }
        }
        // ---- C: phi*, psi* at row y0 - 11 + i ------------------------------------
        {
            const int r = y0 - 11 + i;
            if (i >= 9 && inC && r < yend + 2) {
                const int sr = (r & (LD - 1)) * NT;
                const int srm = ((r - 1) & (LD - 1)) * NT, srp = ((r + 1) & (LD - 1)) * NT;
                const int su = (r & (RD - 1)) * NT;
                const T uxc = ux2;
                const T ue = T(0.5) * (uxc + s_ux[su + c + 1]);
                const T uw = T(0.5) * (s_ux[su + c - 1] + uxc);
                const T un = T(0.5) * (uy2 + uy1);
                const T us = T(0.5) * (uy3 + uy2);
                const T P0 = s_phi[sr + c], PE = s_phi[sr + c + 1], PW = s_phi[sr + c - 1];
                const T PN = s_phi[srp + c], PS_ = s_phi[srm + c];
                const T C0 = s_psi[sr + c], CE = s_psi[sr + c + 1], CW = s_psi[sr + c - 1];
                const T CN = s_psi[srp + c], CS = s_psi[srm + c];
                const bool pe = ue > T(0), pw = uw > T(0), pn = un > T(0), ps = us > T(0);
                const T fe = ue * (pe ? P0 : PE), fw = uw * (pw ? PW : P0);
                const T fn = un * (pn ? P0 : PN), fs = us * (ps ? PS_ : P0);
                const T ge = ue * (pe ? C0 : CE), gw = uw * (pw ? CW : C0);
                const T gn = un * (pn ? C0 : CN), gs = us * (ps ? CS : C0);
                const int so = (r & (CD - 1)) * NT + c;
                s_phs[so] = P0 - ((fe - fw) + (fn - fs));
                s_pss[so] = C0 - ((ge - gw) + (gn - gs));
            }
        }
        // ---- B: force, moments, collision at row y0 - 9 + i -----------------------
        {
            const int r = y0 - 9 + i;
            T ux = T(0), uy = T(0);
            if (i >= 4 && inB && r < yend + 3) {
                const int s1 = ((r + 1) & (RD - 1)) * NT;
                T mx, my, mc, nx_, ny_, nc;
                wMuB.push_grad(s_mu[s1 + c], s_mu[s1 + cl], s_mu[s1 + cr], mx, my, mc);
                wMB.push_grad(s_m[s1 + c], s_m[s1 + cl], s_m[s1 + cr], nx_, ny_, nc);
                if (i >= 6) {
                    const int sr = (r & (LD - 1)) * NT + c;
                    const T ph = s_phi[sr], ps = s_psi[sr];
                    // Eq. (14) with psi grad mu_psi = grad psi + psi grad m
                    T Fx = -ph * mx - (gpx2 + ps * nx_);
                    T Fy = -ph * my - (gpy2 + ps * ny_);
                    if (p.flags & LBD_BODY_FORCE) {
                        Fx += p.fx;
                        Fy += p.fy;
                    }
                    const T *G = s_pop + (i % PS) * 9 * NT + c;
                    const T g0 = G[0], g1 = G[NT], g2 = G[2 * NT], g3 = G[3 * NT], g4 = G[4 * NT];
                    const T g5 = G[5 * NT], g6 = G[6 * NT], g7 = G[7 * NT], g8 = G[8 * NT];
                    // Eq. (11) on the deviations g = f - w
                    const T dn = g0 + ((g1 + g2) + (g3 + g4)) + ((g5 + g6) + (g7 + g8));
                    const T jx = (g1 - g3) + (g5 - g6) + (g8 - g7);
                    const T jy = (g2 - g4) + (g5 + g6) - (g7 + g8);
                    const T n = T(1) + dn;
                    const T inv = T(1) / n;
                    ux = (jx + T(0.5) * Fx) * inv;
                    uy = (jy + T(0.5) * Fy) * inv;
                    if (r >= y0 && r < yend && inE) {
                        // BGK + Guo (Eqs. 10, 12, 13), opposite directions paired:
                        // post_i = (1-w) g_i + W (K + eu (c1 eu + c2 eF)) +- W (c3 eu + c4 eF)
                        const T om = p.omega, gk = p.guo, om1 = T(1) - om;
                        const T usq = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
                        const T K = om * (dn - T(1.5) * n * usq) - T(3) * gk * uF;
                        const T c1 = T(4.5) * om * n, c2 = T(9) * gk;
                        const T c3 = T(3) * om * n, c4 = T(3) * gk;
                        T *Go = p.g_out + (long long)r * pitch + (x0 + c - 5);
                        Go[0] = om1 * g0 + T(4.0 / 9.0) * K;
#define LBD_PAIR(I, J, W, EU, EF)                                       \
    {                                                                   \
        const T eu = (EU), eF = (EF);                                   \
        const T sym = T(W) * (K + eu * (c1 * eu + c2 * eF));            \
        const T anti = T(W) * (c3 * eu + c4 * eF);                      \
        Go[(I) * plane] = om1 * g##I + (sym + anti);                    \
        Go[(J) * plane] = om1 * g##J + (sym - anti);                    \
    }
                        LBD_PAIR(1, 3, 1.0 / 9.0, ux, Fx)
                        LBD_PAIR(2, 4, 1.0 / 9.0, uy, Fy)
                        LBD_PAIR(5, 7, 1.0 / 36.0, ux + uy, Fx + Fy)
                        LBD_PAIR(6, 8, 1.0 / 36.0, uy - ux, Fy - Fx)
#undef LBD_PAIR
                    }
                    if (p.flags & LBD_FROZEN_U) {
                        ux = p.ux0;
                        uy = p.uy0;
                    }
                    s_ux[(r & (RD - 1)) * NT + c] = ux;
                }
            }
            // own-column u history for stage C (rows r-1, r-2, r-3 next iteration)
            uy3 = uy2; uy2 = uy1; uy1 = uy;
            ux2 = ux1; ux1 = ux;
        }
        // ---- A: mu_phi, m, grad psi at row y0 - 7 + i -----------------------------
        {
            const int r = y0 - 7 + i;
            T gx = T(0), gy = T(0);
            if (i >= 1 && inA && r < yend + 4) {
                const int s1 = ((r + 1) & (LD - 1)) * NT;
                T px, py, plap, ph, cs;
                wPhiA.push(s_phi[s1 + c], s_phi[s1 + cl], s_phi[s1 + cr], px, py, plap, ph);
                wPsiA.push_grad(s_psi[s1 + c], s_psi[s1 + cl], s_psi[s1 + cr], gx, gy, cs);
                if (i >= 3) {
                    const int so = (r & (RD - 1)) * NT + c;
                    s_mu[so] = a * ph + b * (ph * ph * ph) - (B0 + B1 * cs) * plap -
                               B1 * (px * gx + py * gy);
                    s_m[so] = T(0.5) * B1 * (px * px + py * py);
                }
            }
            gpx2 = gpx1; gpy2 = gpy1; gpx1 = gx; gpy1 = gy;
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, StripeOcc<T, NT>::value)
    stripe_kernel(const StepArgs<T> p, const int seg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stripe_body<T, NT>(p, blockIdx.x * (NT - 10), blockIdx.y * seg, seg, p.A, p.gamma, smem_raw);
}

// Batched step: CTAs walk the work list; the arguments of the item's instance
// are staged in shared memory and the activity is evaluated from the device
// step count (so that the launch can be replayed from a CUDA graph).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, StripeOcc<T, NT>::value)
    stripe_batch_kernel(const StepArgs<T> *args, const BatchItem *items, const int n_items,
                        const long long *t_dev, const int t_off) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StepArgs<T> sp;
    __shared__ T s_A, s_gamma;
    const long long t = *t_dev + t_off;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem item = items[it];
        if (threadIdx.x == 0) {
            sp = args[item.k];
            double A = 0.0, g = 0.0;
            if (t >= sp.t_on) {
                A = sp.A0 * (double)(t - sp.t_on);
                A = A < sp.A_max ? A : sp.A_max;
                g = sp.gamma_on;
            }
            s_A = (T)A;
            s_gamma = (T)g;
        }
        __syncthreads();
        stripe_body<T, NT>(sp, item.x0, item.y0, item.rows, s_A, s_gamma, smem_raw);
        __syncthreads();
    }
}

__global__ void time_advance_kernel(long long *t, long long add) { *t += add; }
__global__ void time_set_kernel(long long *t, long long v) { *t = v; }

}  // namespace

template <typename T>
size_t stripe_smem_bytes(int nt) {
    return sizeof(T) * StripeSmem<T>::floats(nt);
}

template <typename T>
cudaError_t launch_stripe(const StepArgs<T> &a, int nt, int seg, cudaStream_t s) {
    const size_t smem = stripe_smem_bytes<T>(nt);
    static unsigned long long configured[2] = {0, 0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int which = nt == 128 ? 0 : 1;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured[which] & bit)) {
        e = nt == 128 ? cudaFuncSetAttribute(stripe_kernel<T, 128>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(stripe_kernel<T, 256>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[which] |= bit;
    }
    dim3 grid((a.nx + (nt - 10) - 1) / (nt - 10), (a.ny + seg - 1) / seg);
    if (nt == 128)
        stripe_kernel<T, 128><<<grid, 128, smem, s>>>(a, seg);
    else if (nt == 256)
        stripe_kernel<T, 256><<<grid, 256, smem, s>>>(a, seg);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stripe_batch(const StepArgs<T> *args, const BatchItem *items, int n_items,
                                int nt, int ctas, const long long *t_dev, int t_off,
                                cudaStream_t s) {
    const size_t smem = stripe_smem_bytes<T>(nt);
    static unsigned long long configured[2] = {0, 0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int which = nt == 128 ? 0 : 1;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured[which] & bit)) {
        e = nt == 128
                ? cudaFuncSetAttribute(stripe_batch_kernel<T, 128>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                : cudaFuncSetAttribute(stripe_batch_kernel<T, 256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[which] |= bit;
    }
    if (nt == 128)
        stripe_batch_kernel<T, 128><<<ctas, 128, smem, s>>>(args, items, n_items, t_dev, t_off);
    else if (nt == 256)
        stripe_batch_kernel<T, 256><<<ctas, 256, smem, s>>>(args, items, n_items, t_dev, t_off);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
int stripe_batch_ctas_per_sm(int nt) {
    int n = 0;
    const size_t smem = stripe_smem_bytes<T>(nt);
    cudaError_t e = nt == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &n, stripe_batch_kernel<T, 128>, 128, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &n, stripe_batch_kernel<T, 256>, 256, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}
template int stripe_batch_ctas_per_sm<float>(int);
template int stripe_batch_ctas_per_sm<double>(int);

cudaError_t launch_time_advance(long long *t_dev, long long add, cudaStream_t s) {
    time_advance_kernel<<<1, 1, 0, s>>>(t_dev, add);
    return cudaGetLastError();
}
cudaError_t launch_time_set(long long *t_dev, long long value, cudaStream_t s) {
    time_set_kernel<<<1, 1, 0, s>>>(t_dev, value);
    return cudaGetLastError();
}

template cudaError_t launch_stripe_batch<float>(const StepArgs<float> *, const BatchItem *, int,
                                                int, int, const long long *, int, cudaStream_t);
template cudaError_t launch_stripe_batch<double>(const StepArgs<double> *, const BatchItem *, int,
                                                 int, int, const long long *, int, cudaStream_t);
template cudaError_t launch_stripe<float>(const StepArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stripe<double>(const StepArgs<double> &, int, int, cudaStream_t);
template size_t stripe_smem_bytes<float>(int);
template size_t stripe_smem_bytes<double>(int);

}  // namespace lbd

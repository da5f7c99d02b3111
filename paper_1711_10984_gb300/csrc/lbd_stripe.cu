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
#include <type_traits>

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
    // rings of padded rows (NT + 2 elements: a pad on each side, so that the
    // x-neighbours of every thread are in bounds) plus the population staging
    static constexpr size_t floats(int nt) {
        return (size_t)(nt + 2) * (2 * LD + 6 * RD + 2 * CD) + (size_t)nt * PS * 9;
    }
};

// Resident CTAs per SM the register allocation is held to: 4 (FP32) or 2 (FP64)
// CTAs of 128 threads, i.e. at most 128 / 255 registers per thread.
template <typename T, int NT>
struct StripeOcc {
    static constexpr int value = (sizeof(T) == 4 ? 512 : 256) / NT;
};

template <int OFF>
__device__ __forceinline__ void cp4(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0+%2], [%1], 4;\n" ::"r"(dst), "l"(src), "n"(OFF));
}
template <int OFF>
__device__ __forceinline__ void cp8(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0+%2], [%1], 8;\n" ::"r"(dst), "l"(src), "n"(OFF));
}

template <typename T, int NT>
__device__ __forceinline__ void stripe_body(const StepArgs<T> &p, const int x0, const int y0,
                                            const int seg, const T A_t, const T gamma_t,
                                            unsigned char *smem_raw) {
    constexpr int RS = NT + 2;  // padded ring row
    const int c = threadIdx.x;
    // this thread's element in slot 0 of each ring (x-neighbours at -1, +1)
    T *const s_phi = reinterpret_cast<T *>(smem_raw) + 1 + c;  // [LD] rows
    T *const s_psi = s_phi + LD * RS;                            // [LD]
    T *const s_mu = s_psi + LD * RS;                             // [RD]  mu_phi   (A -> B)
    T *const s_m = s_mu + RD * RS;                               // [RD]  m        (A -> B)
    T *const s_ux = s_m + RD * RS;                               // [RD]  u_x      (B -> C)
    T *const s_mus = s_ux + RD * RS;                             // [RD]  mu*      (D -> E)
    T *const s_ms = s_mus + RD * RS;                             // [RD]  m*       (D -> E)
    T *const s_ps = s_ms + RD * RS;                              // [RD]  psi* m*  (D -> E)
    T *const s_phs = s_ps + RD * RS;                             // [CD]  phi*     (C -> D, E)
    T *const s_pss = s_phs + CD * RS;                            // [CD]  psi*     (C -> D, E)
    T *const s_pop = reinterpret_cast<T *>(smem_raw) + (2 * LD + 6 * RD + 2 * CD) * RS + c;
    const unsigned u_phi = (unsigned)__cvta_generic_to_shared(s_phi);
    const unsigned u_psi = (unsigned)__cvta_generic_to_shared(s_psi);
    const unsigned u_pop = (unsigned)__cvta_generic_to_shared(s_pop);

    const int nx = p.nx, ny = p.ny;
    constexpr unsigned TB = sizeof(T);
    // byte offsets fit 32 bits (the host routes larger lattices to the tiled kernel)
    const unsigned pitch_b = (unsigned)p.pitch * TB, plane_b = (unsigned)p.plane * TB;
    const unsigned rows_b = (unsigned)ny * pitch_b;
    const int xg = wrapi(x0 - 5 + c, nx);
    const unsigned xg_b = (unsigned)xg * TB;
    const unsigned xm_b = (unsigned)(xg == 0 ? nx - 1 : xg - 1) * TB;
    const unsigned xp_b = (unsigned)(xg == nx - 1 ? 0 : xg + 1) * TB;
    const bool inA = c >= 1 && c < NT - 1;
    const bool inB = c >= 2 && c < NT - 2;
    const bool inC = c >= 3 && c < NT - 3;
    const bool inD = c >= 4 && c < NT - 4;
    const int xo = x0 + c - 5;  // output column of this thread
    const bool inE = c >= 5 && c < NT - 5 && xo < nx;
    const unsigned xo_b = (unsigned)xo * TB;
    const int yend = min(y0 + seg, ny);  // owned rows [y0, yend)

    // Byte offsets of the asynchronously loaded rows, advanced by one row per
    // iteration: loader row y0 - 5 + k and the rows rb - 1, rb, rb + 1 around
    // stage-B row rb = y0 - 9 + k.
    unsigned lo_b = (unsigned)wrapi(y0 - 5, ny) * pitch_b + xg_b;
    unsigned rm_b = (unsigned)wrapi(y0 - 10, ny) * pitch_b;
    unsigned r0_b = (unsigned)wrapi(y0 - 9, ny) * pitch_b;
    unsigned rp_b = (unsigned)wrapi(y0 - 8, ny) * pitch_b;
    auto adv = [&](unsigned &o) {
        o += pitch_b;
        if (o >= rows_b) o -= rows_b;
    };
    const char *const phi_in = reinterpret_cast<const char *>(p.phi_in);
    const char *const psi_in = reinterpret_cast<const char *>(p.psi_in);
    const char *const g_in = reinterpret_cast<const char *>(p.g_in);

    // Issue the asynchronous loads of iteration k: phi^n, psi^n of loader row
    // y0 - 5 + k, and the pulled populations f_i(x - e_i) of stage-B row y0 - 9 + k.
    auto issue = [&](int k) {
        const int rl = y0 - 5 + k;
        if (rl < yend + 5) {
            const unsigned so = (unsigned)((rl & (LD - 1)) * RS) * TB;
            if (TB == 8) {
                cp8<0>(u_phi + so, phi_in + lo_b);
                cp8<0>(u_psi + so, psi_in + lo_b);
            } else {
                cp4<0>(u_phi + so, phi_in + lo_b);
                cp4<0>(u_psi + so, psi_in + lo_b);
            }
        }
        const int rb = y0 - 9 + k;
        if (inB && rb >= y0 - 3 && rb < yend + 3) {
            const unsigned d = u_pop + (unsigned)((k % PS) * 9 * NT) * TB;
            constexpr int P = NT * (int)sizeof(T);
#define LBD_PULL(I, ROW, COL)                                                              \
    if (TB == 8) cp8<(I) * P>(d, g_in + ((I) * plane_b + ROW + COL));                     \
    else cp4<(I) * P>(d, g_in + ((I) * plane_b + ROW + COL));
            LBD_PULL(0, r0_b, xg_b)  // e = ( 0, 0)
            LBD_PULL(1, r0_b, xm_b)  // e = ( 1, 0) from x - 1
            LBD_PULL(2, rm_b, xg_b)  // e = ( 0, 1) from y - 1
            LBD_PULL(3, r0_b, xp_b)  // e = (-1, 0) from x + 1
            LBD_PULL(4, rp_b, xg_b)  // e = ( 0,-1) from y + 1
            LBD_PULL(5, rm_b, xm_b)  // e = ( 1, 1)
            LBD_PULL(6, rm_b, xp_b)  // e = (-1, 1)
            LBD_PULL(7, rp_b, xp_b)  // e = (-1,-1)
            LBD_PULL(8, rp_b, xm_b)  // e = ( 1,-1)
#undef LBD_PULL
        }
        cp_commit();
        adv(lo_b);
        adv(rm_b);
        adv(r0_b);
        adv(rp_b);
    };

    WinFull<T> wPhiA, wPsiA, wMuB, wMB, wPhsD, wPssD;
    WinLap<T> wMusE, wMsE, wPssE, wPsE;
    wPhiA.reset(); wPsiA.reset(); wMuB.reset(); wMB.reset(); wPhsD.reset(); wPssD.reset();
    wMusE.reset(); wMsE.reset(); wPssE.reset(); wPsE.reset();
    T gpx1 = 0, gpy1 = 0, gpx2 = 0, gpy2 = 0;  // grad psi from A, 1 and 2 iterations old
    T ux1 = 0, ux2 = 0, uy1 = 0, uy2 = 0, uy3 = 0;  // own u from B, 1..3 iterations old

    const T a = p.a, b = p.b, B0 = p.B0, B1 = p.B1;
    char *const g_out = reinterpret_cast<char *>(p.g_out);
    char *const phi_out = reinterpret_cast<char *>(p.phi_out);
    char *const psi_out = reinterpret_cast<char *>(p.psi_out);
    issue(0);
    issue(1);
    const int iters = (yend - y0) + 15;
    // One pipeline iteration; with GUARD false (steady state: every stage active,
    // every row written is owned) the row conditions vanish at compile time.
    auto body = [&](auto guard_tag, const int i) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        cp_wait1();
        __syncthreads();
        issue(i + 2);

        // ---- E: phi^{n+1}, psi^{n+1} at row y0 - 15 + i --------------------------
        {
            const int r = y0 - 15 + i;   // output row; pushes row r + 1
            if ((!GUARD || i >= 13) && inE) {
                const T *M1 = s_mus + ((r + 1) & (RD - 1)) * RS;
                const T *N1 = s_ms + ((r + 1) & (RD - 1)) * RS;
                const T *P1 = s_ps + ((r + 1) & (RD - 1)) * RS;
                const T *C1 = s_pss + ((r + 1) & (CD - 1)) * RS;
                const T lmu = wMusE.push(M1[0], M1[-1], M1[1]);
                const T mc = wMsE.c0;
                const T lm = wMsE.push(N1[0], N1[-1], N1[1]);
                const T psc = wPssE.c0;
                const T lps = wPssE.push(C1[0], C1[-1], C1[1]);
                const T lp = wPsE.push(P1[0], P1[-1], P1[1]);
                if (!GUARD || r >= y0) {
                    const T phs = s_phs[(r & (CD - 1)) * RS];
                    // Eq. (18): phi* + M lap mu*
                    const T phi_new = phs + p.M * lmu;
                    // Eq. (19): div(D psi grad mu_psi) in the log-free form
                    const T div = lps + T(0.5) * ((psc * lm + lp) - mc * lps);
                    T src = T(0);
                    if (p.theta) {
                        const uint32_t w = p.theta[r * p.theta_words + (xo >> 5)];
                        if ((w >> (xo & 31)) & 1u) src = A_t;
                    }
                    const T psi_new = psc + (p.D * div - gamma_t * (psc - p.c0) + src);
                    const unsigned o = (unsigned)r * pitch_b + xo_b;
                    *reinterpret_cast<T *>(phi_out + o) = phi_new;
                    *reinterpret_cast<T *>(psi_out + o) = psi_new;
                }
            }
        }
        // ---- D: mu*, m*, p* at row y0 - 13 + i -----------------------------------
        {
            const int r = y0 - 13 + i;
            if ((!GUARD || (i >= 10 && r < yend + 1)) && inD) {
                const T *F1 = s_phs + ((r + 1) & (CD - 1)) * RS;
                const T *S1 = s_pss + ((r + 1) & (CD - 1)) * RS;
                T px, py, plap, ph, cx, cy, cs;
                wPhsD.push(F1[0], F1[-1], F1[1], px, py, plap, ph);
                wPssD.push_grad(S1[0], S1[-1], S1[1], cx, cy, cs);
                if (!GUARD || i >= 12) {
                    const T pn = s_phi[(r & (LD - 1)) * RS];  // phi^n for the cubic
                    const T mus = a * ph + b * (pn * pn * pn) - (B0 + B1 * cs) * plap -
                                  B1 * (px * cx + py * cy);
                    const T ms = T(0.5) * B1 * (px * px + py * py);
                    const int so = (r & (RD - 1)) * RS;
                    s_mus[so] = mus;
                    s_ms[so] = ms;
                    s_ps[so] = cs * ms;
                }
            }
        }
        // ---- C: phi*, psi* at row y0 - 11 + i ------------------------------------
        {
            const int r = y0 - 11 + i;
            if ((!GUARD || (i >= 9 && r < yend + 2)) && inC) {
                const T *P = s_phi + (r & (LD - 1)) * RS, *Q = s_psi + (r & (LD - 1)) * RS;
                const T *Pn = s_phi + ((r + 1) & (LD - 1)) * RS, *Qn = s_psi + ((r + 1) & (LD - 1)) * RS;
                const T *Ps = s_phi + ((r - 1) & (LD - 1)) * RS, *Qs = s_psi + ((r - 1) & (LD - 1)) * RS;
                const T *U = s_ux + (r & (RD - 1)) * RS;
                const T uxc = ux2;
                const T ue = T(0.5) * (uxc + U[1]);
                const T uw = T(0.5) * (U[-1] + uxc);
                const T un = T(0.5) * (uy2 + uy1);
                const T us = T(0.5) * (uy3 + uy2);
                const T P0 = P[0], PE = P[1], PW = P[-1], PN = Pn[0], PS_ = Ps[0];
                const T C0 = Q[0], CE = Q[1], CW = Q[-1], CN = Qn[0], CS = Qs[0];
                const bool pe = ue > T(0), pw = uw > T(0), pn = un > T(0), ps = us > T(0);
                const T fe = ue * (pe ? P0 : PE), fw = uw * (pw ? PW : P0);
                const T fn = un * (pn ? P0 : PN), fs = us * (ps ? PS_ : P0);
                const T ge = ue * (pe ? C0 : CE), gw = uw * (pw ? CW : C0);
                const T gn = un * (pn ? C0 : CN), gs = us * (ps ? CS : C0);
                const int so = (r & (CD - 1)) * RS;
                s_phs[so] = P0 - ((fe - fw) + (fn - fs));
                s_pss[so] = C0 - ((ge - gw) + (gn - gs));
            }
        }
        // ---- B: force, moments, collision at row y0 - 9 + i -----------------------
        {
            const int r = y0 - 9 + i;
            T ux = T(0), uy = T(0);
            if ((!GUARD || (i >= 4 && r < yend + 3)) && inB) {
                const T *M1 = s_mu + ((r + 1) & (RD - 1)) * RS;
                const T *N1 = s_m + ((r + 1) & (RD - 1)) * RS;
                T mx, my, mc, nx_, ny_, nc;
                wMuB.push_grad(M1[0], M1[-1], M1[1], mx, my, mc);
                wMB.push_grad(N1[0], N1[-1], N1[1], nx_, ny_, nc);
                if (!GUARD || i >= 6) {
                    const int sr = (r & (LD - 1)) * RS;
                    const T ph = s_phi[sr], ps = s_psi[sr];
                    // Eq. (14) with psi grad mu_psi = grad psi + psi grad m
                    T Fx = -ph * mx - (gpx2 + ps * nx_);
                    T Fy = -ph * my - (gpy2 + ps * ny_);
                    if (p.flags & LBD_BODY_FORCE) {
                        Fx += p.fx;
                        Fy += p.fy;
                    }
                    const T *G = s_pop + (i % PS) * 9 * NT;
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
                    if ((!GUARD || (r >= y0 && r < yend)) && inE) {
                        // BGK + Guo (Eqs. 10, 12, 13), opposite directions paired:
                        // post_i = (1-w) g_i + W (K + eu (c1 eu + c2 eF)) +- W (c3 eu + c4 eF)
                        const T om = p.omega, gk = p.guo, om1 = T(1) - om;
                        const T usq = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
                        const T K = om * (dn - T(1.5) * n * usq) - T(3) * gk * uF;
                        const T c1 = T(4.5) * om * n, c2 = T(9) * gk;
                        const T c3 = T(3) * om * n, c4 = T(3) * gk;
                        char *Go = g_out + ((unsigned)r * pitch_b + xo_b);
#define LBD_OUT(I) (*reinterpret_cast<T *>(Go + (I) * plane_b))
                        LBD_OUT(0) = om1 * g0 + T(4.0 / 9.0) * K;
#define LBD_PAIR(I, J, W, EU, EF)                                       \
    {                                                                   \
        const T eu = (EU), eF = (EF);                                   \
        const T sym = T(W) * (K + eu * (c1 * eu + c2 * eF));            \
        const T anti = T(W) * (c3 * eu + c4 * eF);                      \
        LBD_OUT(I) = om1 * g##I + (sym + anti);                         \
        LBD_OUT(J) = om1 * g##J + (sym - anti);                         \
    }
                        LBD_PAIR(1, 3, 1.0 / 9.0, ux, Fx)
                        LBD_PAIR(2, 4, 1.0 / 9.0, uy, Fy)
                        LBD_PAIR(5, 7, 1.0 / 36.0, ux + uy, Fx + Fy)
                        LBD_PAIR(6, 8, 1.0 / 36.0, uy - ux, Fy - Fx)
#undef LBD_PAIR
#undef LBD_OUT
                    }
                    if (p.flags & LBD_FROZEN_U) {
                        ux = p.ux0;
                        uy = p.uy0;
                    }
                    s_ux[(r & (RD - 1)) * RS] = ux;
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
            if ((!GUARD || (i >= 1 && r < yend + 4)) && inA) {
                const T *F1 = s_phi + ((r + 1) & (LD - 1)) * RS;
                const T *S1 = s_psi + ((r + 1) & (LD - 1)) * RS;
                T px, py, plap, ph, cs;
                wPhiA.push(F1[0], F1[-1], F1[1], px, py, plap, ph);
                wPsiA.push_grad(S1[0], S1[-1], S1[1], gx, gy, cs);
                if (!GUARD || i >= 3) {
                    const int so = (r & (RD - 1)) * RS;
                    s_mu[so] = a * ph + b * (ph * ph * ph) - (B0 + B1 * cs) * plap -
                               B1 * (px * gx + py * gy);
                    s_m[so] = T(0.5) * B1 * (px * px + py * py);
                }
            }
            gpx2 = gpx1; gpy2 = gpy1; gpx1 = gx; gpy1 = gy;
        }
    };
    const std::integral_constant<bool, true> guarded;
    const std::integral_constant<bool, false> steady;
    const int s1 = (yend - y0) + 9;
    int i = 0;
    for (; i < 15 && i < iters; ++i) body(guarded, i);
#pragma unroll 2
    for (; i < s1; ++i) body(steady, i);
    for (; i < iters; ++i) body(guarded, i);
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

// lbd_stripe2.cu -- FP32 coupled step (arXiv 1711.10984, Sections 2.1-2.3) with
// two lattice columns per thread and packed FP32x2 arithmetic (sm_100+ FADD2 /
// FMUL2 / FFMA2 through __fadd2_rn, __fmul2_rn, __ffma2_rn).
//
// Same stripe-marching pipeline as lbd_stripe.cu (loader, A..E, two rows of lag
// per stage, one barrier per row); a CTA of NT = 128 threads covers W = 256
// columns x0 - 8 .. x0 + 247 and writes the 240 columns x0 .. x0 + 239.  Thread t
// owns the column pair (2t, 2t + 1): every per-site formula runs once on the
// pair, own values move as 8-byte shared-memory words and only the two outer
// neighbours are fetched separately.  Rows of phi^n, psi^n and the nine pulled
// population planes are staged by 16-byte cp.async copies (cache-global),
// which needs nx to be a multiple of 4 and at least W + 8 (otherwise the
// library uses the one-column kernel).
#include <cstdint>
#include <type_traits>

#include "lbd_internal.h"

namespace lbd {
namespace {

constexpr int NT2 = 128;        // threads per CTA
constexpr int W2C = 2 * NT2;    // columns per CTA
constexpr int HX = 8;           // halo columns on each side (16-byte aligned)
constexpr int SW = W2C + 8;     // staged population row: columns x0 - 12 .. x0 + 251
constexpr int LD2 = 16, RD2 = 4, CD2 = 8, PS2 = 3;

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one packed FMA: fma(b, -1, a) rounds once, like a subtraction
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 S2(float s) { return make_float2(s, s); }

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp16(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

// Register stencil history of a column pair (see lbd_stripe.cu for the form).
struct Win2 {
    float2 cm, c0, tm, t0, dm, d0;
    __device__ __forceinline__ void reset() {
        cm = c0 = tm = t0 = dm = d0 = S2(0.f);
    }
    __device__ __forceinline__ void push(float2 c, float2 l, float2 r, float2 &gx, float2 &gy,
                                         float2 &lap, float2 &mid) {
        const float2 t = fma2(c, S2(-2.f), l + r);
        const float2 d = r - l;
        gx = fma2(d0, S2(4.f), dm + d) * S2(1.f / 12.f);
        gy = fma2(c - cm, S2(0.5f), (t - tm) * S2(1.f / 12.f));
        lap = fma2(t0, S2(2.f / 3.f), fma2(tm + t, S2(1.f / 6.f), (c - c0) - (c0 - cm)));
        mid = c0;
        cm = c0; c0 = c; tm = t0; t0 = t; dm = d0; d0 = d;
    }
    __device__ __forceinline__ void push_grad(float2 c, float2 l, float2 r, float2 &gx, float2 &gy,
                                              float2 &mid) {
        const float2 t = fma2(c, S2(-2.f), l + r);
        const float2 d = r - l;
        gx = fma2(d0, S2(4.f), dm + d) * S2(1.f / 12.f);
        gy = fma2(c - cm, S2(0.5f), (t - tm) * S2(1.f / 12.f));
        mid = c0;
        cm = c0; c0 = c; tm = t0; t0 = t; dm = d0; d0 = d;
    }
};

struct WinLap2 {
    float2 cm, c0, tm, t0;
    __device__ __forceinline__ void reset() { cm = c0 = tm = t0 = S2(0.f); }
    __device__ __forceinline__ float2 push(float2 c, float2 l, float2 r) {
        const float2 t = fma2(c, S2(-2.f), l + r);
        const float2 lap =
            fma2(t0, S2(2.f / 3.f), fma2(tm + t, S2(1.f / 6.f), (c - c0) - (c0 - cm)));
        cm = c0; c0 = c; tm = t0; t0 = t;
        return lap;
    }
};

// Own pair and its two outer neighbours from a shared row of W2C floats.
struct Nb {
    float2 c, l, r;
};
__device__ __forceinline__ Nb nb(const float *row, int t) {
    Nb n;
    n.c = *reinterpret_cast<const float2 *>(row + 2 * t);
    const float lo = row[t > 0 ? 2 * t - 1 : 0];
    const float hi = row[t < NT2 - 1 ? 2 * t + 2 : W2C - 1];
    n.l = make_float2(lo, n.c.x);
    n.r = make_float2(n.c.y, hi);
    return n;
}
__device__ __forceinline__ float2 ld2(const float *row, int t) {
    return *reinterpret_cast<const float2 *>(row + 2 * t);
}
__device__ __forceinline__ void st2(float *row, int t, float2 v) {
    *reinterpret_cast<float2 *>(row + 2 * t) = v;
}

constexpr size_t kSmemFloats =
    (size_t)2 * LD2 * W2C + (size_t)6 * RD2 * W2C + (size_t)2 * CD2 * W2C + (size_t)PS2 * 9 * SW;

__global__ void __launch_bounds__(NT2, 2) pair_kernel(const StepArgs<float> p, const int seg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_phi = reinterpret_cast<float *>(smem_raw);  // [LD2][W2C]
    float *s_psi = s_phi + LD2 * W2C;
    float *s_mu = s_psi + LD2 * W2C;                     // [RD2][W2C]
    float *s_m = s_mu + RD2 * W2C;
    float *s_ux = s_m + RD2 * W2C;
    float *s_mus = s_ux + RD2 * W2C;
    float *s_ms = s_mus + RD2 * W2C;
    float *s_ps = s_ms + RD2 * W2C;
    float *s_phs = s_ps + RD2 * W2C;                     // [CD2][W2C]
    float *s_pss = s_phs + CD2 * W2C;
    float *s_pop = s_pss + CD2 * W2C;                    // [PS2][9][SW]

    const int t = threadIdx.x;
    const int nx = p.nx, ny = p.ny;
    const long long pitch = p.pitch, plane = p.plane;
    const int x0 = blockIdx.x * (W2C - 2 * HX);
    const int y0 = blockIdx.y * seg;
    const int yend = min(y0 + seg, ny);
    const int xo = x0 - HX + 2 * t;                     // global column of .x (unwrapped)
    const bool out = t >= HX / 2 && t < NT2 - HX / 2 && xo < nx;

    // loader: thread t copies 16 bytes (4 columns) of phi (t < 64) or psi (t >= 64)
    const int lchunk = t & 63;
    int lx = x0 - HX + 4 * lchunk;
    lx = lx < 0 ? lx + nx : (lx >= nx ? lx - nx : lx);
    const float *lsrc = (t < 64 ? p.phi_in : p.psi_in) + lx;
    float *ldst = (t < 64 ? s_phi : s_psi) + 4 * lchunk;

    int yl = wrapi(y0 - 5, ny);
    int ybm = wrapi(y0 - 10, ny), yb0 = wrapi(y0 - 9, ny), ybp = wrapi(y0 - 8, ny);
    auto adv = [&](int &y) { y = (y + 1 == ny) ? 0 : y + 1; };

    auto issue = [&](int k) {
        const int rl = y0 - 5 + k;
        if (rl < yend + 5) cp16(ldst + (rl & (LD2 - 1)) * W2C, lsrc + (long long)yl * pitch);
        const int rb = y0 - 9 + k;
        if (rb >= y0 - 3 && rb < yend + 3) {
            const long long om = (long long)ybm * pitch, o0 = (long long)yb0 * pitch,
                            op = (long long)ybp * pitch;
            float *dst = s_pop + (k % PS2) * 9 * SW;
            // 9 planes x 66 chunks of 16 bytes, columns x0 - 12 + 4 j
            for (int q = t; q < 9 * (SW / 4); q += NT2) {
                const int i = q / (SW / 4), j = q - i * (SW / 4);
                // source row of plane i: y - e_y (rows rb - 1, rb, rb + 1 -> index 0, 1, 2)
                const int ey = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
                int xs = x0 - 12 + 4 * j;
                xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                const long long ro = ey > 0 ? om : (ey < 0 ? op : o0);
                cp16(dst + i * SW + 4 * j, p.g_in + i * plane + ro + xs);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
        adv(yl); adv(ybm); adv(yb0); adv(ybp);
    };

    Win2 wPhiA, wPsiA, wMuB, wMB, wPhsD, wPssD;
    WinLap2 wMusE, wMsE, wPssE, wPsE;
    wPhiA.reset(); wPsiA.reset(); wMuB.reset(); wMB.reset(); wPhsD.reset(); wPssD.reset();
    wMusE.reset(); wMsE.reset(); wPssE.reset(); wPsE.reset();
    float2 gpx1 = S2(0.f), gpy1 = S2(0.f), gpx2 = S2(0.f), gpy2 = S2(0.f);
    float2 ux1 = S2(0.f), ux2 = S2(0.f), uy1 = S2(0.f), uy2 = S2(0.f), uy3 = S2(0.f);

    const float2 a2 = S2(p.a), b2 = S2(p.b), B02 = S2(p.B0), B12 = S2(p.B1);
    const float2 hB1 = S2(0.5f * p.B1);
    issue(0);
    issue(1);
    const int iters = (yend - y0) + 15;
    // One pipeline iteration.  With GUARD false (the steady state, where every
    // stage is active and every row it writes is owned) the stage conditions
    // vanish at compile time, so the compiler can interleave the stages.
    auto body = [&](auto guard_tag, const int i) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        asm volatile("cp.async.wait_group 1;\n" ::);
        __syncthreads();
        issue(i + 2);

        // ---- E: phi^{n+1}, psi^{n+1} ---------------------------------------------
        {
            const int r = y0 - 15 + i;
            if (!GUARD || (i >= 13 && r < yend)) {
                const Nb mu = nb(s_mus + ((r + 1) & (RD2 - 1)) * W2C, t);
                const Nb ms = nb(s_ms + ((r + 1) & (RD2 - 1)) * W2C, t);
                const Nb ps = nb(s_pss + ((r + 1) & (CD2 - 1)) * W2C, t);
                const Nb pp = nb(s_ps + ((r + 1) & (RD2 - 1)) * W2C, t);
                const float2 mc = wMsE.c0, psc = wPssE.c0;
                const float2 lmu = wMusE.push(mu.c, mu.l, mu.r);
                const float2 lm = wMsE.push(ms.c, ms.l, ms.r);
                const float2 lps = wPssE.push(ps.c, ps.l, ps.r);
                const float2 lp = wPsE.push(pp.c, pp.l, pp.r);
                if ((!GUARD || r >= y0) && out) {
                    const float2 phs = ld2(s_phs + (r & (CD2 - 1)) * W2C, t);
                    const float2 phi_new = fma2(S2(p.M), lmu, phs);
                    // lap psi + (psi lap m + lap(psi m) - m lap psi) / 2
                    const float2 div = fma2(S2(0.5f), (fma2(psc, lm, lp) - mc * lps), lps);
                    float2 src = S2(0.f);
                    if (p.theta) {
                        const uint32_t w = p.theta[(long long)r * p.theta_words + (xo >> 5)];
                        src.x = ((w >> (xo & 31)) & 1u) ? p.A : 0.f;
                        src.y = ((w >> ((xo + 1) & 31)) & 1u) ? p.A : 0.f;
                    }
                    const float2 sink = S2(p.gamma) * (psc - S2(p.c0));
                    const float2 psi_new = psc + (fma2(S2(p.D), div, src) - sink);
                    const long long o = (long long)r * pitch + xo;
                    *reinterpret_cast<float2 *>(p.phi_out + o) = phi_new;
                    *reinterpret_cast<float2 *>(p.psi_out + o) = psi_new;
                }
            }
        }
        // ---- D: mu*, m*, p* ----------------------------------------------------------
        {
            const int r = y0 - 13 + i;
            if (!GUARD || (i >= 10 && r < yend + 1)) {
                const Nb ph = nb(s_phs + ((r + 1) & (CD2 - 1)) * W2C, t);
                const Nb cs = nb(s_pss + ((r + 1) & (CD2 - 1)) * W2C, t);
                float2 px, py, plap, phm, cx, cy, csm;
                wPhsD.push(ph.c, ph.l, ph.r, px, py, plap, phm);
                wPssD.push_grad(cs.c, cs.l, cs.r, cx, cy, csm);
                if (!GUARD || i >= 12) {
                    const float2 pn = ld2(s_phi + (r & (LD2 - 1)) * W2C, t);
                    const float2 B = fma2(B12, csm, B02);
                    const float2 mus = fma2(a2, phm, b2 * (pn * pn * pn)) - B * plap -
                                       B12 * fma2(px, cx, py * cy);
                    const float2 ms = hB1 * fma2(px, px, py * py);
                    const int so = (r & (RD2 - 1)) * W2C;
                    st2(s_mus + so, t, mus);
                    st2(s_ms + so, t, ms);
                    st2(s_ps + so, t, csm * ms);
                }
            }
        }
        // ---- C: phi*, psi* (donor-cell fluxes) ----------------------------------------
        {
            const int r = y0 - 11 + i;
            if (!GUARD || (i >= 9 && r < yend + 2)) {
                const float *urow = s_ux + (r & (RD2 - 1)) * W2C;
                const float ulo = urow[t > 0 ? 2 * t - 1 : 0];
                const float uhi = urow[t < NT2 - 1 ? 2 * t + 2 : W2C - 1];
                const float2 uxc = ux2;
                const float2 ue = S2(0.5f) * (uxc + make_float2(uxc.y, uhi));
                const float2 uw = S2(0.5f) * (make_float2(ulo, uxc.x) + uxc);
                const float2 un = S2(0.5f) * (uy2 + uy1);
                const float2 us = S2(0.5f) * (uy3 + uy2);
                const Nb P = nb(s_phi + (r & (LD2 - 1)) * W2C, t);
                const Nb C = nb(s_psi + (r & (LD2 - 1)) * W2C, t);
                const float2 PN = ld2(s_phi + ((r + 1) & (LD2 - 1)) * W2C, t);
                const float2 PS = ld2(s_phi + ((r - 1) & (LD2 - 1)) * W2C, t);
                const float2 CN = ld2(s_psi + ((r + 1) & (LD2 - 1)) * W2C, t);
                const float2 CS = ld2(s_psi + ((r - 1) & (LD2 - 1)) * W2C, t);
                auto up = [](float2 u, float2 a, float2 b) {
                    return make_float2(u.x > 0.f ? a.x : b.x, u.y > 0.f ? a.y : b.y);
                };
                const float2 fe = ue * up(ue, P.c, P.r), fw = uw * up(uw, P.l, P.c);
                const float2 fn = un * up(un, P.c, PN), fs = us * up(us, PS, P.c);
                const float2 ge = ue * up(ue, C.c, C.r), gw = uw * up(uw, C.l, C.c);
                const float2 gn = un * up(un, C.c, CN), gs = us * up(us, CS, C.c);
                const int so = (r & (CD2 - 1)) * W2C;
                st2(s_phs + so, t, P.c - ((fe - fw) + (fn - fs)));
                st2(s_pss + so, t, C.c - ((ge - gw) + (gn - gs)));
            }
        }
        // ---- B: force, moments, collision ------------------------------------------------
        {
            const int r = y0 - 9 + i;
            float2 ux = S2(0.f), uy = S2(0.f);
            if (!GUARD || (i >= 4 && r < yend + 3)) {
                const Nb mu = nb(s_mu + ((r + 1) & (RD2 - 1)) * W2C, t);
                const Nb mm = nb(s_m + ((r + 1) & (RD2 - 1)) * W2C, t);
                float2 mx, my, mc, nx2, ny2, nc;
                wMuB.push_grad(mu.c, mu.l, mu.r, mx, my, mc);
                wMB.push_grad(mm.c, mm.l, mm.r, nx2, ny2, nc);
                if (!GUARD || i >= 6) {
                    const float2 ph = ld2(s_phi + (r & (LD2 - 1)) * W2C, t);
                    const float2 ps = ld2(s_psi + (r & (LD2 - 1)) * W2C, t);
                    // Eq. (14): F = -phi grad mu - (grad psi + psi grad m)
                    float2 Fx = S2(0.f) - fma2(ph, mx, fma2(ps, nx2, gpx2));
                    float2 Fy = S2(0.f) - fma2(ph, my, fma2(ps, ny2, gpy2));
                    if (p.flags & LBD_BODY_FORCE) {
                        Fx = Fx + S2(p.fx);
                        Fy = Fy + S2(p.fy);
                    }
                    const float *G = s_pop + (i % PS2) * 9 * SW + 2 * t + 4;
                    // plane i, column pair: staged index 2t + 4 - e_x
                    const float2 g0 = *reinterpret_cast<const float2 *>(G);
                    const float2 g1 = make_float2(G[SW - 1], G[SW]);
                    const float2 g2 = *reinterpret_cast<const float2 *>(G + 2 * SW);
                    const float2 g3 = make_float2(G[3 * SW + 1], G[3 * SW + 2]);
                    const float2 g4 = *reinterpret_cast<const float2 *>(G + 4 * SW);
                    const float2 g5 = make_float2(G[5 * SW - 1], G[5 * SW]);
                    const float2 g6 = make_float2(G[6 * SW + 1], G[6 * SW + 2]);
                    const float2 g7 = make_float2(G[7 * SW + 1], G[7 * SW + 2]);
                    const float2 g8 = make_float2(G[8 * SW - 1], G[8 * SW]);
                    const float2 dn = g0 + ((g1 + g2) + (g3 + g4)) + ((g5 + g6) + (g7 + g8));
                    const float2 jx = (g1 - g3) + (g5 - g6) + (g8 - g7);
                    const float2 jy = (g2 - g4) + (g5 + g6) - (g7 + g8);
                    const float2 n = S2(1.f) + dn;
                    const float2 inv = make_float2(__frcp_rn(n.x), __frcp_rn(n.y));
                    ux = fma2(S2(0.5f), Fx, jx) * inv;
                    uy = fma2(S2(0.5f), Fy, jy) * inv;
                    if ((!GUARD || (r >= y0 && r < yend)) && out) {
                        const float om = p.omega, gk = p.guo;
                        const float2 om1 = S2(1.f - om);
                        const float2 usq = fma2(ux, ux, uy * uy);
                        const float2 uF = fma2(ux, Fx, uy * Fy);
                        const float2 K = fma2(S2(om), fma2(S2(-1.5f) * n, usq, dn), S2(-3.f * gk) * uF);
                        const float2 c1 = S2(4.5f * om) * n, c2 = S2(9.f * gk);
                        const float2 c3 = S2(3.f * om) * n, c4 = S2(3.f * gk);
                        float *Go = p.g_out + (long long)r * pitch + xo;
                        *reinterpret_cast<float2 *>(Go) = fma2(om1, g0, S2(4.f / 9.f) * K);
#define LBD_PAIR2(I, J, W, EU, EF)                                                   \
    {                                                                                \
        const float2 eu = (EU), eF = (EF);                                           \
        const float2 sym = S2(W) * fma2(eu, fma2(c1, eu, c2 * eF), K);               \
        const float2 anti = S2(W) * fma2(c3, eu, c4 * eF);                           \
        *reinterpret_cast<float2 *>(Go + (I) * plane) = fma2(om1, g##I, sym + anti); \
        *reinterpret_cast<float2 *>(Go + (J) * plane) = fma2(om1, g##J, sym - anti); \
    }
                        LBD_PAIR2(1, 3, 1.f / 9.f, ux, Fx)
                        LBD_PAIR2(2, 4, 1.f / 9.f, uy, Fy)
                        LBD_PAIR2(5, 7, 1.f / 36.f, ux + uy, Fx + Fy)
                        LBD_PAIR2(6, 8, 1.f / 36.f, uy - ux, Fy - Fx)
#undef LBD_PAIR2
                    }
                    if (p.flags & LBD_FROZEN_U) {
                        ux = S2(p.ux0);
                        uy = S2(p.uy0);
                    }
                    st2(s_ux + (r & (RD2 - 1)) * W2C, t, ux);
                }
            }
            uy3 = uy2; uy2 = uy1; uy1 = uy;
            ux2 = ux1; ux1 = ux;
        }
        // ---- A: mu_phi, m, grad psi ----------------------------------------------------
        {
            const int r = y0 - 7 + i;
            float2 gx = S2(0.f), gy = S2(0.f);
            if (!GUARD || (i >= 1 && r < yend + 4)) {
                const Nb ph = nb(s_phi + ((r + 1) & (LD2 - 1)) * W2C, t);
                const Nb cs = nb(s_psi + ((r + 1) & (LD2 - 1)) * W2C, t);
                float2 px, py, plap, phm, csm;
                wPhiA.push(ph.c, ph.l, ph.r, px, py, plap, phm);
                wPsiA.push_grad(cs.c, cs.l, cs.r, gx, gy, csm);
                if (!GUARD || i >= 3) {
                    const int so = (r & (RD2 - 1)) * W2C;
                    const float2 B = fma2(B12, csm, B02);
                    st2(s_mu + so, t,
                        fma2(a2, phm, b2 * (phm * phm * phm)) - B * plap - B12 * fma2(px, gx, py * gy));
                    st2(s_m + so, t, hB1 * fma2(px, px, py * py));
                }
            }
            gpx2 = gpx1; gpy2 = gpy1; gpx1 = gx; gpy1 = gy;
        }
    };
    // prologue and epilogue guarded, steady state [15, rows + 9) unguarded
    const std::integral_constant<bool, true> guarded;
    const std::integral_constant<bool, false> steady;
    const int s1 = (yend - y0) + 9;
    int i = 0;
    for (; i < 15 && i < iters; ++i) body(guarded, i);
#pragma unroll 1
    for (; i < s1; ++i) body(steady, i);
    for (; i < iters; ++i) body(guarded, i);
    asm volatile("cp.async.wait_all;\n" ::);
}

}  // namespace

size_t pair_smem_bytes() { return kSmemFloats * sizeof(float); }

bool pair_supported(int nx) { return nx % 4 == 0 && nx >= SW; }

cudaError_t launch_pair(const StepArgs<float> &a, int seg, cudaStream_t s) {
    if (!pair_supported(a.nx) || (a.pitch % 4) != 0) return cudaErrorInvalidValue;
    static unsigned long long configured = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_smem_bytes());
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    const int bxo = W2C - 2 * HX;
    dim3 grid((a.nx + bxo - 1) / bxo, (a.ny + seg - 1) / seg);
    pair_kernel<<<grid, NT2, pair_smem_bytes(), s>>>(a, seg);
    return cudaGetLastError();
}

}  // namespace lbd

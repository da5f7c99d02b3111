// lbd_vstripe.cu -- the coupled time step (arXiv 1711.10984, Sections 2.1-2.3) as
// a stripe-marching kernel for FP32 periodic lattices whose width is a multiple
// of 4, with the population rows staged by 16-byte copies.
//
// The arithmetic per site is that of the stripe kernel (lbd_stripe.cu): a CTA
// of 128 threads owns a stripe of 116 output columns (x0 = 116 k, so every
// 4-column chunk of a row starts on a 16-byte boundary) and a segment of rows;
// thread c owns column x0 - 6 + c and marches down the rows through the same
// five-stage row pipeline (mu/m -> force, pull, collision -> advection ->
// mu*/m* -> phi/psi update), one barrier per row.  What differs is the
// bookkeeping around the arithmetic:
//
//  * Populations.  Stage B of row rb pulls f_i(x - e_i): planes with e_y = +1
//    from row rb - 1, e_y = 0 from rb, e_y = -1 from rb + 1.  The nine plane
//    rows a row needs are copied into shared memory as 16-byte chunks over the
//    columns x0 - 8 .. x0 + 127 (34 chunks per plane row).  Thread t < 102
//    copies chunk t % 34 of the (t / 34)-th plane of each of the three source
//    rows, so its three source offsets (plane and wrapped chunk column) are
//    fixed for the whole launch and only the row offset advances.  The width
//    being a multiple of 4, a chunk never straddles the periodic seam.
//  * Rings.  The small row rings ((mu, m), u_x, (phi*, psi*), (mu*, m*),
//    (psi*, p*)) and the population stage are 3 rows deep and the steady loop
//    is unrolled 3 times, so every slot is a compile-time constant and the
//    three-row stencil windows in registers advance without register moves.
//    The (phi^n, psi^n) ring has 12 slots and every row is copied into two,
//    s and s + 12: the eight rows an iteration reads (y0 - 13 + i ..
//    y0 - 6 + i) then sit at fixed offsets from one base slot, which advances
//    by one slot per iteration, with no wrap to compute per read.
//  * Launch.  A 1-D grid of (stripe, row segment) CTAs.  Where ceil(ny / by)
//    segments per stripe would leave resident CTA slots free (2048^2 at by = 64:
//    576 CTAs for 608 slots, so that 32 SMs would run one CTA fewer than the
//    rest while the others set the time), the stripes are cut into more,
//    shorter segments (down to by / 2 rows) until the CTAs fill the slots.
#include <cstdint>
#include <type_traits>

#include "lbd_internal.h"

namespace lbd {
namespace {

constexpr int NT = 128;       // threads per CTA
constexpr int W = NT - 12;    // output columns per stripe
constexpr int LD = 12;        // rows in the (phi^n, psi^n) ring (each row stored twice)
constexpr int R3 = 3;         // rows in the small rings and the population stage
constexpr int RS = NT + 2;    // ring row: one padding column on each side
constexpr int PW = NT + 8;    // staged population row: columns x0 - 8 .. x0 + 127
constexpr int NCH = PW / 4;   // 16-byte chunks per staged plane row
constexpr int NCP = 3 * NCH;  // copying threads (three planes per source row)

// (phi, psi) ring, four pair rings, the u_x ring, then the population stage on
// a 128-byte boundary (the 16-byte copies need 16-byte aligned destinations)
constexpr size_t RING_FLOATS = ((size_t)RS * (4 * LD + 2 * 4 * R3 + R3) + 31) / 32 * 32;
constexpr size_t SMEM_FLOATS = RING_FLOATS + (size_t)R3 * 9 * PW;

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsplat(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 vmake(float a, float b) { return make_float2(a, b); }

// Three-row stencil window of one column for a pair of fields, in the form
// T = L + R - 2C, D = R - L plus the centre C (isotropic D2Q9 weights: 1/3,
// 1/12 for the gradient, 2/3, 1/6 for the Laplacian links):
//   d/dx = (4 D_r + D_{r-1} + D_{r+1}) / 12
//   d/dy = (C_{r+1} - C_{r-1}) / 2 + (T_{r+1} - T_{r-1}) / 12
//   lap  = (2/3) T_r + (T_{r-1} + T_{r+1}) / 6 + (C_{r+1} - 2 C_r + C_{r-1})
struct Win {
    // partial sums of the outputs at the last row n (kept values are all
    // recomputed at each arrival, none is copied from another):
    //   ax = (D_{n-1} + 4 D_n) / 12, bx = D_n / 12,
    //   ay = (C_n - C_{n-1}) / 2 - T_{n-1} / 12,
    //   al = (2/3) T_n + T_{n-1} / 6 - (C_n - C_{n-1}),
    //   tp = T_n, cp = C_n
    float2 ax, bx, ay, al, tp, cp;
    __device__ __forceinline__ void reset() {
        ax = bx = ay = al = tp = cp = vsplat(0.f);
    }
    __device__ __forceinline__ void push(float2 c, float2 l, float2 r, float2 &gx, float2 &gy,
                                         float2 &lap, float2 &mid) {
        const float2 t = vfma(c, vsplat(-2.f), l + r);
        const float2 d = r - l;
        const float2 e = c - cp;
        const float2 q = tp * vsplat(1.f / 6.f);
        gx = vfma(d, vsplat(1.f / 12.f), ax);
        ax = vfma(d, vsplat(1.f / 3.f), bx);
        bx = d * vsplat(1.f / 12.f);
        gy = vfma(e, vsplat(0.5f), vfma(t, vsplat(1.f / 12.f), ay));
        ay = vfma(q, vsplat(-0.5f), e * vsplat(0.5f));
        lap = vfma(t, vsplat(1.f / 6.f), al + e);
        al = vfma(t, vsplat(2.f / 3.f), q - e);
        mid = cp;
        tp = t;
        cp = c;
    }
    __device__ __forceinline__ void push_grad(float2 c, float2 l, float2 r, float2 &gx, float2 &gy,
                                              float2 &mid) {
        const float2 t = vfma(c, vsplat(-2.f), l + r);
        const float2 d = r - l;
        const float2 e = c - cp;
        gx = vfma(d, vsplat(1.f / 12.f), ax);
        ax = vfma(d, vsplat(1.f / 3.f), bx);
        bx = d * vsplat(1.f / 12.f);
        gy = vfma(e, vsplat(0.5f), vfma(t, vsplat(1.f / 12.f), ay));
        ay = vfma(tp, vsplat(-1.f / 12.f), e * vsplat(0.5f));
        mid = cp;
        tp = t;
        cp = c;
    }
};

struct WinLap {
    float2 al, tp, cp;  // as in Win
    __device__ __forceinline__ void reset() { al = tp = cp = vsplat(0.f); }
    __device__ __forceinline__ float2 push(float2 c, float2 l, float2 r) {
        const float2 t = vfma(c, vsplat(-2.f), l + r);
        const float2 e = c - cp;
        const float2 lap = vfma(t, vsplat(1.f / 6.f), al + e);
        al = vfma(t, vsplat(2.f / 3.f), vfma(tp, vsplat(1.f / 6.f), vsplat(0.f) - e));
        tp = t;
        cp = c;
        return lap;
    }
};

template <int OFF>
__device__ __forceinline__ void cp4(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0+%2], [%1], 4;\n" ::"r"(dst), "l"(src), "n"(OFF));
}
template <int OFF>
__device__ __forceinline__ void cp16(unsigned dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0+%2], [%1], 16;\n" ::"r"(dst), "l"(src), "n"(OFF));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Phase i % 3 of a pipeline iteration: a compile-time constant (Ph<V>) in the
// unrolled steady loop, a run-time int elsewhere.
template <int V>
struct Ph {};

// Slot of a 3-deep ring for the row y0 + K + i at phase ph = i % 3; K >= -30.
template <int K, int V>
__device__ __forceinline__ constexpr int s3(Ph<V>) {
    return (V + K + 30) % 3;
}
template <int K>
__device__ __forceinline__ int s3(int ph) {
    return (ph + K + 30) % 3;
}

// The pipeline of one CTA.
__device__ __forceinline__ void vstripe_body(const StepArgs<float> &p, const int x0, const int y0,
                                             const int seg, unsigned char *smem_raw) {
    const int c = threadIdx.x;
    float2 *const r_ps = reinterpret_cast<float2 *>(smem_raw) + 1 + c;  // [LD] (phi^n, psi^n)
    float2 *const r_mm = r_ps + 2 * LD * RS;                                 // [R3] (mu, m)       A -> B
    float2 *const r_st = r_mm + R3 * RS;                                 // [R3] (phi*, psi*)  C -> D
    float2 *const r_ms = r_st + R3 * RS;                                 // [R3] (mu*, m*)     D -> E
    float2 *const r_pp = r_ms + R3 * RS;                                 // [R3] (psi*, p*)    D -> E
    float *const r_ux = reinterpret_cast<float *>(r_pp - 1 - c + R3 * RS) + 1 + c;  // [R3] u_x
    float *const s_pop = reinterpret_cast<float *>(smem_raw) + RING_FLOATS;
    const unsigned u_ps = (unsigned)__cvta_generic_to_shared(r_ps);
    // this thread's chunk destination in stage slot 0, group 0
    const unsigned u_chunk = (unsigned)__cvta_generic_to_shared(s_pop) + 16u * (unsigned)c;
    // this thread's column in the population stage
    const float *const s_own = s_pop + c + 2;

    const int nx = p.nx, ny = p.ny;
    const unsigned pitch_b = (unsigned)p.pitch * 4u, plane_b = (unsigned)p.plane * 4u;
    const unsigned rows_b = (unsigned)ny * pitch_b;
    const unsigned xg_b = (unsigned)wrapi(x0 - 6 + c, nx) * 4u;
    const bool copier = c < NCP;
    // source offsets (plane + wrapped chunk column) of the three chunks this
    // thread copies: groups by source row -1, 0, +1 relative to the stage-B row
    unsigned so0 = 0, so1 = 0, so2 = 0;
    {
        const int pl = c / NCH, ch = c - (c / NCH) * NCH;
        const unsigned xb = (unsigned)wrapi(x0 - 8 + 4 * ch, nx) * 4u;
        const int pA = pl == 0 ? 2 : (pl == 1 ? 5 : 6);  // e_y = +1: from row rb - 1
        const int pB = pl == 0 ? 0 : (pl == 1 ? 1 : 3);  // e_y =  0: from row rb
        const int pC = pl == 0 ? 4 : (pl == 1 ? 7 : 8);  // e_y = -1: from row rb + 1
        so0 = (unsigned)pA * plane_b + xb;
        so1 = (unsigned)pB * plane_b + xb;
        so2 = (unsigned)pC * plane_b + xb;
    }
    const char *const gp0 = reinterpret_cast<const char *>(p.g_in) + so0;
    const char *const gp1 = reinterpret_cast<const char *>(p.g_in) + so1;
    const char *const gp2 = reinterpret_cast<const char *>(p.g_in) + so2;
    const int xo = x0 + c - 6;  // output column of this thread
    const bool inE = c >= 6 && c < NT - 6 && xo < nx;
    const unsigned xo_b = (unsigned)xo * 4u;

    const int yend = min(y0 + seg, ny);

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

    // Asynchronous loads of iteration k into stage slot `slot`: (phi^n, psi^n)
    // of loader row y0 - 5 + k, and the populations pulled by stage-B row
    // y0 - 9 + k.
    auto issue = [&](int k, int slot, int ws) {
        const int rl = y0 - 5 + k;
        if (rl < yend + 5) {
            const unsigned so = u_ps + (unsigned)(ws * RS) * 8u;
            cp4<0>(so, phi_in + lo_b);
            cp4<4>(so, psi_in + lo_b);
            cp4<LD * RS * 8>(so, phi_in + lo_b);
            cp4<LD * RS * 8 + 4>(so, psi_in + lo_b);
        }
        const int rb = y0 - 9 + k;
        if (copier && rb >= y0 - 3 && rb < yend + 3) {
            const unsigned d = u_chunk + (unsigned)(slot * 9 * PW) * 4u;
            cp16<0 * 3 * PW * 4>(d, gp0 + rm_b);
            cp16<1 * 3 * PW * 4>(d, gp1 + r0_b);
            cp16<2 * 3 * PW * 4>(d, gp2 + rp_b);
        }
        cp_commit();
        adv(lo_b);
        rm_b = r0_b;
        r0_b = rp_b;
        adv(rp_b);
    };

    uint32_t theta_w = 0;
    float phs_e = 0.f, phs_n = 0.f;
    Win wA, wB, wD;
    WinLap wEm, wEp;
    wA.reset(); wB.reset(); wD.reset(); wEm.reset(); wEp.reset();
    float2 gps1 = vsplat(0.f), gps2 = vsplat(0.f);
    float ux1 = 0, ux2 = 0, uy1 = 0, uy2 = 0, uy3 = 0;

    const float a = p.a, b = p.b, B0 = p.B0, B1 = p.B1;
    char *const g_out = reinterpret_cast<char *>(p.g_out);
    char *const phi_out = reinterpret_cast<char *>(p.phi_out);
    char *const psi_out = reinterpret_cast<char *>(p.psi_out);
    const float A_t = p.A, gamma_t = p.gamma;
    issue(0, 0, 0);
    issue(1, 1, 1);
    // slot of ring row y0 - 13 + i (loader index i - 8) at iteration i
    int bq = 4;
    const int iters = (yend - y0) + 15;

    // One pipeline iteration i (ph = i % 3); with GUARD false every stage is
    // active and every written row is owned, so the row conditions vanish.
    auto body = [&](auto guard_tag, const int i, auto ph) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        cp_wait1();
        __syncthreads();
        issue(i + 2, s3<2>(ph), bq < 2 ? bq + 10 : bq - 2);
        const float2 *const Bp = r_ps + bq * RS;  // rows y0 - 13 + i .. y0 - 6 + i at Bp[j RS]

        // ---- E: phi^{n+1} (Eq. 18), psi^{n+1} (Eq. 19 + source, sink), row y0 - 15 + i
        {
            const int r = y0 - 15 + i;
            if (!GUARD || i >= 13) {
                const float2 *M1 = r_ms + s3<-14>(ph) * RS;
                const float2 *P1 = r_pp + s3<-14>(ph) * RS;
                const float2 mc = wEm.cp, pc = wEp.cp;
                const float2 lm = wEm.push(M1[0], M1[-1], M1[1]);
                const float2 lp = wEp.push(P1[0], P1[-1], P1[1]);
                if ((!GUARD || r >= y0) && inE) {
                const float phi_new = phs_e + p.M * lm.x;
                const float psc = pc.x;
                const float div = lp.x + 0.5f * ((psc * lm.y + lp.y) - mc.y * lp.x);
                const float src = ((theta_w >> (xo & 31)) & 1u) ? A_t : 0.f;
                const float psi_new = psc + (p.D * div - gamma_t * (psc - p.c0) + src);
                    const unsigned o = (unsigned)r * pitch_b + xo_b;
                    *reinterpret_cast<float *>(phi_out + o) = phi_new;
                    *reinterpret_cast<float *>(psi_out + o) = psi_new;
                }
            }
        }
        if (inE) {
            const int rn = y0 - 14 + i;
            theta_w = (rn >= y0 && rn < yend) ? p.theta[rn * p.theta_words + (xo >> 5)] : 0u;
        }
        // ---- D: mu*, m*, p* at row y0 - 13 + i (Eq. 3 on phi*, psi*; Eq. 5) ----
        {
            const int r = y0 - 13 + i;
            if (!GUARD || (i >= 10 && r < yend + 1)) {
                const float2 *S1 = r_st + s3<-12>(ph) * RS;
                float2 gx, gy, lap, mid;
                wD.push(S1[0], S1[-1], S1[1], gx, gy, lap, mid);
                phs_e = phs_n;  // phi* of row y0 - 14 + i, for stage E next iteration
                phs_n = mid.x;
                if (!GUARD || i >= 12) {
                    const float pn = Bp[0].x;
                    const float mus = a * mid.x + b * (pn * pn * pn) - (B0 + B1 * mid.y) * lap.x -
                                      B1 * (gx.x * gx.y + gy.x * gy.y);
                    const float ms = 0.5f * B1 * (gx.x * gx.x + gy.x * gy.x);
                    const int so = s3<-13>(ph) * RS;
                    r_ms[so] = vmake(mus, ms);
                    r_pp[so] = vmake(mid.y, mid.y * ms);
                }
            }
        }
        // ---- C: phi*, psi* at row y0 - 11 + i (donor-cell fluxes, Eqs. 16-17) ----
        {
            const int r = y0 - 11 + i;
            if (!GUARD || (i >= 9 && r < yend + 2)) {
                const float2 *Q = Bp + 2 * RS;
                const float2 QN = Bp[3 * RS];
                const float2 QS = Bp[1 * RS];
                const float *U = r_ux + s3<-11>(ph) * RS;
                const float uxc = ux2;
                const float ue = 0.5f * (uxc + U[1]);
                const float uw = 0.5f * (U[-1] + uxc);
                const float un = 0.5f * (uy2 + uy1);
                const float us = 0.5f * (uy3 + uy2);
                const float2 Q0 = Q[0], QE = Q[1], QW = Q[-1];
                const float2 fe = vsplat(ue) * (ue > 0.f ? Q0 : QE);
                const float2 fw = vsplat(uw) * (uw > 0.f ? QW : Q0);
                const float2 fn = vsplat(un) * (un > 0.f ? Q0 : QN);
                const float2 fs = vsplat(us) * (us > 0.f ? QS : Q0);
                r_st[s3<-11>(ph) * RS] = Q0 - ((fe - fw) + (fn - fs));
            }
        }
        // ---- B: force (Eq. 14), moments (Eq. 11), collision (Eqs. 10, 12, 13) ----
        {
            const int r = y0 - 9 + i;
            float ux = 0.f, uy = 0.f;
            if (!GUARD || (i >= 4 && r < yend + 3)) {
                const float2 *M1 = r_mm + s3<-8>(ph) * RS;
                float2 gx, gy, mid;
                wB.push_grad(M1[0], M1[-1], M1[1], gx, gy, mid);
                if (!GUARD || i >= 6) {
                    const float2 pp = Bp[4 * RS];
                    float2 F = vmake(fmaf(-pp.x, gx.x, fmaf(-pp.y, gx.y, -gps2.x)),
                                     fmaf(-pp.x, gy.x, fmaf(-pp.y, gy.y, -gps2.y)));
                    F = F + vmake(p.fx, p.fy);
                    // pulled populations: group 0 = planes (2, 5, 6) from row r - 1,
                    // group 1 = (0, 1, 3) from row r, group 2 = (4, 7, 8) from r + 1;
                    // f_i(x) = buffer_i(x - e_i), stage column c + 2 - e_ix
                    const float *G = s_own + s3<0>(ph) * 9 * PW;
                    const float g0 = G[3 * PW + 0 * PW];
                    const float g1 = G[3 * PW + 1 * PW - 1], g3 = G[3 * PW + 2 * PW + 1];
                    const float g2 = G[0 * PW], g5 = G[1 * PW - 1], g6 = G[2 * PW + 1];
                    const float g4 = G[6 * PW], g7 = G[7 * PW + 1], g8 = G[8 * PW - 1];
                    const float2 g12 = vmake(g1, g2), g34 = vmake(g3, g4);
                    const float2 g56 = vmake(g5, g6), g78 = vmake(g7, g8);
                    const float2 s1 = (g12 + g34) + (g56 + g78);
                    const float dn = g0 + (s1.x + s1.y);
                    const float2 a13 = g12 - g34;
                    const float jx = a13.x + ((g56.x - g56.y) + (g78.y - g78.x));
                    const float jy = a13.y + ((g56.x + g56.y) - (g78.x + g78.y));
                    const float n = 1.f + dn;
                    const float inv = __fdividef(1.f, n);  // fast reciprocal, <= 2 ulp
                    const float2 u = vfma(vsplat(0.5f), F, vmake(jx, jy)) * vsplat(inv);
                    ux = u.x;
                    uy = u.y;
                    if ((!GUARD || (r >= y0 && r < yend)) && inE) {
                        const float om = p.omega, gk = p.guo;
                        const float2 om1 = vsplat(1.f - om);
                        const float usq = ux * ux + uy * uy, uF = ux * F.x + uy * F.y;
                        const float K = om * (dn - 1.5f * n * usq) - 3.f * gk * uF;
                        const float2 c1 = vsplat(4.5f * om * n), c2 = vsplat(9.f * gk);
                        const float2 c3 = vsplat(3.f * om * n), c4 = vsplat(3.f * gk);
                        const float2 Kv = vsplat(K);
                        char *Go = g_out + ((unsigned)r * pitch_b + xo_b);
#define LBD_OUT(I) *reinterpret_cast<float *>(Go + (I) * plane_b)
                        LBD_OUT(0) = (1.f - om) * g0 + (4.f / 9.f) * K;
                        {
                            const float2 eu = u, eF = F, Wt = vsplat(1.f / 9.f);
                            const float2 sym = Wt * vfma(eu, vfma(c1, eu, c2 * eF), Kv);
                            const float2 anti = Wt * vfma(c3, eu, c4 * eF);
                            const float2 pos = vfma(om1, g12, sym + anti);
                            const float2 neg = vfma(om1, g34, sym - anti);
                            LBD_OUT(1) = pos.x; LBD_OUT(2) = pos.y;
                            LBD_OUT(3) = neg.x; LBD_OUT(4) = neg.y;
                        }
                        {
                            const float2 eu = vmake(ux + uy, uy - ux), eF = vmake(F.x + F.y, F.y - F.x);
                            const float2 Wt = vsplat(1.f / 36.f);
                            const float2 sym = Wt * vfma(eu, vfma(c1, eu, c2 * eF), Kv);
                            const float2 anti = Wt * vfma(c3, eu, c4 * eF);
                            const float2 pos = vfma(om1, g56, sym + anti);
                            const float2 neg = vfma(om1, g78, sym - anti);
                            LBD_OUT(5) = pos.x; LBD_OUT(6) = pos.y;
                            LBD_OUT(7) = neg.x; LBD_OUT(8) = neg.y;
                        }
#undef LBD_OUT
                    }
                    if (p.flags & LBD_FROZEN_U) {
                        ux = p.ux0;
                        uy = p.uy0;
                    }
                    r_ux[s3<-9>(ph) * RS] = ux;
                }
            }
            uy3 = uy2; uy2 = uy1; uy1 = uy;
            ux2 = ux1; ux1 = ux;
        }
        // ---- A: mu_phi (Eq. 3), m (Eq. 5), grad psi at row y0 - 7 + i -----------
        {
            const int r = y0 - 7 + i;
            float2 gp = vsplat(0.f);
            if (!GUARD || (i >= 1 && r < yend + 4)) {
                const float2 *F1 = Bp + 7 * RS;
                float2 gx, gy, lap, mid;
                wA.push(F1[0], F1[-1], F1[1], gx, gy, lap, mid);
                gp = vmake(gx.y, gy.y);
                if (!GUARD || i >= 3) {
                    const float ph_ = mid.x;
                    const float mu = a * ph_ + b * (ph_ * ph_ * ph_) - (B0 + B1 * mid.y) * lap.x -
                                     B1 * (gx.x * gx.y + gy.x * gy.y);
                    const float m = 0.5f * B1 * (gx.x * gx.x + gy.x * gy.x);
                    r_mm[s3<-7>(ph) * RS] = vmake(mu, m);
                }
            }
            gps2 = gps1; gps1 = gp;
        }
        bq = bq == LD - 1 ? 0 : bq + 1;
    };
    const std::integral_constant<bool, true> guarded;
    const std::integral_constant<bool, false> steady;
    const Ph<0> ph0;
    const Ph<1> ph1;
    const Ph<2> ph2;
    // steady iterations, i in [15, nrows + 9): every stage active (E from
    // i = 13, writing owned rows from i = 15) and every written row owned (B's
    // last row at i = nrows + 8); 15 is a multiple of 3, as the unrolled loop needs
    const int s1 = (yend - y0) + 9;
    int i = 0;
    for (; i < 15 && i < iters; ++i) body(guarded, i, i % 3);
#pragma unroll 1
    for (; i + 3 <= s1; i += 3) {
        body(steady, i, ph0);
        body(steady, i + 1, ph1);
        body(steady, i + 2, ph2);
    }
    for (; i < iters; ++i) body(guarded, i, i % 3);
    asm volatile("cp.async.wait_all;\n" ::);
}

// One CTA per (stripe, row segment) on a 1-D grid, stripes fastest (as a 2-D
// grid would run them): the first `rem` stripes are cut into base + 1 row
// segments, the others into base, the heights of a stripe's segments differing
// by at most one row.
__global__ void __launch_bounds__(NT, 4) vstripe_kernel(const StepArgs<float> p, const int stripes,
                                                        const int base, const int rem) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int b = blockIdx.x;
    int s, j;
    if (b < stripes * base) {
        j = b / stripes;
        s = b - j * stripes;
    } else {
        s = b - stripes * base;
        j = base;
    }
    const int n = s < rem ? base + 1 : base;
    // the first ny % n segments one row taller
    const int q = p.ny / n, r = p.ny - q * n;
    vstripe_body(p, s * W, j * q + min(j, r), q + (j < r ? 1 : 0), smem_raw);
}

// Batched step: a persistent grid walks the work items of periodic FP32
// instances; the arguments of the item's instance are staged in shared memory
// with the activity of this step, evaluated from the device step count, so
// that the launch can be replayed from a CUDA graph.
__global__ void __launch_bounds__(NT, 4)
    vstripe_batch_kernel(const StepArgs<float> *args, const BatchItem *items, const int n_items,
                         const long long *t_dev, const int t_off) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ StepArgs<float> sp;
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
            sp.A = (float)A;
            sp.gamma = (float)g;
        }
        __syncthreads();
        vstripe_body(sp, item.x0, item.y0, item.rows, smem_raw);
        __syncthreads();
    }
}

}  // namespace

bool vstripe_supported(int nx, long long plane) {
    return nx % 4 == 0 && 9.0 * (double)plane * 4.0 < 4294967295.0;
}

size_t vstripe_smem_bytes() { return sizeof(float) * SMEM_FLOATS; }

cudaError_t launch_vstripe(const StepArgs<float> &a, int seg, cudaStream_t s) {
    if (!vstripe_supported(a.nx, a.plane) || (a.flags & LBD_WALLS)) return cudaErrorInvalidValue;
    const size_t smem = vstripe_smem_bytes();
    static unsigned long long configured = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(vstripe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    // ceil(ny / seg) segments per stripe; when that leaves resident CTA slots
    // free, more segments (equal heights, at least half a segment each), so
    // that every SM holds as many CTAs as the others
    static int slots[64] = {0};
    if (!slots[dev & 63]) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vstripe_kernel, NT, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        slots[dev & 63] = per_sm * sms > 0 ? per_sm * sms : 1;
    }
    const int stripes = (a.nx + W - 1) / W;
    const int per = (a.ny + seg - 1) / seg;
    long long total = (long long)stripes * per;
    const long long cap = (long long)stripes * (2 * a.ny / seg > per ? 2 * a.ny / seg : per);
    if (total < slots[dev & 63]) total = slots[dev & 63] < cap ? slots[dev & 63] : cap;
    const int base = (int)(total / stripes), rem = (int)(total % stripes);
    vstripe_kernel<<<(unsigned)total, NT, smem, s>>>(a, stripes, base, rem);
    return cudaGetLastError();
}

}  // namespace lbd

namespace lbd {

cudaError_t launch_vstripe_batch(const StepArgs<float> *args, const BatchItem *items, int n_items,
                                 int ctas, const long long *t_dev, int t_off, cudaStream_t s) {
    const size_t smem = vstripe_smem_bytes();
    static unsigned long long configured = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(vstripe_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    vstripe_batch_kernel<<<ctas, NT, smem, s>>>(args, items, n_items, t_dev, t_off);
    return cudaGetLastError();
}

int vstripe_batch_ctas_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, vstripe_batch_kernel, NT,
                                                      vstripe_smem_bytes()) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace lbd

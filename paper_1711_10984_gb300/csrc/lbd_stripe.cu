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
//
// With plates at y = -1/2 and ny - 1/2 (WALLS): the loader reads rows beyond a
// plate mirrored, so stage A produces mirrored mu, m there; the pulls at rows 0
// and ny - 1 take the site's own reversed population (halfway bounce-back); the
// advective flux through a plate face is zero; stages D and E, whose inputs come
// from the LB velocity, never use rows beyond a plate: at row 0 the window's
// row -1 is set to row 0, at row ny - 1 the window pushes its own row again.
#include <cstdint>
#include <type_traits>

#include "lbd_internal.h"

namespace lbd {
namespace {

constexpr int LD = 16;  // rows in the (phi^n, psi^n) ring
constexpr int RD = 4;   // rows in the u_x ring
constexpr int RM = 2;   // rows in the (mu, m), (mu*, m*), (psi*, p*) rings
constexpr int CD = 2;   // rows in the (phi*, psi*) ring
constexpr int PS = 3;   // population staging depth (rows in flight)

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Two fields of one site in the two lanes of a vector: FP32 pairs use the packed
// FP32x2 instructions of sm_100+ (FADD2 / FMUL2 / FFMA2); FP64 pairs are plain
// component-wise arithmetic.
template <typename T>
struct V2t;
template <>
struct V2t<float> {
    using type = float2;
};
template <>
struct V2t<double> {
    using type = double2;
};

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, rounded once
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsplat(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 vmake(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ double2 operator+(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 operator-(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 operator*(double2 a, double2 b) {
    return make_double2(a.x * b.x, a.y * b.y);
}
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vsplat(double s) { return make_double2(s, s); }

// 1 / x for the density in Eq. 11: in FP32 the fast reciprocal (within 2 ulp;
// x = rho is near 1), which made the FP32 step 2 % faster than the correctly
// rounded one; in FP64 the division itself
__device__ __forceinline__ float rcp_rn(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp_rn(double x) { return 1.0 / x; }
__device__ __forceinline__ double2 vmake(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 vneg(double2 a) { return make_double2(-a.x, -a.y); }

// Stencil history of one column for a pair of fields, for the isotropic D2Q9
// stencils (1/3, 1/12 gradient weights; 2/3, 1/6 Laplacian link weights).  With
// T = L + R - 2C, D = R - L and C the centre of row n, arriving row n + 1 gives
// the derivatives at row n:
//   12 d/dx = D_{n-1} + 4 D_n + D_{n+1}
//   12 d/dy = 6 (C_{n+1} - C_{n-1}) + T_{n+1} - T_{n-1}
//   lap     = (2/3) T_n + (T_{n-1} + T_{n+1}) / 6 + (C_{n+1} - 2 C_n + C_{n-1})
// The gradients come out 12 times too large: their users fold the 1/12 into
// their own constants, which saves a multiply per gradient component on the
// FP64 pipe.  The window keeps partial sums of the outputs at row n, each
// recomputed at every arrival (nothing is shifted from one kept value to
// another), with e_n = C_n - C_{n-1}:
//   ax = D_{n-1} + 4 D_n,   bx = D_n,   ay = 6 e_n - T_{n-1},
//   al = (2/3) T_n + T_{n-1} / 6 - e_n,   tp = T_n,   cp = C_n,
// so that 12 d/dx = ax + D_{n+1}, 12 d/dy = ay + T_{n+1} + 6 e_{n+1} and
// lap = al + T_{n+1} / 6 + e_{n+1}: one FP64 operation per lane fewer than
// differencing a window of raw rows.
template <typename V>
struct Win2 {
    V ax, bx, ay, al, tp, cp;
    __device__ __forceinline__ void reset() {
        ax = bx = ay = al = tp = cp = vsplat(decltype(ax.x)(0));
    }
    // row n + 1 as (C, T, D)
    __device__ __forceinline__ void arrive(V c, V t, V d, V &gx, V &gy, V &lap, V &mid) {
        using S = decltype(ax.x);
        const V e = c - cp;
        gx = ax + d;
        gy = vfma(e, vsplat(S(6)), ay + t);
        lap = vfma(t, vsplat(S(1.0 / 6.0)), al + e);
        mid = cp;
        ax = vfma(d, vsplat(S(4)), bx);
        bx = d;
        ay = vfma(e, vsplat(S(6)), vneg(tp));
        al = vfma(t, vsplat(S(2.0 / 3.0)), vfma(tp, vsplat(S(1.0 / 6.0)), vneg(e)));
        tp = t;
        cp = c;
    }
    __device__ __forceinline__ void push(V c, V l, V r, V &gx, V &gy, V &lap, V &mid) {
        using S = decltype(ax.x);
        arrive(c, vfma(c, vsplat(S(-2)), l + r), r - l, gx, gy, lap, mid);
    }
    // the row below the current one is the current row mirrored (a plate
    // between): D_{n-1} = D_n, T_{n-1} = T_n, e_n = 0
    __device__ __forceinline__ void mirror_below() {
        using S = decltype(ax.x);
        ax = bx * vsplat(S(5));
        ay = vneg(tp);
        al = tp * vsplat(S(5.0 / 6.0));
    }
    // push(n + 1) where row n + 1 is row n mirrored (a plate above)
    __device__ __forceinline__ void push_mirror(V &gx, V &gy, V &lap, V &mid) {
        arrive(cp, tp, bx, gx, gy, lap, mid);
    }
};

// Gradients only, for (mu, m): a window of raw rows (rows n - 1 and n as C, T
// and D), which costs one operation per lane fewer than partial sums when no
// Laplacian is formed.
template <typename V>
struct WinG2 {
    V cm, c0, tm, t0, dm, d0;
    __device__ __forceinline__ void reset() { cm = c0 = tm = t0 = dm = d0 = vsplat(decltype(cm.x)(0)); }
    __device__ __forceinline__ void push_grad(V c, V l, V r, V &gx, V &gy, V &mid) {
        using S = decltype(cm.x);
        const V t = vfma(c, vsplat(S(-2)), l + r);
        const V d = r - l;
        gx = vfma(d0, vsplat(S(4)), dm + d);
        gy = vfma(c - cm, vsplat(S(6)), t - tm);
        mid = c0;
        cm = c0; c0 = c; tm = t0; t0 = t; dm = d0; d0 = d;
    }
};

// Laplacian only, in the partial-sum form of Win2: al, tp, cp.
template <typename V>
struct WinLap2 {
    V al, tp, cp;
    __device__ __forceinline__ void reset() { al = tp = cp = vsplat(decltype(al.x)(0)); }
    __device__ __forceinline__ V arrive(V c, V t) {
        using S = decltype(al.x);
        const V e = c - cp;
        const V lap = vfma(t, vsplat(S(1.0 / 6.0)), al + e);
        al = vfma(t, vsplat(S(2.0 / 3.0)), vfma(tp, vsplat(S(1.0 / 6.0)), vneg(e)));
        tp = t;
        cp = c;
        return lap;
    }
    __device__ __forceinline__ V push(V c, V l, V r) {
        using S = decltype(al.x);
        return arrive(c, vfma(c, vsplat(S(-2)), l + r));
    }
    __device__ __forceinline__ void mirror_below() {
        using S = decltype(al.x);
        al = tp * vsplat(S(5.0 / 6.0));
    }
    __device__ __forceinline__ V push_mirror() { return arrive(cp, tp); }
};

template <typename T>
struct StripeSmem {
    // Pair rings (two fields interleaved per column) and one scalar ring, each row
    // padded by one column on each side so the x-neighbours of every thread are in
    // bounds; then the population staging.
    static constexpr size_t floats(int nt) {
        return (size_t)(nt + 2) * (2 * (LD + RM + RM + RM + CD) + RD) + (size_t)nt * PS * 9;
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

template <typename T, int NT, bool WALLS>
__device__ __forceinline__ void stripe_body(const StepArgs<T> &p, const int x0, const int y0,
                                            const int seg, const T A_t, const T gamma_t,
                                            unsigned char *smem_raw) {
    using V = typename V2t<T>::type;
    constexpr int RS = NT + 2;  // padded ring row (columns)
    const int c = threadIdx.x;
    // this thread's element in slot 0 of each ring (x-neighbours at -1, +1)
    V *const r_ps = reinterpret_cast<V *>(smem_raw) + 1 + c;  // [LD] (phi^n, psi^n)
    V *const r_mm = r_ps + LD * RS;                             // [RD] (mu, m)       A -> B
    V *const r_ms = r_mm + RM * RS;                             // [RD] (mu*, m*)     D -> E
    V *const r_pp = r_ms + RM * RS;                             // [RD] (psi*, p*)    D -> E
    V *const r_st = r_pp + RM * RS;                             // [CD] (phi*, psi*)  C -> D
    T *const r_ux = reinterpret_cast<T *>(r_st - 1 - c + CD * RS) + 1 + c;  // [RD] u_x  B -> C
    T *const s_pop = reinterpret_cast<T *>(smem_raw) + 2 * (LD + 3 * RM + CD) * RS + RD * RS + c;
    const unsigned u_ps = (unsigned)__cvta_generic_to_shared(r_ps);
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
    // Every thread runs every stage: stage k's results are valid on columns
    // [k, NT - k) and the columns outside are read only by threads whose own
    // results are outside the next stage's valid range (the ring rows carry a
    // padding column on each side, so every read stays inside shared memory).
    const bool inB = c >= 2 && c < NT - 2;
    const int xo = x0 + c - 5;  // output column of this thread
    const bool inE = c >= 5 && c < NT - 5 && xo < nx;
    const unsigned xo_b = (unsigned)xo * TB;
    const int yend = min(y0 + seg, ny);  // owned rows [y0, yend)

    // Byte offsets of the asynchronously loaded rows, advanced one row per
    // iteration: loader row y0 - 5 + k and rows rb - 1, rb, rb + 1 around stage-B
    // row rb = y0 - 9 + k.
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

    // Asynchronous loads of iteration k: (phi^n, psi^n) of loader row y0 - 5 + k
    // into the two lanes of the pair ring, and the pulled populations f_i(x - e_i)
    // of stage-B row y0 - 9 + k.
    auto issue = [&](int k, int slot) {  // slot = k % PS
        const int rl = y0 - 5 + k;
        if (rl < yend + 5) {
            const unsigned so = (unsigned)(((rl - y0) & (LD - 1)) * RS) * (2 * TB);
            unsigned lo = lo_b;
            if (WALLS)  // rows beyond a plate are the mirrored rows inside
                lo = (unsigned)(rl < 0 ? -1 - rl : (rl >= ny ? 2 * ny - 1 - rl : rl)) * pitch_b + xg_b;
            if (TB == 8) {
                cp8<0>(u_ps + so, phi_in + lo);
                cp8<8>(u_ps + so, psi_in + lo);
            } else {
                cp4<0>(u_ps + so, phi_in + lo);
                cp4<4>(u_ps + so, psi_in + lo);
            }
        }
        const int rb = y0 - 9 + k;
        if (inB && rb >= y0 - 3 && rb < yend + 3) {
            const unsigned d = u_pop + (unsigned)(slot * 9 * NT) * TB;
            constexpr int P = NT * (int)sizeof(T);
#define LBD_PULL(I, ROW, COL)                                                              \
    if (TB == 8) cp8<(I) * P>(d, g_in + ((I) * plane_b + (ROW) + (COL)));                 \
    else cp4<(I) * P>(d, g_in + ((I) * plane_b + (ROW) + (COL)));
#define LBD_PULL_FROM(I, J, ROW, COL)                                                      \
    if (TB == 8) cp8<(I) * P>(d, g_in + ((J) * plane_b + (ROW) + (COL)));                 \
    else cp4<(I) * P>(d, g_in + ((J) * plane_b + (ROW) + (COL)));
            LBD_PULL(0, r0_b, xg_b)  // e = ( 0, 0)
            LBD_PULL(1, r0_b, xm_b)  // e = ( 1, 0) from x - 1
            LBD_PULL(3, r0_b, xp_b)  // e = (-1, 0) from x + 1
            if (WALLS && (rb == 0 || rb == ny - 1)) {
                // halfway bounce-back: at row 0 the populations with e_y = 1, at
                // row ny - 1 those with e_y = -1 are the site's own reversed ones
                const bool bot = rb == 0, top = rb == ny - 1;
                const unsigned rmw = bot ? r0_b : rm_b, rpw = top ? r0_b : rp_b;
                LBD_PULL_FROM(2, bot ? 4u : 2u, rmw, xg_b)
                LBD_PULL_FROM(5, bot ? 7u : 5u, rmw, bot ? xg_b : xm_b)
                LBD_PULL_FROM(6, bot ? 8u : 6u, rmw, bot ? xg_b : xp_b)
                LBD_PULL_FROM(4, top ? 2u : 4u, rpw, xg_b)
                LBD_PULL_FROM(7, top ? 5u : 7u, rpw, top ? xg_b : xp_b)
                LBD_PULL_FROM(8, top ? 6u : 8u, rpw, top ? xg_b : xm_b)
            } else {
                LBD_PULL(2, rm_b, xg_b)  // e = ( 0, 1) from y - 1
                LBD_PULL(4, rp_b, xg_b)  // e = ( 0,-1) from y + 1
                LBD_PULL(5, rm_b, xm_b)  // e = ( 1, 1)
                LBD_PULL(6, rm_b, xp_b)  // e = (-1, 1)
                LBD_PULL(7, rp_b, xp_b)  // e = (-1,-1)
                LBD_PULL(8, rp_b, xm_b)  // e = ( 1,-1)
            }
#undef LBD_PULL_FROM
#undef LBD_PULL
        }
        cp_commit();
        adv(lo_b);
        adv(rm_b);
        adv(r0_b);
        adv(rp_b);
    };

    uint32_t theta_w = 0;         // source-mask word of stage E's current row
    T phs_e = T(0), phs_n = T(0); // phi* of stage E's next row and the row after
    Win2<V> wA, wD;               // (phi, psi), (phi*, psi*)
    WinG2<V> wB;                  // (mu, m)
    WinLap2<V> wEm, wEp;          // (mu*, m*), (psi*, p*)
    wA.reset(); wB.reset(); wD.reset(); wEm.reset(); wEp.reset();
    V gps1 = vsplat(T(0)), gps2 = vsplat(T(0));  // grad psi (x, y) from A, 1 and 2 iterations old
    T ux1 = 0, ux2 = 0, uy1 = 0, uy2 = 0, uy3 = 0;  // own u from B, 1..3 iterations old

    const T a = p.a, b = p.b, B0 = p.B0, B1 = p.B1;
    // B1 with the 1/12 of each of two gradient factors (the windows return 12 grad)
    const T B1g = B1 * T(1.0 / 144.0), B1h = B1 * T(0.5 / 144.0);
    char *const g_out = reinterpret_cast<char *>(p.g_out);
    char *const phi_out = reinterpret_cast<char *>(p.phi_out);
    char *const psi_out = reinterpret_cast<char *>(p.psi_out);
    issue(0, 0);
    issue(1, 1);
    int ps = 0;  // population staging slot of the current iteration, i % PS
    const int iters = (yend - y0) + 15;
    // One pipeline iteration; with GUARD false (steady state: every stage active,
    // every row written is owned) the row conditions vanish at compile time.
    auto body = [&](auto guard_tag, const int i) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        cp_wait1();
        __syncthreads();
        issue(i + 2, ps == 0 ? PS - 1 : ps - 1);

        // ---- E: phi^{n+1} (Eq. 18), psi^{n+1} (Eq. 19 + source, sink), row y0 - 15 + i
        {
            const int r = y0 - 15 + i;   // output row; pushes row r + 1
            if ((!GUARD || i >= 13) && inE) {
                // with plates, row -1 mirrors row 0 and row ny mirrors row ny - 1
                const V *M1 = r_ms + ((r + 1 - y0) & (RM - 1)) * RS;
                const V *P1 = r_pp + ((r + 1 - y0) & (RM - 1)) * RS;
                if (WALLS && r == 0) {
                    wEm.mirror_below();
                    wEp.mirror_below();
                }
                const V mc = wEm.cp, pc = wEp.cp;            // (mu*, m*), (psi*, p*) at r
                V lm, lp;                                     // (lap mu*, lap m*), (lap psi*, lap p*)
                if (WALLS && r == ny - 1) {
                    lm = wEm.push_mirror();
                    lp = wEp.push_mirror();
                } else {
                    lm = wEm.push(M1[0], M1[-1], M1[1]);
                    lp = wEp.push(P1[0], P1[-1], P1[1]);
                }
                if (!GUARD || r >= y0) {
                    const T phs = phs_e;
                    const T phi_new = phs + p.M * lm.x;
                    // lap psi + (psi lap m + lap(psi m) - m lap psi) / 2
                    const T psc = pc.x;
                    const T div = lp.x + T(0.5) * ((psc * lm.y + lp.y) - mc.y * lp.x);
                    T src = T(0);
                    if ((theta_w >> (xo & 31)) & 1u) src = A_t;
                    const T psi_new = psc + (p.D * div - gamma_t * (psc - p.c0) + src);
                    const unsigned o = (unsigned)r * pitch_b + xo_b;
                    *reinterpret_cast<T *>(phi_out + o) = phi_new;
                    *reinterpret_cast<T *>(psi_out + o) = psi_new;
                }
            }
        }
        // source-mask word of the next output row, loaded one iteration ahead
        if (inE) {
            const int rn = y0 - 14 + i;
            theta_w = (rn >= y0 && rn < yend) ? p.theta[rn * p.theta_words + (xo >> 5)] : 0u;
        }
        // ---- D: mu*, m*, p* at row y0 - 13 + i (Eq. 3 on phi*, psi*; Eq. 5) ----
        {
            const int r = y0 - 13 + i;
            if (!GUARD || (i >= 10 && r < yend + 1)) {
                const V *S1 = r_st + ((r + 1 - y0) & (CD - 1)) * RS;
                V gx, gy, lap, mid;
                if (WALLS && r == 0) wD.mirror_below();
                if (WALLS && r == ny - 1)
                    wD.push_mirror(gx, gy, lap, mid);
                else
                    wD.push(S1[0], S1[-1], S1[1], gx, gy, lap, mid);  // lanes: phi*, psi*
                phs_e = phs_n;  // phi* at row r - 1: stage E's row in the next iteration
                phs_n = mid.x;
                if (!GUARD || i >= 12) {
                    const T pn = r_ps[((r - y0) & (LD - 1)) * RS].x;  // phi^n for the cubic
                    const T mus = a * mid.x + b * (pn * pn * pn) - (B0 + B1 * mid.y) * lap.x -
                                  B1g * (gx.x * gx.y + gy.x * gy.y);
                    const T ms = B1h * (gx.x * gx.x + gy.x * gy.x);
                    const int so = ((r - y0) & (RM - 1)) * RS;
                    r_ms[so] = vmake(mus, ms);
                    r_pp[so] = vmake(mid.y, mid.y * ms);
                }
            }
        }
        // ---- C: phi*, psi* at row y0 - 11 + i (donor-cell fluxes, Eqs. 16-17) ----
        {
            const int r = y0 - 11 + i;
            if (!GUARD || (i >= 9 && r < yend + 2)) {
                const V *Q = r_ps + ((r - y0) & (LD - 1)) * RS;
                const V QN = r_ps[((r + 1 - y0) & (LD - 1)) * RS], QS = r_ps[((r - 1 - y0) & (LD - 1)) * RS];
                const T *U = r_ux + ((r - y0) & (RD - 1)) * RS;
                const T uxc = ux2;
                const T ue = T(0.5) * (uxc + U[1]);
                const T uw = T(0.5) * (U[-1] + uxc);
                T un = T(0.5) * (uy2 + uy1);
                T us = T(0.5) * (uy3 + uy2);
                if (WALLS && r == ny - 1) un = T(0);  // no flux through a plate
                if (WALLS && r == 0) us = T(0);
                const V Q0 = Q[0], QE = Q[1], QW = Q[-1];
                // face flux = u_f * upwind value, both fields of the pair at once
                const V fe = vsplat(ue) * (ue > T(0) ? Q0 : QE);
                const V fw = vsplat(uw) * (uw > T(0) ? QW : Q0);
                const V fn = vsplat(un) * (un > T(0) ? Q0 : QN);
                const V fs = vsplat(us) * (us > T(0) ? QS : Q0);
                r_st[((r - y0) & (CD - 1)) * RS] = Q0 - ((fe - fw) + (fn - fs));
            }
        }
        // ---- B: force (Eq. 14), moments (Eq. 11), collision (Eqs. 10, 12, 13) ----
        {
            const int r = y0 - 9 + i;
            T ux = T(0), uy = T(0);
            if (!GUARD || (i >= 4 && r < yend + 3)) {
                const V *M1 = r_mm + ((r + 1 - y0) & (RM - 1)) * RS;
                V gx, gy, mid;
                wB.push_grad(M1[0], M1[-1], M1[1], gx, gy, mid);  // lanes: mu, m
                if (!GUARD || i >= 6) {
                    const V pp = r_ps[((r - y0) & (LD - 1)) * RS];  // (phi, psi) at r
                    // F = -phi grad mu - (grad psi + psi grad m); lanes x, y (the
                    // gradients 12 times too large, hence the 1/12)
                    V F = vmake(fma(-pp.x, gx.x, fma(-pp.y, gx.y, -gps2.x)),
                                fma(-pp.x, gy.x, fma(-pp.y, gy.y, -gps2.y)));
                    F = vfma(F, vsplat(T(1.0 / 12.0)), vmake(p.fx, p.fy));  // fx, fy: LBD_BODY_FORCE
                    const T *G = s_pop + ps * 9 * NT;
                    const T g0 = G[0];
                    const V g12 = vmake(G[NT], G[2 * NT]), g34 = vmake(G[3 * NT], G[4 * NT]);
                    const V g56 = vmake(G[5 * NT], G[6 * NT]), g78 = vmake(G[7 * NT], G[8 * NT]);
                    // Eq. (11) on the deviations g = f - w; j = (jx, jy)
                    const V s1 = (g12 + g34) + (g56 + g78);
                    const T dn = g0 + (s1.x + s1.y);
                    const V a13 = g12 - g34;  // (g1 - g3, g2 - g4)
                    const T jx = a13.x + ((g56.x - g56.y) + (g78.y - g78.x));
                    const T jy = a13.y + ((g56.x + g56.y) - (g78.x + g78.y));
                    const T n = T(1) + dn;
                    const T inv = rcp_rn(n);
                    const V u = vfma(vsplat(T(0.5)), F, vmake(jx, jy)) * vsplat(inv);
                    ux = u.x;
                    uy = u.y;
                    if ((!GUARD || (r >= y0 && r < yend)) && inE) {
                        // post_i = (1-w) g_i + W (K + eu (c1 eu + c2 eF)) +- W (c3 eu + c4 eF),
                        // opposite directions paired; axis pairs (1,3), (2,4) in the lanes of
                        // one vector, diagonal pairs (5,7), (6,8) in another
                        const T om = p.omega, gk = p.guo;
                        const V om1 = vsplat(T(1) - om);
                        const T usq = ux * ux + uy * uy, uF = ux * F.x + uy * F.y;
                        const T K = om * (dn - T(1.5) * n * usq) - T(3) * gk * uF;
                        const V c1 = vsplat(T(4.5) * om * n), c2 = vsplat(T(9) * gk);
                        const V c3 = vsplat(T(3) * om * n), c4 = vsplat(T(3) * gk);
                        const V Kv = vsplat(K);
                        char *Go = g_out + ((unsigned)r * pitch_b + xo_b);
#define LBD_OUT(I) (*reinterpret_cast<T *>(Go + (I) * plane_b))
                        LBD_OUT(0) = (T(1) - om) * g0 + T(4.0 / 9.0) * K;
                        {   // e = (1,0) and (0,1) in the lanes, opposites (-1,0), (0,-1)
                            const V eu = u, eF = F, W = vsplat(T(1.0 / 9.0));
                            const V sym = W * vfma(eu, vfma(c1, eu, c2 * eF), Kv);
                            const V anti = W * vfma(c3, eu, c4 * eF);
                            const V pos = vfma(om1, g12, sym + anti);
                            const V neg = vfma(om1, g34, sym - anti);
                            LBD_OUT(1) = pos.x; LBD_OUT(2) = pos.y;
                            LBD_OUT(3) = neg.x; LBD_OUT(4) = neg.y;
                        }
                        {   // e = (1,1) and (-1,1) in the lanes, opposites (-1,-1), (1,-1)
                            const V eu = vmake(ux + uy, uy - ux), eF = vmake(F.x + F.y, F.y - F.x);
                            const V W = vsplat(T(1.0 / 36.0));
                            const V sym = W * vfma(eu, vfma(c1, eu, c2 * eF), Kv);
                            const V anti = W * vfma(c3, eu, c4 * eF);
                            const V pos = vfma(om1, g56, sym + anti);
                            const V neg = vfma(om1, g78, sym - anti);
                            LBD_OUT(5) = pos.x; LBD_OUT(6) = pos.y;
                            LBD_OUT(7) = neg.x; LBD_OUT(8) = neg.y;
                        }
#undef LBD_OUT
                    }
                    if (p.flags & LBD_FROZEN_U) {
                        ux = p.ux0;
                        uy = p.uy0;
                    }
                    r_ux[((r - y0) & (RD - 1)) * RS] = ux;
                }
            }
            // own-column u history for stage C (rows r-1, r-2, r-3 next iteration)
            uy3 = uy2; uy2 = uy1; uy1 = uy;
            ux2 = ux1; ux1 = ux;
        }
        // ---- A: mu_phi (Eq. 3), m (Eq. 5), grad psi at row y0 - 7 + i -----------
        {
            const int r = y0 - 7 + i;
            V gp = vsplat(T(0));
            if (!GUARD || (i >= 1 && r < yend + 4)) {
                const V *F1 = r_ps + ((r + 1 - y0) & (LD - 1)) * RS;
                V gx, gy, lap, mid;
                wA.push(F1[0], F1[-1], F1[1], gx, gy, lap, mid);  // lanes: phi, psi
                gp = vmake(gx.y, gy.y);
                if (!GUARD || i >= 3) {
                    const T ph = mid.x;
                    const T mu = a * ph + b * (ph * ph * ph) - (B0 + B1 * mid.y) * lap.x -
                                 B1g * (gx.x * gx.y + gy.x * gy.y);
                    const T m = B1h * (gx.x * gx.x + gy.x * gy.x);
                    r_mm[((r - y0) & (RM - 1)) * RS] = vmake(mu, m);
                }
            }
            gps2 = gps1; gps1 = gp;
        }
        ps = ps == PS - 1 ? 0 : ps + 1;
    };
    const std::integral_constant<bool, true> guarded;
    const std::integral_constant<bool, false> steady;
    // steady iterations, i in [15, nrows + 9): every stage active (E writes
    // owned rows from i = 15) and every written row owned (B's last at nrows + 8)
    const int s1 = (yend - y0) + 9;
    int i = 0;
    for (; i < 15 && i < iters; ++i) body(guarded, i);
#pragma unroll 2
    for (; i < s1; ++i) body(steady, i);
    for (; i < iters; ++i) body(guarded, i);
    asm volatile("cp.async.wait_all;\n" ::);
}

// One CTA per (stripe, row segment) on a 1-D grid, stripes fastest: the first
// `rem` stripes are cut into base + 1 row segments, the others into base, the
// heights of a stripe's segments differing by at most one row.
template <typename T, int NT, bool WALLS>
__global__ void __launch_bounds__(NT, StripeOcc<T, NT>::value)
    stripe_kernel(const StepArgs<T> p, const int stripes, const int base, const int rem) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
    const int q = p.ny / n, r = p.ny - q * n;  // the first ny % n segments one row taller
    stripe_body<T, NT, WALLS>(p, s * (NT - 10), j * q + min(j, r), q + (j < r ? 1 : 0), p.A,
                              p.gamma, smem_raw);
}

// Batched step: CTAs walk the work list; the arguments of the item's instance
// are staged in shared memory and the activity is evaluated from the device
// step count (so that the launch can be replayed from a CUDA graph).
template <typename T, int NT, bool WALLS>
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
        stripe_body<T, NT, WALLS>(sp, item.x0, item.y0, item.rows, s_A, s_gamma, smem_raw);
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

template <typename T, int NT, bool WALLS>
cudaError_t launch_stripe_as(const StepArgs<T> &a, int seg, cudaStream_t s) {
    const size_t smem = stripe_smem_bytes<T>(NT);
    static unsigned long long configured = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(stripe_kernel<T, NT, WALLS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    // ceil(ny / seg) segments per stripe; when that leaves resident CTA slots
    // free, more segments (at least half a segment high), so that every SM
    // holds as many CTAs as the others
    static int slots[64] = {0};
    if (!slots[dev & 63]) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stripe_kernel<T, NT, WALLS>, NT,
                                                          smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        slots[dev & 63] = per_sm * sms > 0 ? per_sm * sms : 1;
    }
    const int stripes = (a.nx + (NT - 10) - 1) / (NT - 10);
    const int per = (a.ny + seg - 1) / seg;
    long long total = (long long)stripes * per;
    const long long cap = (long long)stripes * (2 * a.ny / seg > per ? 2 * a.ny / seg : per);
    if (total < slots[dev & 63]) total = slots[dev & 63] < cap ? slots[dev & 63] : cap;
    const int base = (int)(total / stripes), rem = (int)(total % stripes);
    stripe_kernel<T, NT, WALLS><<<(unsigned)total, NT, smem, s>>>(a, stripes, base, rem);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stripe(const StepArgs<T> &a, int nt, int seg, cudaStream_t s) {
    const bool walls = (a.flags & LBD_WALLS) != 0;
    if (nt == 128) return walls ? launch_stripe_as<T, 128, true>(a, seg, s)
                                : launch_stripe_as<T, 128, false>(a, seg, s);
    if (nt == 256) return walls ? launch_stripe_as<T, 256, true>(a, seg, s)
                                : launch_stripe_as<T, 256, false>(a, seg, s);
    return cudaErrorInvalidValue;
}

// One launch of the batch walk over n_items items of one variant (periodic, or
// with plates: each is its own instantiation, so that an instance computes
// exactly as it would in a context of its own).
template <typename T, int NT, bool WALLS>
cudaError_t launch_stripe_batch_as(const StepArgs<T> *args, const BatchItem *items, int n_items,
                                   int ctas, const long long *t_dev, int t_off, cudaStream_t s) {
    const size_t smem = stripe_smem_bytes<T>(NT);
    static unsigned long long configured = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(stripe_batch_kernel<T, NT, WALLS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    stripe_batch_kernel<T, NT, WALLS><<<ctas, NT, smem, s>>>(args, items, n_items, t_dev, t_off);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stripe_batch(const StepArgs<T> *args, const BatchItem *items, int n_items,
                                int nt, bool walls, int ctas, const long long *t_dev, int t_off,
                                cudaStream_t s) {
    if (nt == 128)
        return walls ? launch_stripe_batch_as<T, 128, true>(args, items, n_items, ctas, t_dev, t_off, s)
                     : launch_stripe_batch_as<T, 128, false>(args, items, n_items, ctas, t_dev, t_off, s);
    if (nt == 256)
        return walls ? launch_stripe_batch_as<T, 256, true>(args, items, n_items, ctas, t_dev, t_off, s)
                     : launch_stripe_batch_as<T, 256, false>(args, items, n_items, ctas, t_dev, t_off, s);
    return cudaErrorInvalidValue;
}

template <typename T>
int stripe_batch_ctas_per_sm(int nt) {
    int n = 0;
    const size_t smem = stripe_smem_bytes<T>(nt);
    cudaError_t e = nt == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &n, stripe_batch_kernel<T, 128, false>, 128, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &n, stripe_batch_kernel<T, 256, false>, 256, smem);
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
                                                int, bool, int, const long long *, int,
                                                cudaStream_t);
template cudaError_t launch_stripe_batch<double>(const StepArgs<double> *, const BatchItem *, int,
                                                 int, bool, int, const long long *, int,
                                                 cudaStream_t);
template cudaError_t launch_stripe<float>(const StepArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stripe<double>(const StepArgs<double> &, int, int, cudaStream_t);
template size_t stripe_smem_bytes<float>(int);
template size_t stripe_smem_bytes<double>(int);

}  // namespace lbd

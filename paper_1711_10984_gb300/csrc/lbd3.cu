// lbd3.cu -- the coupled step of arXiv 1711.10984 (Section 2) on the D3Q19
// lattice, and the C ABI of include/lbd3.h.
//
// One step is five kernels; each CTA walks a run of z planes of a 32 x 8 tile
// (32 x 16 for the advection, two rows per thread), the differentiated fields
// staged in a ring of shared-memory halo planes:
//   k_chem    mu_phi (Eq. 3), m (Eq. 5) at t^n                       -> mu, m
//   k_lb      F (Eq. 14), pull f_i, u (Eq. 11), BGK + Guo collision
//             (Eqs. 10, 12, 13), u for the advection                 -> f, u
//   k_advect  phi*, psi* by donor-cell fluxes on 6 faces (Eqs. 16-17)
//   k_chem2   mu*, m* from phi*, psi* (cubic from phi^n)
//   k_update  phi^{n+1} (Eq. 18), psi^{n+1} (Eq. 19 in link form, sink, source)
// Populations are stored as deviations g_i = f_i - w_i (pull layout: buffer_i(x)
// is read by site x + e_i); x rows are padded to 128 bytes.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>

#include "lbd3.h"

namespace lbd {
// device and pinned-host allocation through the library-wide failure hook (lbd_api.cu)
cudaError_t dev_malloc(void **p, size_t bytes);
}  // namespace lbd

namespace {

constexpr int Q = 19;
// D3Q19 velocity components of direction i (the order of include/lbd3.h), as
// compile-time functions so that unrolled loops fold every neighbour index
__host__ __device__ constexpr int c_ex(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int c_ey(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int c_ez(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}

__host__ __device__ inline double wq(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Lattice geometry and the scalars of one step.
template <typename T>
struct Arg3 {
    int nx, ny, nz;
    int zl;                       // planes per CTA of the marching kernels
    long long pitch, plane, vol;  // row pitch, pitch * ny, plane * nz (elements)
    const T *g_in;
    T *g_out;
    const T *phi, *psi;  // phi^n, psi^n
    T *phi_o, *psi_o;    // phi^{n+1}, psi^{n+1}
    T *mu, *mm, *ux, *uy, *uz, *phs, *pss, *mus, *mms;  // intermediates
    const uint32_t *theta;  // source balls, one bit per site (words per row (nx+31)/32)
    T a, b, B0, B1, M, D, omega, guo, gamma, c0, A;
    T fx, fy, fz, ux0, uy0, uz0;
    int frozen;
};

// ------------------------------------------------------ z-marching kernels
// Each CTA of NT = TX x TY threads owns a TX x (TY RY) tile of the xy plane (RY
// rows per thread) and a run of zl planes, and walks the run in z.  The fields
// it differentiates pass through a ring of SLOTS shared-memory planes, each the
// tile with a one-site periodic halo, so that a value is loaded from global
// memory about HP / (TX TY RY) + 2 / zl times per step instead of once per
// neighbour (nine xy rows per value with one thread
// per site).  The planes arrive by cp.async, AHEAD planes ahead of the ones
// being read.  One barrier per plane: at plane k, after each thread has waited
// for its own copies of plane k + 1, the barrier makes every copy of plane
// k + 1 visible and ends every read of plane k - 2, whose slot then receives
// plane k + 3.  Two fields that are differentiated alike are stored as a pair
// (interleaved), read with one shared-memory access and, in FP32, combined with
// the packed FP32x2 instructions.
constexpr int TX = 32, TY = 8, NT = TX * TY;  // threads of a CTA
constexpr int HX = TX + 2;                     // halo row length
constexpr int AHEAD = 2;
constexpr int SLOTS = 3 + AHEAD;  // planes k - 1, k, k + 1 read, the rest in flight

// A tile of TX x (TY RY) sites: thread (tx, ty) computes rows ty + TY r, r < RY.
template <int RY>
struct Tile {
    static constexpr int H = TY * RY;              // rows of the tile
    static constexpr int HP = HX * (H + 2);        // values per halo plane
    static constexpr int LPT = (HP + NT - 1) / NT;  // halo values a thread copies per plane
};

// rows per thread of the step kernels (k_lb keeps one: its 19 pulls per site
// are held in registers across the barrier)
constexpr int R_LB = 1, R_ADVECT = 2;

extern __shared__ __align__(16) unsigned char lbd3_smem[];

// NP pair fields and NS single fields
template <int NP, int NS, int RY>
constexpr size_t ring_bytes(size_t esz) {
    return (size_t)(2 * NP + NS) * SLOTS * Tile<RY>::HP * esz;
}

// Two values of one site in the lanes of a vector: FP32 uses the packed FP32x2
// instructions (FMUL2 / FFMA2), FP64 plain component-wise arithmetic;
// every lane is rounded as the scalar operation would be.
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
template <typename T>
using V2 = typename V2t<T>::type;

__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, rounded once
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 operator-(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 operator*(double2 a, double2 b) {
    return make_double2(a.x * b.x, a.y * b.y);
}
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// the lane type of V and a lane value broadcast to V
template <typename V>
struct Lane {
    using type = V;
    static __device__ __forceinline__ V splat(V s) { return s; }
};
template <>
struct Lane<float2> {
    using type = float;
    static __device__ __forceinline__ float2 splat(float s) { return make_float2(s, s); }
};
template <>
struct Lane<double2> {
    using type = double;
    static __device__ __forceinline__ double2 splat(double s) { return make_double2(s, s); }
};

template <int BYTES>
__device__ __forceinline__ void cp_async(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The three halo planes around the site being computed.
template <typename T, int HP>
struct Planes {
    const V2<T> *pp;  // pair fields, NP x SLOTS x HP pairs, offset by the site's index
    const T *ps;      // single fields, NS x SLOTS x HP values, offset likewise
    int om, o0, op;   // slot offsets of planes z - 1, z, z + 1
    __device__ int off(int ex, int ey, int ez) const {
        return (ez < 0 ? om : (ez > 0 ? op : o0)) + ey * HX + ex;
    }
    __device__ V2<T> pair(int f, int ex, int ey, int ez) const {
        return pp[f * SLOTS * HP + off(ex, ey, ez)];
    }
    __device__ T one(int f, int ex, int ey, int ez) const {
        return ps[f * SLOTS * HP + off(ex, ey, ez)];
    }
};

// Walk the CTA's run of planes; site(x, y, z, s, planes) is called for every
// lattice site of the tile, s its element offset, and pre(x, y, z, s) before
// the wait for the plane (loads that need no ring).  src lists the two fields
// of each pair, then the single fields.
template <typename T, int NP, int NS, int RY, class Pre, class Site>
__device__ __forceinline__ void march(const Arg3<T> &p, const T *const (&src)[2 * NP + NS],
                                      Pre pre, Site site) {
    constexpr int HP = Tile<RY>::HP, LPT = Tile<RY>::LPT;
    constexpr int SINGLES = 2 * NP * SLOTS * HP;  // element offset of the single fields
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    T *sm = reinterpret_cast<T *>(lbd3_smem);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * Tile<RY>::H;
    const int z0 = blockIdx.z * p.zl;
    const int z1 = min(nz, z0 + p.zl);
    const int x = x0 + tid % TX, y = y0 + tid / TX;
    const unsigned pitch = (unsigned)p.pitch, plane = (unsigned)p.plane;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(sm);
    unsigned hxy[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int e = tid + j * NT;
        int gx = (x0 + e % HX - 1) % nx, gy = (y0 + e / HX - 1) % ny;
        gx += gx < 0 ? nx : 0;
        gy += gy < 0 ? ny : 0;
        hxy[j] = (unsigned)gy * pitch + (unsigned)gx;
    }
    // copy plane k (k in [z0 - 1, z1], periodic) into the slot at element offset o
    auto issue = [&](int k, int o) {
        if (k <= z1) {
            const unsigned zo = (unsigned)(k < 0 ? k + nz : (k >= nz ? k - nz : k)) * plane;
#pragma unroll
            for (int j = 0; j < LPT; ++j) {
                const int e = tid + j * NT;
                if (e < HP) {
#pragma unroll
                    for (int f = 0; f < NP; ++f)
#pragma unroll
                        for (int c = 0; c < 2; ++c)
                            cp_async<sizeof(T)>(
                                sbase + (unsigned)((2 * (f * SLOTS * HP + o + e) + c) * sizeof(T)),
                                src[2 * f + c] + zo + hxy[j]);
#pragma unroll
                    for (int f = 0; f < NS; ++f)
                        cp_async<sizeof(T)>(
                            sbase + (unsigned)((SINGLES + f * SLOTS * HP + o + e) * sizeof(T)),
                            src[2 * NP + f] + zo + hxy[j]);
                }
            }
        }
        cp_commit();
    };
    int o[SLOTS];  // slot offsets of planes k - 1, k, k + 1, ..., k + AHEAD, and the free slot
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) o[q] = q * HP;
#pragma unroll
    for (int q = 0; q < SLOTS - 1; ++q) issue(z0 - 1 + q, o[q]);
    const int c = (tid / TX + 1) * HX + tid % TX + 1;
    const bool xin = x < nx;
    for (int k = z0; k < z1; ++k) {
        const unsigned s = (unsigned)k * plane + (unsigned)y * pitch + (unsigned)x;
#pragma unroll
        for (int r = 0; r < RY; ++r)
            if (xin && y + TY * r < ny) pre(x, y + TY * r, k, s + (unsigned)(TY * r) * pitch);
        cp_wait<AHEAD - 1>();  // this thread's copies of plane k + 1 have landed
        __syncthreads();
        issue(k + SLOTS - 2, o[SLOTS - 1]);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            Planes<T, HP> pl;
            pl.pp = reinterpret_cast<const V2<T> *>(sm) + c + TY * r * HX;
            pl.ps = sm + SINGLES + c + TY * r * HX;
            pl.om = o[0];
            pl.o0 = o[1];
            pl.op = o[2];
            if (xin && y + TY * r < ny)
                site(x, y + TY * r, k, s + (unsigned)(TY * r) * pitch, pl);
        }
        const int freed = o[0];
#pragma unroll
        for (int q = 0; q < SLOTS - 1; ++q) o[q] = o[q + 1];
        o[SLOTS - 1] = freed;
    }
    cp_wait<0>();
}

// The z-window form of march for kernels that need the D3Q19 gradient or
// Laplacian of ring fields (and nothing else of the neighbours).  The 19-point
// stencil splits into per-plane sums over the in-plane 3 x 3 neighbourhood
// (ZWin below), so each plane is read once, when it arrives, and a thread
// keeps in registers the partial sums of its outputs at the plane before it:
// at the arrival of plane k the output is plane k - 1.  The ring holds the arriving plane and
// AHEAD planes in flight.  arrive(nb, out, x, y, z, s) receives the arriving
// plane's neighbourhood (nb.pair(f, ex, ey), nb.one(f, ex, ey)); out says
// whether plane z = k - 1 (element offset s) is one of the CTA's planes;
// pre(x, y, z, s) runs for that plane before the wait.
constexpr int ZSLOTS = 1 + AHEAD;

template <int NP, int NS>
constexpr size_t zring_bytes(size_t esz) {
    return (size_t)(2 * NP + NS) * ZSLOTS * Tile<1>::HP * esz;
}

template <typename T>
struct ZNb {
    const V2<T> *pp;
    const T *ps;
    int o;
    __device__ V2<T> pair(int f, int ex, int ey) const {
        return pp[f * ZSLOTS * Tile<1>::HP + o + ey * HX + ex];
    }
    __device__ T one(int f, int ex, int ey) const {
        return ps[f * ZSLOTS * Tile<1>::HP + o + ey * HX + ex];
    }
};

template <typename T, int NP, int NS, class Pre, class Arrive>
__device__ __forceinline__ void march_zw(const Arg3<T> &p, const T *const (&src)[2 * NP + NS],
                                         Pre pre, Arrive arrive) {
    constexpr int HP = Tile<1>::HP, LPT = Tile<1>::LPT;
    constexpr int SINGLES = 2 * NP * ZSLOTS * HP;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    T *sm = reinterpret_cast<T *>(lbd3_smem);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * p.zl;
    const int z1 = min(nz, z0 + p.zl);
    const int x = x0 + tid % TX, y = y0 + tid / TX;
    const unsigned pitch = (unsigned)p.pitch, plane = (unsigned)p.plane;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(sm);
    unsigned hxy[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int e = tid + j * NT;
        int gx = (x0 + e % HX - 1) % nx, gy = (y0 + e / HX - 1) % ny;
        gx += gx < 0 ? nx : 0;
        gy += gy < 0 ? ny : 0;
        hxy[j] = (unsigned)gy * pitch + (unsigned)gx;
    }
    // copy plane k (k in [z0 - 1, z1], periodic) into the slot at element offset o
    auto issue = [&](int k, int o) {
        if (k <= z1) {
            const unsigned zo = (unsigned)(k < 0 ? k + nz : (k >= nz ? k - nz : k)) * plane;
#pragma unroll
            for (int j = 0; j < LPT; ++j) {
                const int e = tid + j * NT;
                if (e < HP) {
#pragma unroll
                    for (int f = 0; f < NP; ++f)
#pragma unroll
                        for (int c = 0; c < 2; ++c)
                            cp_async<sizeof(T)>(
                                sbase + (unsigned)((2 * (f * ZSLOTS * HP + o + e) + c) * sizeof(T)),
                                src[2 * f + c] + zo + hxy[j]);
#pragma unroll
                    for (int f = 0; f < NS; ++f)
                        cp_async<sizeof(T)>(
                            sbase + (unsigned)((SINGLES + f * ZSLOTS * HP + o + e) * sizeof(T)),
                            src[2 * NP + f] + zo + hxy[j]);
                }
            }
        }
        cp_commit();
    };
    int o[ZSLOTS];  // slot offsets of planes k, k + 1, ..., k + AHEAD - 1, and the free slot
#pragma unroll
    for (int q = 0; q < ZSLOTS; ++q) o[q] = q * HP;
#pragma unroll
    for (int q = 0; q < ZSLOTS - 1; ++q) issue(z0 - 1 + q, o[q]);
    const int c = (tid / TX + 1) * HX + tid % TX + 1;
    const bool in = x < nx && y < ny;
    for (int k = z0 - 1; k <= z1; ++k) {
        const bool out = k > z0;
        const unsigned s = (unsigned)(out ? k - 1 : 0) * plane + (unsigned)y * pitch + (unsigned)x;
        if (in && out) pre(x, y, k - 1, s);
        cp_wait<AHEAD - 1>();  // this thread's copies of plane k have landed
        __syncthreads();       // ... and everyone's; plane k - 1 has been read
        issue(k + AHEAD, o[ZSLOTS - 1]);
        ZNb<T> nb;
        nb.pp = reinterpret_cast<const V2<T> *>(sm) + c;
        nb.ps = sm + SINGLES + c;
        nb.o = o[0];
        if (in) arrive(nb, out, x, y, k - 1, s);
        const int freed = o[0];
#pragma unroll
        for (int q = 0; q < ZSLOTS - 1; ++q) o[q] = o[q + 1];
        o[ZSLOTS - 1] = freed;
    }
    cp_wait<0>();
}

// Per-plane sums of a pair field for the isotropic D3Q19 gradient and Laplacian
// (weights 1/18 for the 6 faces, 1/36 for the 12 edges).  For plane z, with C
// the value at (x, y, z) and the in-plane neighbours x+-1, y+-1 and diagonals:
//   T  = (x+1) + (x-1) + (y+1) + (y-1) - 4 C,    E  = (four diagonals) - 4 C,
//   DX = (x+1) - (x-1),   DY = (y+1) - (y-1),
//   EX = (x+1,y+1) + (x+1,y-1) - (x-1,y+1) - (x-1,y-1),   EY likewise in y.
// With m, 0, p the planes z - 1, z, z + 1:
//   d/dx = DX_0 / 6 + (EX_0 + DX_m + DX_p) / 12,   d/dy likewise,
//   d/dz = (C_p - C_m) / 2 + (T_p - T_m) / 12,
//   lap  = T_0 / 3 + (E_0 + T_m + T_p) / 6 + (C_p - C_0) - (C_0 - C_m),
// which is 3 sum_i w_i e_i v_i and 6 sum_i w_i (v_i - v_0) term by term.
template <typename V, bool GRAD, bool LAP>
struct ZWin {
    using S = typename Lane<V>::type;
    // Kept as partial sums of the outputs at plane z (the last plane before the
    // arriving one), so that each arrival recomputes every kept value instead of
    // shifting a window (no register moves in the plane loop).  With D = C - C_prev:
    //   ax = DX_z / 6 + EX_z / 12 + DX_{z-1} / 12     (d/dx at z = ax + DX_{z+1} / 12)
    //   ay likewise                                    (d/dy)
    //   az = D_z / 2 - T_{z-1} / 12                    (d/dz = az + D_{z+1} / 2 + T_{z+1} / 12)
    //   al = T_z / 3 + E_z / 6 + T_{z-1} / 6 - D_z     (lap = al + T_{z+1} / 6 + D_{z+1})
    // and bx = DX_z / 12, by = DY_z / 12, tp = T_z, cp = C_z.
    V ax, ay, az, al, bx, by, tp, cp;
    __device__ __forceinline__ void reset() {
        ax = ay = az = al = bx = by = tp = cp = Lane<V>::splat(S(0));
    }
    // the arriving plane z + 1 (values from get(ex, ey)); with out, the
    // gradient and Laplacian at plane z and its centre value
    template <class Get>
    __device__ __forceinline__ void arrive(Get get, bool out, V &gx, V &gy, V &gz, V &lap,
                                           V &mid) {
        const V k6 = Lane<V>::splat(S(1) / S(6)), k12 = Lane<V>::splat(S(1) / S(12));
        const V c = get(0, 0);
        const V xp = get(1, 0), xm = get(-1, 0), yp = get(0, 1), ym = get(0, -1);
        const V pp = get(1, 1), pm = get(1, -1), mp = get(-1, 1), mn = get(-1, -1);
        const V t = vfma(c, Lane<V>::splat(S(-4)), (xp + xm) + (yp + ym));
        const V a = pp + pm, b = mp + mn;
        const V d = c - cp;
        if (out) {
            if (GRAD) {
                gx = vfma(xp - xm, k12, ax);
                gy = vfma(yp - ym, k12, ay);
                gz = az + vfma(d, Lane<V>::splat(S(0.5)), t * k12);
            }
            if (LAP) lap = al + vfma(t, k6, d);
            mid = cp;
        }
        if (GRAD) {
            const V dx = xp - xm, dy = yp - ym;
            ax = vfma(dx, k6, vfma(a - b, k12, bx));
            ay = vfma(dy, k6, vfma((pp + mp) - (pm + mn), k12, by));
            az = vfma(d, Lane<V>::splat(S(0.5)), tp * Lane<V>::splat(S(-1) / S(12)));
            bx = dx * k12;
            by = dy * k12;
        }
        if (LAP) {
            const V e = vfma(c, Lane<V>::splat(S(-4)), a + b);
            al = vfma(t, Lane<V>::splat(S(1) / S(3)), vfma(e + tp, k6, Lane<V>::splat(S(0)) - d));
        }
        tp = t;
        cp = c;
    }
};

// Offsets of the 27 sites around (x, y, z) (periodic), ox/oy/oz index -1, 0, 1;
// 32-bit (the host keeps 19 * vol below 2^32).
struct Nb {
    unsigned ox[3], oy[3], oz[3];
    __device__ unsigned at(int ex, int ey, int ez) const {
        return ox[ex + 1] + oy[ey + 1] + oz[ez + 1];
    }
};

template <typename T>
__device__ inline Nb neighbours(const Arg3<T> &p, int x, int y, int z) {
    Nb n;
    n.ox[0] = x ? x - 1 : p.nx - 1;
    n.ox[1] = x;
    n.ox[2] = x + 1 < p.nx ? x + 1 : 0;
    const unsigned pitch = (unsigned)p.pitch, plane = (unsigned)p.plane;
    n.oy[0] = (unsigned)(y ? y - 1 : p.ny - 1) * pitch;
    n.oy[1] = (unsigned)y * pitch;
    n.oy[2] = (unsigned)(y + 1 < p.ny ? y + 1 : 0) * pitch;
    n.oz[0] = (unsigned)(z ? z - 1 : p.nz - 1) * plane;
    n.oz[1] = (unsigned)z * plane;
    n.oz[2] = (unsigned)(z + 1 < p.nz ? z + 1 : 0) * plane;
    return n;
}

// The 19 values of ring pair f (single field f) around the site, in the D3Q19 order.
template <typename V, class P>
__device__ inline void gather_pair(const P &pl, int f, V v[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = pl.pair(f, c_ex(i), c_ey(i), c_ez(i));
}
template <typename T, class P>
__device__ inline void gather_one(const P &pl, int f, T v[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = pl.one(f, c_ex(i), c_ey(i), c_ez(i));
}

// acc + c * v for a compile-time velocity component c in {-1, 0, 1}: no code for
// c = 0 (IEEE arithmetic cannot drop an explicit 0 * v), a sign for c = -1;
// the value is the one of acc + (T)c * v.
template <int C, typename T>
__device__ __forceinline__ T acc_e(T acc, T v) {
    return C > 0 ? acc + v : (C < 0 ? acc - v : acc);
}
// acc + c w v, rounded once, for scalars and pairs
template <int C, typename V, typename S>
__device__ __forceinline__ V acc_we(V acc, S w, V v) {
    return C > 0 ? vfma(Lane<V>::splat(w), v, acc)
                 : (C < 0 ? vfma(Lane<V>::splat(-w), v, acc) : acc);
}
// (T)c * v for a compile-time component
template <int C, typename T>
__device__ __forceinline__ T mul_e(T v) {
    return C > 0 ? v : (C < 0 ? -v : T(0));
}

// f(std::integral_constant<int, i>) for i = I .. N-1, so that each direction's
// velocity components are template arguments
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// Isotropic D3Q19 gradient and Laplacian of the gathered values (scalars or pairs).
template <typename V>
__device__ inline void grad_lap(const V v[Q], V &gx, V &gy, V &gz, V &lap) {
    using S = typename Lane<V>::type;
    V sx = Lane<V>::splat(S(0)), sy = sx, sz = sx, sl = sx;
    static_for<1, Q>([&](auto k) {
        constexpr int i = decltype(k)::value;
        const S w = (S)wq(i);
        sx = acc_we<c_ex(i)>(sx, w, v[i]);
        sy = acc_we<c_ey(i)>(sy, w, v[i]);
        sz = acc_we<c_ez(i)>(sz, w, v[i]);
        sl = vfma(Lane<V>::splat(w), v[i] - v[0], sl);
    });
    gx = Lane<V>::splat(S(3)) * sx;
    gy = Lane<V>::splat(S(3)) * sy;
    gz = Lane<V>::splat(S(3)) * sz;
    lap = Lane<V>::splat(S(6)) * sl;
}

template <typename V>
__device__ inline void grad3(const V v[Q], V &gx, V &gy, V &gz) {
    V lap;
    grad_lap(v, gx, gy, gz, lap);
}

// mu_phi and m at t^n (Eqs. 3, 5); ring: the pair (phi, psi), z-window form
template <typename T>
__global__ void __launch_bounds__(NT) k_chem(const Arg3<T> p) {
    const T *const src[2] = {p.phi, p.psi};
    ZWin<V2<T>, true, true> w;
    w.reset();
    march_zw<T, 1, 0>(p, src, [](int, int, int, unsigned) {}, [&](const ZNb<T> &nb, bool out, int, int, int, unsigned s) {
        V2<T> gx, gy, gz, lap, mid;
        w.arrive([&](int ex, int ey) { return nb.pair(0, ex, ey); }, out, gx, gy, gz, lap, mid);
        if (out) {
            const T ph = mid.x, c = mid.y;
            p.mu[s] = p.a * ph + p.b * (ph * ph * ph) - (p.B0 + p.B1 * c) * lap.x -
                      p.B1 * (gx.x * gx.y + gy.x * gy.y + gz.x * gz.y);
            p.mm[s] = T(0.5) * p.B1 * (gx.x * gx.x + gy.x * gy.x + gz.x * gz.x);
        }
    });
}

// F (Eq. 14), pulled populations, u (Eq. 11) and the BGK + Guo collision
// (Eqs. 10, 12, 13) on the deviations g = f - w; with FIELDS, rho and u of the
// current state to dense doubles (rho, ux, uy, uz at d, N + d, 2N + d, 3N + d).
// Ring: the pair (mu, m) and psi.
template <typename T, int FIELDS>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) k_lb(const Arg3<T> p, double *out) {
    const T *const src[3] = {p.mu, p.mm, p.psi};
    T g[Q];
    auto pull = [&](int x, int y, int z, unsigned) {
        const Nb n = neighbours(p, x, y, z);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            g[i] = p.g_in[i * (unsigned)p.vol + n.at(-c_ex(i), -c_ey(i), -c_ez(i))];  // x - e_i
    };
    march<T, 1, 1, R_LB>(p, src, pull, [&](int x, int y, int z, unsigned s, const auto &pl) {
        T Fx, Fy, Fz;
        {
            V2<T> v[Q], gx, gy, gz;
            gather_pair(pl, 0, v);
            grad3(v, gx, gy, gz);
            T C[Q], gcx, gcy, gcz;
            gather_one(pl, 0, C);
            grad3(C, gcx, gcy, gcz);
            const T ph = p.phi[s], c = C[0];
            // psi grad mu_psi = grad psi + psi grad m; (fx, fy, fz) is zero without a body force
            Fx = -ph * gx.x - (gcx + c * gx.y) + p.fx;
            Fy = -ph * gy.x - (gcy + c * gy.y) + p.fy;
            Fz = -ph * gz.x - (gcz + c * gz.y) + p.fz;
        }
        T dn = 0, jx = 0, jy = 0, jz = 0;
        static_for<0, Q>([&](auto k) {
            constexpr int i = decltype(k)::value;
            dn += g[i];
            jx = acc_e<c_ex(i)>(jx, g[i]);
            jy = acc_e<c_ey(i)>(jy, g[i]);
            jz = acc_e<c_ez(i)>(jz, g[i]);
        });
        const T rho = T(1) + dn;
        const T ux = (jx + T(0.5) * Fx) / rho, uy = (jy + T(0.5) * Fy) / rho,
                uz = (jz + T(0.5) * Fz) / rho;
        if (FIELDS) {
            const long long N = (long long)p.nx * p.ny * p.nz;
            const long long d = ((long long)z * p.ny + y) * p.nx + x;
            out[d] = (double)rho;
            out[N + d] = (double)ux;
            out[2 * N + d] = (double)uy;
            out[3 * N + d] = (double)uz;
            return;
        }
        const T usq = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
        static_for<0, Q>([&](auto k) {
            constexpr int i = decltype(k)::value;
            const T w = (T)wq(i);
            const T eu = acc_e<c_ez(i)>(acc_e<c_ey(i)>(mul_e<c_ex(i)>(ux), uy), uz);
            const T eF = acc_e<c_ez(i)>(acc_e<c_ey(i)>(mul_e<c_ex(i)>(Fx), Fy), Fz);
            const T geq = w * (dn + rho * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * usq));
            const T Fi = p.guo * w * (T(3) * (eF - uF) + T(9) * eu * eF);
            p.g_out[i * (unsigned)p.vol + s] = g[i] - p.omega * (g[i] - geq) + Fi;
        });
        p.ux[s] = p.frozen ? p.ux0 : ux;
        p.uy[s] = p.frozen ? p.uy0 : uy;
        p.uz[s] = p.frozen ? p.uz0 : uz;
    });
}

// phi*, psi* (Eqs. 16-17): g* = g - sum over the 6 faces of the outgoing flux
// u_f g_upwind, u_f the mean of the two sites' normal velocities.
// Ring: the pair (phi, psi), ux, uy, uz.
template <typename T>
__global__ void __launch_bounds__(NT) k_advect(const Arg3<T> p) {
    constexpr int ROWS = R_ADVECT;
    const T *const src[5] = {p.phi, p.psi, p.ux, p.uy, p.uz};
    march<T, 1, 3, ROWS>(p, src, [](int, int, int, unsigned) {}, [=](int, int, int, unsigned s, const auto &pl) {
        T netp = 0, netc = 0;
        const V2<T> c0 = pl.pair(0, 0, 0, 0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ex = a == 0, ey = a == 1, ez = a == 2;
            const T Us = pl.one(a, 0, 0, 0);
            const T fp = T(0.5) * (Us + pl.one(a, ex, ey, ez)),
                    fm = T(0.5) * (pl.one(a, -ex, -ey, -ez) + Us);
            const V2<T> up = fp > T(0) ? c0 : pl.pair(0, ex, ey, ez);
            const V2<T> dn = fm > T(0) ? pl.pair(0, -ex, -ey, -ez) : c0;
            netp += fp * up.x - fm * dn.x;
            netc += fp * up.y - fm * dn.y;
        }
        p.phs[s] = c0.x - netp;
        p.pss[s] = c0.y - netc;
    });
}

// mu*, m* from phi*, psi* (Eqs. 3, 5), the cubic from phi^n (Eq. 18); ring: the
// pair (phi*, psi*), z-window form
template <typename T>
__global__ void __launch_bounds__(NT) k_chem2(const Arg3<T> p) {
    const T *const src[2] = {p.phs, p.pss};
    ZWin<V2<T>, true, true> w;
    w.reset();
    T pn = 0;
    march_zw<T, 1, 0>(p, src, [&](int, int, int, unsigned s) { pn = p.phi[s]; },
                      [&](const ZNb<T> &nb, bool out, int, int, int, unsigned s) {
        V2<T> gx, gy, gz, lap, mid;
        w.arrive([&](int ex, int ey) { return nb.pair(0, ex, ey); }, out, gx, gy, gz, lap, mid);
        if (out) {
            p.mus[s] = p.a * mid.x + p.b * (pn * pn * pn) - (p.B0 + p.B1 * mid.y) * lap.x -
                       p.B1 * (gx.x * gx.y + gy.x * gy.y + gz.x * gz.y);
            p.mms[s] = T(0.5) * p.B1 * (gx.x * gx.x + gy.x * gy.x + gz.x * gz.x);
        }
    });
}

// phi^{n+1} = phi* + M lap mu* (Eq. 18); psi^{n+1} = psi* + D sum_j 6 w_j
// [(psi*_j - psi*) + (psi* + psi*_j)(m*_j - m*)/2] - gamma (psi* - c0) + A Theta
// (Eq. 19).  With L the D3Q19 Laplacian and p* = psi* m*, the link sum is
// L psi* + (psi* L m* + L p* - m* L psi*) / 2, so that every neighbour term is a
// linear stencil: z-window form on the pairs (psi*, m*) and (mu*, p*), p* formed
// from each neighbour's psi* and m*.  Ring: the pair (psi*, m*) and mu*.
template <typename T>
__global__ void __launch_bounds__(NT) k_update(const Arg3<T> p) {
    const T *const src[3] = {p.pss, p.mms, p.mus};
    ZWin<V2<T>, false, true> wpm, wup;
    wpm.reset();
    wup.reset();
    T phs = 0;
    uint32_t word = 0;
    const int words = (p.nx + 31) / 32;
    march_zw<T, 1, 1>(p, src, [&](int x, int y, int z, unsigned s) {
        phs = p.phs[s];
        word = p.theta[((long long)z * p.ny + y) * words + (x >> 5)];
    }, [&](const ZNb<T> &nb, bool out, int x, int, int, unsigned s) {
        V2<T> g, lpm, lup, mpm, mup;
        wpm.arrive([&](int ex, int ey) { return nb.pair(0, ex, ey); }, out, g, g, g, lpm, mpm);
        wup.arrive([&](int ex, int ey) {
            const V2<T> q = nb.pair(0, ex, ey);
            V2<T> r;
            r.x = nb.one(0, ex, ey);
            r.y = q.x * q.y;
            return r;
        }, out, g, g, g, lup, mup);
        if (out) {
            p.phi_o[s] = phs + p.M * lup.x;
            const T C0 = mpm.x, m0 = mpm.y;
            const T div = lpm.x + T(0.5) * ((C0 * lpm.y + lup.y) - m0 * lpm.x);
            const bool bit = (word >> (x & 31)) & 1u;
            p.psi_o[s] = C0 + (p.D * div - p.gamma * (C0 - p.c0) + (bit ? p.A : T(0)));
        }
    });
}

// ------------------------------------------------------------ utility kernels

struct Geo3 {
    int nx, ny, nz;
    long long pitch, plane, vol;
};

__device__ inline void coords(const Geo3 &G, long long d, int &x, int &y, int &z) {
    const long long r = d / G.nx;
    x = (int)(d - r * G.nx);
    y = (int)(r % G.ny);
    z = (int)(r / G.ny);
}

__device__ inline int pw(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The first invalid site of an upload (dense doubles rho, ux, uy, uz, phi, psi at
// d, N + d, ..., 5N + d), in index order, as 4 d + reason: 1 a non-finite value,
// 2 psi <= 0 or B(psi) = B0 + B1 psi <= 0, 3 rho <= 0.  *first must hold all
// bits set on entry.
__global__ void k_check(long long N, const double *in, double B0, double B1,
                        unsigned long long *first) {
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < N;
         d += (long long)gridDim.x * blockDim.x) {
        const double n = in[d], ps = in[5 * N + d];
        unsigned code = 0;
        if (!isfinite(n) || !isfinite(in[N + d]) || !isfinite(in[2 * N + d]) ||
            !isfinite(in[3 * N + d]) || !isfinite(in[4 * N + d]) || !isfinite(ps))
            code = 1;
        else if (!(ps > 0.0) || !(__dadd_rn(B0, __dmul_rn(B1, ps)) > 0.0))
            code = 2;
        else if (!(n > 0.0))
            code = 3;
        if (code) atomicMin(first, (unsigned long long)d * 4ull + code);
    }
}

__global__ void k_fill(long long n, double v, double *a) {
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < n;
         d += (long long)gridDim.x * blockDim.x)
        a[d] = v;
}

// f_i = f_i^eq(rho, u) (Eq. 12) in the pull layout: buffer_i(x) holds the value
// site x + e_i reads, f_i^eq at x + e_i; phi, psi copied.  Inputs: dense doubles
// rho, ux, uy, uz, phi, psi at d, N + d, ..., 5N + d.
// Nothing is written unless *bad holds no invalid site (all bits set).
template <typename T>
__global__ void k_init(const Geo3 G, const double *in, const unsigned long long *bad, T *g, T *phi,
                       T *psi) {
    if (*bad != ~0ull) return;
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < N;
         d += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(G, d, x, y, z);
        const long long s = (long long)z * G.plane + (long long)y * G.pitch + x;
        phi[s] = (T)in[4 * N + d];
        psi[s] = (T)in[5 * N + d];
        for (int i = 0; i < Q; ++i) {
            const int xs = pw(x + c_ex(i), G.nx), ys = pw(y + c_ey(i), G.ny), zs = pw(z + c_ez(i), G.nz);
            const long long q = ((long long)zs * G.ny + ys) * G.nx + xs;
            const double n = in[q], u = in[N + q], v = in[2 * N + q], w = in[3 * N + q];
            const double eu = c_ex(i) * u + c_ey(i) * v + c_ez(i) * w, usq = u * u + v * v + w * w;
            g[i * G.vol + s] = (T)(wq(i) * ((n - 1.0) + n * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq)));
        }
    }
}

// pre-collision f_i(x) = w_i + buffer_i(x - e_i), and phi, psi, as dense doubles
template <typename T>
__global__ void k_pops(const Geo3 G, const T *g, double *f) {
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < N;
         d += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(G, d, x, y, z);
        for (int i = 0; i < Q; ++i) {
            const long long s = (long long)pw(z - c_ez(i), G.nz) * G.plane +
                                (long long)pw(y - c_ey(i), G.ny) * G.pitch + pw(x - c_ex(i), G.nx);
            f[i * N + d] = wq(i) + (double)g[i * G.vol + s];
        }
    }
}

template <typename T>
__global__ void k_dense(const Geo3 G, const T *phi, const T *psi, double *out_phi, double *out_psi) {
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < N;
         d += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(G, d, x, y, z);
        const long long s = (long long)z * G.plane + (long long)y * G.pitch + x;
        out_phi[d] = (double)phi[s];
        out_psi[d] = (double)psi[s];
    }
}

struct Balls {
    lbd3_source s[LBD_MAX_SOURCES];
};

// Theta of the source balls, one bit per site: inclusive, periodic minimum
// image, union; the test in double without contraction into FMAs.
__global__ void k_theta(const Geo3 G, int n_src, Balls b, uint32_t *mask) {
    const int words = (G.nx + 31) / 32;
    const long long total = (long long)words * G.ny * G.nz;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const long long r = w / words;
        const int y = (int)(r % G.ny), z = (int)(r / G.ny), x0 = (int)(w - r * words) * 32;
        uint32_t bits = 0;
        for (int k = 0; k < 32 && x0 + k < G.nx; ++k)
            for (int j = 0; j < n_src; ++j) {
                double d[3] = {(double)(x0 + k) - b.s[j].x, (double)y - b.s[j].y,
                               (double)z - b.s[j].z};
                const int L[3] = {G.nx, G.ny, G.nz};
                for (int a = 0; a < 3; ++a) {
                    if (d[a] > 0.5 * L[a]) d[a] -= L[a];
                    else if (d[a] < -0.5 * L[a]) d[a] += L[a];
                }
                const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                            __dmul_rn(d[2], d[2]));
                if (r2 <= __dmul_rn(b.s[j].R, b.s[j].R)) {
                    bits |= 1u << k;
                    break;
                }
            }
        mask[w] = bits;
    }
}

constexpr int NRED3 = 8;  // sum g, sum phi, sum psi, phi dx, phi dy, phi dz, phi, nonfinite
constexpr int RED3_BLOCKS = 608, RED3_THREADS = 256;

// Per-block sums over a fixed set of sites (block b: sites b, b + B, ...), tree
// reduced in shared memory: the result does not depend on scheduling.
template <typename T>
__global__ void k_red(const Geo3 G, const T *g, const T *phi, const T *psi, double rx, double ry,
                      double rz, double *partial) {
    __shared__ double sh[NRED3][RED3_THREADS];
    double v[NRED3] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long N = (long long)G.nx * G.ny * G.nz;
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < N;
         d += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(G, d, x, y, z);
        const long long s = (long long)z * G.plane + (long long)y * G.pitch + x;
        double dn = 0;
        for (int i = 0; i < Q; ++i) dn += (double)g[i * G.vol + s];
        const double ph = (double)phi[s], c = (double)psi[s];
        v[0] += dn;
        v[1] += ph;
        v[2] += c;
        if (!isfinite(dn) || !isfinite(ph) || !isfinite(c)) v[7] += 1;
        if (ph >= 0) {
            double e[3] = {x - rx, y - ry, z - rz};
            const int L[3] = {G.nx, G.ny, G.nz};
            for (int a = 0; a < 3; ++a) {
                if (e[a] >= 0.5 * L[a]) e[a] -= L[a];
                else if (e[a] < -0.5 * L[a]) e[a] += L[a];
            }
            v[3] += ph * e[0];
            v[4] += ph * e[1];
            v[5] += ph * e[2];
            v[6] += ph;
        }
    }
    for (int k = 0; k < NRED3; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int h = RED3_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int k = 0; k < NRED3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NRED3; ++k) partial[k * gridDim.x + blockIdx.x] = sh[k][0];
}

__global__ void k_red_final(int nb, const double *partial, double *out) {
    const int k = threadIdx.x;
    if (k >= NRED3) return;
    double a = 0;
    for (int b = 0; b < nb; ++b) a += partial[k * nb + b];
    out[k] = a;
}

}  // namespace

// ---------------------------------------------------------------- host side

struct lbd3_ctx {
    int dev = 0;
    lbd3_grid grid{};
    lbd3_params params{};
    cudaStream_t stream = nullptr;
    long long pitch = 0, plane = 0, vol = 0, N = 0;
    size_t esz = 0;
    void *g[2] = {nullptr, nullptr}, *phi[2] = {nullptr, nullptr}, *psi[2] = {nullptr, nullptr};
    void *work = nullptr;            // mu, m, ux, uy, uz, phi*, psi*, mu*, m* (9 fields)
    uint32_t *theta = nullptr;
    double *staging = nullptr;       // 6N dense doubles
    double *pop_staging = nullptr;   // 19N, on demand
    double *red = nullptr;           // NRED3 * RED3_BLOCKS partials + NRED3 results
    int zl = 0;                      // planes per CTA of the marching kernels
    int sms = 1;
    int cur = 0;
    int64_t t = 0;
    int sticky = 0;
    std::string msg;
};

namespace {

int fail3(lbd3_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->msg = buf;
        if (code == LBD_ECUDA) c->sticky = LBD_ECUDA;
    }
    return code;
}

#define CK3(ctx, call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail3(ctx, LBD_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                         __FILE__, __LINE__);                                               \
    } while (0)

int check3(lbd3_ctx *c, const lbd3_params *q) {
    if (!q) return fail3(c, LBD_EINVAL, "params is NULL");
    const lbd_params &p = q->base;
    if (!(p.tau > 0.5)) return fail3(c, LBD_EINVAL, "tau must be > 1/2");
    if (!(p.b >= 0.0)) return fail3(c, LBD_EINVAL, "b must be >= 0");
    const double vals[] = {p.a, p.b, p.B0, p.B1, p.M, p.D, p.tau, p.gamma, p.c0, p.A0, p.A_max,
                           p.fx, p.fy, p.ux0, p.uy0, q->fz, q->uz0};
    for (double v : vals)
        if (!std::isfinite(v)) return fail3(c, LBD_EINVAL, "non-finite parameter");
    if (p.precision != LBD_FP64 && p.precision != LBD_FP32)
        return fail3(c, LBD_EINVAL, "precision must be LBD_FP64 or LBD_FP32");
    if (p.flags & ~(LBD_FROZEN_U | LBD_BODY_FORCE))
        return fail3(c, LBD_EINVAL, "unknown or unsupported flags (3D has no walls)");
    if (q->n_src < 0 || q->n_src > LBD_MAX_SOURCES)
        return fail3(c, LBD_EINVAL, "n_src must be in [0, %d]", LBD_MAX_SOURCES);
    for (int k = 0; k < q->n_src; ++k) {
        const lbd3_source &b = q->src[k];
        if (!std::isfinite(b.x) || !std::isfinite(b.y) || !std::isfinite(b.z) || !(b.R >= 0.0))
            return fail3(c, LBD_EINVAL, "bad source %d", k);
    }
    return LBD_OK;
}

int theta3(lbd3_ctx *c) {
    Balls b;
    const lbd3_params &q = c->params;
    const double L[3] = {(double)c->grid.nx, (double)c->grid.ny, (double)c->grid.nz};
    for (int k = 0; k < q.n_src; ++k) {
        double v[3] = {q.src[k].x, q.src[k].y, q.src[k].z};
        for (int a = 0; a < 3; ++a) {
            v[a] = std::fmod(v[a], L[a]);
            if (v[a] < 0) v[a] += L[a];
        }
        b.s[k] = lbd3_source{v[0], v[1], v[2], q.src[k].R};
    }
    const Geo3 G{c->grid.nx, c->grid.ny, c->grid.nz, c->pitch, c->plane, c->vol};
    k_theta<<<1024, 256, 0, c->stream>>>(G, q.n_src, b, c->theta);
    CK3(c, cudaGetLastError());
    return LBD_OK;
}

Geo3 geo(const lbd3_ctx *c) {
    return Geo3{c->grid.nx, c->grid.ny, c->grid.nz, c->pitch, c->plane, c->vol};
}

template <typename T>
Arg3<T> args3(const lbd3_ctx *c) {
    Arg3<T> a;
    memset(&a, 0, sizeof a);
    a.nx = c->grid.nx;
    a.ny = c->grid.ny;
    a.nz = c->grid.nz;
    a.zl = c->zl;
    a.pitch = c->pitch;
    a.plane = c->plane;
    a.vol = c->vol;
    a.g_in = (const T *)c->g[c->cur];
    a.g_out = (T *)c->g[1 - c->cur];
    a.phi = (const T *)c->phi[c->cur];
    a.psi = (const T *)c->psi[c->cur];
    a.phi_o = (T *)c->phi[1 - c->cur];
    a.psi_o = (T *)c->psi[1 - c->cur];
    T *w = (T *)c->work;
    T **f[9] = {&a.mu, &a.mm, &a.ux, &a.uy, &a.uz, &a.phs, &a.pss, &a.mus, &a.mms};
    for (int k = 0; k < 9; ++k) *f[k] = w + k * c->vol;
    a.theta = c->theta;
    const lbd_params &p = c->params.base;
    a.a = (T)p.a;
    a.b = (T)p.b;
    a.B0 = (T)p.B0;
    a.B1 = (T)p.B1;
    a.M = (T)p.M;
    a.D = (T)p.D;
    a.omega = (T)(1.0 / p.tau);
    a.guo = (T)(1.0 - 0.5 / p.tau);
    a.c0 = (T)p.c0;
    double A = 0, gm = 0;
    if (c->t >= p.t_on) {
        A = p.A0 * (double)(c->t - p.t_on);
        A = A < p.A_max ? A : p.A_max;
        gm = p.gamma;
    }
    a.A = (T)A;
    a.gamma = (T)gm;
    const bool body = (p.flags & LBD_BODY_FORCE) != 0;
    a.fx = body ? (T)p.fx : T(0);
    a.fy = body ? (T)p.fy : T(0);
    a.fz = body ? (T)c->params.fz : T(0);
    a.frozen = (p.flags & LBD_FROZEN_U) ? 1 : 0;
    a.ux0 = (T)p.ux0;
    a.uy0 = (T)p.uy0;
    a.uz0 = (T)c->params.uz0;
    return a;
}

// Planes per CTA of the marching kernels: enough CTAs for about sixteen per SM
// over the whole lattice, runs of at least four planes.
int auto_zrun(const lbd3_grid &g, int sms) {
    const long long tiles = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    long long runs = (16LL * sms + tiles - 1) / tiles;
    const long long most = (g.nz + 3) / 4;
    runs = runs < 1 ? 1 : (runs > most ? most : runs);
    return (int)((g.nz + runs - 1) / runs);
}

template <int RY, typename T>
dim3 march_grid(const Arg3<T> &a) {
    return dim3((a.nx + TX - 1) / TX, (a.ny + Tile<RY>::H - 1) / Tile<RY>::H,
                (a.nz + a.zl - 1) / a.zl);
}

template <typename T>
cudaError_t launch_step3(const Arg3<T> &a, cudaStream_t s) {
    const size_t e = sizeof(T);
    k_chem<T><<<march_grid<1>(a), NT, zring_bytes<1, 0>(e), s>>>(a);
    k_lb<T, 0><<<march_grid<R_LB>(a), NT, ring_bytes<1, 1, R_LB>(e), s>>>(a, nullptr);
    k_advect<T><<<march_grid<R_ADVECT>(a), NT, ring_bytes<1, 3, R_ADVECT>(e), s>>>(a);
    k_chem2<T><<<march_grid<1>(a), NT, zring_bytes<1, 0>(e), s>>>(a);
    k_update<T><<<march_grid<1>(a), NT, zring_bytes<1, 1>(e), s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fields3(const Arg3<T> &a, const Geo3 &G, double *out, cudaStream_t s) {
    const size_t e = sizeof(T);
    const long long N = (long long)a.nx * a.ny * a.nz;
    k_chem<T><<<march_grid<1>(a), NT, zring_bytes<1, 0>(e), s>>>(a);
    k_lb<T, 1><<<march_grid<R_LB>(a), NT, ring_bytes<1, 1, R_LB>(e), s>>>(a, out);
    k_dense<T><<<1024, 256, 0, s>>>(G, a.phi, a.psi, out + 4 * N, out + 5 * N);
    return cudaGetLastError();
}

// Rings above the default 48 KB of dynamic shared memory (the FP64 ones).
template <typename T>
cudaError_t ring_limits() {
    const size_t e = sizeof(T);
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t r = cudaFuncSetAttribute(k_chem<T>, A, (int)zring_bytes<1, 0>(e));
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_lb<T, 0>, A, (int)ring_bytes<1, 1, R_LB>(e));
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_lb<T, 1>, A, (int)ring_bytes<1, 1, R_LB>(e));
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_advect<T>, A, (int)ring_bytes<1, 3, R_ADVECT>(e));
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_chem2<T>, A, (int)zring_bytes<1, 0>(e));
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_update<T>, A, (int)zring_bytes<1, 1>(e));
    return r;
}

int ensure_staging3(lbd3_ctx *c) {
    if (c->staging) return LBD_OK;
    // six fields of doubles, then the first-invalid-site word of an upload
    if (lbd::dev_malloc((void **)&c->staging, sizeof(double) * (6 * c->N + 1)) != cudaSuccess) {
        cudaGetLastError();
        c->staging = nullptr;
        return fail3(c, LBD_ENOMEM, "staging allocation failed");
    }
    return LBD_OK;
}

}  // namespace

extern "C" {

const char *lbd3_last_error(const lbd3_ctx *c) { return c ? c->msg.c_str() : "null context"; }

void lbd3_destroy(lbd3_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->g[k]);
        cudaFree(c->phi[k]);
        cudaFree(c->psi[k]);
    }
    cudaFree(c->work);
    cudaFree(c->theta);
    cudaFree(c->staging);
    cudaFree(c->pop_staging);
    cudaFree(c->red);
    cudaGetLastError();
    delete c;
}

int lbd3_create(const lbd3_grid *grid, const lbd3_params *params, void *stream, lbd3_ctx **out) {
    if (!grid || !params || !out) return LBD_EINVAL;
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->nx > 4096 || grid->ny > 4096 ||
        grid->nz > 4096 || (long long)grid->nx * grid->ny * grid->nz > (1LL << 31))
        return LBD_EINVAL;
    {   // the kernels index the 19 population planes with 32-bit offsets
        const long long al = 128 / (params->base.precision == LBD_FP64 ? 8 : 4);
        const long long vol = (grid->nx + al - 1) / al * al * grid->ny * grid->nz;
        if (19 * vol >= (1LL << 32)) return LBD_EINVAL;
    }
    if (check3(nullptr, params) != LBD_OK) return LBD_EINVAL;
    lbd3_ctx *c = new (std::nothrow) lbd3_ctx();
    if (!c) return LBD_ENOMEM;
    c->grid = *grid;
    c->params = *params;
    c->stream = (cudaStream_t)stream;
    c->esz = params->base.precision == LBD_FP64 ? sizeof(double) : sizeof(float);
    const long long align = 128 / (long long)c->esz;
    c->pitch = (grid->nx + align - 1) / align * align;
    c->plane = c->pitch * grid->ny;
    c->vol = c->plane * grid->nz;
    c->N = (long long)grid->nx * grid->ny * grid->nz;
    int sms = 0;
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess ||
        (c->esz == sizeof(double) ? ring_limits<double>() : ring_limits<float>()) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LBD_ECUDA;
    }
    c->sms = sms;
    c->zl = auto_zrun(c->grid, sms);
    const size_t fb = (size_t)c->vol * c->esz;
    const size_t words = (size_t)((grid->nx + 31) / 32) * grid->ny * grid->nz;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok &= lbd::dev_malloc((void **)&c->g[k], (size_t)Q * fb) == cudaSuccess;
        ok &= ok && lbd::dev_malloc((void **)&c->phi[k], fb) == cudaSuccess;
        ok &= ok && lbd::dev_malloc((void **)&c->psi[k], fb) == cudaSuccess;
    }
    ok &= ok && lbd::dev_malloc((void **)&c->work, 9 * fb) == cudaSuccess;
    ok &= ok && lbd::dev_malloc((void **)&c->theta, 4 * words) == cudaSuccess;
    ok &= ok && lbd::dev_malloc((void **)&c->red, sizeof(double) * NRED3 * (RED3_BLOCKS + 1)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbd3_destroy(c);
        return LBD_ENOMEM;
    }
    // rest state; the work fields are zeroed so that padding columns stay finite
    for (int k = 0; k < 2; ++k)
        ok &= cudaMemsetAsync(c->g[k], 0, Q * fb, c->stream) == cudaSuccess &&
              cudaMemsetAsync(c->phi[k], 0, fb, c->stream) == cudaSuccess &&
              cudaMemsetAsync(c->psi[k], 0, fb, c->stream) == cudaSuccess;
    ok &= cudaMemsetAsync(c->work, 0, 9 * fb, c->stream) == cudaSuccess;
    if (!ok || theta3(c) != LBD_OK || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        lbd3_destroy(c);
        return LBD_ECUDA;
    }
    *out = c;
    return LBD_OK;
}

int lbd3_set_params(lbd3_ctx *c, const lbd3_params *p) {
    if (!c) return LBD_EINVAL;
    int rc = check3(c, p);
    if (rc != LBD_OK) return rc;
    if (p->base.precision != c->params.base.precision)
        return fail3(c, LBD_EINVAL, "precision cannot change after creation");
    c->params = *p;
    CK3(c, cudaSetDevice(c->dev));
    return theta3(c);
}

int lbd3_set_fields(lbd3_ctx *c, const double *rho, const double *ux, const double *uy,
                    const double *uz, const double *phi, const double *psi) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (!phi || !psi) return fail3(c, LBD_EINVAL, "phi and psi are required");
    const long long N = c->N;
    const lbd_params &p = c->params.base;
    int rc = ensure_staging3(c);
    if (rc != LBD_OK) return rc;
    CK3(c, cudaSetDevice(c->dev));
    // upload into the staging area, validate there, and build the state only if
    // every site is valid (the state is left as it was otherwise)
    double *d = c->staging;
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(d + 6 * N);
    const size_t B = sizeof(double) * N;
    CK3(c, cudaMemsetAsync(bad, 0xFF, sizeof *bad, c->stream));
    if (rho) CK3(c, cudaMemcpyAsync(d, rho, B, cudaMemcpyHostToDevice, c->stream));
    else k_fill<<<1024, 256, 0, c->stream>>>(N, 1.0, d);
    const double *u[3] = {ux, uy, uz};
    for (int k = 0; k < 3; ++k)
        if (u[k]) CK3(c, cudaMemcpyAsync(d + (k + 1) * N, u[k], B, cudaMemcpyHostToDevice, c->stream));
        else CK3(c, cudaMemsetAsync(d + (k + 1) * N, 0, B, c->stream));
    CK3(c, cudaMemcpyAsync(d + 4 * N, phi, B, cudaMemcpyHostToDevice, c->stream));
    CK3(c, cudaMemcpyAsync(d + 5 * N, psi, B, cudaMemcpyHostToDevice, c->stream));
    k_check<<<1024, 256, 0, c->stream>>>(N, d, p.B0, p.B1, bad);
    CK3(c, cudaGetLastError());
    const Geo3 G = geo(c);
    if (p.precision == LBD_FP64)
        k_init<double><<<1024, 256, 0, c->stream>>>(G, d, bad, (double *)c->g[c->cur],
                                                    (double *)c->phi[c->cur], (double *)c->psi[c->cur]);
    else
        k_init<float><<<1024, 256, 0, c->stream>>>(G, d, bad, (float *)c->g[c->cur],
                                                   (float *)c->phi[c->cur], (float *)c->psi[c->cur]);
    CK3(c, cudaGetLastError());
    unsigned long long first = 0;
    CK3(c, cudaMemcpyAsync(&first, bad, sizeof first, cudaMemcpyDeviceToHost, c->stream));
    CK3(c, cudaStreamSynchronize(c->stream));
    if (first != ~0ull) {
        const long long site = (long long)(first >> 2);
        switch ((int)(first & 3ull)) {
            case 1: return fail3(c, LBD_ENONFINITE, "non-finite value at site %lld", site);
            case 2: return fail3(c, LBD_EUNSTABLE, "B(psi) <= 0 or psi <= 0 at site %lld", site);
            default: return fail3(c, LBD_EINVAL, "rho <= 0 at site %lld", site);
        }
    }
    return LBD_OK;
}

int lbd3_step(lbd3_ctx *c, int64_t n) {
    if (!c || n < 0) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK3(c, cudaSetDevice(c->dev));
    for (int64_t k = 0; k < n; ++k) {
        if (c->params.base.precision == LBD_FP64)
            CK3(c, launch_step3<double>(args3<double>(c), c->stream));
        else
            CK3(c, launch_step3<float>(args3<float>(c), c->stream));
        c->cur = 1 - c->cur;
        c->t += 1;
    }
    return LBD_OK;
}

int lbd3_get_fields(lbd3_ctx *c, double *rho, double *ux, double *uy, double *uz, double *phi,
                    double *psi) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    int rc = ensure_staging3(c);
    if (rc != LBD_OK) return rc;
    CK3(c, cudaSetDevice(c->dev));
    const Geo3 G = geo(c);
    if (c->params.base.precision == LBD_FP64)
        CK3(c, launch_fields3<double>(args3<double>(c), G, c->staging, c->stream));
    else
        CK3(c, launch_fields3<float>(args3<float>(c), G, c->staging, c->stream));
    double *outs[6] = {rho, ux, uy, uz, phi, psi};
    for (int k = 0; k < 6; ++k)
        if (outs[k])
            CK3(c, cudaMemcpyAsync(outs[k], c->staging + k * c->N, sizeof(double) * c->N,
                                   cudaMemcpyDeviceToHost, c->stream));
    CK3(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}

int lbd3_get_populations(lbd3_ctx *c, double *f) {
    if (!c || !f) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK3(c, cudaSetDevice(c->dev));
    if (!c->pop_staging && lbd::dev_malloc((void **)&c->pop_staging, sizeof(double) * Q * c->N) != cudaSuccess) {
        cudaGetLastError();
        c->pop_staging = nullptr;
        return fail3(c, LBD_ENOMEM, "population staging allocation failed");
    }
    const Geo3 G = geo(c);
    if (c->params.base.precision == LBD_FP64)
        k_pops<double><<<1024, 256, 0, c->stream>>>(G, (const double *)c->g[c->cur], c->pop_staging);
    else
        k_pops<float><<<1024, 256, 0, c->stream>>>(G, (const float *)c->g[c->cur], c->pop_staging);
    CK3(c, cudaGetLastError());
    CK3(c, cudaMemcpyAsync(f, c->pop_staging, sizeof(double) * Q * c->N, cudaMemcpyDeviceToHost,
                           c->stream));
    CK3(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}

int lbd3_diagnostics(lbd3_ctx *c, double rx, double ry, double rz, lbd3_diag *out) {
    if (!c || !out) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (!(rx >= 0 && rx < c->grid.nx && ry >= 0 && ry < c->grid.ny && rz >= 0 && rz < c->grid.nz))
        return fail3(c, LBD_EINVAL, "reference point outside the lattice");
    CK3(c, cudaSetDevice(c->dev));
    const Geo3 G = geo(c);
    if (c->params.base.precision == LBD_FP64)
        k_red<double><<<RED3_BLOCKS, RED3_THREADS, 0, c->stream>>>(
            G, (const double *)c->g[c->cur], (const double *)c->phi[c->cur],
            (const double *)c->psi[c->cur], rx, ry, rz, c->red);
    else
        k_red<float><<<RED3_BLOCKS, RED3_THREADS, 0, c->stream>>>(
            G, (const float *)c->g[c->cur], (const float *)c->phi[c->cur],
            (const float *)c->psi[c->cur], rx, ry, rz, c->red);
    CK3(c, cudaGetLastError());
    k_red_final<<<1, 32, 0, c->stream>>>(RED3_BLOCKS, c->red, c->red + NRED3 * RED3_BLOCKS);
    CK3(c, cudaGetLastError());
    double h[NRED3];
    CK3(c, cudaMemcpyAsync(h, c->red + NRED3 * RED3_BLOCKS, sizeof h, cudaMemcpyDeviceToHost,
                           c->stream));
    CK3(c, cudaStreamSynchronize(c->stream));
    out->sum_rho = (double)c->N + h[0];
    out->sum_phi = h[1];
    out->sum_psi = h[2];
    out->mass_pos = h[6];
    out->cm_x = h[6] > 0 ? rx + h[3] / h[6] : NAN;
    out->cm_y = h[6] > 0 ? ry + h[4] / h[6] : NAN;
    out->cm_z = h[6] > 0 ? rz + h[5] / h[6] : NAN;
    out->nonfinite = (int64_t)h[7];
    return LBD_OK;
}

int lbd3_synchronize(lbd3_ctx *c) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK3(c, cudaSetDevice(c->dev));
    CK3(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}

int lbd3_get_time(const lbd3_ctx *c, int64_t *t) {
    if (!c || !t) return LBD_EINVAL;
    *t = c->t;
    return LBD_OK;
}

int lbd3_set_zrun(lbd3_ctx *c, int32_t planes) {
    if (!c) return LBD_EINVAL;
    if (planes < 0 || planes > c->grid.nz)
        return fail3(c, LBD_EINVAL, "planes must be in [0, nz]");
    c->zl = planes ? planes : auto_zrun(c->grid, c->sms);
    return LBD_OK;
}

int lbd3_get_zrun(const lbd3_ctx *c, int32_t *planes) {
    if (!c || !planes) return LBD_EINVAL;
    *planes = c->zl;
    return LBD_OK;
}

}  // extern "C"

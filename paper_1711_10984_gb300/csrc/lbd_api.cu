// lbd_api.cu -- the C ABI of include/lbd.h: context management, state upload,
// field read-back, populations, and the FP64 diagnostic reductions.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "lbd_internal.h"

using lbd::StepArgs;
using lbd::Tile;

namespace {

constexpr int NRED = 9;      // reduction slots, see reduce_partial
constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int RED32_BLOCKS = 456;  // FP32 reduction: 3 resident blocks on each of 152 SMs

}  // namespace

struct lbd_ctx {
    int dev = 0;
    lbd_grid grid{};
    lbd_params params{};
    cudaStream_t stream = nullptr;
    long long pitch = 0, plane = 0;
    size_t N = 0, esz = 0;
    void *g[2] = {nullptr, nullptr};
    void *phi[2] = {nullptr, nullptr};
    void *psi[2] = {nullptr, nullptr};
    int cur = 0;
    double *staging = nullptr;   // dense doubles, 5*N
    float *staging32 = nullptr;  // dense floats, 5*N (FP32 host I/O, on demand)
    // a second stream and two events (on demand): lbd_get_fields_f32 reads phi
    // and psi back on it while rho and u are evaluated on the context's stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_main = nullptr, ev_side = nullptr;
    unsigned long long *word = nullptr;  // verdict of a float rest-state upload (on demand)
    double *pop_staging = nullptr;  // dense doubles, 9*N (on demand)
    double *red_partial = nullptr, *red_out = nullptr, *h_red = nullptr;
    uint32_t *theta = nullptr;      // source indicator, one bit per site
    double *drop_dev = nullptr;     // droplet sums: block partials, results, references
    double *h_drop = nullptr;       // pinned: results and references
    int64_t t = 0;
    Tile tile{118, 64};
    int sticky = 0;
    std::string msg;
    // Run-time checks (lbd_set_check): every `check_every` steps lbd_step queues
    // the diagnostics reduction into one of NCHECK result slots (device result,
    // pinned host copy, completion event) without a host synchronisation; the
    // verdicts are read as the slots complete.  `flagged` holds the first
    // failure found (LBD_ENONFINITE or LBD_EUNSTABLE) until the state is reset.
    static constexpr int NCHECK = 4;
    int64_t check_every = 0;
    struct CheckSlot {
        double *d = nullptr, *h = nullptr;
        cudaEvent_t ev = nullptr;
        int64_t t = 0;
        bool pending = false;
    } chk[NCHECK];
    int chk_next = 0;
    int flagged = 0;
};


struct lbd_batch {
    int n = 0;
    std::vector<lbd_ctx *> ctx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int prec = LBD_FP32;
    void *args_dev[2] = {nullptr, nullptr};  // StepArgs<T>[n] for buffer parity 0 / 1
    lbd::BatchItem *items_dev = nullptr;  // periodic instances' items, then those with plates
    int n_items = 0;
    int n_plain = 0;                       // items of periodic instances
    int ctas_walls = 1;
    long long *t_dev = nullptr;
    Tile tile{118, 64};
    int ctas = 1;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps = 100;
    int64_t t = 0;
    int sticky = 0;
    std::string msg;
};

namespace {

int bfail(lbd_batch *b, int code, const char *fmt, ...) {
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->msg = buf;
        if (code == LBD_ECUDA) b->sticky = LBD_ECUDA;
    }
    return code;
}

#define BCK(b, call)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail(b, LBD_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                         __FILE__, __LINE__);                                             \
    } while (0)

int fail(lbd_ctx *c, int code, const char *fmt, ...) {
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

#define CK(ctx, call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, LBD_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                               \
    } while (0)

// ---------------------------------------------------------------- kernels

// The first invalid site of an upload, in index order, as 4 s + reason:
// 1 a non-finite value, 2 psi <= 0 or B(psi) = B0 + B1 psi <= 0, 3 rho <= 0 (the
// first failing test of the site).  *first must hold all bits set on entry.
__global__ void check_fields_kernel(long long N, const double *rho, const double *ux,
                                    const double *uy, const double *phi, const double *psi,
                                    int has_rho, int has_ux, int has_uy, double B0, double B1,
                                    unsigned long long *first) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const double ph = phi[s], ps = psi[s];
        unsigned code = 0;
        if (!isfinite(ph) || !isfinite(ps) || (has_rho && !isfinite(rho[s])) ||
            (has_ux && !isfinite(ux[s])) || (has_uy && !isfinite(uy[s])))
            code = 1;
        else if (!(ps > 0.0) || !(__dadd_rn(B0, __dmul_rn(B1, ps)) > 0.0))
            code = 2;
        else if (has_rho && !(rho[s] > 0.0))
            code = 3;
        if (code) atomicMin(first, (unsigned long long)s * 4ull + code);
    }
}

// The same test of phi and psi in place, for pitched FP32 planes (rest-state
// upload of an FP32 context: rho = 1 and u = 0 are valid).  The values are
// widened to double first, so the verdict is that of check_fields_kernel on the
// same values.
__global__ void check_state_kernel(int nx, int ny, long long pitch, const float *phi,
                                   const float *psi, double B0, double B1,
                                   unsigned long long *first) {
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const long long y = s / nx, o = y * pitch + (s - y * nx);
        const double ph = (double)phi[o], ps = (double)psi[o];
        unsigned code = 0;
        if (!isfinite(ph) || !isfinite(ps))
            code = 1;
        else if (!(ps > 0.0) || !(__dadd_rn(B0, __dmul_rn(B1, ps)) > 0.0))
            code = 2;
        if (code) atomicMin(first, (unsigned long long)s * 4ull + code);
    }
}

// f_i = f_i^eq(rho, u) of Eq. (12) stored as g_i = f_i - w_i in the pull
// layout: buffer_i(x) is what site x + e_i reads, so it holds f_i^eq at x + e_i;
// with walls, a buffer whose reader lies beyond a plate is read back by its own
// site as the reversed population (bounce-back), so it holds f_{-i}^eq at x.
// Nothing is written unless *bad holds no invalid site (all bits set).
template <typename T>
__global__ void init_kernel(int nx, int ny, long long pitch, long long plane, const double *rho,
                            const double *ux, const double *uy, const double *phi,
                            const double *psi, int walls, const unsigned long long *bad, T *g,
                            T *phi_o, T *psi_o) {
    if (*bad != ~0ull) return;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                         1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        const long long o = (long long)y * pitch + x;
        phi_o[o] = (T)phi[s];
        psi_o[o] = (T)psi[s];
        for (int i = 0; i < 9; ++i) {
            int xs = x + ex[i], ys = y + ey[i];
            int k = i;  // population stored
            if (walls && (ys < 0 || ys >= ny)) {
                xs = x;
                ys = y;
                k = i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
            }
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
            const long long q = (long long)ys * nx + xs;
            const double n = rho[q], u = ux[q], v = uy[q];
            const double eu = ex[k] * u + ey[k] * v, usq = u * u + v * v;
            g[i * plane + o] = (T)(w[i] * ((n - 1.0) + n * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq)));
        }
    }
}

// The rest state rho = 1, u = 0 with the uploaded phi, psi: f_i^eq(1, 0) = w_i, so
// every deviation g_i is exactly +0 (the value init_kernel's formula gives for
// rho = 1, u = 0, bit for bit), plates or not.  Nothing is written unless *bad
// holds no invalid site.
template <typename T>
__global__ void init_rest_kernel(int nx, int ny, long long pitch, long long plane, const double *phi,
                                 const double *psi, const unsigned long long *bad, T *g, T *phi_o,
                                 T *psi_o) {
    if (*bad != ~0ull) return;
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        const long long o = (long long)y * pitch + x;
        phi_o[o] = (T)phi[s];
        psi_o[o] = (T)psi[s];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i * plane + o] = T(0);
    }
}

struct DropInits {
    lbd_droplet_init d[LBD_MAX_DROPLETS];
};

__device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ inline double min_image_even(double d, double L) { return d - L * rint(d / L); }

// phi and psi of the seeded droplets (lbd_init_droplets) into the pitched buffers
template <typename T>
__global__ void init_droplets_kernel(int nx, int ny, long long pitch, int n, DropInits D,
                                     double phieq, double xi, double psi_bg, uint64_t seed,
                                     T *phi, T *psi) {
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        double best = -INFINITY, bdx = 0, bdy = 0;
        int owner = -1;
        for (int k = 0; k < n; ++k) {
            const double dx = min_image_even(x - D.d[k].x, nx), dy = min_image_even(y - D.d[k].y, ny);
            const double v = D.d[k].R - sqrt(dx * dx + dy * dy);
            if (v > best) {
                best = v;
                owner = k;
                bdx = dx;
                bdy = dy;
            }
        }
        const long long o = (long long)y * pitch + x;
        phi[o] = (T)(phieq * tanh(best / xi));
        double c = psi_bg;
        if (owner >= 0 && best > 0) {
            const lbd_droplet_init &d = D.d[owner];
            const double u = (double)(splitmix64_at(seed, (uint64_t)s) >> 11) * 0x1.0p-53;
            c = d.psi_mean + d.psi_noise * (2.0 * u - 1.0) + d.gx * bdx / d.R + d.gy * bdy / d.R;
        }
        psi[o] = (T)c;
    }
}

__global__ void to_double_kernel(long long n, const float *a, double *b) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        b[s] = (double)a[s];
}

__global__ void to_float_kernel(long long n, const double *a, float *b) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        b[s] = (float)a[s];
}

__global__ void fill_kernel(double *a, long long n, double v) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        a[s] = v;
}

// Pre-collision populations f_i(x) = w_i + buffer_i(x - e_i) as dense doubles
// (with walls, w_i + buffer_{-i}(x) where x - e_i lies beyond a plate).
template <typename T>
__global__ void populations_kernel(int nx, int ny, long long pitch, long long plane, int walls,
                                   const T *g, double *f) {
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                         1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        for (int i = 0; i < 9; ++i) {
            int xs = x - ex[i], ys = y - ey[i];
            int k = i;  // buffer read
            if (walls && (ys < 0 || ys >= ny)) {
                xs = x;
                ys = y;
                k = i < 5 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5;
            }
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
            f[i * N + s] = w[i] + (double)g[k * plane + (long long)ys * pitch + xs];
        }
    }
}

// Inverse of populations_kernel: pre-collision f_i(x) (dense doubles) into the
// pull layout, buffer_i(x - e_i) = f_i(x) - w_i (with walls, buffer_{-i}(x) where
// x - e_i lies beyond a plate).
template <typename T>
__global__ void set_populations_kernel(int nx, int ny, long long pitch, long long plane, int walls,
                                       const double *f, T *g) {
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                         1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        for (int i = 0; i < 9; ++i) {
            int xs = x - ex[i], ys = y - ey[i];
            int k = i;
            if (walls && (ys < 0 || ys >= ny)) {
                xs = x;
                ys = y;
                k = i < 5 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5;
            }
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
            g[k * plane + (long long)ys * pitch + xs] = (T)(f[i * N + s] - w[i]);
        }
    }
}

// Block-wide reduction of the NRED slots (sums, then two minima).
__device__ void block_reduce(double v[NRED], double *smem /* [NRED][32] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < NRED; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            x = (k == 6 || k == 7) ? fmin(x, y) : x + y;
        }
        if (lane == 0) smem[k * 32 + warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < NRED; ++k) {
            const bool mn = (k == 6 || k == 7);
            double x = lane < nw ? smem[k * 32 + lane] : (mn ? INFINITY : 0.0);
            for (int o = 16; o > 0; o >>= 1) {
                double y = __shfl_down_sync(0xffffffffu, x, o);
                x = mn ? fmin(x, y) : x + y;
            }
            if (lane == 0) v[k] = x;
        }
    }
}

// Slots: 0 sum of all g_i (so sum rho = N + slot 0), 1 sum phi, 2 sum psi,
// 3-4 sum phi*dx, phi*dy over phi >= 0 (minimum image about the reference),
// 5 sum phi over phi >= 0, 6 min B(psi), 7 min psi, 8 non-finite count.
template <typename T>
__global__ void reduce_partial(int nx, int ny, long long pitch, long long plane, const T *g,
                               const T *phi, const T *psi, double B0, double B1, double refx,
                               double refy, double *partial) {
    __shared__ double smem[NRED * 32];
    double v[NRED] = {0, 0, 0, 0, 0, 0, INFINITY, INFINITY, 0};
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        double dy = y - refy;
        if (dy >= 0.5 * ny) dy -= ny; else if (dy < -0.5 * ny) dy += ny;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long o = (long long)y * pitch + x;
            double sg = 0.0;
            int bad = 0;
            for (int i = 0; i < 9; ++i) {
                const double gi = (double)g[i * plane + o];
                bad |= !isfinite(gi);
                sg += gi;
            }
            const double ph = (double)phi[o], c = (double)psi[o];
            bad |= !isfinite(ph) | !isfinite(c);
            v[0] += sg;
            v[1] += ph;
            v[2] += c;
            if (ph >= 0.0) {
                double dx = x - refx;
                if (dx >= 0.5 * nx) dx -= nx; else if (dx < -0.5 * nx) dx += nx;
                v[3] += ph * dx;
                v[4] += ph * dy;
                v[5] += ph;
            }
            v[6] = fmin(v[6], B0 + B1 * c);
            v[7] = fmin(v[7], c);
            v[8] += bad;
        }
    }
    block_reduce(v, smem);
    if (threadIdx.x == 0)
        for (int k = 0; k < NRED; ++k) partial[k * gridDim.x + blockIdx.x] = v[k];
}

// Exact sum of two floats: s + e == a + b (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Reference point of the minimum image, split on the host into its integer
// part and fraction, with the integer thresholds that reproduce the FP64 test
// d = x - ref >= n/2 (d -= n), d < -n/2 (d += n) for d = k - frac, k = x - floor(ref):
// k >= hi wraps down, k < lo wraps up.
struct RefImage {
    int ix, iy, hix, lox, hiy, loy;
    double frx, fry;
};

RefImage ref_image(int nx, int ny, double refx, double refy) {
    RefImage r;
    const double fx = std::floor(refx), fy = std::floor(refy);
    r.ix = (int)fx;
    r.iy = (int)fy;
    r.frx = refx - fx;
    r.fry = refy - fy;
    r.hix = (int)std::ceil(0.5 * nx + r.frx);
    r.lox = (int)std::ceil(r.frx - 0.5 * nx);
    r.hiy = (int)std::ceil(0.5 * ny + r.fry);
    r.loy = (int)std::ceil(r.fry - 0.5 * ny);
    return r;
}

// The FP32 form of the diagnostics reduction, with the results of the FP64
// form up to rounding, in one launch of RED32_BLOCKS (<= RED_BLOCKS) blocks:
//  * each thread walks 4-site row chunks (16-byte loads where rows and planes
//    are 16-byte aligned), sums each chunk's four sites in FP32 and adds the
//    chunk sums to six Neumaier-compensated FP32 sums; the warps merge the
//    (sum, compensation) pairs by TwoSum over shuffles, and so do the blocks
//    (into partial, one float2 slot per value and block) and the last block;
//    only the final totals are formed in FP64;
//  * min and max psi stay in FP32: min B = B0 + B1 psi is monotone in psi, so
//    it is evaluated once, at the extreme psi (max for B1 < 0);
//  * the minimum-image displacements are integers (RefImage); slots 3-4 of the
//    totals are shifted by the fraction of ref times the phi >= 0 mass in FP64;
//  * a chunk whose values do not add up to a finite number is re-examined
//    value by value, so the count is that of sites holding a non-finite value;
//  * the block that finishes last (a counter at partial[NRED * RED_BLOCKS],
//    zero between calls) combines the block partials in a fixed order and
//    writes the NRED results to out, so the results do not depend on which
//    block finishes last.
__global__ void __launch_bounds__(RED_THREADS, 3) reduce_f32(
    int nx, int ny, long long pitch, long long plane, const float *g, const float *phi,
    const float *psi, double B0, double B1, RefImage ri, int vec, double *partial, double *out) {
    constexpr int NW = RED_THREADS / 32;
    __shared__ float2 wsum[6][NW];  // (sum, compensation) of each warp
    __shared__ float wext[3][NW];   // min psi, max psi, bad count
    __shared__ float2 bres[NRED];   // the block's results
    __shared__ bool last;
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, cmp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto add = [&](int k, float x) {
        const float t = s[k] + x;
        cmp[k] += fabsf(s[k]) >= fabsf(x) ? (s[k] - t) + x : (x - t) + s[k];
        s[k] = t;
    };
    float pmin = INFINITY, pmax = -INFINITY, bad = 0.f;
    const int nq = (nx + 3) >> 2;
    const long long nchunks = (long long)nq * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nchunks;
         q += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(q / nq), x0 = (int)(q - (long long)y * nq) * 4;
        int ky = y - ri.iy;
        if (ky >= ri.hiy) ky -= ny; else if (ky < ri.loy) ky += ny;
        const long long o = (long long)y * pitch + x0;
        const int cnt = nx - x0 < 4 ? nx - x0 : 4;
        float gv[4] = {0.f, 0.f, 0.f, 0.f}, pv[4] = {0.f, 0.f, 0.f, 0.f}, cv[4] = {0.f, 0.f, 0.f, 0.f};
        if (vec && cnt == 4) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(g + i * plane + o));
                gv[0] += v.x; gv[1] += v.y; gv[2] += v.z; gv[3] += v.w;
            }
            const float4 a = __ldcs(reinterpret_cast<const float4 *>(phi + o));
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(psi + o));
            pv[0] = a.x; pv[1] = a.y; pv[2] = a.z; pv[3] = a.w;
            cv[0] = b.x; cv[1] = b.y; cv[2] = b.z; cv[3] = b.w;
        } else {
            for (int k = 0; k < cnt; ++k) {
                for (int i = 0; i < 9; ++i) gv[k] += g[i * plane + o + k];
                pv[k] = phi[o + k];
                cv[k] = psi[o + k];
            }
        }
        // the chunk's sites are summed first, in a fixed order, then each sum
        // takes one compensated add per chunk
        const float g4 = (gv[0] + gv[1]) + (gv[2] + gv[3]);
        const float p4 = (pv[0] + pv[1]) + (pv[2] + pv[3]);
        const float c4 = (cv[0] + cv[1]) + (cv[2] + cv[3]);
        if (!isfinite(g4 + p4 + c4)) {
            for (int k = 0; k < cnt; ++k) {
                bool nf = !isfinite(pv[k]) || !isfinite(cv[k]);
                for (int i = 0; i < 9; ++i) nf |= !isfinite(g[i * plane + o + k]);
                bad += nf ? 1.f : 0.f;
            }
        }
        float cx = 0.f, cw = 0.f;  // phi >= 0: sum of phi x, sum of phi (the row's y is common)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < cnt) {
                const float ph = pv[k], c = cv[k];
                if (ph >= 0.f) {
                    int kx = x0 + k - ri.ix;
                    if (kx >= ri.hix) kx -= nx; else if (kx < ri.lox) kx += nx;
                    cx = fmaf(ph, (float)kx, cx);
                    cw += ph;
                }
                pmin = fminf(pmin, c);
                pmax = fmaxf(pmax, c);
            }
        }
        add(0, g4);
        add(1, p4);
        add(2, c4);
        add(3, cx);
        add(4, cw * (float)ky);
        add(5, cw);
    }
    // warp: merge the compensated pairs (TwoSum of the sums, compensations added)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float s2 = __shfl_down_sync(0xffffffffu, s[k], o);
            const float c2 = __shfl_down_sync(0xffffffffu, cmp[k], o);
            float t, e;
            two_sum(s[k], s2, t, e);
            s[k] = t;
            cmp[k] = (cmp[k] + c2) + e;
        }
        pmin = fminf(pmin, __shfl_down_sync(0xffffffffu, pmin, o));
        pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        for (int k = 0; k < 6; ++k) wsum[k][warp] = make_float2(s[k], cmp[k]);
        wext[0][warp] = pmin;
        wext[1][warp] = pmax;
        wext[2][warp] = bad;
    }
    __syncthreads();
    // The block's totals, then the grid's, stay (sum, compensation) pairs of
    // floats merged by TwoSum in a fixed order: the FP64 pipe is a small
    // fraction of the FP32 one, and a few thousand dependent double operations in
    // one block used to be the kernel's tail.  Each value takes one float2 slot
    // of the partial array (extremes and the count in .x).
    const int nb = gridDim.x;
    float2 *const pp = reinterpret_cast<float2 *>(partial);
    // the completion counter sits after the RED_BLOCKS partials of either form
    unsigned long long *counter =
        reinterpret_cast<unsigned long long *>(partial + NRED * RED_BLOCKS);
    if (threadIdx.x < NRED) {
        const int k = threadIdx.x;
        float hi, lo = 0.f;
        if (k < 6) {
            hi = wsum[k][0].x;
            lo = wsum[k][0].y;
            for (int w = 1; w < NW; ++w) {
                float t, e;
                two_sum(hi, wsum[k][w].x, t, e);
                hi = t;
                lo = (lo + wsum[k][w].y) + e;
            }
        } else {
            hi = wext[k - 6][0];
            for (int w = 1; w < NW; ++w)
                hi = k == 6 ? fminf(hi, wext[0][w]) : (k == 7 ? fmaxf(hi, wext[1][w]) : hi + wext[2][w]);
        }
        bres[k] = make_float2(hi, lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NRED; ++k) pp[k * nb + blockIdx.x] = bres[k];
        asm volatile("fence.acq_rel.gpu;\n" ::: "memory");  // release the block's partials
        last = atomicAdd(counter, 1ull) == (unsigned long long)(nb - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last block: thread t merges the partials of blocks t, t + 256, ...,
    // then the warps by shuffles and the warp totals in warp order; the order
    // does not depend on which block finished last
    asm volatile("fence.acq_rel.gpu;\n" ::: "memory");  // acquire every block's partials
    float hi[NRED], lo[NRED];
    for (int k = 0; k < NRED; ++k) {
        hi[k] = k == 6 ? INFINITY : (k == 7 ? -INFINITY : 0.f);
        lo[k] = 0.f;
    }
    auto merge = [](int k, float &h, float &l, float xh, float xl) {
        if (k == 6) {
            h = fminf(h, xh);
        } else if (k == 7) {
            h = fmaxf(h, xh);
        } else {
            float t, e;
            two_sum(h, xh, t, e);
            h = t;
            l = (l + xl) + e;
        }
    };
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NRED; ++k) {
            const float2 x = __ldcg(pp + k * nb + b);
            merge(k, hi[k], lo[k], x.x, x.y);
        }
    __shared__ float2 tree[NRED][NW];
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            const float yh = __shfl_down_sync(0xffffffffu, hi[k], o);
            const float yl = __shfl_down_sync(0xffffffffu, lo[k], o);
            merge(k, hi[k], lo[k], yh, yl);
        }
        if (lane == 0) tree[k][warp] = make_float2(hi[k], lo[k]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[NRED];
        for (int k = 0; k < NRED; ++k) {
            float h = tree[k][0].x, l = tree[k][0].y;
            for (int w = 1; w < NW; ++w) merge(k, h, l, tree[k][w].x, tree[k][w].y);
            r[k] = (double)h + (double)l;
        }
        // the minimum-image shift by the fraction of ref, on the totals
        r[3] -= ri.frx * r[5];
        r[4] -= ri.fry * r[5];
        for (int k = 0; k < 6; ++k) out[k] = r[k];
        // min B = B0 + B1 psi at the extreme psi; +inf without any site
        const double ext = B1 < 0.0 ? r[7] : r[6];
        out[6] = isinf(ext) ? INFINITY : (B1 == 0.0 ? B0 : B0 + B1 * ext);
        out[7] = r[6];
        out[8] = r[8];
        *counter = 0ull;
    }
}

__global__ void reduce_final(int nb, const double *partial, double *out) {
    __shared__ double smem[NRED * 32];
    double v[NRED] = {0, 0, 0, 0, 0, 0, INFINITY, INFINITY, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int k = 0; k < NRED; ++k) {
            const double x = partial[k * nb + b];
            v[k] = (k == 6 || k == 7) ? fmin(v[k], x) : v[k] + x;
        }
    block_reduce(v, smem);
    if (threadIdx.x == 0)
        for (int k = 0; k < NRED; ++k) out[k] = v[k];
}

// The diagnostics reduction of the state in (g, phi, psi) on stream st into
// out[NRED]: the FP64 form takes the FP64 block kernel and reduce_final, the
// FP32 form the compensated FP32 kernel, which finishes in its last block.
// partial holds NRED * RED_BLOCKS + 1 doubles (the last one a counter that is
// zero between calls).
cudaError_t launch_reduce(int prec, int nx, int ny, long long pitch, long long plane, const void *g,
                          const void *phi, const void *psi, double B0, double B1, double refx,
                          double refy, double *partial, double *out, cudaStream_t st) {
    if (prec == LBD_FP64) {
        reduce_partial<double><<<RED_BLOCKS, RED_THREADS, 0, st>>>(
            nx, ny, pitch, plane, (const double *)g, (const double *)phi, (const double *)psi, B0,
            B1, refx, refy, partial);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        reduce_final<<<1, RED_THREADS, 0, st>>>(RED_BLOCKS, partial, out);
    } else {
        const int vec = pitch % 4 == 0 && ((uintptr_t)g | (uintptr_t)phi | (uintptr_t)psi) % 16 == 0;
        reduce_f32<<<RED32_BLOCKS, RED_THREADS, 0, st>>>(
            nx, ny, pitch, plane, (const float *)g, (const float *)phi, (const float *)psi, B0, B1,
            ref_image(nx, ny, refx, refy), vec, partial, out);
    }
    return cudaGetLastError();
}

// -------------------------------------------- scratch of lbd_diagnostics_static
// Partial sums of the RED_BLOCKS reduction blocks, the FP32 form's completion
// counter, then the NRED results: 5482 doubles = 43,856 bytes.  Every GPU that
// loads this library holds the array until the process exits.  Each call
// overwrites every slot it reads (each block writes all of its partials, the
// final step writes all results); the counter starts at zero (the array is
// zero-initialised when the library's device code loads) and every FP32 call
// leaves it at zero.
constexpr int kStaticScratchDoubles = NRED * RED_BLOCKS + 1 + NRED;
static __device__ __align__(256) double g_diag_static_scratch[kStaticScratchDoubles];

// Device address of the static scratch on the current device and context.  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up with cudaGetSymbolAddress on every call: the lookup allocates
// nothing and does not synchronise, and it cannot go stale (a cached address
// would be wrong after cudaDeviceReset, which reloads the module in a new
// primary context, or under a caller's own non-primary context).  The first
// lookup on a device loads the library's device code there if lazy module
// loading has not done so yet.
cudaError_t static_scratch(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_diag_static_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

// Whether p is memory that kernels on the current device can read: device
// memory of that device, or managed memory.
bool on_current_device(const void *p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// ------------------------------------------------ allocation failure hook
// Allocations still to go before the one that fails (0: none fails).
std::atomic<int> g_fail_countdown{0};

bool fail_this_allocation() {
    int n = g_fail_countdown.load();
    while (n > 0) {
        if (g_fail_countdown.compare_exchange_weak(n, n - 1)) return n == 1;
    }
    return false;
}

// ---------------------------------------------------------------- helpers

int check_params(lbd_ctx *c, const lbd_grid *gr, const lbd_params *p) {
    if (!p) return fail(c, LBD_EINVAL, "params is NULL");
    if (!(p->tau > 0.5)) return fail(c, LBD_EINVAL, "tau must be > 1/2 (got %g)", p->tau);
    if (!(p->b >= 0.0)) return fail(c, LBD_EINVAL, "b must be >= 0 (got %g)", p->b);
    const double vals[] = {p->a, p->b, p->B0, p->B1, p->M, p->D, p->tau, p->gamma,
                           p->c0, p->A0, p->A_max, p->fx, p->fy, p->ux0, p->uy0};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(c, LBD_EINVAL, "non-finite parameter");
    if (p->precision != LBD_FP64 && p->precision != LBD_FP32)
        return fail(c, LBD_EINVAL, "precision must be LBD_FP64 or LBD_FP32");
    if (p->n_src < 0 || p->n_src > LBD_MAX_SOURCES)
        return fail(c, LBD_EINVAL, "n_src must be in [0, %d]", LBD_MAX_SOURCES);
    if (p->flags & ~(LBD_FROZEN_U | LBD_BODY_FORCE | LBD_WALLS))
        return fail(c, LBD_EINVAL, "unknown flags");
    const int ny = gr ? gr->ny : (c ? c->grid.ny : 0);
    if ((p->flags & LBD_WALLS) && ny < 8) return fail(c, LBD_EINVAL, "walls need ny >= 8");
    for (int k = 0; k < p->n_src; ++k) {
        const lbd_source &s = p->src[k];
        if (!std::isfinite(s.x) || !std::isfinite(s.y) || !(s.R >= 0.0))
            return fail(c, LBD_EINVAL, "bad source %d", k);
    }
    if (gr && (gr->nx < 4 || gr->ny < 4 || gr->nx > (1 << 20) || gr->ny > (1 << 20)))
        return fail(c, LBD_EINVAL, "grid must be within [4, 2^20] per side");
    return LBD_OK;
}

template <typename T>
StepArgs<T> make_args(const lbd_ctx *c, int cur = -1) {
    StepArgs<T> a;
    memset(&a, 0, sizeof a);
    const lbd_params &p = c->params;
    if (cur < 0) cur = c->cur;
    a.nx = c->grid.nx;
    a.ny = c->grid.ny;
    a.pitch = c->pitch;
    a.plane = c->plane;
    a.g_in = (const T *)c->g[cur];
    a.g_out = (T *)c->g[1 - cur];
    a.phi_in = (const T *)c->phi[cur];
    a.psi_in = (const T *)c->psi[cur];
    a.phi_out = (T *)c->phi[1 - cur];
    a.psi_out = (T *)c->psi[1 - cur];
    a.A0 = p.A0;
    a.A_max = p.A_max;
    a.t_on = p.t_on;
    a.gamma_on = p.gamma;
    a.a = (T)p.a;
    a.b = (T)p.b;
    a.B0 = (T)p.B0;
    a.B1 = (T)p.B1;
    a.M = (T)p.M;
    a.D = (T)p.D;
    a.omega = (T)(1.0 / p.tau);
    a.guo = (T)(1.0 - 0.5 / p.tau);
    a.c0 = (T)p.c0;
    // zero unless LBD_BODY_FORCE: the stripe kernel adds (fx, fy) unconditionally
    a.fx = (p.flags & LBD_BODY_FORCE) ? (T)p.fx : T(0);
    a.fy = (p.flags & LBD_BODY_FORCE) ? (T)p.fy : T(0);
    a.ux0 = (T)p.ux0;
    a.uy0 = (T)p.uy0;
    a.flags = p.flags;
    a.theta = c->theta;  // always valid (all zero without sources)
    a.theta_words = (a.nx + 31) / 32;
    return a;
}


// The verdict of a completed check: the first failure is kept in c->flagged.
void judge_check(lbd_ctx *c, const double *r, int64_t t) {
    if (c->flagged) return;
    if (r[8] > 0) {
        c->flagged = LBD_ENONFINITE;
        c->msg = "run-time check: " + std::to_string((long long)r[8]) +
                 " sites hold a non-finite value at step " + std::to_string((long long)t);
    } else if (!(r[6] > 0) || !(r[7] > 0)) {
        char buf[160];
        snprintf(buf, sizeof buf, "run-time check: min B(psi) = %g, min psi = %g at step %lld",
                 r[6], r[7], (long long)t);
        c->flagged = LBD_EUNSTABLE;
        c->msg = buf;
    }
}

// Read the verdicts of the completed checks, in the order they were queued;
// with wait, wait for all of them.  Returns an LBD code for a CUDA failure.
int poll_checks(lbd_ctx *c, bool wait) {
    for (int k = 0; k < lbd_ctx::NCHECK; ++k) {
        lbd_ctx::CheckSlot &s = c->chk[(c->chk_next + k) % lbd_ctx::NCHECK];
        if (!s.pending) continue;
        cudaError_t e = wait ? cudaEventSynchronize(s.ev) : cudaEventQuery(s.ev);
        if (e == cudaErrorNotReady) break;  // later slots completed no earlier
        if (e != cudaSuccess) return fail(c, LBD_ECUDA, "check: %s", cudaGetErrorString(e));
        s.pending = false;
        judge_check(c, s.h, s.t);
    }
    return LBD_OK;
}

// Queue one check of the current state (after the step that reached c->t).
int queue_check(lbd_ctx *c) {
    lbd::NvtxRange range("lbd check reduction");
    lbd_ctx::CheckSlot &s = c->chk[c->chk_next];
    if (!s.d) {
        if (lbd::dev_malloc((void **)&s.d, NRED * sizeof(double)) != cudaSuccess ||
            lbd::host_malloc((void **)&s.h, NRED * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(s.d);
            s.d = nullptr;
            return fail(c, LBD_ENOMEM, "check slot allocation failed");
        }
        CK(c, cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
    }
    if (s.pending) {  // every slot in flight: wait for the oldest
        CK(c, cudaEventSynchronize(s.ev));
        s.pending = false;
        judge_check(c, s.h, s.t);
    }
    const lbd_params &p = c->params;
    CK(c, launch_reduce(p.precision, c->grid.nx, c->grid.ny, c->pitch, c->plane, c->g[c->cur],
                        c->phi[c->cur], c->psi[c->cur], p.B0, p.B1, 0.0, 0.0, c->red_partial, s.d,
                        c->stream));
    CK(c, cudaMemcpyAsync(s.h, s.d, NRED * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaEventRecord(s.ev, c->stream));
    s.t = c->t;
    s.pending = true;
    c->chk_next = (c->chk_next + 1) % lbd_ctx::NCHECK;
    return LBD_OK;
}

// Forget queued checks and a flagged failure (the state was replaced).
int reset_checks(lbd_ctx *c) {
    int rc = poll_checks(c, true);
    c->flagged = 0;
    return rc;
}

template <typename T>
int run_steps(lbd_ctx *c, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        StepArgs<T> a = make_args<T>(c);
        double A, gm;
        lbd::activity_at(c->params, c->t, &A, &gm);
        a.A = (T)A;
        a.gamma = (T)gm;
        CK(c, lbd::launch_step<T>(a, lbd::MODE_STEP, c->tile, c->stream));
        c->cur = 1 - c->cur;
        c->t += 1;
        if (c->check_every > 0 && c->t % c->check_every == 0) {
            const int rc = queue_check(c);
            if (rc != LBD_OK) return rc;
        }
    }
    return LBD_OK;
}

// Source disks with centres wrapped into [0, nx) x [0, ny), then the bit mask.
int update_theta(lbd_ctx *c) {
    const lbd_params &p = c->params;
    lbd_source src[LBD_MAX_SOURCES];
    for (int k = 0; k < p.n_src; ++k) {
        double x = std::fmod(p.src[k].x, (double)c->grid.nx);
        double y = std::fmod(p.src[k].y, (double)c->grid.ny);
        src[k].x = x < 0 ? x + c->grid.nx : x;
        src[k].y = y < 0 ? y + c->grid.ny : y;
        if (p.flags & LBD_WALLS) src[k].y = p.src[k].y;  // no periodic image across a plate
        src[k].R = p.src[k].R;
    }
    CK(c, lbd::launch_theta_mask(c->grid.nx, c->grid.ny, p.n_src, src, (p.flags & LBD_WALLS) == 0,
                                 c->theta, c->stream));
    return LBD_OK;
}

// Whether launch shape t can run this context's steps: compiled in, valid for
// its precision and lattice, and a stripe shape when the lattice has walls.
bool tile_ok(const lbd_ctx *c, Tile t) {
    if (!lbd::tile_valid(t, c->params.precision == LBD_FP32, c->grid.nx, c->plane)) return false;
    // no walls in the 16-byte staged stripe kernel
    return !(c->params.flags & LBD_WALLS) || t.bx != 116;
}

int ensure_staging(lbd_ctx *c) {
    if (c->staging) return LBD_OK;
    // five fields of doubles, then the first-invalid-site word of an upload
    if (lbd::dev_malloc((void **)&c->staging, (5 * c->N + 1) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->staging = nullptr;
        return fail(c, LBD_ENOMEM, "staging allocation of %zu bytes failed",
                    (5 * c->N + 1) * sizeof(double));
    }
    return LBD_OK;
}

int ensure_staging32(lbd_ctx *c) {
    if (c->staging32) return LBD_OK;
    if (lbd::dev_malloc((void **)&c->staging32, 5 * c->N * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        c->staging32 = nullptr;
        return fail(c, LBD_ENOMEM, "float staging allocation of %zu bytes failed",
                    5 * c->N * sizeof(float));
    }
    return LBD_OK;
}

int ensure_side(lbd_ctx *c) {
    if (c->side) return LBD_OK;
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_side, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->side) cudaStreamDestroy(c->side);
        if (c->ev_main) cudaEventDestroy(c->ev_main);
        if (c->ev_side) cudaEventDestroy(c->ev_side);
    cudaFree(c->word);
        c->side = nullptr;
        c->ev_main = c->ev_side = nullptr;
        return fail(c, LBD_ECUDA, "stream or event creation failed");
    }
    return LBD_OK;
}

int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

}  // namespace

namespace lbd {
cudaError_t dev_malloc(void **p, size_t bytes) {
    if (fail_this_allocation()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
cudaError_t host_malloc(void **p, size_t bytes) {
    if (fail_this_allocation()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}
}  // namespace lbd

namespace {

template <typename T>
int adjoint_impl(lbd_ctx *c, int64_t nsteps, int32_t ckpt_every, double refx, double *loss,
                 double *dpsi, double *dB1) {
    lbd::AdjointJob<T> job;
    const lbd_params &p = c->params;
    job.nx = c->grid.nx;
    job.ny = c->grid.ny;
    job.pitch = c->pitch;
    job.plane = c->plane;
    job.args = make_args<T>(c);
    job.tile = c->tile;
    job.stream = c->stream;
    job.params = &c->params;
    job.g0 = (const T *)c->g[c->cur];
    job.phi0 = (const T *)c->phi[c->cur];
    job.psi0 = (const T *)c->psi[c->cur];
    job.g_final = (T *)c->g[c->cur];
    job.phi_final = (T *)c->phi[c->cur];
    job.psi_final = (T *)c->psi[c->cur];
    job.t0 = c->t;
    job.nsteps = nsteps;
    job.ckpt_every = ckpt_every;
    job.refx = refx;
    job.a = p.a; job.b = p.b; job.B0 = p.B0; job.B1 = p.B1; job.M = p.M; job.D = p.D;
    job.tau = p.tau; job.c0 = p.c0; job.fx = p.fx; job.fy = p.fy;
    job.body = (p.flags & LBD_BODY_FORCE) ? 1 : 0;
    job.loss = loss;
    job.dB1 = dB1;
    job.dpsi_host = dpsi;
    const int rc = lbd::adjoint_run<T>(job);
    if (rc == LBD_ECUDA) return fail(c, LBD_ECUDA, "adjoint: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == LBD_ENOMEM) return fail(c, LBD_ENOMEM, "adjoint: device allocation failed");
    if (rc == LBD_OK) c->t += nsteps;
    return rc;
}


// ---------------------------------------------------------------- batches

void batch_drop_graphs(lbd_batch *b) {
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) {
            cudaGraphExecDestroy(b->graph[p]);
            b->graph[p] = nullptr;
        }
}

// Device tables of step arguments (one per buffer parity) and the work list of
// the current launch shape.
template <typename T>
int batch_build(lbd_batch *b) {
    const size_t bytes = sizeof(StepArgs<T>) * (size_t)b->n;
    std::vector<StepArgs<T>> host(b->n);
    for (int p = 0; p < 2; ++p) {
        if (!b->args_dev[p]) BCK(b, lbd::dev_malloc((void **)&b->args_dev[p], bytes));
        for (int k = 0; k < b->n; ++k) host[k] = make_args<T>(b->ctx[k], p);
        BCK(b, cudaMemcpyAsync(b->args_dev[p], host.data(), bytes, cudaMemcpyHostToDevice, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
    }
    // Periodic instances take stripes of the launch shape's width; with the
    // 16-byte staged kernel (bx 116) the instances with plates take the stripe
    // kernel's 118-column stripes.
    const int seg = b->tile.by;
    const int w_plain = b->tile.bx, w_walls = b->tile.bx == 116 ? 118 : b->tile.bx;
    std::vector<lbd::BatchItem> plain, walled;
    for (int k = 0; k < b->n; ++k) {
        const int nx = b->ctx[k]->grid.nx, ny = b->ctx[k]->grid.ny;
        const bool walls = (b->ctx[k]->params.flags & LBD_WALLS) != 0;
        const int bxo = walls ? w_walls : w_plain;
        // ceil(ny / seg) row segments of equal height (within one row), so that
        // no instance leaves a short tail segment that costs a full pipeline fill
        const int nseg = (ny + seg - 1) / seg;
        for (int j = 0; j < nseg; ++j) {
            const int y0 = (int)((long long)ny * j / nseg), y1 = (int)((long long)ny * (j + 1) / nseg);
            for (int x0 = 0; x0 < nx; x0 += bxo)
                (walls ? walled : plain).push_back(lbd::BatchItem{k, x0, y0, y1 - y0});
        }
    }
    int sms = 0;
    BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx[0]->dev));
    const int per_sm_plain = w_plain == 116 ? lbd::vstripe_batch_ctas_per_sm()
                                            : lbd::stripe_batch_ctas_per_sm<T>(w_plain + 10);
    const int per_sm_walls = lbd::stripe_batch_ctas_per_sm<T>(w_walls + 10);
    b->ctas = std::min((int)plain.size(), sms * per_sm_plain);
    b->ctas_walls = std::min((int)walled.size(), sms * per_sm_walls);
    // CTA j of a persistent launch takes items j, j + P, j + 2P, ... (P CTAs).
    // An item costs about its rows plus the pipeline fill, so the items are
    // sorted by rows, largest first, and dealt in boustrophedon order: CTA j
    // gets the j-th item of even rounds and the j-th from the end of odd ones,
    // which evens the CTAs' totals out (greedy longest-first in effect).
    auto deal = [](std::vector<lbd::BatchItem> &v, int P) {
        std::stable_sort(v.begin(), v.end(), [](const lbd::BatchItem &u, const lbd::BatchItem &w) {
            return u.rows > w.rows;
        });
        if (P < 1) return;
        std::vector<lbd::BatchItem> out(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            const size_t r = i / (size_t)P, k = i % (size_t)P;
            const size_t cnt = std::min((size_t)P, v.size() - r * (size_t)P);
            out[i] = v[r * (size_t)P + ((r & 1) ? cnt - 1 - k : k)];
        }
        v.swap(out);
    };
    deal(plain, b->ctas);
    deal(walled, b->ctas_walls);
    // periodic instances first: the plates take a launch of their own
    std::vector<lbd::BatchItem> items(plain);
    items.insert(items.end(), walled.begin(), walled.end());
    if (b->items_dev) cudaFree(b->items_dev);
    b->items_dev = nullptr;
    BCK(b, lbd::dev_malloc((void **)&b->items_dev, sizeof(lbd::BatchItem) * items.size()));
    BCK(b, cudaMemcpyAsync(b->items_dev, items.data(), sizeof(lbd::BatchItem) * items.size(),
                           cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->n_items = (int)items.size();
    b->n_plain = (int)plain.size();
    batch_drop_graphs(b);
    return LBD_OK;
}

template <typename T>
cudaError_t launch_vstripe_batch_if_float(const StepArgs<T> *, const lbd::BatchItem *, int, int,
                                         const long long *, int, cudaStream_t) {
    return cudaErrorInvalidValue;
}
template <>
cudaError_t launch_vstripe_batch_if_float<float>(const StepArgs<float> *args,
                                                 const lbd::BatchItem *items, int n, int ctas,
                                                 const long long *t_dev, int t_off,
                                                 cudaStream_t s) {
    return lbd::launch_vstripe_batch(args, items, n, ctas, t_dev, t_off, s);
}

template <typename T>
cudaError_t batch_launch(lbd_batch *b, int parity, int t_off) {
    const StepArgs<T> *args = (const StepArgs<T> *)b->args_dev[parity];
    cudaError_t e = cudaSuccess;
    const int w_walls = b->tile.bx == 116 ? 118 : b->tile.bx;
    if (b->n_plain > 0) {
        if (b->tile.bx == 116)
            e = launch_vstripe_batch_if_float<T>(args, b->items_dev, b->n_plain, b->ctas, b->t_dev,
                                                 t_off, b->stream);
        else
            e = lbd::launch_stripe_batch<T>(args, b->items_dev, b->n_plain, b->tile.bx + 10,
                                            false, b->ctas, b->t_dev, t_off, b->stream);
    }
    if (e == cudaSuccess && b->n_items > b->n_plain)
        e = lbd::launch_stripe_batch<T>(args, b->items_dev + b->n_plain, b->n_items - b->n_plain,
                                        w_walls + 10, true, b->ctas_walls, b->t_dev, t_off,
                                        b->stream);
    return e;
}

template <typename T>
int batch_run(lbd_batch *b, int64_t nsteps) {
    BCK(b, lbd::launch_time_set(b->t_dev, (long long)b->t, b->stream));
    int parity = b->ctx[0]->cur;
    int64_t done = 0;
    const int G = b->graph_steps;  // even, so a replay returns to the same parity
    while (nsteps - done >= G) {
        if (!b->graph[parity]) {
            cudaGraph_t g = nullptr;
            BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int j = 0; j < G && e == cudaSuccess; ++j)
                e = batch_launch<T>(b, (parity + j) & 1, j);
            if (e == cudaSuccess) e = lbd::launch_time_advance(b->t_dev, G, b->stream);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return bfail(b, LBD_ECUDA, "graph capture: %s",
                             cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&b->graph[parity], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return bfail(b, LBD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        BCK(b, cudaGraphLaunch(b->graph[parity], b->stream));
        done += G;
    }
    const int64_t r = nsteps - done;
    for (int64_t j = 0; j < r; ++j) BCK(b, batch_launch<T>(b, (int)((parity + j) & 1), (int)j));
    if (r) BCK(b, lbd::launch_time_advance(b->t_dev, r, b->stream));
    for (lbd_ctx *c : b->ctx) {
        if (nsteps & 1) c->cur = 1 - c->cur;
        c->t += nsteps;
    }
    b->t += nsteps;
    return LBD_OK;
}
}  // namespace

// ====================================================================== C ABI

extern "C" {

const char *lbd_strerror(int code) {
    switch (code) {
        case LBD_OK: return "LBD_OK";
        case LBD_EINVAL: return "LBD_EINVAL: invalid argument";
        case LBD_ENOMEM: return "LBD_ENOMEM: out of memory";
        case LBD_ECUDA: return "LBD_ECUDA: CUDA error";
        case LBD_ENONFINITE: return "LBD_ENONFINITE: non-finite value";
        case LBD_EUNSTABLE: return "LBD_EUNSTABLE: B(psi) <= 0 or psi <= 0";
        case LBD_ETIMEOUT: return "LBD_ETIMEOUT: device wait timed out";
        default: return "unknown lbd error";
    }
}

const char *lbd_last_error(const lbd_ctx *ctx) { return ctx ? ctx->msg.c_str() : ""; }

void lbd_destroy(lbd_ctx *c) {
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->g[k]);
        cudaFree(c->phi[k]);
        cudaFree(c->psi[k]);
    }
    cudaFree(c->staging);
    cudaFree(c->staging32);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_main) cudaEventDestroy(c->ev_main);
    if (c->ev_side) cudaEventDestroy(c->ev_side);
    cudaFree(c->word);
    cudaFree(c->pop_staging);
    cudaFree(c->drop_dev);
    cudaFreeHost(c->h_drop);
    cudaFree(c->red_partial);
    cudaFree(c->red_out);
    cudaFree(c->theta);
    cudaFreeHost(c->h_red);
    for (auto &k : c->chk) {
        cudaFree(k.d);
        cudaFreeHost(k.h);
        if (k.ev) cudaEventDestroy(k.ev);
    }
    cudaSetDevice(prev);
    delete c;
}

int lbd_create(const lbd_grid *grid, const lbd_params *params, void *stream, lbd_ctx **out) {
    if (!out || !grid) return LBD_EINVAL;
    *out = nullptr;
    lbd_ctx *c = new (std::nothrow) lbd_ctx();
    if (!c) return LBD_ENOMEM;
    int rc = check_params(c, grid, params);
    if (rc == LBD_OK && params->reserved != 0) rc = LBD_EINVAL;
    if (rc != LBD_OK) {
        delete c;
        return rc;
    }
    c->grid = *grid;
    c->params = *params;
    c->stream = (cudaStream_t)stream;
    c->esz = params->precision == LBD_FP64 ? sizeof(double) : sizeof(float);
    // rows padded to 128 bytes
    const long long align = 128 / (long long)c->esz;
    c->pitch = (grid->nx + align - 1) / align * align;
    c->plane = c->pitch * grid->ny;
    c->N = (size_t)grid->nx * grid->ny;
    if (cudaGetDevice(&c->dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LBD_ECUDA;
    }
    const size_t fbytes = (size_t)c->plane * c->esz;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok &= lbd::dev_malloc((void **)&c->g[k], 9 * fbytes) == cudaSuccess;
        ok &= ok && lbd::dev_malloc((void **)&c->phi[k], fbytes) == cudaSuccess;
        ok &= ok && lbd::dev_malloc((void **)&c->psi[k], fbytes) == cudaSuccess;
    }
    // block partials plus the FP32 reduction's completion counter (zeroed below)
    ok &= ok && lbd::dev_malloc((void **)&c->red_partial, (NRED * RED_BLOCKS + 1) * sizeof(double)) == cudaSuccess;
    ok &= ok && lbd::dev_malloc((void **)&c->red_out, NRED * sizeof(double)) == cudaSuccess;
    ok &= ok && lbd::host_malloc((void **)&c->h_red, NRED * sizeof(double)) == cudaSuccess;
    ok &= ok && lbd::dev_malloc((void **)&c->theta, (size_t)((grid->nx + 31) / 32) * grid->ny * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbd_destroy(c);
        return LBD_ENOMEM;
    }
    // the reduction's completion counter starts at zero
    if (cudaMemsetAsync(c->red_partial + NRED * RED_BLOCKS, 0, sizeof(double), c->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        lbd_destroy(c);
        return LBD_ECUDA;
    }
    // rest state: g = 0 (f = w_i, rho = 1, u = 0), phi = psi = 0
    for (int k = 0; k < 2; ++k) {
        if (cudaMemsetAsync(c->g[k], 0, 9 * fbytes, c->stream) != cudaSuccess ||
            cudaMemsetAsync(c->phi[k], 0, fbytes, c->stream) != cudaSuccess ||
            cudaMemsetAsync(c->psi[k], 0, fbytes, c->stream) != cudaSuccess) {
            cudaGetLastError();
            lbd_destroy(c);
            return LBD_ECUDA;
        }
    }
    // Default launch shape: the stripe kernel (fastest measured on large
    // lattices) unless it would leave most SMs idle, then the tiled kernel with
    // its smallest tiles; lbd_autotune refines the choice.
    // FP32 on periodic lattices of width 4k: the stripe kernel with 16-byte
    // population staging; otherwise the plain stripe kernel.
    c->tile = Tile{116, 64};
    if (!tile_ok(c, c->tile)) c->tile = Tile{118, 64};
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 1;
        }
        const int w = c->tile.bx;
        const long long stripe_ctas = (long long)((grid->nx + w - 1) / w) * ((grid->ny + 63) / 64);
        if (stripe_ctas < 2LL * sms || !tile_ok(c, c->tile)) c->tile = Tile{32, 8};
    }
    if (update_theta(c) != LBD_OK) {
        lbd_destroy(c);
        return LBD_ECUDA;
    }
    *out = c;
    return LBD_OK;
}

int lbd_set_params(lbd_ctx *c, const lbd_params *p) {
    if (!c) return LBD_EINVAL;
    int rc = check_params(c, nullptr, p);
    if (rc != LBD_OK) return rc;
    if (p->precision != c->params.precision)
        return fail(c, LBD_EINVAL, "precision cannot change after creation");
    const lbd_params keep = c->params;
    c->params = *p;
    if ((p->flags & LBD_WALLS) && !tile_ok(c, c->tile)) {  // a shape without walls
        c->tile = Tile{118, 64};
        if (!tile_ok(c, c->tile)) c->tile = Tile{32, 8};
        if (!tile_ok(c, c->tile)) {
            c->params = keep;
            return fail(c, LBD_EINVAL, "no launch shape runs walls on this lattice");
        }
    }
    CK(c, cudaSetDevice(c->dev));
    return update_theta(c);
}

}  // extern "C"

namespace {
// Upload the host fields (element type In: double or float) into the dense
// double staging area, validate them there and build the state only if every
// site is valid (the state is left as it was otherwise).  Float input is
// copied as is and widened on the device (exact).
template <typename In>
int set_fields_impl(lbd_ctx *c, const In *rho, const In *ux, const In *uy, const In *phi,
                    const In *psi) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (!phi || !psi) return fail(c, LBD_EINVAL, "phi and psi are required");
    const size_t N = c->N;
    const lbd_params &p = c->params;
    constexpr bool F32 = std::is_same<In, float>::value;
    if (F32 && !rho && !ux && !uy && p.precision == LBD_FP32) {
        // Float phi and psi into an FP32 context's rest state: copied straight
        // into the second buffer set (scratch between steps), checked there,
        // and, if every site is valid, copied into the state with g = 0 (the
        // buffer parity is kept).  Same state and verdicts as the staged path.
        if (!c->word && lbd::dev_malloc((void **)&c->word, sizeof *c->word) != cudaSuccess) {
            cudaGetLastError();
            c->word = nullptr;
            return fail(c, LBD_ENOMEM, "upload verdict allocation failed");
        }
        CK(c, cudaSetDevice(c->dev));
        const int back = 1 - c->cur;
        float *ph = (float *)c->phi[back], *ps = (float *)c->psi[back];
        const size_t w = (size_t)c->grid.nx * sizeof(float), pb = (size_t)c->pitch * sizeof(float);
        const size_t fb = (size_t)c->plane * sizeof(float);
        CK(c, cudaMemcpy2DAsync(ph, pb, phi, w, w, c->grid.ny, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpy2DAsync(ps, pb, psi, w, w, c->grid.ny, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemsetAsync(c->word, 0xFF, sizeof *c->word, c->stream));
        check_state_kernel<<<grid_for(N), 256, 0, c->stream>>>(c->grid.nx, c->grid.ny, c->pitch,
                                                               ph, ps, p.B0, p.B1, c->word);
        CK(c, cudaGetLastError());
        unsigned long long first = 0;
        CK(c, cudaMemcpyAsync(&first, c->word, sizeof first, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        if (first != ~0ull) {
            const size_t site = (size_t)(first >> 2);
            if ((first & 3ull) == 1ull)
                return fail(c, LBD_ENONFINITE, "non-finite initial value at site %zu", site);
            return fail(c, LBD_EUNSTABLE, "psi <= 0 or B(psi) <= 0 at site %zu", site);
        }
        CK(c, cudaMemcpyAsync(c->phi[c->cur], ph, fb, cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->psi[c->cur], ps, fb, cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaMemsetAsync(c->g[c->cur], 0, 9 * fb, c->stream));
        return reset_checks(c);
    }
    int rc = ensure_staging(c);
    if (rc != LBD_OK) return rc;
    if (F32) {
        rc = ensure_staging32(c);
        if (rc != LBD_OK) return rc;
    }
    CK(c, cudaSetDevice(c->dev));
    double *d = c->staging;
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(d + 5 * N);
    const size_t B = N * sizeof(double);
    const int nb = grid_for(N);
    // without rho and u the populations are the rest state: no equilibrium to evaluate
    const bool rest = !rho && !ux && !uy;
    auto upload = [&](const In *h, int k) -> int {
        if (F32) {
            float *t = c->staging32 + k * N;
            CK(c, cudaMemcpyAsync(t, h, N * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            to_double_kernel<<<nb, 256, 0, c->stream>>>((long long)N, t, d + k * N);
            CK(c, cudaGetLastError());
        } else {
            CK(c, cudaMemcpyAsync(d + k * N, h, B, cudaMemcpyHostToDevice, c->stream));
        }
        return LBD_OK;
    };
    CK(c, cudaMemsetAsync(bad, 0xFF, sizeof *bad, c->stream));
    if (rho) {
        if ((rc = upload(rho, 0)) != LBD_OK) return rc;
    } else if (!rest) {
        fill_kernel<<<nb, 256, 0, c->stream>>>(d, (long long)N, 1.0);
        CK(c, cudaGetLastError());
    }
    if (ux) {
        if ((rc = upload(ux, 1)) != LBD_OK) return rc;
    } else if (!rest) CK(c, cudaMemsetAsync(d + N, 0, B, c->stream));
    if (uy) {
        if ((rc = upload(uy, 2)) != LBD_OK) return rc;
    } else if (!rest) CK(c, cudaMemsetAsync(d + 2 * N, 0, B, c->stream));
    if ((rc = upload(phi, 3)) != LBD_OK) return rc;
    if ((rc = upload(psi, 4)) != LBD_OK) return rc;
    check_fields_kernel<<<nb, 256, 0, c->stream>>>((long long)N, d, d + N, d + 2 * N, d + 3 * N,
                                                   d + 4 * N, rho != nullptr, ux != nullptr,
                                                   uy != nullptr, p.B0, p.B1, bad);
    CK(c, cudaGetLastError());
    if (rest && p.precision == LBD_FP64)
        init_rest_kernel<double><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, d + 3 * N, d + 4 * N, bad,
            (double *)c->g[c->cur], (double *)c->phi[c->cur], (double *)c->psi[c->cur]);
    else if (rest)
        init_rest_kernel<float><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, d + 3 * N, d + 4 * N, bad,
            (float *)c->g[c->cur], (float *)c->phi[c->cur], (float *)c->psi[c->cur]);
    else if (p.precision == LBD_FP64)
        init_kernel<double><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, d, d + N, d + 2 * N, d + 3 * N, d + 4 * N,
            (p.flags & LBD_WALLS) ? 1 : 0, bad, (double *)c->g[c->cur], (double *)c->phi[c->cur],
            (double *)c->psi[c->cur]);
    else
        init_kernel<float><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, d, d + N, d + 2 * N, d + 3 * N, d + 4 * N,
            (p.flags & LBD_WALLS) ? 1 : 0, bad, (float *)c->g[c->cur], (float *)c->phi[c->cur],
            (float *)c->psi[c->cur]);
    CK(c, cudaGetLastError());
    unsigned long long first = 0;
    CK(c, cudaMemcpyAsync(&first, bad, sizeof first, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (first == ~0ull) {  // the state was replaced: earlier check verdicts no longer apply
        rc = reset_checks(c);
        if (rc != LBD_OK) return rc;
    }
    if (first != ~0ull) {
        const size_t site = (size_t)(first >> 2);
        switch ((int)(first & 3ull)) {
            case 1: return fail(c, LBD_ENONFINITE, "non-finite initial value at site %zu", site);
            case 2: return fail(c, LBD_EUNSTABLE, "psi <= 0 or B(psi) <= 0 at site %zu", site);
            default: return fail(c, LBD_EINVAL, "rho <= 0 at site %zu", site);
        }
    }
    return LBD_OK;
}
}  // namespace

extern "C" {

int lbd_set_fields(lbd_ctx *c, const double *rho, const double *ux, const double *uy,
                   const double *phi, const double *psi) {
    return set_fields_impl<double>(c, rho, ux, uy, phi, psi);
}

int lbd_set_fields_f32(lbd_ctx *c, const float *rho, const float *ux, const float *uy,
                       const float *phi, const float *psi) {
    return set_fields_impl<float>(c, rho, ux, uy, phi, psi);
}

int lbd_step(lbd_ctx *c, int64_t n) {
    if (!c || n < 0) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK(c, cudaSetDevice(c->dev));
    int rc = poll_checks(c, false);
    if (rc != LBD_OK) return rc;
    if (c->flagged) return c->flagged;
    if (n == 0) return LBD_OK;
    lbd::NvtxRange range("lbd_step");
    rc = c->params.precision == LBD_FP64 ? run_steps<double>(c, n) : run_steps<float>(c, n);
    if (rc != LBD_OK) return rc;
    rc = poll_checks(c, false);
    if (rc != LBD_OK) return rc;
    return c->flagged;
}

int lbd_set_check(lbd_ctx *c, int64_t every) {
    if (!c || every < 0) return LBD_EINVAL;
    c->check_every = every;
    return LBD_OK;
}

}  // extern "C"

namespace {
// Fields of the current state (rho, ux, uy, phi, psi: dense doubles, Eq. 11 for
// u) into the device staging area, queued on the context's stream.
int eval_fields(lbd_ctx *c) {
    int rc = ensure_staging(c);
    if (rc != LBD_OK) return rc;
    CK(c, cudaSetDevice(c->dev));
    const size_t N = c->N;
    double *d = c->staging;
    if (c->params.precision == LBD_FP64) {
        StepArgs<double> a = make_args<double>(c);
        a.rho_f = d; a.ux_f = d + N; a.uy_f = d + 2 * N; a.phi_f = d + 3 * N; a.psi_f = d + 4 * N;
        CK(c, lbd::launch_step<double>(a, lbd::MODE_FIELDS, c->tile, c->stream));
    } else {
        StepArgs<float> a = make_args<float>(c);
        a.rho_f = d; a.ux_f = d + N; a.uy_f = d + 2 * N; a.phi_f = d + 3 * N; a.psi_f = d + 4 * N;
        CK(c, lbd::launch_step<float>(a, lbd::MODE_FIELDS, c->tile, c->stream));
    }
    return LBD_OK;
}

// Per-droplet sums (tracking, or the squirmer fit) of the current state for n
// references of `stride` doubles each (host); the n * DROP_SUMS results land in
// c->h_drop.  Synchronises.
int droplet_sums(lbd_ctx *c, int n, const double *ref, int stride, bool squirm) {
    int rc = eval_fields(c);
    if (rc != LBD_OK) return rc;
    const size_t m = (size_t)LBD_MAX_DROPLETS * lbd::DROP_SUMS;
    if (!c->drop_dev) {
        if (lbd::dev_malloc((void **)&c->drop_dev, sizeof(double) * (m * (RED_BLOCKS + 1) + 4 * LBD_MAX_DROPLETS)) !=
                cudaSuccess ||
            lbd::host_malloc((void **)&c->h_drop, sizeof(double) * (m + 4 * LBD_MAX_DROPLETS)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->drop_dev);
            c->drop_dev = nullptr;
            return fail(c, LBD_ENOMEM, "droplet scratch allocation failed");
        }
    }
    double *partial = c->drop_dev, *out = partial + m * RED_BLOCKS, *dref = out + m;
    double *href = c->h_drop + m;
    for (int k = 0; k < n * stride; ++k) href[k] = ref[k];
    CK(c, cudaMemcpyAsync(dref, href, sizeof(double) * n * stride, cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, lbd::launch_droplet_sums(c->grid.nx, c->grid.ny, !(c->params.flags & LBD_WALLS),
                                   c->staging, n, dref, squirm, partial, RED_BLOCKS, out,
                                   c->stream));
    CK(c, cudaMemcpyAsync(c->h_drop, out, sizeof(double) * n * lbd::DROP_SUMS,
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}
}  // namespace

extern "C" {

int lbd_get_fields(lbd_ctx *c, double *rho, double *ux, double *uy, double *phi, double *psi) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    int rc = eval_fields(c);
    if (rc != LBD_OK) return rc;
    const size_t N = c->N;
    double *d = c->staging;
    double *outs[5] = {rho, ux, uy, phi, psi};
    for (int k = 0; k < 5; ++k)
        if (outs[k])
            CK(c, cudaMemcpyAsync(outs[k], d + k * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}

int lbd_get_fields_f32(lbd_ctx *c, float *rho, float *ux, float *uy, float *phi, float *psi) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (c->params.precision == LBD_FP32) {
        // phi and psi are the state itself: read back on the side stream while
        // rho and u are evaluated and read back on the context's stream
        int rc = ensure_side(c);
        if (rc != LBD_OK) return rc;
        CK(c, cudaSetDevice(c->dev));
        const size_t w = (size_t)c->grid.nx * sizeof(float), pb = (size_t)c->pitch * sizeof(float);
        const bool side = phi || psi;
        if (side) {
            CK(c, cudaEventRecord(c->ev_main, c->stream));
            CK(c, cudaStreamWaitEvent(c->side, c->ev_main, 0));
            if (phi)
                CK(c, cudaMemcpy2DAsync(phi, w, c->phi[c->cur], pb, w, c->grid.ny,
                                        cudaMemcpyDeviceToHost, c->side));
            if (psi)
                CK(c, cudaMemcpy2DAsync(psi, w, c->psi[c->cur], pb, w, c->grid.ny,
                                        cudaMemcpyDeviceToHost, c->side));
        }
        if (rho || ux || uy) {
            rc = eval_fields(c);
            if (rc == LBD_OK) rc = ensure_staging32(c);
            const size_t N = c->N;
            float *outs[3] = {rho, ux, uy};
            for (int k = 0; k < 3 && rc == LBD_OK; ++k)
                if (outs[k]) {
                    to_float_kernel<<<grid_for(N), 256, 0, c->stream>>>(
                        (long long)N, c->staging + k * N, c->staging32 + k * N);
                    if (cudaGetLastError() != cudaSuccess ||
                        cudaMemcpyAsync(outs[k], c->staging32 + k * N, N * sizeof(float),
                                        cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
                        rc = fail(c, LBD_ECUDA, "field read-back failed");
                }
        }
        // the caller's arrays are complete when this returns, on success or not
        if (side && cudaStreamSynchronize(c->side) != cudaSuccess && rc == LBD_OK)
            rc = fail(c, LBD_ECUDA, "field read-back failed");
        if (cudaStreamSynchronize(c->stream) != cudaSuccess && rc == LBD_OK)
            rc = fail(c, LBD_ECUDA, "field read-back failed");
        return rc;
    }
    int rc = eval_fields(c);
    if (rc == LBD_OK) rc = ensure_staging32(c);
    if (rc != LBD_OK) return rc;
    const size_t N = c->N;
    float *outs[5] = {rho, ux, uy, phi, psi};
    for (int k = 0; k < 5; ++k)
        if (outs[k]) {
            to_float_kernel<<<grid_for(N), 256, 0, c->stream>>>((long long)N, c->staging + k * N,
                                                              c->staging32 + k * N);
            CK(c, cudaGetLastError());
            CK(c, cudaMemcpyAsync(outs[k], c->staging32 + k * N, N * sizeof(float),
                                  cudaMemcpyDeviceToHost, c->stream));
        }
    CK(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}

int lbd_init_droplets(lbd_ctx *c, int32_t n, const lbd_droplet_init *d, double psi_bg, double xi,
                      uint64_t seed) {
    if (!c || !d) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (n < 1 || n > LBD_MAX_DROPLETS)
        return fail(c, LBD_EINVAL, "n must be in [1, %d]", LBD_MAX_DROPLETS);
    const lbd_params &p = c->params;
    if (!(p.a < 0) || !(p.b > 0)) return fail(c, LBD_EINVAL, "droplets need a < 0 < b");
    if (!std::isfinite(psi_bg) || !std::isfinite(xi)) return fail(c, LBD_EINVAL, "non-finite psi_bg or xi");
    // bounds of psi: inside |x - x0|, |y - y0| < R, so each ramp term is below |g|
    double lo = psi_bg, hi = psi_bg;
    DropInits D;
    for (int k = 0; k < n; ++k) {
        const lbd_droplet_init &q = d[k];
        const double v[7] = {q.x, q.y, q.R, q.psi_mean, q.psi_noise, q.gx, q.gy};
        for (double e : v)
            if (!std::isfinite(e)) return fail(c, LBD_EINVAL, "droplet %d: non-finite value", k);
        if (!(q.R > 0)) return fail(c, LBD_EINVAL, "droplet %d: R must be > 0", k);
        const double w = std::fabs(q.psi_noise) + std::fabs(q.gx) + std::fabs(q.gy);
        lo = std::min(lo, q.psi_mean - w);
        hi = std::max(hi, q.psi_mean + w);
        D.d[k] = q;
    }
    if (!(lo > 0) || !(p.B0 + p.B1 * lo > 0) || !(p.B0 + p.B1 * hi > 0))
        return fail(c, LBD_EUNSTABLE, "the droplets' psi range reaches psi <= 0 or B(psi) <= 0");
    const double kappa = p.B0 + p.B1 * psi_bg;
    const double w0 = xi > 0 ? xi : std::sqrt(2.0 * kappa / -p.a);
    if (!(w0 > 0)) return fail(c, LBD_EINVAL, "interface width must be > 0");
    CK(c, cudaSetDevice(c->dev));
    const size_t fbytes = (size_t)c->plane * c->esz;
    CK(c, cudaMemsetAsync(c->g[c->cur], 0, 9 * fbytes, c->stream));  // f = w_i: rho = 1, u = 0
    const int nb = grid_for(c->N);
    const double phieq = std::sqrt(-p.a / p.b);
    if (p.precision == LBD_FP64)
        init_droplets_kernel<double><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, n, D, phieq, w0, psi_bg, seed,
            (double *)c->phi[c->cur], (double *)c->psi[c->cur]);
    else
        init_droplets_kernel<float><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, n, D, phieq, w0, psi_bg, seed,
            (float *)c->phi[c->cur], (float *)c->psi[c->cur]);
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(c->stream));
    return reset_checks(c);
}

int lbd_get_fields_device(lbd_ctx *c, void *rho, void *ux, void *uy, void *phi, void *psi) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    int rc = eval_fields(c);
    if (rc != LBD_OK) return rc;
    void *outs[5] = {rho, ux, uy, phi, psi};
    const long long N = (long long)c->N;
    for (int k = 0; k < 5; ++k) {
        if (!outs[k]) continue;
        const double *src = c->staging + k * N;
        if (c->params.precision == LBD_FP64) {
            CK(c, cudaMemcpyAsync(outs[k], src, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                  c->stream));
        } else {
            to_float_kernel<<<grid_for(c->N), 256, 0, c->stream>>>(N, src, (float *)outs[k]);
            CK(c, cudaGetLastError());
        }
    }
    return LBD_OK;
}

int lbd_set_populations(lbd_ctx *c, const double *f) {
    if (!c || !f) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    const size_t n9 = 9 * c->N;
    for (size_t k = 0; k < n9; ++k)
        if (!std::isfinite(f[k])) return fail(c, LBD_ENONFINITE, "non-finite population %zu", k);
    CK(c, cudaSetDevice(c->dev));
    if (!c->pop_staging) {
        if (lbd::dev_malloc((void **)&c->pop_staging, 9 * c->N * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->pop_staging = nullptr;
            return fail(c, LBD_ENOMEM, "population staging allocation failed");
        }
    }
    CK(c, cudaMemcpyAsync(c->pop_staging, f, n9 * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
    const int nb = grid_for(c->N);
    const int walls = (c->params.flags & LBD_WALLS) ? 1 : 0;
    if (c->params.precision == LBD_FP64)
        set_populations_kernel<double><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, walls, c->pop_staging, (double *)c->g[c->cur]);
    else
        set_populations_kernel<float><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, walls, c->pop_staging, (float *)c->g[c->cur]);
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(c->stream));
    return reset_checks(c);
}

int lbd_get_populations(lbd_ctx *c, double *f) {
    if (!c || !f) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK(c, cudaSetDevice(c->dev));
    if (!c->pop_staging) {
        if (lbd::dev_malloc((void **)&c->pop_staging, 9 * c->N * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->pop_staging = nullptr;
            return fail(c, LBD_ENOMEM, "population staging allocation failed");
        }
    }
    const int nb = grid_for(c->N);
    if (c->params.precision == LBD_FP64)
        populations_kernel<double><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, (c->params.flags & LBD_WALLS) ? 1 : 0,
            (const double *)c->g[c->cur], c->pop_staging);
    else
        populations_kernel<float><<<nb, 256, 0, c->stream>>>(
            c->grid.nx, c->grid.ny, c->pitch, c->plane, (c->params.flags & LBD_WALLS) ? 1 : 0,
            (const float *)c->g[c->cur], c->pop_staging);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(f, c->pop_staging, 9 * c->N * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBD_OK;
}

int lbd_diagnostics(lbd_ctx *c, double refx, double refy, lbd_diag *out) {
    if (!c || !out) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (!(refx >= 0 && refx < c->grid.nx && refy >= 0 && refy < c->grid.ny))
        return fail(c, LBD_EINVAL, "reference point outside the lattice");
    lbd::NvtxRange range("lbd_diagnostics");
    CK(c, cudaSetDevice(c->dev));
    const lbd_params &p = c->params;
    CK(c, launch_reduce(p.precision, c->grid.nx, c->grid.ny, c->pitch, c->plane, c->g[c->cur],
                        c->phi[c->cur], c->psi[c->cur], p.B0, p.B1, refx, refy, c->red_partial,
                        c->red_out, c->stream));
    CK(c, cudaMemcpyAsync(c->h_red, c->red_out, NRED * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double *r = c->h_red;
    out->sum_rho = (double)c->N + r[0];
    out->sum_phi = r[1];
    out->sum_psi = r[2];
    out->mass_pos = r[5];
    out->cm_x = r[5] > 0 ? refx + r[3] / r[5] : NAN;
    out->cm_y = r[5] > 0 ? refy + r[4] / r[5] : NAN;
    out->min_B = r[6];
    out->min_psi = r[7];
    out->nonfinite = (int64_t)r[8];
    if (out->nonfinite > 0)
        return fail(c, LBD_ENONFINITE, "%lld sites hold a non-finite value",
                    (long long)out->nonfinite);
    if (!(out->min_B > 0) || !(out->min_psi > 0))
        return fail(c, LBD_EUNSTABLE, "min B(psi) = %g, min psi = %g", out->min_B, out->min_psi);
    return LBD_OK;
}

int lbd_droplets(lbd_ctx *c, int32_t n, const double *ref_xy, lbd_droplet *out) {
    if (!c || !ref_xy || !out) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (n < 1 || n > LBD_MAX_DROPLETS)
        return fail(c, LBD_EINVAL, "n must be in [1, %d]", LBD_MAX_DROPLETS);
    const int nx = c->grid.nx, ny = c->grid.ny;
    for (int k = 0; k < n; ++k)
        if (!(ref_xy[2 * k] >= 0 && ref_xy[2 * k] < nx && ref_xy[2 * k + 1] >= 0 &&
              ref_xy[2 * k + 1] < ny))
            return fail(c, LBD_EINVAL, "reference point %d outside the lattice", k);
    int rc = droplet_sums(c, n, ref_xy, 2, false);
    if (rc != LBD_OK) return rc;
    const bool walls = (c->params.flags & LBD_WALLS) != 0;
    for (int k = 0; k < n; ++k) {
        const double *a = c->h_drop + k * lbd::DROP_SUMS;
        lbd_droplet &d = out[k];
        d.mass = a[0];
        d.sites = (int64_t)a[5];
        if (a[0] > 0) {
            double x = std::fmod(ref_xy[2 * k] + a[1] / a[0], (double)nx);
            double y = ref_xy[2 * k + 1] + a[2] / a[0];
            if (x < 0) x += nx;
            if (!walls) {
                y = std::fmod(y, (double)ny);
                if (y < 0) y += ny;
            }
            d.x = x;
            d.y = y;
            d.ux = a[3] / a[0];
            d.uy = a[4] / a[0];
        } else {
            d.x = d.y = d.ux = d.uy = NAN;
        }
    }
    return LBD_OK;
}

int lbd_squirmer(lbd_ctx *c, int32_t n, const lbd_droplet *drops, double *b1, double *b2,
                 int64_t *points) {
    if (!c || !drops || !b1 || !b2) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (n < 1 || n > LBD_MAX_DROPLETS)
        return fail(c, LBD_EINVAL, "n must be in [1, %d]", LBD_MAX_DROPLETS);
    double cen[4 * LBD_MAX_DROPLETS];
    for (int k = 0; k < n; ++k) {
        const lbd_droplet &d = drops[k];
        if (!std::isfinite(d.x) || !std::isfinite(d.y) || !std::isfinite(d.ux) ||
            !std::isfinite(d.uy))
            return fail(c, LBD_EINVAL, "droplet %d has a non-finite centre or velocity", k);
        cen[4 * k] = d.x;
        cen[4 * k + 1] = d.y;
        cen[4 * k + 2] = d.ux;
        cen[4 * k + 3] = d.uy;
    }
    int rc = droplet_sums(c, n, cen, 4, true);
    if (rc != LBD_OK) return rc;
    for (int k = 0; k < n; ++k) {
        // normal equations [S11 S12; S12 S22] (b1, b2) = (U1, U2)
        const double *a = c->h_drop + k * lbd::DROP_SUMS;
        const double det = a[0] * a[2] - a[1] * a[1];
        if (a[5] >= 2 && det != 0.0) {
            b1[k] = (a[3] * a[2] - a[4] * a[1]) / det;
            b2[k] = (a[0] * a[4] - a[1] * a[3]) / det;
        } else {
            b1[k] = b2[k] = NAN;
        }
        if (points) points[k] = (int64_t)a[5];
    }
    return LBD_OK;
}

int lbd_set_tile(lbd_ctx *c, int32_t bx, int32_t by) {
    if (!c) return LBD_EINVAL;
    const Tile t{bx, by};
    if (!tile_ok(c, t))
        return fail(c, LBD_EINVAL, "launch shape %dx%d is not available for this precision and lattice",
                    bx, by);
    c->tile = t;
    return LBD_OK;
}

int lbd_autotune(lbd_ctx *c, int32_t reps, int32_t *bx, int32_t *by) {
    if (!c || reps < 1) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK(c, cudaSetDevice(c->dev));
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    float best = 1e30f;
    Tile keep = c->tile;
    int rc = LBD_OK;
    for (int k = 0; k < lbd::n_tiles() && rc == LBD_OK; ++k) {
        const Tile t = lbd::tile_at(k);
        if (!tile_ok(c, t)) continue;
        // The trial launches read the current buffers and write the others; the
        // buffers are not swapped, so the state and t are unchanged.
        auto launch = [&]() -> cudaError_t {
            if (c->params.precision == LBD_FP64) {
                StepArgs<double> a = make_args<double>(c);
                return lbd::launch_step<double>(a, lbd::MODE_STEP, t, c->stream);
            }
            StepArgs<float> a = make_args<float>(c);
            return lbd::launch_step<float>(a, lbd::MODE_STEP, t, c->stream);
        };
        cudaError_t e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(c, LBD_ECUDA, "autotune: %s", cudaGetErrorString(e));
            break;
        }
        if (ms < best) {
            best = ms;
            keep = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBD_OK) return rc;
    c->tile = keep;
    if (bx) *bx = keep.bx;
    if (by) *by = keep.by;
    return LBD_OK;
}

int lbd_tiles(int32_t *bx, int32_t *by, int32_t cap) {
    const int n = lbd::n_tiles();
    for (int k = 0; k < n && k < cap; ++k) {
        if (bx) bx[k] = lbd::tile_at(k).bx;
        if (by) by[k] = lbd::tile_at(k).by;
    }
    return n;
}

int lbd_diagnostics_static(int32_t nx, int32_t ny, int64_t pitch, int32_t precision,
                           const void *g, const void *phi, const void *psi, double B0, double B1,
                           double ref_x, double ref_y, void *stream, lbd_diag *out) {
    if (!g || !phi || !psi || !out) return LBD_EINVAL;
    if (nx < 1 || ny < 1 || nx > (1 << 20) || ny > (1 << 20) || pitch < nx) return LBD_EINVAL;
    // the nine planes span 9 * pitch * ny elements: keep every index in range
    if (pitch > (int64_t(1) << 40) || 9.0 * (double)pitch * (double)ny >= 0x1p52) return LBD_EINVAL;
    if (precision != LBD_FP64 && precision != LBD_FP32) return LBD_EINVAL;
    if (!(ref_x >= 0 && ref_x < nx && ref_y >= 0 && ref_y < ny)) return LBD_EINVAL;
    // a host pointer or another GPU's buffer would fault the kernel: refuse it
    if (!on_current_device(g) || !on_current_device(phi) || !on_current_device(psi))
        return LBD_EINVAL;
    double *scratch = nullptr;
    if (static_scratch(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return LBD_ECUDA;
    }
    double *partial = scratch, *res = scratch + NRED * RED_BLOCKS + 1;
    cudaStream_t s = (cudaStream_t)stream;
    const long long plane = (long long)pitch * ny;
    if (launch_reduce(precision, nx, ny, pitch, plane, g, phi, psi, B0, B1, ref_x, ref_y, partial,
                      res, s) != cudaSuccess)
        return LBD_ECUDA;
    double r[NRED];
    if (cudaMemcpyAsync(r, res, sizeof r, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return LBD_ECUDA;
    }
    out->sum_rho = (double)nx * (double)ny + r[0];
    out->sum_phi = r[1];
    out->sum_psi = r[2];
    out->mass_pos = r[5];
    out->cm_x = r[5] > 0 ? ref_x + r[3] / r[5] : NAN;
    out->cm_y = r[5] > 0 ? ref_y + r[4] / r[5] : NAN;
    out->min_B = r[6];
    out->min_psi = r[7];
    out->nonfinite = (int64_t)r[8];
    if (out->nonfinite > 0) return LBD_ENONFINITE;
    if (!(out->min_B > 0) || !(out->min_psi > 0)) return LBD_EUNSTABLE;
    return LBD_OK;
}

int lbd_adjoint(lbd_ctx *c, int64_t nsteps, int32_t ckpt_every, double ref_x, double *loss,
                double *dL_dpsi0, double *dL_dB1) {
    lbd::NvtxRange range("lbd_adjoint");
    if (!c || !loss || !dL_dB1) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    if (nsteps < 1 || ckpt_every < 1) return fail(c, LBD_EINVAL, "nsteps and ckpt_every must be >= 1");
    if (!(ref_x >= 0 && ref_x < c->grid.nx)) return fail(c, LBD_EINVAL, "ref_x outside the lattice");
    if (c->params.flags & LBD_FROZEN_U)
        return fail(c, LBD_EINVAL, "the adjoint is defined for the coupled velocity only");
    if (c->params.flags & LBD_WALLS)
        return fail(c, LBD_EINVAL, "the adjoint is defined for periodic lattices only");
    CK(c, cudaSetDevice(c->dev));
    const int64_t K = ckpt_every < nsteps ? ckpt_every : nsteps;
    return c->params.precision == LBD_FP64
               ? adjoint_impl<double>(c, nsteps, (int32_t)K, ref_x, loss, dL_dpsi0, dL_dB1)
               : adjoint_impl<float>(c, nsteps, (int32_t)K, ref_x, loss, dL_dpsi0, dL_dB1);
}


void lbd_batch_destroy(lbd_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (lbd_ctx *c : b->ctx) lbd_destroy(c);
    cudaFree(b->args_dev[0]);
    cudaFree(b->args_dev[1]);
    cudaFree(b->items_dev);
    cudaFree(b->t_dev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int lbd_batch_create(int32_t n, const lbd_grid *grids, const lbd_params *params, void *stream,
                     lbd_batch **out) {
    if (!out || !grids || !params || n < 1) return LBD_EINVAL;
    *out = nullptr;
    for (int k = 0; k < n; ++k)
        if (params[k].precision != params[0].precision) return LBD_EINVAL;
    lbd_batch *b = new (std::nothrow) lbd_batch();
    if (!b) return LBD_ENOMEM;
    b->n = n;
    b->prec = params[0].precision;
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return LBD_ECUDA;
        }
        b->own_stream = true;
    }
    for (int k = 0; k < n; ++k) {
        lbd_ctx *c = nullptr;
        const int rc = lbd_create(&grids[k], &params[k], b->stream, &c);
        if (rc != LBD_OK) {
            lbd_batch_destroy(b);
            return rc;
        }
        b->ctx.push_back(c);
    }
    for (lbd_ctx *c : b->ctx)
        if (!lbd::tile_valid(b->tile, b->prec == LBD_FP32, c->grid.nx, c->plane)) {
            lbd_batch_destroy(b);
            return LBD_EINVAL;
        }
    // FP32 batches whose periodic instances are all 4k wide start on the 16-byte
    // staged stripe kernel (lbd_batch_autotune refines the choice)
    if (b->prec == LBD_FP32) {
        bool all = true;
        for (lbd_ctx *c : b->ctx)
            if (!(c->params.flags & LBD_WALLS))
                all &= lbd::tile_valid(Tile{116, 64}, true, c->grid.nx, c->plane);
        if (all) b->tile = Tile{116, 64};
    }
    if (lbd::dev_malloc((void **)&b->t_dev, sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        lbd_batch_destroy(b);
        return LBD_ENOMEM;
    }
    const int rc = b->prec == LBD_FP64 ? batch_build<double>(b) : batch_build<float>(b);
    if (rc != LBD_OK) {
        lbd_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBD_OK;
}

const char *lbd_batch_last_error(const lbd_batch *b) { return b ? b->msg.c_str() : ""; }

int lbd_batch_set_fields(lbd_batch *b, int32_t k, const double *rho, const double *ux,
                         const double *uy, const double *phi, const double *psi) {
    if (!b || k < 0 || k >= b->n) return LBD_EINVAL;
    const int rc = lbd_set_fields(b->ctx[k], rho, ux, uy, phi, psi);
    if (rc != LBD_OK) bfail(b, rc, "instance %d: %s", k, b->ctx[k]->msg.c_str());
    return rc;
}

int lbd_batch_get_fields(lbd_batch *b, int32_t k, double *rho, double *ux, double *uy,
                         double *phi, double *psi) {
    if (!b || k < 0 || k >= b->n) return LBD_EINVAL;
    return lbd_get_fields(b->ctx[k], rho, ux, uy, phi, psi);
}

int lbd_batch_diagnostics(lbd_batch *b, int32_t k, double ref_x, double ref_y, lbd_diag *out) {
    if (!b || k < 0 || k >= b->n) return LBD_EINVAL;
    return lbd_diagnostics(b->ctx[k], ref_x, ref_y, out);
}

int lbd_batch_step(lbd_batch *b, int64_t nsteps) {
    if (!b || nsteps < 0) return LBD_EINVAL;
    if (b->sticky) return b->sticky;
    if (nsteps == 0) return LBD_OK;
    BCK(b, cudaSetDevice(b->ctx[0]->dev));
    return b->prec == LBD_FP64 ? batch_run<double>(b, nsteps) : batch_run<float>(b, nsteps);
}

int lbd_batch_set_tile(lbd_batch *b, int32_t bx, int32_t by) {
    if (!b) return LBD_EINVAL;
    if (!((bx == 118 || bx == 246 || bx == 116) && (by == 32 || by == 64 || by == 128)))
        return bfail(b, LBD_EINVAL,
                     "batched steps use a stripe kernel: bx 116, 118 or 246, by 32, 64 or 128");
    for (lbd_ctx *c : b->ctx) {
        // instances with plates run the 118-column stripe kernel under bx 116
        const bool walls = (c->params.flags & LBD_WALLS) != 0;
        const Tile t{bx == 116 && walls ? 118 : bx, by};
        if (!lbd::tile_valid(t, b->prec == LBD_FP32, c->grid.nx, c->plane))
            return bfail(b, LBD_EINVAL, "launch shape %dx%d is not valid for an instance", bx, by);
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    b->tile = Tile{bx, by};
    return b->prec == LBD_FP64 ? batch_build<double>(b) : batch_build<float>(b);
}

int lbd_batch_autotune(lbd_batch *b, int32_t reps, int32_t *bx, int32_t *by) {
    if (!b || reps < 1) return LBD_EINVAL;
    if (b->sticky) return b->sticky;
    const Tile cand[] = {{118, 32}, {118, 64}, {118, 128}, {246, 32}, {246, 64},
                         {116, 32}, {116, 64}, {116, 96},  {116, 128}};
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    float best = 1e30f;
    Tile keep = b->tile;
    int rc = LBD_OK;
    for (const Tile &t : cand) {
        rc = lbd_batch_set_tile(b, t.bx, t.by);
        if (rc == LBD_EINVAL) {  // not valid for these instances (e.g. 116 with FP64)
            rc = LBD_OK;
            continue;
        }
        if (rc != LBD_OK) break;
        // trial launches read the current buffers and write the others: no state change
        const int parity = b->ctx[0]->cur;
        cudaError_t e = cudaSuccess;
        e = lbd::launch_time_set(b->t_dev, (long long)b->t, b->stream);
        auto go = [&]() {
            return b->prec == LBD_FP64 ? batch_launch<double>(b, parity, 0)
                                       : batch_launch<float>(b, parity, 0);
        };
        if (e == cudaSuccess) e = go();
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = go();
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = bfail(b, LBD_ECUDA, "batch autotune: %s", cudaGetErrorString(e));
            break;
        }
        if (ms < best) {
            best = ms;
            keep = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBD_OK) return rc;
    rc = lbd_batch_set_tile(b, keep.bx, keep.by);
    if (bx) *bx = keep.bx;
    if (by) *by = keep.by;
    return rc;
}

int lbd_batch_get_tile(const lbd_batch *b, int32_t *bx, int32_t *by) {
    if (!b) return LBD_EINVAL;
    if (bx) *bx = b->tile.bx;
    if (by) *by = b->tile.by;
    return LBD_OK;
}

int lbd_get_tile(const lbd_ctx *c, int32_t *bx, int32_t *by) {
    if (!c) return LBD_EINVAL;
    if (bx) *bx = c->tile.bx;
    if (by) *by = c->tile.by;
    return LBD_OK;
}

int lbd_batch_synchronize(lbd_batch *b) {
    if (!b) return LBD_EINVAL;
    if (b->sticky) return b->sticky;
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBD_OK;
}

int lbd_batch_get_time(const lbd_batch *b, int64_t *t) {
    if (!b || !t) return LBD_EINVAL;
    *t = b->t;
    return LBD_OK;
}

int lbd_get_time(const lbd_ctx *c, int64_t *t) {
    if (!c || !t) return LBD_EINVAL;
    *t = c->t;
    return LBD_OK;
}

int lbd_set_time(lbd_ctx *c, int64_t t) {
    if (!c) return LBD_EINVAL;
    c->t = t;
    return LBD_OK;
}

int lbd_synchronize(lbd_ctx *c) {
    if (!c) return LBD_EINVAL;
    if (c->sticky) return c->sticky;
    CK(c, cudaSetDevice(c->dev));
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaGetLastError());
    const int rc = poll_checks(c, true);
    if (rc != LBD_OK) return rc;
    return c->flagged;
}

int lbd_debug_fail_alloc(int32_t nth) {
    if (nth < 0) return LBD_EINVAL;
    g_fail_countdown.store(nth);
    return LBD_OK;
}

}  // extern "C"

// lbd_droplets.cu -- per-droplet tracking and the squirmer fit of Section 4
// (arXiv 1711.10984, Eq. 21) on the dense double fields of the fields
// evaluation (rho, u_x, u_y, phi, psi; site y * nx + x).
//
// Tracking: every site with phi >= 0 belongs to the nearest reference point
// (minimum image in x, and in y unless plates bound the lattice; ties to the
// lower index) and adds phi, phi * (displacement from the reference), phi * u
// and 1 to that droplet's sums.
//
// Squirmer fit: the phi = 0 contour is sampled where phi changes sign along a
// lattice link (x to x+1 and y to y+1, none through a plate), the point and its
// velocity interpolated linearly along the link; each point belongs to the
// nearest droplet centre.  In the droplet frame (u - U), with theta from the
// swimming direction e = U / |U| towards e_perp = z x e, the polar component is
// u_theta = (u - U) . (-sin(theta) e + cos(theta) e_perp); the point adds to the
// normal equations of the least-squares fit u_theta = b1 s + b2 s c (s, c =
// sin, cos theta): sums s^2, s^2 c, s^2 c^2, u_theta s, u_theta s c and 1.
//
// Both reductions accumulate per block in shared memory (double atomics, so
// the order inside a block is not fixed) and then over blocks in a fixed order.
#include <cstdint>

#include "lbd_internal.h"

namespace lbd {
namespace {

__device__ __forceinline__ double min_image(double d, int n) {
    if (d > 0.5 * n) return d - n;
    if (d < -0.5 * n) return d + n;
    return d;
}

__device__ __forceinline__ int nearest(double x, double y, int n, const double *ref, int stride,
                                       int nx, int ny, int wrap_y) {
    int best = 0;
    double bd = 1e300;
    for (int k = 0; k < n; ++k) {
        const double dx = min_image(x - ref[k * stride], nx);
        const double dy = wrap_y ? min_image(y - ref[k * stride + 1], ny) : y - ref[k * stride + 1];
        const double d2 = dx * dx + dy * dy;
        if (d2 < bd) {
            bd = d2;
            best = k;
        }
    }
    return best;
}

__global__ void drop_partial(int nx, int ny, int wrap_y, const double *ux, const double *uy,
                             const double *phi, int n, const double *ref, double *partial) {
    extern __shared__ double acc[];  // [n][DROP_SUMS]
    for (int j = threadIdx.x; j < n * DROP_SUMS; j += blockDim.x) acc[j] = 0.0;
    __syncthreads();
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const double p = phi[s];
        if (!(p >= 0.0)) continue;
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        const int k = nearest(x, y, n, ref, 2, nx, ny, wrap_y);
        const double dx = min_image(x - ref[2 * k], nx);
        const double dy = wrap_y ? min_image(y - ref[2 * k + 1], ny) : y - ref[2 * k + 1];
        double *a = acc + k * DROP_SUMS;
        atomicAdd(a + 0, p);
        atomicAdd(a + 1, p * dx);
        atomicAdd(a + 2, p * dy);
        atomicAdd(a + 3, p * ux[s]);
        atomicAdd(a + 4, p * uy[s]);
        atomicAdd(a + 5, 1.0);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n * DROP_SUMS; j += blockDim.x)
        partial[(long long)blockIdx.x * n * DROP_SUMS + j] = acc[j];
}

// one interface point (x, y) with velocity (u, v): its droplet's fit sums
__device__ __forceinline__ void squirm_point(double x, double y, double u, double v, int n,
                                             const double *cen, int nx, int ny, int wrap_y,
                                             double *acc) {
    const int k = nearest(x, y, n, cen, 4, nx, ny, wrap_y);
    const double *c = cen + 4 * k;
    const double dx = min_image(x - c[0], nx);
    const double dy = wrap_y ? min_image(y - c[1], ny) : y - c[1];
    const double U = c[2], V = c[3];
    const double sp = sqrt(U * U + V * V);
    const double ex = sp > 0.0 ? U / sp : 1.0, ey = sp > 0.0 ? V / sp : 0.0;
    const double px = -ey, py = ex;  // e_perp
    const double r = sqrt(dx * dx + dy * dy);
    const double cs = (dx * ex + dy * ey) / r, sn = (dx * px + dy * py) / r;
    const double wx = u - U, wy = v - V;
    const double ut = wx * (-sn * ex + cs * px) + wy * (-sn * ey + cs * py);
    const double g1 = sn, g2 = sn * cs;  // columns of the design matrix
    double *a = acc + k * DROP_SUMS;
    atomicAdd(a + 0, g1 * g1);
    atomicAdd(a + 1, g1 * g2);
    atomicAdd(a + 2, g2 * g2);
    atomicAdd(a + 3, ut * g1);
    atomicAdd(a + 4, ut * g2);
    atomicAdd(a + 5, 1.0);
}

__global__ void squirm_partial(int nx, int ny, int wrap_y, const double *ux, const double *uy,
                               const double *phi, int n, const double *cen, double *partial) {
    extern __shared__ double acc[];  // [n][DROP_SUMS]
    for (int j = threadIdx.x; j < n * DROP_SUMS; j += blockDim.x) acc[j] = 0.0;
    __syncthreads();
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
        const double a = phi[s];
        // link to x + 1 (periodic)
        {
            const long long q = (long long)y * nx + (x + 1 < nx ? x + 1 : 0);
            const double b = phi[q];
            if ((a >= 0.0) != (b >= 0.0)) {
                const double t = a / (a - b);
                squirm_point(x + t, y, (1 - t) * ux[s] + t * ux[q], (1 - t) * uy[s] + t * uy[q],
                             n, cen, nx, ny, wrap_y, acc);
            }
        }
        // link to y + 1 (periodic unless a plate is in between)
        if (y + 1 < ny || wrap_y) {
            const long long q = (long long)(y + 1 < ny ? y + 1 : 0) * nx + x;
            const double b = phi[q];
            if ((a >= 0.0) != (b >= 0.0)) {
                const double t = a / (a - b);
                squirm_point(x, y + t, (1 - t) * ux[s] + t * ux[q], (1 - t) * uy[s] + t * uy[q],
                             n, cen, nx, ny, wrap_y, acc);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n * DROP_SUMS; j += blockDim.x)
        partial[(long long)blockIdx.x * n * DROP_SUMS + j] = acc[j];
}

// out[j] = sum over blocks of partial[b][j], blocks in order
__global__ void drop_final(int nblocks, int m, const double *partial, double *out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partial[(long long)b * m + j];
        out[j] = v;
    }
}

}  // namespace

cudaError_t launch_droplet_sums(int nx, int ny, bool wrap_y, const double *fields, int n,
                                const double *ref, bool squirm, double *partial, int nblocks,
                                double *out, cudaStream_t s) {
    const long long N = (long long)nx * ny;
    const double *ux = fields + N, *uy = fields + 2 * N, *phi = fields + 3 * N;
    const size_t smem = sizeof(double) * (size_t)n * DROP_SUMS;
    if (squirm)
        squirm_partial<<<nblocks, 256, smem, s>>>(nx, ny, wrap_y ? 1 : 0, ux, uy, phi, n, ref,
                                                  partial);
    else
        drop_partial<<<nblocks, 256, smem, s>>>(nx, ny, wrap_y ? 1 : 0, ux, uy, phi, n, ref,
                                                partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    drop_final<<<(n * DROP_SUMS + 127) / 128, 128, 0, s>>>(nblocks, n * DROP_SUMS, partial, out);
    return cudaGetLastError();
}

}  // namespace lbd

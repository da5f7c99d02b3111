// lbd_internal.h -- device-side argument blocks and launcher declarations shared
// by the kernels (lbd_step.cu, lbd_aux.cu) and the C ABI (lbd_api.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lbd.h"

namespace lbd {

// NVTX range over a host scope (header-only NVTX v3: free when no tool is
// attached); names the library's phases in Nsight timelines.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Arguments of the fused coupled-step kernel.  Arrays are pitched: site (x, y)
// at y*pitch + x, population i at offset i*plane with plane = pitch*ny.
// Populations are stored as deviations g_i = f_i - w_i from the rest weights,
// in the pull layout: buffer_i(x) holds the post-collision value that site
// x + e_i reads at the next step.
template <typename T>
struct StepArgs {
    int nx, ny;
    long long pitch, plane;
    const T *g_in;
    T *g_out;
    const T *phi_in, *psi_in;
    T *phi_out, *psi_out;
    // fields mode: dense double outputs (index y*nx + x)
    double *rho_f, *ux_f, *uy_f, *phi_f, *psi_f;
    // model
    T a, b, B0, B1, M, D, omega, guo;  // omega = 1/tau, guo = 1 - 1/(2 tau)
    T gamma, c0, A;                    // activity at this step
    T fx, fy, ux0, uy0;
    uint32_t flags;
    // Source indicator Theta as a bit mask: bit (x & 31) of word y*theta_words + x/32
    // (all zero when there is no source).
    const uint32_t *theta;
    int theta_words;
    // Activity schedule, used by the batched kernel, which reads the step count
    // from device memory: A(t) = min(A0 (t - t_on), A_max), gamma(t) = gamma_on
    // for t >= t_on, both 0 before.
    double A0, A_max;
    long long t_on;
    double gamma_on;
};

// Work item of the batched step: instance, first output column, first row, rows.
struct BatchItem {
    int k, x0, y0, rows;
};

enum { MODE_STEP = 0, MODE_FIELDS = 1 };

// Launch shape of the step: bx output columns by by output rows per CTA.
//   bx in {32, 64}:   tiled kernel (lbd_step.cu), bx x by tiles;
//   bx in {118, 246}: stripe-marching kernel (lbd_stripe.cu), bx + 10 threads,
//                     segments of by rows;
//   bx == 116:        FP32 stripe kernel with 16-byte population staging
//                     (lbd_vstripe.cu), 128 threads, segments of at most by
//                     rows, shorter (down to by / 2) where that fills the
//                     resident CTA slots evenly (periodic lattices with
//                     nx % 4 == 0 only).
struct Tile {
    int bx, by;
};

// Whether a launch shape can run a step of this precision on an nx-wide lattice
// whose population planes hold `plane` elements (the stripe kernels address the
// nine planes with 32-bit byte offsets).
bool tile_valid(Tile t, bool fp32, int nx, long long plane);

// Launch one coupled step (mode MODE_STEP) or the fields evaluation
// (MODE_FIELDS) with tile shape `tile`; returns the launch error.
template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, int mode, Tile tile, cudaStream_t s);

// Launch one coupled step with the stripe-marching kernel (nt threads, seg rows).
template <typename T>
cudaError_t launch_stripe(const StepArgs<T> &a, int nt, int seg, cudaStream_t s);

template <typename T>
size_t stripe_smem_bytes(int nt);

// One step of the instances of a batch that share one variant (walls false:
// periodic; true: with plates): a persistent grid of ctas CTAs walks the n_items
// work items; instance k reads its arguments from args[k]; the step count of
// this launch is *t_dev + t_off.
template <typename T>
cudaError_t launch_stripe_batch(const StepArgs<T> *args, const BatchItem *items, int n_items,
                                int nt, bool walls, int ctas, const long long *t_dev, int t_off,
                                cudaStream_t s);

// Resident CTAs per SM of the batched kernel (occupancy calculator).
template <typename T>
int stripe_batch_ctas_per_sm(int nt);

// t_dev += add (one thread)
cudaError_t launch_time_advance(long long *t_dev, long long add, cudaStream_t s);
cudaError_t launch_time_set(long long *t_dev, long long value, cudaStream_t s);

// FP32 stripe kernel with 16-byte population row staging (lbd_vstripe.cu):
// periodic lattices with nx % 4 == 0 whose nine planes fit 32-bit byte offsets.
bool vstripe_supported(int nx, long long plane);
size_t vstripe_smem_bytes();
cudaError_t launch_vstripe(const StepArgs<float> &a, int seg, cudaStream_t s);
// The batched form (periodic FP32 instances; items 116 columns wide) and its
// resident CTAs per SM.
cudaError_t launch_vstripe_batch(const StepArgs<float> *args, const BatchItem *items, int n_items,
                                 int ctas, const long long *t_dev, int t_off, cudaStream_t s);
int vstripe_batch_ctas_per_sm();


// Per-droplet sums (lbd_droplets.cu) on the dense fields of the fields
// evaluation (5 arrays of nx*ny doubles: rho, ux, uy, phi, psi).  Tracking
// (squirm false): ref holds n (x, y) reference points; per droplet sum phi,
// sum phi dx, sum phi dy, sum phi ux, sum phi uy, sites.  Squirmer fit (squirm
// true): ref holds n (x, y, ux, uy) centres; per droplet sum s^2, sum s^2 c,
// sum s^2 c^2, sum u_theta s, sum u_theta s c, points.  partial holds
// nblocks * n * DROP_SUMS doubles; out receives n * DROP_SUMS.
constexpr int DROP_SUMS = 6;
cudaError_t launch_droplet_sums(int nx, int ny, bool wrap_y, const double *fields, int n,
                                const double *ref, bool squirm, double *partial, int nblocks,
                                double *out, cudaStream_t s);

// Fill the source indicator bit mask (words per row = (nx + 31) / 32) for the
// disks (x, y, R) with the exact inclusive double-precision test, periodic in
// x and, if wrap_y, in y.
cudaError_t launch_theta_mask(int nx, int ny, int n_src, const lbd_source *src, bool wrap_y,
                              uint32_t *mask, cudaStream_t s);

// Activity at step t (Section 4): off before t_on, then the sink rate gamma and
// the source strength A(t) = min(A0 (t - t_on), A_max).
inline void activity_at(const lbd_params &p, int64_t t, double *A, double *gamma) {
    if (t < p.t_on) {
        *A = 0.0;
        *gamma = 0.0;
        return;
    }
    const double a = p.A0 * (double)(t - p.t_on);
    *A = a < p.A_max ? a : p.A_max;
    *gamma = p.gamma;
}

// One adjoint computation (lbd_adjoint): the state at t0 is read from g0, phi0,
// psi0; the state at t0 + nsteps is written to the *_final buffers (which may
// alias the inputs).
template <typename T>
struct AdjointJob {
    int nx, ny;
    long long pitch, plane;
    StepArgs<T> args;  // model arguments of the step kernel; buffers are replaced
    Tile tile;
    cudaStream_t stream;
    const lbd_params *params;
    const T *g0, *phi0, *psi0;
    T *g_final, *phi_final, *psi_final;
    int64_t t0, nsteps, ckpt_every;
    double refx;
    double a, b, B0, B1, M, D, tau, c0, fx, fy;
    int body;
    double *loss, *dB1, *dpsi_host;
};

template <typename T>
int adjoint_run(const AdjointJob<T> &job);

// Shared memory bytes the fused kernel needs for a tile shape.
template <typename T>
size_t step_smem_bytes(Tile tile);

// Every device and pinned-host allocation of the library goes through these,
// so that the test hook lbd_debug_fail_alloc can make the n-th one fail as if
// the memory were exhausted (cudaErrorMemoryAllocation, nothing allocated).
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t host_malloc(void **p, size_t bytes);

// Tile shapes compiled into the library.
int n_tiles();
Tile tile_at(int k);

}  // namespace lbd

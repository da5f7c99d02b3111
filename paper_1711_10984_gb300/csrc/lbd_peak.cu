// lbd_peak.cu -- measurement support: the FP64 FMA rate of the device the
// library runs on, the denominator of the FP64 step's ALU roofline (the FP64
// form of the coupled step is bound by the FP64 pipe, not by HBM).
#include <cstdint>

#include "lbd_internal.h"

namespace {

constexpr int PEAK_CHAINS = 8;   // independent FMA chains per thread
constexpr int PEAK_THREADS = 256;

// Each thread runs PEAK_CHAINS independent chains a <- a * b + c for iters
// rounds (2 flops per FMA); the final values are written out so that nothing
// is optimised away.
__global__ void __launch_bounds__(PEAK_THREADS) fp64_fma_kernel(int iters, double b, double c,
                                                                 double *out) {
    double a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int lbd_fp64_peak(int32_t iters, double *flops_per_s) {
    if (!flops_per_s || iters < 1) return LBD_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBD_ECUDA;
    }
    const int blocks = sms * 8;
    double *out = nullptr;
    if (lbd::dev_malloc((void **)&out, sizeof(double) * blocks * PEAK_THREADS) != cudaSuccess) {
        cudaGetLastError();
        return LBD_ENOMEM;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBD_OK;
    float ms = 0.f;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = LBD_ECUDA;
    } else {
        // b slightly below 1 keeps the chains finite for any iteration count
        fp64_fma_kernel<<<blocks, PEAK_THREADS, 0, s>>>(iters / 4 + 1, 0.999999, 1e-6, out);
        cudaEventRecord(e0, s);
        fp64_fma_kernel<<<blocks, PEAK_THREADS, 0, s>>>(iters, 0.999999, 1e-6, out);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || !(ms > 0.f))
            rc = LBD_ECUDA;
    }
    if (rc == LBD_OK)
        *flops_per_s = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_THREADS / (ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    cudaGetLastError();
    return rc;
}

// sphst_peak.cu -- FMA throughput of this GPU, measured: the denominator of
// the roofline of the pair sweeps, which are bound by FP32 (FP64) arithmetic
// rather than by HBM bandwidth.
//
// Every thread runs CHAINS independent chains x <- x * a + b for `iters`
// rounds (a and b chosen so the values stay finite), on enough blocks to fill
// every SM several times over; the work is 2 * CHAINS * iters flops per
// thread.  The result of each thread is stored so that nothing is removed.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/sphst.h"
#include "sphst_engine.cuh"

namespace sphst {

constexpr int PEAK_CHAINS = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, int iters, T a, T b) {
    T x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int fma_peak(double *tflops, double *ms_out) {
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const int threads = 256, blocks = n_sm * 16;
    const int iters = sizeof(T) == 4 ? 8192 : 512;
    T *out = nullptr;
    e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads);
    if (e != cudaSuccess) return cuda_fail(e, "peak buffer");
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {      // first launch warms up
        cudaEventRecord(ev[0]);
        k_fma_peak<T><<<blocks, threads>>>(out, iters, T(0.9999999), T(1e-7));
        cudaEventRecord(ev[1]);
        e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "peak kernel");
    const double flops = 2.0 * PEAK_CHAINS * (double)iters * threads * (double)blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return SPHST_OK;
}

}  // namespace sphst

extern "C" int sphst_fma_peak(int32_t precision, double *tflops, double *kernel_ms) {
    if (!tflops || (precision != 32 && precision != 64)) {
        sphst::set_error("precision must be 32 or 64 and tflops non-NULL");
        return SPHST_ERR_INVALID_ARG;
    }
    return precision == 32 ? sphst::fma_peak<float>(tflops, kernel_ms) : sphst::fma_peak<double>(tflops, kernel_ms);
}

extern "C" int sphst_device_info(int32_t *sm_count, int32_t *max_sm_clock_khz, int32_t *cc_major,
                                 int32_t *cc_minor) {
    if (!sm_count || !max_sm_clock_khz) {
        sphst::set_error("sm_count and max_sm_clock_khz must be non-NULL");
        return SPHST_ERR_INVALID_ARG;
    }
    int dev = 0, v[4] = {0, 0, 0, 0};
    cudaError_t e = cudaGetDevice(&dev);
    const cudaDeviceAttr attrs[4] = {cudaDevAttrMultiProcessorCount, cudaDevAttrClockRate,
                                     cudaDevAttrComputeCapabilityMajor, cudaDevAttrComputeCapabilityMinor};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaDeviceGetAttribute(&v[k], attrs[k], dev);
    if (e != cudaSuccess) return sphst::cuda_fail(e, "device attribute query");
    *sm_count = v[0];
    *max_sm_clock_khz = v[1];
    if (cc_major) *cc_major = v[2];
    if (cc_minor) *cc_minor = v[3];
    return SPHST_OK;
}

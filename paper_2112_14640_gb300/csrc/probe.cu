// probe.cu -- a measured FP32 FMA peak, the denominator of the ALU roofline
// that the Brillouin stencil is reported against (the stencil's arithmetic
// intensity, ~45 flop/B at N_v = 12, puts it above the machine balance).
//
// Every thread runs eight independent FMA chains (enough independent work to
// hide the FMA latency at full occupancy); the grid is 8 blocks of 256 threads
// per SM, sized from the device's multiprocessor count.
#include <limits>

#include "internal.h"

namespace dgb {

constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

// the chains' sum is stored here when it equals `never` (a NaN at run time,
// so never); the store keeps ptxas from removing the unused arithmetic
static __device__ float g_ffma_sink;

__global__ void __launch_bounds__(256) ffma_peak_kernel(int iters, float a, float b, float never) {
    float x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i];
    if (s == never) g_ffma_sink = s;
}

}  // namespace dgb

extern "C" int dirac_measure_fp32_peak(int iters, double *tflops, int *sm_count, void *stream) {
    using namespace dgb;
    if (!tflops || iters < 1) return DIRAC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "multiProcessorCount");
    if (rc) return rc;
    if (sm_count) *sm_count = sms;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 8 * sms, threads = 256;
    cudaEvent_t e0, e1;
    rc = cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
    if (rc) return rc;
    rc = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
    if (rc) {
        cudaEventDestroy(e0);
        return rc;
    }
    // warm-up launch, then the timed one
    ffma_peak_kernel<<<blocks, threads, 0, s>>>(iters / 8 + 1, 0.999999f, 1e-6f, std::numeric_limits<float>::quiet_NaN());
    cudaEventRecord(e0, s);
    ffma_peak_kernel<<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-6f, std::numeric_limits<float>::quiet_NaN());
    cudaEventRecord(e1, s);
    rc = launch_check("ffma_peak_kernel");
    if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double flop = 2.0 * kPeakChains * kPeakUnroll * (double)iters * blocks * threads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return DIRAC_OK;
}

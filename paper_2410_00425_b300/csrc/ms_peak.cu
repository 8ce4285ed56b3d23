// ms_measure_fp32_peak: the measured FP32 FMA rate of the current device,
// the denominator of the batched step's ALU roofline.
//
// Every thread of a full-occupancy grid runs CHAINS independent chains of
// dependent fused multiply-adds (a <- a * b + c, written out as fmaf: the
// library is compiled without automatic contraction, so each is one FFMA).
// With 8 chains per thread and every warp slot of every SM filled, the FMA
// pipes, not the dependent latency, bound the rate.  Each FMA counts 2 flop.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/ms.h"
#include "ms_internal.h"

namespace ms {

static constexpr int PEAK_CHAINS = 8;
static constexpr int PEAK_UNROLL = 16;
static constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) k_fma_chains(float* out, int iters, float b, float c) {
    float a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; k++) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; u++) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; k++) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; k++) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;      // keeps the chains live
}

}  // namespace ms

using namespace ms;

#define PK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            char m_[256];                                                                 \
            snprintf(m_, sizeof m_, "ms_measure_fp32_peak: %s", cudaGetErrorString(e_)); \
            set_last_error(m_);                                                           \
            rc = MS_ERR_CUDA;                                                             \
            goto done;                                                                    \
        }                                                                                 \
    } while (0)

extern "C" ms_status ms_measure_fp32_peak(double seconds, double* flops_per_s, int* sm_count, double* measured_s) {
    if (!flops_per_s || !(seconds > 0.0) || seconds > 10.0) {
        set_last_error("ms_measure_fp32_peak: flops_per_s must be non-null and seconds in (0, 10]");
        return MS_ERR_INVALID_ARG;
    }
    ms_status rc = MS_OK;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0, per_sm = 0, grid = 0, iters = 64;
    float ms_ = 0.f;
    double flop = 0.0;
    PK(cudaGetDevice(&dev));
    PK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains, PEAK_THREADS, 0));
    grid = sms * (per_sm > 0 ? per_sm : 1);
    PK(cudaMalloc(&out, (size_t)grid * PEAK_THREADS * sizeof(float)));
    PK(cudaEventCreate(&e0));
    PK(cudaEventCreate(&e1));
    // grow the launch until it runs for a tenth of the requested time, then
    // time enough launches to fill it
    for (;;) {
        k_fma_chains<<<grid, PEAK_THREADS>>>(out, iters, 0.99999f, 1e-6f);
        PK(cudaGetLastError());
        PK(cudaEventRecord(e0));
        k_fma_chains<<<grid, PEAK_THREADS>>>(out, iters, 0.99999f, 1e-6f);
        PK(cudaEventRecord(e1));
        PK(cudaEventSynchronize(e1));
        PK(cudaEventElapsedTime(&ms_, e0, e1));
        if (ms_ * 1e-3 >= 0.1 * seconds || iters >= (1 << 24)) break;
        iters *= 4;
    }
    {
        int reps = (int)(seconds / (ms_ * 1e-3)) + 1;
        if (reps > 1000) reps = 1000;
        PK(cudaEventRecord(e0));
        for (int r = 0; r < reps; r++) k_fma_chains<<<grid, PEAK_THREADS>>>(out, iters, 0.99999f, 1e-6f);
        PK(cudaEventRecord(e1));
        PK(cudaEventSynchronize(e1));
        PK(cudaGetLastError());
        PK(cudaEventElapsedTime(&ms_, e0, e1));
        flop = 2.0 * PEAK_CHAINS * PEAK_UNROLL * (double)iters * (double)grid * PEAK_THREADS * reps;
    }
    *flops_per_s = flop / (ms_ * 1e-3);
    if (sm_count) *sm_count = sms;
    if (measured_s) *measured_s = ms_ * 1e-3;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}

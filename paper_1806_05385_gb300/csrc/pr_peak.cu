// pr_peak.cu -- FP32 fused multiply-add throughput of the device, measured.
// It cross-checks the peak of the fragment stage's ALU roofline, which is
// derived from the unit counts (SMs x 128 FP32 lanes x 2 FLOP) and the SM
// clock.
#include <cmath>

#include "pr_launch.h"

namespace pr {

constexpr int kPeakChains = 8;     // independent FMA chains per thread (hides the FMA latency)
constexpr int kPeakIters = 4096;   // iterations per chain
constexpr int kPeakThreads = 256;
constexpr int kPeakSink = 1024;    // floats of the (never written) result buffer

// Every thread runs kPeakChains independent chains x = x * a + b; the
// result is stored only if it equals a value it never takes, so the work
// cannot be removed while nothing is written.
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float a, float b, float never, float *sink)
{
    float x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c)
        x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c)
            x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c)
        s += x[c];
    if (s == never)
        sink[(blockIdx.x * blockDim.x + threadIdx.x) % kPeakSink] = s;
}

cudaError_t measure_fma_peak(cudaStream_t st, double *tflops)
{
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_peak, kPeakThreads, 0);
    if (e != cudaSuccess)
        return e;
    const int grid = sms * (per > 0 ? per : 1) * 4;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, sizeof(float) * kPeakSink);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        // a, b keep x bounded (|a| < 1), so no value overflows or underflows
        k_fma_peak<<<grid, kPeakThreads, 0, st>>>(0.999f, 1e-3f, -12345.f, sink);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {  // the first launch warms up
            const double flop = 2.0 * kPeakChains * kPeakIters * (double)grid * kPeakThreads;
            best = (float)std::fmax((double)best, flop / (ms * 1e-3) / 1e12);
        }
    }
    if (sink)
        cudaFree(sink);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    *tflops = best;
    return e;
}

}  // namespace pr

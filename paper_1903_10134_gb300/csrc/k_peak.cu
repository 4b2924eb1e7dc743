// Measured FP32 issue rate: the denominator of the ALU roofline the force and
// density passes are reported against.  Every thread runs CHAINS independent
// fused multiply-add chains (enough independent work per warp to cover the
// pipeline latency) for `iters` iterations on a full-occupancy grid; the rate
// is FMA lane-operations per second, one per lane per instruction.
#include <string>

#include "mdpd_internal.cuh"

namespace mdpd {
void set_global_error(const std::string& msg);
}

using namespace mdpd;

namespace {

constexpr int PEAK_BLOCK = 256;
constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(PEAK_BLOCK) k_fma_peak(int iters, float a, float b,
                                                         float* __restrict__ sink)
{
    float x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (float)threadIdx.x * 1e-3f + (float)c;
    // unrolled so that the loop counter costs a few slots per 64 FMAs
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    if (s == -1.0f) sink[blockIdx.x] = s;          // keeps the chains; never true
}

}  // namespace

extern "C" int mdpd_measure_fma_peak(double* lane_ops_per_s, double* best_ms)
{
    if (!lane_ops_per_s) return MDPD_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    auto fail = [](const char* what, cudaError_t e) {
        set_global_error(std::string(what) + ": " + cudaGetErrorString(e));
        return MDPD_ERR_CUDA;
    };
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return fail("device query", e);
    const int blocks = sms * (per_sm / PEAK_BLOCK);
    const int iters = 1 << 14;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float) * (size_t)blocks)) != cudaSuccess) return fail("cudaMalloc", e);
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e300;
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        k_fma_peak<<<blocks, PEAK_BLOCK>>>(iters, 0.9999999f, 1e-7f, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;   // rep 0 warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return fail("FMA peak kernel", e);
    const double ops = (double)blocks * PEAK_BLOCK * (double)iters * PEAK_CHAINS;
    *lane_ops_per_s = ops / (best * 1e-3);
    if (best_ms) *best_ms = best;
    return MDPD_OK;
}

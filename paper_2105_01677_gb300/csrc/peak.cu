// peak.cu -- measured arithmetic peaks of the device (a measuring tool of this library; the
// paper has no counterpart).  The pair sums of the step are bound by FP32 arithmetic in the
// mixed path and by FP64 arithmetic in the FP64 path, so their rooflines are taken against
// these measured rates rather than against figures derived from unit counts and clocks.
//
// Each kernel runs chains of dependent fused multiply-adds, kChains independent chains per
// thread so that every sub-partition has enough independent work to keep its pipe busy, on
// a grid of whole waves (a multiple of the SM count).  The result of every chain is folded
// into a value that is stored only if it equals an impossible sentinel, so the compiler
// keeps every operation and the kernel writes no memory.  One fused multiply-add counts as
// two flops.
#include <cuda_runtime.h>

#include <algorithm>

#include "mps.h"

namespace mps {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;
constexpr int kChains = 8;

static __device__ double g_peak_sink;

// FP32: scalar FFMA
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(int iters, float seed) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed + (float)(threadIdx.x + k);
    const float m = 0.999999f, c = 1e-7f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.2345e30f) g_peak_sink = s;
}

// FP32: packed two-lane FFMA (one instruction, two fused multiply-adds)
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(int iters, float seed) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++)
        a[k] = make_float2(seed + (float)(threadIdx.x + k), seed - (float)(threadIdx.x + k));
    const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = __ffma2_rn(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k].x + a[k].y;
    if (s == -1.2345e30f) g_peak_sink = s;
}

// FP64: DFMA
__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(int iters, double seed) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed + (double)(threadIdx.x + k);
    const double m = 0.999999999, c = 1e-12;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.2345e300) g_peak_sink = s;
}

}  // namespace
}  // namespace mps

extern "C" int mps_measure_peak(int32_t device, int32_t which, int32_t repeats, void* stream,
                                double* tflops, double* ms_per_launch) {
    using namespace mps;
    if (!tflops || repeats < 1 || which < MPS_PEAK_FFMA || which > MPS_PEAK_DFMA)
        return MPS_EINVAL;
    if (cudaPeekAtLastError() != cudaSuccess) return MPS_EDEVICE;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return MPS_EDEVICE;
    if (device != prev && cudaSetDevice(device) != cudaSuccess) return MPS_EDEVICE;
    int rc = MPS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MPS_EDEVICE;
    } else {
        const int blocks = sms * kPeakBlocksPerSm;
        // ~1-2 ms per launch at the expected rates: long enough for events, short for a tool
        const int iters = (which == MPS_PEAK_DFMA) ? 256 : 8192;
        auto launch = [&]() {
            if (which == MPS_PEAK_FFMA)
                k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f);
            else if (which == MPS_PEAK_FFMA2)
                k_peak_ffma2<<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f);
            else
                k_peak_dfma<<<blocks, kPeakThreads, 0, s>>>(iters, 1.0);
        };
        launch();   // warm-up (clocks ramp, module load)
        launch();
        cudaEventRecord(e0, s);
        for (int r = 0; r < repeats; r++) launch();
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
            rc = MPS_EDEVICE;
        } else {
            const double lanes = (which == MPS_PEAK_FFMA2) ? 2.0 : 1.0;
            const double flops = 2.0 * lanes * kChains * (double)iters * kPeakThreads * blocks;
            const double per = (double)ms / repeats;
            *tflops = flops / (per * 1e-3) / 1e12;
            if (ms_per_launch) *ms_per_launch = per;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (device != prev) cudaSetDevice(prev);
    return rc;
}

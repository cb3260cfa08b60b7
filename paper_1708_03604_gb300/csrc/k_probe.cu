// Throughput probes of single arithmetic units (bsm_measure_peak): the
// denominators against which the numeric kernels' rates are read.  Every
// probe is a fixed-length loop of independent instruction chains on every
// SM, with no waits and no memory traffic beyond one conditional store that
// keeps the compiler from removing the chains.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 4096;
constexpr int kChains = 8;

// FP64 FMA on the CUDA cores: kChains independent fma chains per thread
__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(double x, double y, double *sink) {
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (double)(threadIdx.x + c);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 1234.5678) *sink = s;
}

// FP32 FMA on the CUDA cores
__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(float x, float y, float *sink) {
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 1234.5678f) *sink = s;
}

// FP64 tensor-core MMA, m8n8k4 (512 FLOP per instruction per warp)
__global__ void __launch_bounds__(kProbeThreads) k_probe_dmma(double x, double y, double *sink) {
    double d[kChains][2];
#pragma unroll
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 0.0;
    const double a = x * (double)(threadIdx.x & 7), b = y;
    for (int it = 0; it < kProbeIters / 4; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
    if (s == 1234.5678) *sink = s;
}

// TF32 mma.sync m16n8k8 (2048 FLOP per instruction per warp) and BF16
// m16n8k16 (4096 FLOP)
template <bool BF16>
__global__ void __launch_bounds__(kProbeThreads) k_probe_mma(uint32_t abits, uint32_t bbits, float *sink) {
    float d[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0.f;
    const uint32_t a0 = abits ^ (threadIdx.x & 3), b0 = bbits;
    for (int it = 0; it < kProbeIters / 4; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (BF16)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};"
                    : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                    : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
            else
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};"
                    : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                    : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == 1234.5678f) *sink = s;
}

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" bsm_status bsm_measure_peak(int32_t unit, int32_t reps, double *flop_per_s) {
    if (!flop_per_s) return set_error(BSM_ERR_ARG, "flop_per_s is NULL");
    if (unit < BSM_U_FP64_FMA || unit > BSM_U_FP32_FMA) return set_error(BSM_ERR_ARG, "unknown unit");
    if (reps < 1 || reps > 100) return set_error(BSM_ERR_ARG, "reps outside [1, 100]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(e, "device attributes");
    cudaStream_t s = stream();
    // 4 CTAs of 8 warps per SM: enough warps to cover the chains' latency
    const int grid = 4 * sms;
    const double threads = (double)grid * kProbeThreads, warps = threads / 32.0;
    double flop = 0.0;
    switch (unit) {
        case BSM_U_FP64_FMA:
        case BSM_U_FP32_FMA: flop = threads * kProbeIters * kChains * 2.0; break;
        case BSM_U_FP64_MMA: flop = warps * (kProbeIters / 4) * kChains * 512.0; break;
        case BSM_U_TF32_MMA: flop = warps * (kProbeIters / 4) * kChains * 2048.0; break;
        default: flop = warps * (kProbeIters / 4) * kChains * 4096.0; break;
    }
    void *sink = nullptr;
    bsm_status st = dalloc(&sink, 16);
    if (st) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // launch 0 warms up
        cudaEventRecord(e0, s);
        switch (unit) {
            case BSM_U_FP64_FMA:
                k_probe_dfma<<<grid, kProbeThreads, 0, s>>>(0.999999, 1e-7, static_cast<double *>(sink));
                break;
            case BSM_U_FP64_MMA:
                k_probe_dmma<<<grid, kProbeThreads, 0, s>>>(1e-3, 1e-3, static_cast<double *>(sink));
                break;
            case BSM_U_TF32_MMA:
                k_probe_mma<false><<<grid, kProbeThreads, 0, s>>>(0x3a800000u, 0x3a800000u, static_cast<float *>(sink));
                break;
            case BSM_U_BF16_MMA:
                k_probe_mma<true><<<grid, kProbeThreads, 0, s>>>(0x3a803a80u, 0x3a803a80u, static_cast<float *>(sink));
                break;
            default:
                k_probe_ffma<<<grid, kProbeThreads, 0, s>>>(0.999999f, 1e-7f, static_cast<float *>(sink));
                break;
        }
        count_launch(1);
        e = cudaGetLastError();
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess && r > 0) {
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(sink);
    if (e != cudaSuccess) return cuda_check(e, "peak probe");
    *flop_per_s = flop / (best * 1e-3);
    return BSM_OK;
}

// peak.cu -- measured FP32 FMA throughput of the GPU, the denominator of the
// walk's roofline fraction (the walk is bound by the FP32 FMA pipe: Eq. 1 and
// the cell expansion are evaluated with FP32 fused multiply-adds).
//
// Every thread runs kChains independent FMA chains for `iters` rounds on
// register operands only (no memory traffic in the loop); the grid fills
// every SM with resident blocks.  Scalar: fmaf; packed: __ffma2_rn on float2
// (two FMAs per instruction).  flop = 2 per FMA.
#include "common.cuh"

namespace treegb {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_scalar(int iters, float seed, float *out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 1.0000001f, b = -1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live; never true for these operands
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_packed(int iters, float seed, float *out) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
    const float2 m = make_float2(1.0000001f, 1.0000001f), b = make_float2(-1e-7f, -1e-7f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace treegb

extern "C" tree_status_t tree_fp32_peak(double *tflops_scalar, double *tflops_packed) {
    using namespace treegb;
    if (!tflops_scalar && !tflops_packed) return TREE_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TREE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TREE_ERR_CUDA;
    float *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tree_status_t ret = TREE_OK;
    if (cudaMalloc(&out, 65536 * sizeof(float)) != cudaSuccess) return TREE_ERR_ALLOC;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        ret = TREE_ERR_CUDA;
    const int iters = 4096;
    for (int kind = 0; kind < 2 && ret == TREE_OK; ++kind) {
        double *dst = kind == 0 ? tflops_scalar : tflops_packed;
        if (!dst) continue;
        const void *fn = kind == 0 ? (const void *)k_peak_scalar : (const void *)k_peak_packed;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0) != cudaSuccess ||
            per_sm < 1) {
            ret = TREE_ERR_CUDA;
            break;
        }
        const int blocks = per_sm * sms * 4;  // four full waves
        float best = INFINITY;
        for (int rep = 0; rep < 4 && ret == TREE_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(e0, s);
            if (kind == 0) k_peak_scalar<<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f + rep, out);
            else k_peak_packed<<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f + rep, out);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { ret = TREE_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        const double fmas = (double)blocks * kPeakThreads * iters * 16.0 * kChains * (kind == 0 ? 1.0 : 2.0);
        if (ret == TREE_OK) *dst = 2.0 * fmas / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return ret;
}

// Measured FP32 CUDA-core throughput of the current device: the denominator of the FP32
// roofline fractions of the pair kernel and the FP32 contractions. Not part of the
// estimator; the paper has no counterpart.
//
// Every thread runs kChains independent fused multiply-add chains (x <- x a + b), enough
// in flight per warp to cover the FMA latency; four blocks of 256 threads per SM fill every
// scheduler. The chains stay bounded (|a| < 1), and the result is written only under a
// condition the host makes false, so the compiler keeps every FMA.
#include "encore_gpu.h"

#include <cuda_runtime.h>

#include <algorithm>

namespace npcf {
void set_global_error(const char* msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

__global__ void __launch_bounds__(kThreads) k_fma_probe(float* out, int iters, float a, float b, float never) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == never) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" npcf_status npcf_probe_fp32_peak(double* tflops, double* ms_out) {
    if (!tflops) {
        npcf::set_global_error("null output pointer");
        return NPCF_EINVAL;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        npcf::set_global_error("no CUDA device");
        return NPCF_ECUDA;
    }
    const int blocks = nsm * kBlocksPerSM;
    const int iters = 1 << 14;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    npcf_status st = NPCF_OK;
    float best = 0.f;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        npcf::set_global_error("probe set-up failed");
        st = NPCF_ECUDA;
    } else {
        for (int rep = 0; rep < 6 && st == NPCF_OK; ++rep) {
            cudaEventRecord(e0, 0);
            k_fma_probe<<<blocks, kThreads>>>(out, iters, 0.9999f, 1e-4f, -1.0f);
            cudaEventRecord(e1, 0);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                npcf::set_global_error("probe launch failed");
                st = NPCF_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best == 0.f || ms < best)) best = ms;   // first launch is a warm-up
        }
    }
    if (st == NPCF_OK) {
        const double flop = 2.0 * kChains * 4.0 * (double)iters * (double)blocks * kThreads;
        *tflops = flop / (best * 1e-3) / 1e12;
        if (ms_out) *ms_out = best;
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

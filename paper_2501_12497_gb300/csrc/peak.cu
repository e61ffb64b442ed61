// Measured FP32 ceilings of this GPU for the projector pair's roofline (library
// plumbing; the paper has no counterpart): the FP32 FMA rate and the rate of 4-byte
// loads served by L1, each by a kernel that does nothing else, timed with CUDA events.
#include "common.cuh"

#include <algorithm>

namespace mof {

namespace {

constexpr int PK_T = 256;      // threads per block
constexpr int PK_CHAINS = 8;   // independent FMA chains per thread
constexpr int PK_ITERS = 4096; // unrolled steps per chain

// PK_CHAINS x PK_ITERS dependent FMAs per thread (independent across chains); the result
// is stored so the compiler keeps the work
__global__ void __launch_bounds__(PK_T) k_peak_fma(float *out, float a, float b) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-7f;
#pragma unroll 16
    for (int i = 0; i < PK_ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    out[blockIdx.x * PK_T + threadIdx.x] = s;
}

// Each thread sums PK_LOADS 4-byte loads from a 16 KB table (L1 resident after the first
// pass) at addresses that step by one element per lane, as the Joseph taps of adjacent
// rays do
constexpr int PK_LOADS = 8192;
__global__ void __launch_bounds__(PK_T) k_peak_l1(const float *__restrict__ tab, float *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int idx = (w * 37 + lane) & 4095;
#pragma unroll 8
    for (int i = 0; i < PK_LOADS; i += 4) {
        s0 += __ldg(tab + idx);
        s1 += __ldg(tab + ((idx + 1024) & 4095));
        s2 += __ldg(tab + ((idx + 2048) & 4095));
        s3 += __ldg(tab + ((idx + 3072) & 4095));
        idx = (idx + 33) & 4095;
    }
    out[blockIdx.x * PK_T + threadIdx.x] = s0 + s1 + s2 + s3;
}

}  // namespace

}  // namespace mof

using namespace mof;

extern "C" mof_status mof_measure_fp32_peaks(double *fma_tflops, double *l1_gloads_per_s) {
    if (!fma_tflops || !l1_gloads_per_s) return fail(MOF_EINVAL, "null output");
    int dev = 0, sms = 0;
    MOF_CUDA(cudaGetDevice(&dev));
    MOF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    float *out = nullptr, *tab = nullptr;
    MOF_CUDA(cudaMalloc(&out, sizeof(float) * blocks * PK_T));
    MOF_CUDA(cudaMalloc(&tab, sizeof(float) * 4096));
    MOF_CUDA(cudaMemset(tab, 0, sizeof(float) * 4096));
    cudaEvent_t e0, e1;
    MOF_CUDA(cudaEventCreate(&e0));
    MOF_CUDA(cudaEventCreate(&e1));
    float best_fma = 1e30f, best_ld = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {  // best of five after a warm-up launch each
        ::mof::count_launch(), k_peak_fma<<<blocks, PK_T>>>(out, 0.999f, 1e-3f);
        MOF_CUDA(cudaEventRecord(e0));
        ::mof::count_launch(), k_peak_fma<<<blocks, PK_T>>>(out, 0.999f, 1e-3f);
        MOF_CUDA(cudaEventRecord(e1));
        MOF_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MOF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best_fma = std::min(best_fma, ms);
        ::mof::count_launch(), k_peak_l1<<<blocks, PK_T>>>(tab, out);
        MOF_CUDA(cudaEventRecord(e0));
        ::mof::count_launch(), k_peak_l1<<<blocks, PK_T>>>(tab, out);
        MOF_CUDA(cudaEventRecord(e1));
        MOF_CUDA(cudaEventSynchronize(e1));
        MOF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best_ld = std::min(best_ld, ms);
    }
    const double threads = (double)blocks * PK_T;
    *fma_tflops = 2.0 * threads * PK_CHAINS * PK_ITERS / (best_fma * 1e-3) / 1e12;
    *l1_gloads_per_s = threads * PK_LOADS / (best_ld * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(tab);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

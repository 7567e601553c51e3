// Diagnostics: issue-rate microbenchmarks of the two pipes the emission
// kernel lives on (MUFU ex2 and FP32 FMA), used as its roofline denominators.
// Each thread runs 8 independent dependency chains; nothing is read from
// memory and each thread writes one float.
#include "dust_internal.cuh"

namespace dust {
namespace {

constexpr int CH = 8;

__global__ void k_ex2_rate(int iters, float *sink) {
    float x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = 0.01f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[i]));
            x[i] = y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma_rate(int iters, float a, float b, float *sink) {
    float x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = 0.01f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[i]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace dust

using namespace dust;

extern "C" int dust_diag_throughput(int device, double *ex2_per_s, double *ffma_per_s) {
    int prev = 0;
    DUST_CUDA_TRY(cudaGetDevice(&prev));
    DUST_CUDA_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    DUST_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    const int threads = 256, blocks = prop.multiProcessorCount * 8;
    float *sink = nullptr;
    DUST_CUDA_TRY(cudaMalloc(&sink, sizeof(float) * threads * blocks));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 4096;
    double best_ex2 = 0.0, best_fma = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        float ms = 0.f;
        cudaEventRecord(e0);
        k_ex2_rate<<<blocks, threads>>>(iters, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        double ops = (double)blocks * threads * CH * iters;
        if (rep) best_ex2 = std::max(best_ex2, ops / (ms * 1e-3));
        cudaEventRecord(e0);
        k_ffma_rate<<<blocks, threads>>>(iters * 4, 0.999f, 1e-4f, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        ops = (double)blocks * threads * CH * iters * 4;
        if (rep) best_fma = std::max(best_fma, ops / (ms * 1e-3));
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaSetDevice(prev);
    if (err != cudaSuccess) return set_error(DUST_ECUDA, "diag kernels failed: %s", cudaGetErrorString(err));
    if (ex2_per_s) *ex2_per_s = best_ex2;
    if (ffma_per_s) *ffma_per_s = best_fma;
    return DUST_OK;
}

// Diagnostics: issue-rate microbenchmarks of the two pipes the emission
// kernel lives on (MUFU ex2 and FP32 FMA), used as its roofline denominators
// (each thread runs 8 independent dependency chains; nothing is read from
// memory and each thread writes one float), and a probe of the bounded
// mbarrier wait that the tensor-core GEMM relies on for failure detection.
#include "dust_internal.cuh"
#include "mbar.cuh"

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

// One thread waits on phase 0 of an mbarrier that expects one arrival and
// gets none: the wait must give up after limit_ns, record DUST_ETIMEOUT and
// return, exactly as a GEMM warp whose producer stalled would.
__global__ void k_wait_probe(unsigned long long limit_ns, int *status, unsigned long long *elapsed_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer_ns();
        const bool ok = mbar_wait(&bar, 0, &abort_flag, status, limit_ns);
        *elapsed_ns = globaltimer_ns() - t0;
        if (ok) record_status(status, DUST_EINVAL);  // a phase nobody completed completed
    }
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

extern "C" int dust_diag_wait_timeout(int device, double limit_ms, int *device_status, double *elapsed_ms) {
    if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) return set_error(DUST_EINVAL, "limit_ms must lie in (0, 2000]");
    int ndev = 0;
    DUST_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_error(DUST_EINVAL, "device %d of %d", device, ndev);
    int prev = 0;
    DUST_CUDA_TRY(cudaGetDevice(&prev));
    DUST_CUDA_TRY(cudaSetDevice(device));
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 16);
    int st = 0;
    unsigned long long ns = 0;
    if (e == cudaSuccess) e = cudaMemset(buf, 0, 16);
    if (e == cudaSuccess) {
        int *status = static_cast<int *>(buf);
        unsigned long long *el = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf) + 8);
        k_wait_probe<<<1, 32>>>((unsigned long long)(limit_ms * 1e6), status, el);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&ns, el, sizeof(ns), cudaMemcpyDeviceToHost);
    }
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return set_error(DUST_ECUDA, "wait probe failed: %s", cudaGetErrorString(e));
    if (device_status) *device_status = st;
    if (elapsed_ms) *elapsed_ms = (double)ns * 1e-6;
    return DUST_OK;
}

// dust_solve_noalloc: the hot path without any device allocation.
//
// The absorption kernel writes the scaled absorbed powers S[C][Gs] that the
// solve/emission kernel reads back; dust_solve keeps that scratch in a
// context-owned buffer it grows with cudaMalloc.  This entry point instead
// uses one fixed array in the library's own device data, so a caller that may
// not allocate device memory (one whose device memory is owned by a host
// framework's pool, a real-time loop that cannot afford cudaMalloc's implicit
// synchronisation, a memory-capped embedding) can still run the path.
#include "dust_internal.cuh"

#include <mutex>


namespace {

// 64 MiB of scratch, resident on every device that loads the library.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / sizeof(float)];

constexpr int MAX_DEVICES = 64;
std::mutex g_addr_mu;
float *g_addr[MAX_DEVICES] = {};  // device address of the array, per device

// Device address of the scratch array on `device` (which must be current).
// Taken once per device with cudaGetSymbolAddress: in host code the array's
// name is only a host-side stand-in, not a device address.  The address is
// kept for the life of the process, so a device reset (which reloads the
// module) is not supported.
int scratch_address(int device, float **out) {
    if (device < 0 || device >= MAX_DEVICES)
        return dust::set_error(DUST_EINVAL, "device %d beyond the scratch table", device);
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return dust::set_error(DUST_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                                   cudaGetErrorString(e));
        }
        g_addr[device] = static_cast<float *>(p);
    }
    *out = g_addr[device];
    return DUST_OK;
}

int check_ptr(const void *p, int device, const char *name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return dust::set_error(DUST_EINVAL, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return dust::set_error(DUST_EINVAL, "%s must be device memory", name);
    if (a.type == cudaMemoryTypeDevice && a.device != device)
        return dust::set_error(DUST_EINVAL, "%s lives on device %d, the context on device %d", name, a.device,
                               device);
    return DUST_OK;
}

}  // namespace

extern "C" size_t dust_noalloc_max_cells(const dust_ctx *ctx) {
    if (!ctx) return 0;
    // largest C whose scratch (with the emission's part) fits the array
    size_t lo = 0, hi = NOALLOC_SCRATCH_BYTES;
    while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (dust::scratch_bytes(ctx, (int64_t)mid, true) <= NOALLOC_SCRATCH_BYTES) lo = mid; else hi = mid;
    }
    return lo;
}

extern "C" int dust_solve_noalloc(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n,
                                  float *T, float *L, double *resid, uint8_t *flags, void *stream) {
    using namespace dust;
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (n_cells < 0) return set_error(DUST_EINVAL, "n_cells < 0");
    if (ld < ctx->K) return set_error(DUST_EINVAL, "ld=%lld < K=%d", (long long)ld, ctx->K);
    if (n_cells == 0) return DUST_OK;
    // one limit for every mode (the emission's scratch included), so that
    // whether a batch is accepted never depends on which outputs it wants
    const size_t max_cells = dust_noalloc_max_cells(ctx);
    if ((size_t)n_cells > max_cells)
        return set_error(DUST_EINVAL,
                         "n_cells=%lld needs %zu scratch bytes; this entry point has %zu (at most %zu cells "
                         "for this context): split the batch",
                         (long long)n_cells, scratch_bytes(ctx, n_cells, true), NOALLOC_SCRATCH_BYTES, max_cells);
    if (!J || !n || !T) return set_error(DUST_EINVAL, "J, n and T must be non-NULL");
    int rc;
    if ((rc = check_ptr(J, ctx->device, "J")) || (rc = check_ptr(n, ctx->device, "n")) ||
        (rc = check_ptr(T, ctx->device, "T")) || (L && (rc = check_ptr(L, ctx->device, "L"))) ||
        (resid && (rc = check_ptr(resid, ctx->device, "resid"))) ||
        (flags && (rc = check_ptr(flags, ctx->device, "flags"))))
        return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    // the precision is read under the lock: the kernel choice and its checks use one value
    const int precision = ctx->precision;
    if (precision != DUST_PREC_FP32 && (ld % 4 != 0 || ((uintptr_t)J & 15) != 0))
        return set_error(DUST_EINVAL, "tensor-core precisions need ld %% 4 == 0 and a 16-byte aligned J");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DUST_ECUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    float *S = nullptr;
    rc = scratch_address(ctx->device, &S);
    if (rc == DUST_OK) {
        cudaStream_t st = (cudaStream_t)stream;
        // every scratch value a launch reads is written earlier in the same
        // call (S by the absorption kernel, the pairs and cell records by the
        // solve), so nothing needs clearing between calls
        const ScratchView sv = scratch_view(ctx, n_cells, S);
        rc = precision == DUST_PREC_FP32 ? launch_gemm_simt(ctx, n_cells, J, ld, sv.S, st)
                                         : launch_gemm_tc(ctx, precision, n_cells, J, ld, sv.S, st);
        if (rc == DUST_OK) {
            ctx->launches += 1;
            int nl = 0;
            rc = launch_solve_emit(ctx, n_cells, sv, n, T, L, ld, resid, flags, st, &nl);
            ctx->launches += (uint64_t)nl;
        }
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

// Self-absorption: dust that is optically thick to its own emission is heated
// by it too, so the radiation field and the temperatures have to be found
// together by iteration (Section 2; the paper's radiative-transfer code does it
// globally).  This is a local form of that iteration around the hot path:
//   J^(0) = J_ext,   J^(i) = J_ext + E (.) L^(i),   L^(i) = emission of solve(J^(i-1)),
// with a caller-supplied coupling E[c,k] >= 0 (the part of the cell's own
// emission L[c,k] that returns to its mean intensity J[c,k]).  It stops when
// the largest peak-normalised change of L between two iterations,
//   max_c max_k |L^(i)[c,k] - L^(i-1)[c,k]| / max_k L^(i)[c,k],
// falls to `tol`, or after `max_iters` solves.
#include "dust_internal.cuh"

#include <algorithm>
#include <cstring>

namespace dust {
namespace {

constexpr int CPL_TH = 128;

// One warp per cell: the change of L against the previous iterate (folded
// into *change with an integer max on the float's bits, exact for values
// >= 0), then Lprev = L and Jw = J_ext + E L.
__global__ void __launch_bounds__(CPL_TH) k_couple(int64_t C, int K, int64_t ld, const float *Jext,
                                                   const float *E, const float *L, float *Lprev, float *Jw,
                                                   int first, unsigned int *change) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * CPL_TH) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * CPL_TH + threadIdx.x) >> 5; c < C; c += nw) {
        const float *Lr = L + c * ld;
        float *Pr = Lprev + c * ld;
        float peak = 0.f, d = 0.f;
        for (int k = lane; k < K; k += 32) {
            const float v = Lr[k];
            peak = fmaxf(peak, v);
            if (!first) d = fmaxf(d, fabsf(v - Pr[k]));
        }
        for (int o = 16; o; o >>= 1) {
            peak = fmaxf(peak, __shfl_xor_sync(0xffffffffu, peak, o));
            d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
        }
        const float *Jr = Jext + c * ld, *Er = E + c * ld;
        float *Wr = Jw + c * ld;
        for (int k = lane; k < K; k += 32) {
            const float v = Lr[k];
            Pr[k] = v;
            Wr[k] = fmaf(Er[k], v, Jr[k]);
        }
        if (lane == 0 && !first) {
            float ch = d > 0.f ? (peak > 0.f ? d / peak : INFINITY) : 0.f;
            if (!(ch == ch)) ch = INFINITY;  // NaN counts as not converged
            atomicMax(change, __float_as_uint(ch));
        }
    }
}

int check_dev(const void *p, int device, const char *name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DUST_EINVAL, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error(DUST_EINVAL, "%s must be device memory", name);
    if (a.type == cudaMemoryTypeDevice && a.device != device)
        return set_error(DUST_EINVAL, "%s lives on device %d, the context on device %d", name, a.device, device);
    return DUST_OK;
}

}  // namespace
}  // namespace dust

using namespace dust;

extern "C" int dust_solve_coupled(dust_ctx *ctx, int64_t n_cells, const float *J_ext, int64_t ld, const float *E,
                                  const float *n, int max_iters, double tol, float *T, float *L, double *resid,
                                  uint8_t *flags, int *iters_done, double *last_change, void *stream) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (n_cells < 0) return set_error(DUST_EINVAL, "n_cells < 0");
    if (ld < ctx->K) return set_error(DUST_EINVAL, "ld=%lld < K=%d", (long long)ld, ctx->K);
    if (max_iters < 1 || max_iters > 10000) return set_error(DUST_EINVAL, "max_iters outside [1, 10000]");
    if (!(tol >= 0.0)) return set_error(DUST_EINVAL, "tol must be >= 0");
    if (iters_done) *iters_done = 0;
    if (last_change) *last_change = 0.0;
    if (n_cells == 0) return DUST_OK;
    if (!J_ext || !E || !n || !T || !L) return set_error(DUST_EINVAL, "J_ext, E, n, T and L must be non-NULL");
    const int precision = ctx->precision;
    if (precision != DUST_PREC_FP32 && (ld % 4 != 0 || ((uintptr_t)J_ext & 15) != 0))
        return set_error(DUST_EINVAL, "tensor-core precisions need ld %% 4 == 0 and a 16-byte aligned J_ext");
    int rc;
    if ((rc = check_dev(J_ext, ctx->device, "J_ext")) || (rc = check_dev(E, ctx->device, "E")) ||
        (rc = check_dev(n, ctx->device, "n")) || (rc = check_dev(T, ctx->device, "T")) ||
        (rc = check_dev(L, ctx->device, "L")) || (resid && (rc = check_dev(resid, ctx->device, "resid"))) ||
        (flags && (rc = check_dev(flags, ctx->device, "flags"))))
        return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DUST_ECUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // working J, previous L and the change word, grown on demand
    const size_t need = (size_t)2 * n_cells * ld * sizeof(float) + 256;
    rc = DUST_OK;
    if (ctx->cpl_bytes < need) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            cudaFree(ctx->cpl);
            ctx->cpl = nullptr;
            ctx->cpl_bytes = 0;
            e = cudaMalloc(&ctx->cpl, need);
        }
        // columns K..ld of the working J are read as padding by nothing, but keep them defined
        if (e == cudaSuccess) e = cudaMemset(ctx->cpl, 0, need);
        if (e == cudaSuccess) ctx->cpl_bytes = need;
        else rc = set_error(DUST_ENOMEM, "coupled-solve buffers: %s", cudaGetErrorString(e));
    }
    float *Jw = static_cast<float *>(ctx->cpl);
    float *Lprev = Jw + (size_t)n_cells * ld;
    unsigned int *chg = reinterpret_cast<unsigned int *>(Lprev + (size_t)n_cells * ld);
    const float *Jcur = J_ext;
    int it = 0;
    float change = INFINITY;
    if (rc == DUST_OK) rc = ensure_scratch(ctx, n_cells, st);
    const int64_t grid = std::min<int64_t>((n_cells * 32 + CPL_TH - 1) / CPL_TH, (int64_t)ctx->num_sms * 16);
    while (rc == DUST_OK && it < max_iters) {
        rc = solve_device(ctx, precision, n_cells, Jcur, ld, n, T, L, resid, flags, ctx->S, st);
        if (rc != DUST_OK) break;
        ++it;
        cudaError_t e = cudaMemsetAsync(chg, 0, sizeof(unsigned int), st);
        if (e == cudaSuccess) {
            k_couple<<<(unsigned)grid, CPL_TH, 0, st>>>(n_cells, ctx->K, ld, J_ext, E, L, Lprev, Jw, it == 1, chg);
            e = cudaGetLastError();
        }
        unsigned int bits = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, chg, sizeof(bits), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = set_error(DUST_ECUDA, "coupled iteration: %s", cudaGetErrorString(e));
            break;
        }
        if (it > 1) {
            std::memcpy(&change, &bits, sizeof(change));
            if (change <= tol) break;
        }
        Jcur = Jw;
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (iters_done) *iters_done = it;
    if (last_change) *last_change = (double)change;
    return rc;
}

// The paper's own temperature kernel (its kernel 3, Section 4.3), kept as an
// ablation of the table solve: per (cell, grain), Newton-Raphson in T on
// Eq. 7 with the full wavelength quadrature of P_g(T) and dP_g/dT evaluated
// at every iterate, started from the fitted guess of Eqs. 11-12 (floored at
// 5 K) and stopped once the energy non-conservation |P_g(T) - A| / A falls
// below 0.1 %.  As in the paper, a block takes one grain over many cells and
// keeps that grain's cross-section vector in shared memory; threads of a warp
// that need fewer iterations wait for the slowest one.
//
// Scaled units: P_g(T) = 2^Ew / (4 pi) sum_k wq_k Chat[g,k] t/(1-t) with
// t = 2^(nax_k / T) (the emission kernel's weights), so the equation solved is
//   sum_k wq_k Chat[g,k] t_k/(1-t_k) = S sigma_g,  sigma_g = gscale_g 4 pi 2^-Ew,
// where A = S gscale_g.  dP/dT follows from d/dT [t/(1-t)] = t/(1-t)^2 x/T
// with x = -nax ln 2 / T.
#include "dust_internal.cuh"

#include <cmath>
#include <vector>

namespace dust {
namespace {

constexpr int NW_TH = 128;   // cells per block (one grain per block row)
constexpr int NW_MAXIT = 64; // iteration cap; beyond it the grain is flagged

// Eqs. 11-12 (SI units, log base 10): log T ~ k + b1 x + b2 x^2,
// x = log L_h + a1 log a + a2 log^2 a.
constexpr double GUESS_K = 1.86, GUESS_B1 = 0.189, GUESS_B2 = 3.41e-3;
constexpr double GUESS_A1 = -1.39, GUESS_A2 = 0.126;
constexpr float GUESS_FLOOR_K = 5.f;
constexpr float STOP_REL = 1e-3f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ng[g] = (x0_g, sigma_g): x0_g = log10 gscale_g + a1 log10 a_g + a2 log10^2 a_g.
__global__ void __launch_bounds__(NW_TH) k_newton_paper(const DevTables tb, int64_t C, const float *S,
                                                        const float2 *ng, float *T, uint8_t *iters,
                                                        uint8_t *flags) {
    extern __shared__ float sm[];
    const int g = blockIdx.y, K = tb.K;
    float *wC = sm, *nx = sm + K;
    for (int k = threadIdx.x; k < K; k += NW_TH) {
        const float chat = tb.Chat[((size_t)(k / KQ) * tb.G8 + g) * KQ + (k % KQ)];
        wC[k] = tb.wq[k] * chat;
        nx[k] = tb.nax[k];
    }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * NW_TH + threadIdx.x;
    if (c >= C) return;
    const float s = S[c * tb.Gs + g];
    const float4 gr = tb.gres[g];  // z: S of P_g(T_min), w: S of P_g(T_max)
    int fl = (!(s >= 0.f) || isinf(s)) ? DUST_FLAG_INVALID
           : s < gr.z ? DUST_FLAG_LOW
           : s > gr.w ? DUST_FLAG_HIGH : DUST_FLAG_OK;
    float Tv = fl == DUST_FLAG_LOW ? tb.Tmin : fl == DUST_FLAG_HIGH ? tb.Tmax : __int_as_float(0x7fc00000);
    int it = 0;
    if (fl == DUST_FLAG_OK) {
        const float2 q = ng[g];
        const float A = s * q.y;
        const float x = lg2_approx(s) * 0.30102999566f + q.x;  // log10 L_h + size terms
        const float lt = (float)GUESS_K + x * ((float)GUESS_B1 + x * (float)GUESS_B2);
        float Tc = ex2_approx(lt * 3.32192809489f);
        Tc = fminf(fmaxf(Tc, fmaxf(GUESS_FLOOR_K, tb.Tmin)), tb.Tmax);
        for (;; ++it) {
            const float iT = 1.f / Tc;
            float P = 0.f, Q = 0.f;  // sum w C f, and sum w C f/(1-t) a  (a = log2 t)
            for (int k = 0; k < K; ++k) {
                const float a = nx[k] * iT;
                const float t = ex2_approx(a);
                const float r = rcp_approx(1.f - t);
                const float wf = wC[k] * (t * r);
                P += wf;
                Q = fmaf(wf * r, a, Q);
            }
            if (fabsf(P - A) <= STOP_REL * A) break;
            if (it == NW_MAXIT) { fl = DUST_FLAG_NOCONV; break; }
            const float dP = -0.69314718056f * Q * iT;  // dP/dT
            const float Tn = fminf(fmaxf(Tc - (P - A) / dP, tb.Tmin), tb.Tmax);
            if (!(Tn != Tc)) { fl = DUST_FLAG_NOCONV; break; }
            Tc = Tn;
        }
        Tv = Tc;
    }
    const int64_t o = c * tb.G + g;
    T[o] = Tv;
    if (iters) iters[o] = (uint8_t)(it < 255 ? it : 255);
    if (flags) flags[o] = (uint8_t)fl;
}

}  // namespace
}  // namespace dust

using namespace dust;

extern "C" {

int dust_ctx_set_grain_sizes(dust_ctx *ctx, const double *a_m) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (!a_m) return set_error(DUST_EINVAL, "a_m is NULL");
    const int G = ctx->G;
    for (int g = 0; g < G; ++g)
        if (!(a_m[g] > 0.0) || !std::isfinite(a_m[g]))
            return set_error(DUST_EINVAL, "grain %d: size %g is not a positive finite length", g, a_m[g]);
    std::lock_guard<std::mutex> lk(ctx->mu);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DUST_ECUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    std::vector<double> gs(G);
    cudaError_t e = cudaMemcpy(gs.data(), ctx->tb.gscale, sizeof(double) * G, cudaMemcpyDeviceToHost);
    std::vector<float2> ng(G);
    int rc = DUST_OK;
    if (e != cudaSuccess) rc = set_error(DUST_ECUDA, "reading the grain scales failed: %s", cudaGetErrorString(e));
    for (int g = 0; g < G && rc == DUST_OK; ++g) {
        const double la = std::log10(a_m[g]);
        const double x0 = std::log10(gs[g]) + GUESS_A1 * la + GUESS_A2 * la * la;
        const double sg = std::ldexp(gs[g] * 4.0 * 3.14159265358979323846, -ctx->tb.Ew);
        if (!(sg > 1e-37 && sg < 1e37))
            rc = set_error(DUST_EINVAL, "grain %d: scale %g of the quadrature solve is outside FP32", g, sg);
        ng[g] = make_float2((float)x0, (float)sg);
    }
    if (rc == DUST_OK && !ctx->newton_grain) {
        e = cudaMalloc(&ctx->newton_grain, sizeof(float2) * G);
        if (e != cudaSuccess) rc = set_error(DUST_ENOMEM, "cudaMalloc failed: %s", cudaGetErrorString(e));
    }
    if (rc == DUST_OK) {
        e = cudaMemcpy(ctx->newton_grain, ng.data(), sizeof(float2) * G, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = set_error(DUST_ECUDA, "cudaMemcpy failed: %s", cudaGetErrorString(e));
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

int dust_solve_T_newton(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, float *T, uint8_t *iters,
                        uint8_t *flags, void *stream) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (n_cells < 0) return set_error(DUST_EINVAL, "n_cells < 0");
    if (ld < ctx->K) return set_error(DUST_EINVAL, "ld=%lld < K=%d", (long long)ld, ctx->K);
    if (!ctx->newton_grain) return set_error(DUST_EINVAL, "grain sizes not set: call dust_ctx_set_grain_sizes");
    if (n_cells == 0) return DUST_OK;
    if (!J || !T) return set_error(DUST_EINVAL, "J and T must be non-NULL");
    const int precision = ctx->precision;
    if (precision != DUST_PREC_FP32 && (ld % 4 != 0 || ((uintptr_t)J & 15) != 0))
        return set_error(DUST_EINVAL, "tensor-core precisions need ld %% 4 == 0 and a 16-byte aligned J");
    for (const void *p : {(const void *)J, (const void *)T, (const void *)iters, (const void *)flags}) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return set_error(DUST_EINVAL, "an argument is not a CUDA pointer");
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return set_error(DUST_EINVAL, "J, T, iters and flags must be device memory");
        if (a.type == cudaMemoryTypeDevice && a.device != ctx->device)
            return set_error(DUST_EINVAL, "an argument lives on device %d, the context on device %d", a.device,
                             ctx->device);
    }
    if ((uint64_t)(n_cells + NW_TH - 1) / NW_TH > 0x7fffffffull)
        return set_error(DUST_EINVAL, "n_cells too large for one launch");
    std::lock_guard<std::mutex> lk(ctx->mu);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DUST_ECUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_scratch(ctx, n_cells, st);
    if (rc == DUST_OK) {
        float *S = scratch_view(ctx, n_cells, ctx->S).S;
        rc = precision == DUST_PREC_FP32 ? launch_gemm_simt(ctx, n_cells, J, ld, S, st)
                                         : launch_gemm_tc(ctx, precision, n_cells, J, ld, S, st);
        if (rc == DUST_OK) {
            const dim3 grid((unsigned)((n_cells + NW_TH - 1) / NW_TH), (unsigned)ctx->G);
            k_newton_paper<<<grid, NW_TH, sizeof(float) * 2 * ctx->K, st>>>(
                ctx->tb, n_cells, S, reinterpret_cast<const float2 *>(ctx->newton_grain), T, iters, flags);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = set_error(DUST_ECUDA, "Newton kernel launch failed: %s", cudaGetErrorString(e));
        }
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

}  // extern "C"

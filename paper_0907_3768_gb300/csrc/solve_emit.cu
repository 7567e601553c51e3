// Kernel (b): fused equilibrium-temperature solve and emission SED.
//
// A persistent CTA walks tiles of TC cells.  For each tile:
//  phase 0  per-cell exponent m_c of max_g n[c,g] (n is used as n 2^-m_c);
//  phase 1  one thread per (cell, grain): the root of Eq. 7 from the scaled
//           absorbed power S (A / P_g(T_min) = S 2^f_g): an initial guess from
//           the inverse table u(t), then Newton on the FP32 Hermite
//           interpolant of t_g(u) = log2(P_g(2^u) / P_g(T_min)) inside the
//           bracketing table interval (bisection when a Newton step leaves
//           it).  The paper's kernel 3 ran Newton with a fresh quadrature per
//           iteration (Section 4.3); the table removes those exponentials.
//  phase 2  one thread per (cell, 8 consecutive wavelengths): Eq. 10,
//           L[c,k] = 2^(m_c+q_k) sum_g (n 2^-m_c) Chat[g,k] t/(1-t),
//           t = 2^(nax_k / T[c,g]) (one MUFU ex2 per term), with the sum over
//           grains accumulated as a fraction N/D over groups of 8 grains so
//           that each group costs one reciprocal instead of eight:
//             N <- N + t (w D - N),  D <- D - t D   (= sum of w t/(1-t)).
//           Chat is staged in shared memory (in grain chunks when it does not
//           fit), as the paper staged sigma per block (Section 4.4).
//  resid    sum_k w_k L[c,k] / (4 pi sum_g n Pe) - 1 in FP64.
#include "dust_internal.cuh"

namespace dust {
namespace {

constexpr int NTH = 256;
constexpr double FOUR_PI = 12.566370614359172954;

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

// Cubic Hermite on [0,1] with end values p0, p1 and end slopes d0, d1.
__device__ __forceinline__ float hermite(float p0, float d0, float p1, float d1, float x) {
    float d = p1 - p0;
    float c2 = 3.f * d - 2.f * d0 - d1;
    float c3 = d0 + d1 - 2.f * d;
    return p0 + x * (d0 + x * (c2 + x * c3));
}

// Equilibrium temperature of grain g for scaled absorbed power s (see above).
__device__ __forceinline__ float solve_T(const DevTables &tb, int g, float s, int &flag) {
    const float4 gq = __ldg(reinterpret_cast<const float4 *>(tb.gp) + g);  // f, tmax, invdy
    if (!(s >= 0.f) || isinf(s)) { flag = DUST_FLAG_INVALID; return __int_as_float(0x7fc00000); }
    if (s == 0.f) { flag = DUST_FLAG_LOW; return tb.Tmin; }
    const float y = log2f(s) + gq.x;
    if (y < 0.f) { flag = DUST_FLAG_LOW; return tb.Tmin; }
    if (y > gq.y) { flag = DUST_FLAG_HIGH; return tb.Tmax; }
    flag = DUST_FLAG_OK;
    // initial guess u(y) from the inverse table
    const float fy = y * gq.z;
    const int m = min((int)fy, tb.NI - 2);
    const float ty = fminf(fy - (float)m, 1.f);
    const float4 iv = __ldg(tb.inv + (size_t)g * (tb.NI - 1) + m);
    const float ug = hermite(iv.x, iv.y, iv.z, iv.w, ty);
    const float fj = (ug - tb.log2Tmin) / tb.h2;
    int j = min(max((int)floorf(fj), 0), tb.NT - 2);
    float tau = fminf(fmaxf(fj - (float)j, 0.f), 1.f);
    // bracketing interval t_j <= y <= t_j+1
    const float4 *fwg = tb.fw + (size_t)g * (tb.NT - 1);
    float4 f4 = __ldg(fwg + j);
    for (int a = 0; a < 4; ++a) {
        if (y < f4.x && j > 0) { --j; tau = 1.f; }
        else if (y > f4.z && j < tb.NT - 2) { ++j; tau = 0.f; }
        else break;
        f4 = __ldg(fwg + j);
    }
    // Newton on the Hermite cubic q(tau) = t(u_j + tau h2) - t_j = y - t_j
    const float r = y - f4.x, d = f4.z - f4.x, m0 = f4.y, m1 = f4.w;
    const float c2 = 3.f * d - 2.f * m0 - m1, c3 = m0 + m1 - 2.f * d;
    float lo = 0.f, hi = 1.f;
    for (int it = 0; it < 4; ++it) {
        const float q = tau * (m0 + tau * (c2 + tau * c3)) - r;
        const float dq = m0 + tau * (2.f * c2 + 3.f * tau * c3);
        if (q < 0.f) lo = tau; else hi = tau;
        float nt = tau - q / dq;
        if (!(nt >= lo && nt <= hi)) nt = 0.5f * (lo + hi);  // bracketed fallback
        const float step = fabsf(nt - tau);
        tau = nt;
        if (step * tb.h2 < 2e-7f) break;
    }
    return __ldg(tb.Tnode + j) * exp2f(tau * tb.h2);
}

template <int R, bool EMIT, bool RESID, bool STORE_L>
__global__ void __launch_bounds__(NTH, 2)
k_solve_emit(DevTables tb, int64_t C, int TC, int GC, int chat_resident, const float *__restrict__ S,
             const float *__restrict__ n, float *__restrict__ T, float *__restrict__ L, int64_t ld,
             double *__restrict__ resid, uint8_t *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = tb.G, NKG = tb.NKG, K = tb.K, Gs = tb.Gs;
    const int TNS = 2 * G + 2;  // floats per cell row of (1/T, n 2^-m) pairs
    float4 *sC = reinterpret_cast<float4 *>(smem_raw);
    float *sTN = reinterpret_cast<float *>(sC + (EMIT ? (size_t)GC * 2 * NKG : 0));
    int *sM = reinterpret_cast<int *>(sTN + (size_t)TC * TNS);
    double *sAbs = reinterpret_cast<double *>(sM + ((TC + 1) & ~1));
    double *sEm = sAbs + TC;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (C + TC - 1) / TC;

    // phase-2 work items of this thread (fixed across tiles)
    int icell[R], ikg[R];
    float nax[R][KQ];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int it = r * NTH + tid;
        bool ok = it < TC * NKG;
        icell[r] = ok ? it / NKG : -1;
        ikg[r] = ok ? it % NKG : 0;
#pragma unroll
        for (int q = 0; q < KQ; ++q) nax[r][q] = EMIT ? __ldg(tb.nax + ikg[r] * KQ + q) : 0.f;
    }

    if (EMIT && chat_resident) {
        const float4 *src = reinterpret_cast<const float4 *>(tb.Chat);
        for (int i = tid; i < G * 2 * NKG; i += NTH) sC[i] = __ldg(src + i);
    }

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t c0 = tile * TC;
        const int nc = (int)((C - c0) < (int64_t)TC ? (C - c0) : (int64_t)TC);
        __syncthreads();  // previous tile finished with shared memory
        // phases 0 + 1, one warp per cell: exponent of max_g n, then the
        // temperatures (lanes over grains); the absorbed power of the residual
        // is reduced in a fixed order so that results do not depend on timing
        for (int c = warp; c < TC; c += NTH / 32) {
            const int64_t cell = c0 + c;
            float mx = 0.f;
            if (c < nc)
                for (int g = lane; g < G; g += 32) mx = fmaxf(mx, __ldg(n + cell * G + g));
            for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            int mc = 0;
            if (mx > 0.f && mx < INFINITY) frexpf(mx, &mc);
            double ab = 0.0;
            for (int g = lane; g < G; g += 32) {
                float invT = 1.f / tb.Tmax, nn = 0.f;
                if (c < nc) {
                    const float s = __ldg(S + cell * Gs + g);
                    const float nv = __ldg(n + cell * G + g);
                    int flag;
                    const float Tv = solve_T(tb, g, s, flag);
                    T[cell * G + g] = Tv;
                    if (flags) flags[cell * G + g] = (uint8_t)flag;
                    invT = __frcp_rn(Tv);
                    nn = scale2(nv, -mc);
                    if (RESID) {
                        double pe = flag == DUST_FLAG_OK ? (double)s * __ldg(tb.gscale + g)
                                  : flag == DUST_FLAG_LOW ? __ldg(tb.P0 + g)
                                  : flag == DUST_FLAG_HIGH ? __ldg(tb.Pmax + g)
                                  : (double)__int_as_float(0x7fc00000);
                        ab = fma((double)nv, pe, ab);
                    }
                }
                if (EMIT) *reinterpret_cast<float2 *>(sTN + (size_t)c * TNS + 2 * g) = make_float2(invT, nn);
            }
            if (RESID)
                for (int o = 16; o; o >>= 1) ab += __shfl_xor_sync(0xffffffffu, ab, o);
            if (lane == 0) {
                sM[c] = mc;
                if (RESID) sAbs[c] = ab;
            }
        }
        if (!EMIT) continue;
        __syncthreads();
        // phase 2: emission
        float acc[R][KQ], N[R][KQ], D[R][KQ];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < KQ; ++q) acc[r][q] = 0.f;
        for (int g0 = 0; g0 < G; g0 += GC) {
            const int gn = min(GC, G - g0);
            if (!chat_resident) {
                __syncthreads();
                const float4 *src = reinterpret_cast<const float4 *>(tb.Chat) + (size_t)g0 * 2 * NKG;
                for (int i = tid; i < gn * 2 * NKG; i += NTH) sC[i] = __ldg(src + i);
                __syncthreads();
            }
            const float4 *cbase = chat_resident ? sC + (size_t)g0 * 2 * NKG : sC;
            for (int gg0 = 0; gg0 < gn; gg0 += RG) {
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int q = 0; q < KQ; ++q) { N[r][q] = 0.f; D[r][q] = 1.f; }
#pragma unroll
                for (int u = 0; u < RG; ++u) {
                    const int gg = gg0 + u;
                    if (gg < gn) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if (icell[r] < 0) continue;
                            const float2 tn = *reinterpret_cast<const float2 *>(
                                sTN + (size_t)icell[r] * TNS + 2 * (g0 + gg));
                            const float4 ca = cbase[(gg * 2 + 0) * NKG + ikg[r]];
                            const float4 cb = cbase[(gg * 2 + 1) * NKG + ikg[r]];
                            const float cw[KQ] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
                            for (int q = 0; q < KQ; ++q) {
                                const float t = ex2_approx(nax[r][q] * tn.x);
                                const float wq = tn.y * cw[q];
                                const float e = fmaf(wq, D[r][q], -N[r][q]);
                                N[r][q] = fmaf(t, e, N[r][q]);
                                D[r][q] = fmaf(-t, D[r][q], D[r][q]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int q = 0; q < KQ; ++q) acc[r][q] = fmaf(N[r][q], rcp_approx(D[r][q]), acc[r][q]);
            }
        }
        // epilogue: scale, store, residual partials
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int c = icell[r];
            if (c < 0 || c >= nc) continue;
            const int64_t cell = c0 + c;
            const int mc = sM[c];
            double em = 0.0;
            const int kb = ikg[r] * KQ;
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                const int k = kb + q;
                if (k < K) {
                    const float Lv = scale2(acc[r][q], mc + __ldg(tb.qexp + k));
                    if (STORE_L) L[cell * ld + k] = Lv;
                    if (RESID) em = fma(__ldg(tb.w + k), (double)Lv, em);
                }
            }
            if (RESID) sEm[c * NKG + ikg[r]] = em;
        }
        if (RESID) {
            __syncthreads();
            for (int c = tid; c < nc; c += NTH) {
                double e = 0.0;
                for (int kg = 0; kg < NKG; ++kg) e += sEm[c * NKG + kg];
                resid[c0 + c] = e / (FOUR_PI * sAbs[c]) - 1.0;
            }
        }
    }
}

struct Plan {
    int R, TC, GC, resident;
    size_t smem;
};

Plan make_plan(const dust_ctx *ctx, bool emit) {
    const DevTables &tb = ctx->tb;
    Plan p{};
    p.R = 2;
    if (tb.NKG > p.R * NTH) p.R = 4;
    p.TC = emit ? (p.R * NTH) / tb.NKG : 64;
    if (p.TC < 1) p.TC = 1;
    if (p.TC > 64) p.TC = 64;
    const size_t per_cta = (size_t)(ctx->smem_optin ? ctx->smem_optin : 101376);
    const size_t budget = std::min<size_t>(per_cta, 110 * 1024);  // two CTAs per SM
    auto fixed = [&](int TC) {  // sTN, sM, sAbs, sEm (per item)
        return (size_t)TC * (2 * tb.G + 2) * 4 + (size_t)((TC + 1) & ~1) * 4 + (size_t)TC * 8 +
               (size_t)TC * tb.NKG * 8 + 64;
    };
    const size_t per_grain = (size_t)2 * tb.NKG * 16;
    if (!emit) { p.GC = 0; p.resident = 0; p.smem = fixed(p.TC); return p; }
    size_t full = per_grain * tb.G + fixed(p.TC);
    if (full <= budget) { p.GC = tb.G; p.resident = 1; p.smem = full; return p; }
    size_t avail = budget > fixed(p.TC) ? budget - fixed(p.TC) : 0;
    int gc = (int)(avail / per_grain) / RG * RG;
    if (gc < RG) gc = RG;
    p.GC = gc;
    p.resident = 0;
    p.smem = per_grain * gc + fixed(p.TC);
    return p;
}

template <int R, bool EMIT, bool RESID, bool STORE_L>
int launch_t(const dust_ctx *ctx, const Plan &p, int64_t C, const float *S, const float *n, float *T,
             float *L, int64_t ld, double *resid, uint8_t *flags, cudaStream_t st) {
    auto kern = k_solve_emit<R, EMIT, RESID, STORE_L>;
    DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    int64_t ntiles = (C + p.TC - 1) / p.TC;
    int blocks_per_sm = 0;
    DUST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NTH, p.smem));
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    int64_t grid = std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * blocks_per_sm);
    kern<<<(unsigned)grid, NTH, p.smem, st>>>(ctx->tb, C, p.TC, p.GC, p.resident, S, n, T, L, ld, resid,
                                              flags);
    DUST_CUDA_TRY(cudaGetLastError());
    return DUST_OK;
}

template <int R>
int launch_r(const dust_ctx *ctx, const Plan &p, int64_t C, const float *S, const float *n, float *T,
             float *L, int64_t ld, double *resid, uint8_t *flags, cudaStream_t st) {
    const bool emit = L || resid;
    if (!emit) return launch_t<R, false, false, false>(ctx, p, C, S, n, T, L, ld, resid, flags, st);
    if (L && resid) return launch_t<R, true, true, true>(ctx, p, C, S, n, T, L, ld, resid, flags, st);
    if (L) return launch_t<R, true, false, true>(ctx, p, C, S, n, T, L, ld, resid, flags, st);
    return launch_t<R, true, true, false>(ctx, p, C, S, n, T, L, ld, resid, flags, st);
}

}  // namespace

int launch_solve_emit(const dust_ctx *ctx, int64_t C, const float *S, const float *n, float *T,
                      float *L, int64_t ld, double *resid, uint8_t *flags, cudaStream_t st) {
    if (C <= 0) return DUST_OK;
    Plan p = make_plan(ctx, L || resid);
    if (p.R == 2) return launch_r<2>(ctx, p, C, S, n, T, L, ld, resid, flags, st);
    return launch_r<4>(ctx, p, C, S, n, T, L, ld, resid, flags, st);
}

}  // namespace dust

// Absorption contraction on the CUDA cores in FP32 (the plain FP32 path):
//   S[c,g] = sum_k J[c,k] W32[g,k]                          (Eq. 6, scaled)
// The paper's kernel 2 is the same matrix product with shared-memory tiles
// over wavelength intervals (Section 4.2).  Here: 128-cell x (16 TN)-grain CTA
// tiles, 16-wavelength double-buffered stages, an 8 x TN register tile per
// thread, FP32 FMA accumulation in ascending k.
#include "dust_internal.cuh"

namespace dust {
namespace {

constexpr int BM = 128, BK = 16, NTH = 256;

template <int TN, bool VEC>
__global__ void __launch_bounds__(NTH) k_gemm_simt(int64_t C, int K, const float *__restrict__ J,
                                                   int64_t ld, const float *__restrict__ W, int Kw,
                                                   int Gs, float *__restrict__ S) {
    constexpr int BN = 16 * TN;
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ float Bs[2][BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;

    // A loader: row ar, 8 consecutive k from ak
    const int ar = tid >> 1, ak = (tid & 1) * 8;
    const int64_t arow = m0 + ar;
    const bool arow_ok = arow < C;
    const float *Jrow = J + (arow_ok ? arow : 0) * ld;

    float a_reg[8];
    float b_reg[(BN * BK + NTH - 1) / NTH];

    auto load_tile = [&](int k0) {
        if (VEC && arow_ok && k0 + ak + 8 <= K) {
            float4 v0 = __ldg(reinterpret_cast<const float4 *>(Jrow + k0 + ak));
            float4 v1 = __ldg(reinterpret_cast<const float4 *>(Jrow + k0 + ak + 4));
            a_reg[0] = v0.x; a_reg[1] = v0.y; a_reg[2] = v0.z; a_reg[3] = v0.w;
            a_reg[4] = v1.x; a_reg[5] = v1.y; a_reg[6] = v1.z; a_reg[7] = v1.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                int k = k0 + ak + e;
                a_reg[e] = (arow_ok && k < K) ? __ldg(Jrow + k) : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < (BN * BK + NTH - 1) / NTH; ++i) {
            int idx = tid + i * NTH;
            int r = idx / BK, kk = idx % BK;
            int g = n0 + r;
            b_reg[i] = (idx < BN * BK && g < Gs) ? __ldg(W + (size_t)g * Kw + k0 + kk) : 0.f;
        }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
        for (int e = 0; e < 8; ++e) As[buf][ak + e][ar] = a_reg[e];
#pragma unroll
        for (int i = 0; i < (BN * BK + NTH - 1) / NTH; ++i) {
            int idx = tid + i * NTH;
            if (idx < BN * BK) Bs[buf][idx % BK][idx / BK] = b_reg[i];
        }
    };

    float acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    const int nk = (K + BK - 1) / BK;
    load_tile(0);
    store_tile(0);
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
        const int buf = t & 1;
        if (t + 1 < nk) load_tile((t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8 + 4]);
            float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (t + 1 < nk) store_tile(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int64_t row = m0 + ty * 8 + i;
        if (row >= C) break;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int col = n0 + tx + 16 * j;
            if (col < Gs) S[row * Gs + col] = acc[i][j];
        }
    }
}

template <int TN>
int launch_tn(const dust_ctx *ctx, int64_t C, const float *J, int64_t ld, float *S, cudaStream_t st) {
    const int Gs = ctx->tb.Gs;
    dim3 grid((unsigned)((C + BM - 1) / BM), (unsigned)((Gs + 16 * TN - 1) / (16 * TN)));
    bool vec = (ld % 4 == 0) && ((uintptr_t)J % 16 == 0);
    if (vec)
        k_gemm_simt<TN, true><<<grid, NTH, 0, st>>>(C, ctx->K, J, ld, ctx->W32, ctx->Kw, Gs, S);
    else
        k_gemm_simt<TN, false><<<grid, NTH, 0, st>>>(C, ctx->K, J, ld, ctx->W32, ctx->Kw, Gs, S);
    return DUST_OK;
}

}  // namespace

int launch_gemm_simt(const dust_ctx *ctx, int64_t C, const float *J, int64_t ld, float *S,
                     cudaStream_t st) {
    if (C <= 0) return DUST_OK;
    if ((C + BM - 1) / BM > 0x7fffffff) return set_error(DUST_EINVAL, "too many cells");
    int tiles16 = ctx->tb.Gs / 16;  // 1..32
    int ntile = (tiles16 + 7) / 8;
    int TN = (tiles16 + ntile - 1) / ntile;
    int rc;
    switch (TN) {
        case 1: rc = launch_tn<1>(ctx, C, J, ld, S, st); break;
        case 2: rc = launch_tn<2>(ctx, C, J, ld, S, st); break;
        case 3: rc = launch_tn<3>(ctx, C, J, ld, S, st); break;
        case 4: rc = launch_tn<4>(ctx, C, J, ld, S, st); break;
        case 5: rc = launch_tn<5>(ctx, C, J, ld, S, st); break;
        case 6: rc = launch_tn<6>(ctx, C, J, ld, S, st); break;
        case 7: rc = launch_tn<7>(ctx, C, J, ld, S, st); break;
        default: rc = launch_tn<8>(ctx, C, J, ld, S, st); break;
    }
    if (rc != DUST_OK) return rc;
    DUST_CUDA_TRY(cudaGetLastError());
    return DUST_OK;
}

}  // namespace dust

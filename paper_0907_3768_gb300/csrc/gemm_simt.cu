// Absorption contraction on the CUDA cores in FP32 (the plain FP32 path):
//   S[c,g] = sum_k J[c,k] W32[g,k]                          (Eq. 6, scaled)
// The paper's kernel 2 is the same matrix product with shared-memory tiles
// over wavelength intervals (Section 4.2).  Here: 128-cell x (16 TN)-grain CTA
// tiles over a work list of requests, 16-wavelength double-buffered stages,
// an 8 x TN register tile per thread, FP32 FMA accumulation in ascending k
// (so a cell's result does not depend on the tiling or the batch).
#include "dust_internal.cuh"

#include <algorithm>

namespace dust {
namespace {

constexpr int BM = 128, BK = 16, NTH = 256;

template <int TN>
__global__ void __launch_bounds__(NTH, 2) k_gemm_simt(const __grid_constant__ SimtBatch B) {
    constexpr int BN = 16 * TN;
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ float Bs[2][BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    const int64_t tile = blockIdx.x;
    int ri = 0;
    while (ri + 1 < B.nreq && tile >= B.req[ri + 1].tile_begin) ++ri;
    const SimtReq &q = B.req[ri];
    const int64_t local = tile - q.tile_begin;
    const int64_t m0 = (local / q.ntn) * BM;
    const int n0 = (int)(local % q.ntn) * BN;
    const int K = q.K, Kw = q.Kw, Gs = q.Gs;
    const int64_t C = q.C, ld = q.ld;
    const float *__restrict__ W = q.W;
    const bool vec = (ld % 4 == 0) && (((uintptr_t)q.J & 15) == 0);

    // A loader: row ar, 8 consecutive k from ak
    const int ar = tid >> 1, ak = (tid & 1) * 8;
    const int64_t arow = m0 + ar;
    const bool arow_ok = arow < C;
    const float *__restrict__ Jrow = q.J + (arow_ok ? arow : 0) * ld;

    float a_reg[8];
    float b_reg[(BN * BK + NTH - 1) / NTH];

    auto load_tile = [&](int k0) {
        if (vec && arow_ok && k0 + ak + 8 <= K) {
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
            if (col < Gs) q.S[row * Gs + col] = acc[i][j];
        }
    }
}

}  // namespace

void make_simt_req(const dust_ctx *ctx, int64_t C, const float *J, int64_t ld, float *S, SimtReq &r) {
    r.C = C;
    r.ld = ld;
    r.tile_begin = 0;
    r.J = J;
    r.W = ctx->W32;
    r.S = S;
    r.K = ctx->K;
    r.Kw = ctx->Kw;
    r.Gs = ctx->tb.Gs;
    r.ntn = 0;
}

// Picks the register tile width from the widest request, numbers the tiles
// and launches one CTA per (cell tile, grain tile).
int launch_simt_batch(SimtBatch &B, cudaStream_t st) {
    int gmax = 16;
    for (int i = 0; i < B.nreq; ++i) gmax = std::max(gmax, B.req[i].Gs);
    const int t16 = gmax / 16;  // 1..32
    const int ntile = (t16 + 7) / 8;
    const int TN = (t16 + ntile - 1) / ntile;
    int64_t t = 0;
    for (int i = 0; i < B.nreq; ++i) {
        SimtReq &r = B.req[i];
        r.ntn = (r.Gs + 16 * TN - 1) / (16 * TN);
        r.tile_begin = t;
        t += (r.C + BM - 1) / BM * r.ntn;
    }
    B.ntiles = t;
    if (t <= 0) return DUST_OK;
    if (t > 0x7fffffff) return set_error(DUST_EINVAL, "too many cells for one launch");
    const unsigned grid = (unsigned)t;
    switch (TN) {
        case 1: k_gemm_simt<1><<<grid, NTH, 0, st>>>(B); break;
        case 2: k_gemm_simt<2><<<grid, NTH, 0, st>>>(B); break;
        case 3: k_gemm_simt<3><<<grid, NTH, 0, st>>>(B); break;
        case 4: k_gemm_simt<4><<<grid, NTH, 0, st>>>(B); break;
        case 5: k_gemm_simt<5><<<grid, NTH, 0, st>>>(B); break;
        case 6: k_gemm_simt<6><<<grid, NTH, 0, st>>>(B); break;
        case 7: k_gemm_simt<7><<<grid, NTH, 0, st>>>(B); break;
        default: k_gemm_simt<8><<<grid, NTH, 0, st>>>(B); break;
    }
    DUST_CUDA_TRY(cudaGetLastError());
    return DUST_OK;
}

int launch_gemm_simt(const dust_ctx *ctx, int64_t C, const float *J, int64_t ld, float *S, cudaStream_t st) {
    if (C <= 0) return DUST_OK;
    SimtBatch B;
    B.nreq = 1;
    make_simt_req(ctx, C, J, ld, S, B.req[0]);
    return launch_simt_batch(B, st);
}

}  // namespace dust

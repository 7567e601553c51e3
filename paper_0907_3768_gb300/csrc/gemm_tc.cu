// Kernel (a): the absorption contraction of Eq. 6 on the 5th-generation
// tensor cores, S[c,g] = sum_k J[c,k] W32[g,k], with 16-bit operands split
// into hi + lo parts (three products hi.hi + lo.hi + hi.lo, FP32 accumulation
// in tensor memory).  The paper's kernel 2 (Section 4.2) is the same matrix
// product on CUDA cores in FP32.
//
// One persistent CTA per SM walks 128-cell tiles of a work list of requests.
// Warp roles:
//   warp 0      J producer: FP32 tiles of J (128 cells x 32 wavelengths,
//               128-byte swizzle) by TMA into a ring of staging buffers; it
//               runs as far ahead as that ring allows.
//   warp 1      owns tensor memory (two accumulators of 128 lanes x Gs FP32
//               columns when they fit) and issues tcgen05.mma from one thread.
//   warp 2      W producer: the pre-split 16-bit W chunk of each K step by a
//               bulk copy next to the converted A operand.
//   warps 3-6   one thread per cell row: per-cell power-of-two exponent of
//               max_k J[c,k] (first pass over the tile, FP16 only: J spans
//               ~8 decades), conversion of J 2^-e into hi/lo 16-bit values in
//               the K-major core-matrix layout (second pass).
//   warps 7-10  epilogue: tensor memory -> registers -> S = acc 2^(e - offsets),
//               overlapped with the next tile's MMAs in the other accumulator.
// Every mbarrier wait is bounded; on expiry the kernel records DUST_ETIMEOUT
// in the status word and winds down.
//
// k_gemm_tc_t is the grain-major form used when Gs <= 128: W is the MMA's A
// operand (M = 128 grain rows) and 256 cells of J its B operand (N = 256), so
// each MMA covers twice the cells; the issue cost of an MMA, not its
// tensor-pipe time, is what limits the cell-major form at small G.
// k_absorb_solve is the cell-major kernel with the temperature solve as its
// epilogue (S stays in tensor memory).
#include "dust_internal.cuh"
#include "mbar.cuh"
#include "solve_core.cuh"

#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

namespace dust {
namespace {

constexpr int BM = 128;                    // cells per tile (UMMA M)
constexpr int NTHREADS = 352;              // 11 warps
constexpr int NACC_MAX = 4;                // accumulators (and solver groups of the fused kernel), at most
constexpr int NTHREADS_F = (7 + 4 * NACC_MAX) * 32;  // fused kernel: 7 + 4 nacc warps
constexpr int FUSED_NS1 = 2, FUSED_NS2 = 2;          // fused kernel: ring depths, at most
constexpr int STAGE1_BYTES = BM * KC * 4;  // FP32 staging tile: 16 KB
constexpr int A_BYTES = BM * KC * 2;       // one 16-bit A part: 8 KB
// grain-major orientation (Gs <= 128): grains are the MMA's M, cells its N
constexpr int BN_T = 256;                     // cells per tile (UMMA N)
constexpr int MW = 128;                       // grain rows of the W operand (UMMA M; zero past Gs)
constexpr int STAGE1T_BYTES = BN_T * KC * 4;  // FP32 staging tile: 32 KB
constexpr int WA_PART = MW * KC * 2;          // one 16-bit W part: 8 KB
constexpr int JB_PART = BN_T * KC * 2;        // one 16-bit J part: 16 KB
constexpr int TN_NS1 = 4, TN_NS2 = 2;         // its ring depths, at most
constexpr int NCV_T = 8;                      // its converter warps
constexpr int RPT = BN_T / (32 * NCV_T);      // cell rows per converter thread
constexpr int NTHREADS_T = (3 + NCV_T + 4) * 32;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16, FP32 accumulation.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 32 lanes x 32 bits, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 bits, 4 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 bits, 32 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; LBO = byte step between core matrices along K,
// SBO = byte step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
    return d;                // base offset 0, absolute LBO mode, no swizzle
}

// Instruction descriptor of kind::f16: FP32 accumulator, K-major A and B.
__host__ __device__ constexpr uint32_t instr_desc(bool bf16, int M, int N) {
    return (1u << 4)                       // D format: F32
           | ((bf16 ? 1u : 0u) << 7)       // A format: BF16 = 1, F16 = 0
           | ((bf16 ? 1u : 0u) << 10)      // B format
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ uint32_t pack_split(float x0, float x1, bool bf16, uint32_t &lo) {
    uint32_t hi;
    if (bf16) {
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
        float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
    } else {
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
        __half2 h2 = *reinterpret_cast<__half2 *>(&hi);
        float2 hf = __half22float2(h2);
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - hf.y), "f"(x0 - hf.x));
    }
    return hi;
}

// Request of global tile `tile` (tiles of a CTA increase, so the search
// starts from the previous answer).
__device__ __forceinline__ int tc_req_of(const TcBatch &p, int64_t tile, int ri) {
    while (ri + 1 < p.nreq && tile >= p.req[ri + 1].tile_begin) ++ri;
    return ri;
}

// Waits (bounded, ignoring aborts) for the last copy issued into each slot of
// a ring of `ns` slots after `n` copies, so none lands after the CTA exits.
__device__ __forceinline__ void drain_ring(uint64_t *full, int ns, int64_t n, int *status) {
    for (int s = 0; s < ns; ++s) {
        const int64_t last = n - 1 - ((n - 1 - s) % ns + ns) % ns;
        if (last >= 0 && last % ns == s) mbar_drain(&full[s], (uint32_t)((last / ns) & 1), status);
    }
}

// Fused epilogue, one thread per cell row: the stand-alone solve's work for
// that cell, with S read from tensor memory (columns of accumulator `tbase`)
// instead of global memory.  Four grains per step; every result goes through
// the same solve_batch / grain_out arithmetic as the stand-alone solve, so T,
// the flags and the emission pairs are bitwise the same; only the order of the
// cell's absorbed-power sum differs (ascending grains here).  All lanes run
// the tensor-memory loads; rows past the request (valid = false) store nothing.
__device__ __forceinline__ void solve_row(const EmitReq &q, int64_t cell, bool valid, int ex, uint32_t tbase) {
    const DevTables &tb = q.tb;
    const int G = tb.G, G8 = tb.G8;
    const bool emit = (q.mode & EMIT_ON) != 0, rs = (q.mode & EMIT_RESID) != 0, mass = (q.mode & EMIT_MASS) != 0;
    const bool with_n = emit && !mass && valid;
    const int64_t c = valid ? cell : 0;
    const float *nrow = q.n + c * G;
    const bool quad_rows = (G & 3) == 0;  // rows of T, flags and n start on 4-element boundaries
    const bool nvec = quad_rows && ((uintptr_t)q.n & 15) == 0;
    const bool tvec = quad_rows && ((uintptr_t)q.T & 15) == 0;
    const bool fvec = quad_rows && ((uintptr_t)q.flags & 3) == 0;
    int mc = 0;
    float ms = 0.f;  // dust-mass form: m_c = ms 2^mc
    if (emit && valid) {
        if (mass) {
            const float m = __ldg(q.n + c);
            ms = (m != 0.f && isfinite(m)) ? frexpf(m, &mc) : m;
        } else {
            float mx = 0.f;
            if (nvec) {
                for (int g = 0; g < G; g += 4) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(nrow + g));
                    mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
                }
            } else {
                for (int g = 0; g < G; ++g) mx = fmaxf(mx, __ldg(nrow + g));
            }
            if (mx > 0.f && mx < INFINITY) frexpf(mx, &mc);
        }
    }
    float *Trow = q.T + c * G;
    uint8_t *frow = q.flags ? q.flags + c * G : nullptr;
    float ah = 0.f, al = 0.f;  // absorbed power n 2^-m_c Pe 2^-Eg, float-float
    for (int g0 = 0; g0 < G8; g0 += 4) {
        float v[4];
        __syncwarp();
        tmem_ld4(tbase + (uint32_t)g0, v);
        int gi[4], fl[4];
        float sv[4], nv[4] = {0.f, 0.f, 0.f, 0.f}, Tv[4];
        float4 gq[4];
        const bool full = g0 + 4 <= G;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int g = g0 + i;
            gi[i] = g < G ? g : 0;
            sv[i] = g < G ? scale2(v[i], ex) : 0.f;
            gq[i] = __ldg(reinterpret_cast<const float4 *>(tb.gp) + gi[i]);
        }
        if (with_n) {
            if (nvec && full) {
                const float4 n4 = __ldg(reinterpret_cast<const float4 *>(nrow + g0));
                nv[0] = n4.x; nv[1] = n4.y; nv[2] = n4.z; nv[3] = n4.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) nv[i] = g0 + i < G ? __ldg(nrow + g0 + i) : 0.f;
            }
        }
        solve_batch<4>(tb, gi, sv, gq, Tv, fl);
        if (!valid) continue;
        if (tvec && full) {
            *reinterpret_cast<float4 *>(Trow + g0) = make_float4(Tv[0], Tv[1], Tv[2], Tv[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) if (g0 + i < G) Trow[g0 + i] = Tv[i];
        }
        if (frow) {
            if (fvec && full) {
                *reinterpret_cast<uint32_t *>(frow + g0) =
                    (uint32_t)fl[0] | ((uint32_t)fl[1] << 8) | ((uint32_t)fl[2] << 16) | ((uint32_t)fl[3] << 24);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) if (g0 + i < G) frow[g0 + i] = (uint8_t)fl[i];
            }
        }
        if (emit) {
            float invT[4], nn[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                invT[i] = PAD_INV_T;
                nn[i] = 0.f;
                if (g0 + i < G) grain_out(tb, g0 + i, Tv[i], fl[i], sv[i], nv[i], mc, mass, rs, invT[i], nn[i], ah, al);
            }
            // pair rows are G8 (a multiple of 8) long and 16-byte aligned
            if (mass) {
                *reinterpret_cast<float4 *>(reinterpret_cast<float *>(q.prep) + c * G8 + g0) =
                    make_float4(invT[0], invT[1], invT[2], invT[3]);
            } else {
                float4 *dst = reinterpret_cast<float4 *>(q.prep + c * G8 + g0);
                dst[0] = make_float4(invT[0], nn[0], invT[1], nn[1]);
                dst[1] = make_float4(invT[2], nn[2], invT[3], nn[3]);
            }
        }
    }
    if (emit && valid) {
        CellInfo ci;
        ci.mc = mc;
        ci.ah = rs ? ah : 0.f;
        ci.al = rs ? al : 0.f;
        ci.ms_bits = __float_as_int(ms);
        q.cell[c] = ci;
    }
}

// TcBatch fields: GsMax sets the ring layout, ns1 / ns2 the ring depths,
// nacc the accumulators (tmem_cols each), j_off scales J to
// [2^(j_off-1), 2^j_off) per cell, off_exp is the W image scale folded back
// in the epilogue.
template <bool BF16, bool TWO_PASS, bool FUSED>
__device__ __forceinline__ void gemm_body(const TcBatch &p, const SolveList *sl) {
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int B_BYTES = p.GsMax * KC * 2 * 2;  // ring slot of a hi + lo W chunk
    unsigned char *st1 = smem;
    unsigned char *stA = st1 + (size_t)p.ns1 * STAGE1_BYTES;
    unsigned char *stB = stA + (size_t)p.ns2 * 2 * A_BYTES;
    uint64_t *bars = (uint64_t *)(stB + (size_t)p.ns2 * B_BYTES);
    uint64_t *full1 = bars, *empty1 = full1 + p.ns1;
    uint64_t *a_full = empty1 + p.ns1, *b_full = a_full + p.ns2, *ab_empty = b_full + p.ns2;
    uint64_t *acc_full = ab_empty + p.ns2, *acc_empty = acc_full + NACC_MAX;
    uint64_t *e_full = acc_empty + NACC_MAX, *e_empty = e_full + NACC_MAX, *drain = e_empty + NACC_MAX;
    int *e_smem = (int *)(drain + 1);                 // [NACC_MAX][BM] per-cell exponents
    uint32_t *tmem_slot = (uint32_t *)(e_smem + NACC_MAX * BM);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = p.ntiles;
    const int nacc = p.nacc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.ns1; ++s) { mbar_init(&full1[s], 1); mbar_init(&empty1[s], 4); }
        for (int s = 0; s < p.ns2; ++s) { mbar_init(&a_full[s], 4); mbar_init(&b_full[s], 1); mbar_init(&ab_empty[s], 1); }
        for (int b = 0; b < NACC_MAX; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
            mbar_init(&e_full[b], 4);
            mbar_init(&e_empty[b], 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(p.tmem_cols * nacc) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ J producer
        if (lane == 0) {
            int s1 = 0, ri = 0;
            uint32_t ph1 = 0;
            int64_t n1 = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                ri = tc_req_of(p, tile, ri);
                const TcReq &q = p.req[ri];
                const CUtensorMap *tm = &p.tm[ri];
                const int row0 = (int)((tile - q.tile_begin) * BM);
                for (int pass = TWO_PASS ? 0 : 1; pass < 2 && ok; ++pass) {
                    for (int kc = 0; kc < q.nkc && ok; ++kc) {
                        if (!(ok = mbar_wait(&empty1[s1], ph1 ^ 1, abort_flag, p.status))) break;
                        mbar_expect_tx(&full1[s1], STAGE1_BYTES);
                        tma_load_2d(st1 + (size_t)s1 * STAGE1_BYTES, tm, kc * KC, row0, &full1[s1]);
                        ++n1;
                        if (++s1 == p.ns1) { s1 = 0; ph1 ^= 1; }
                    }
                }
            }
            if (!ok) drain_ring(full1, p.ns1, n1, p.status);
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------ W producer
        if (lane == 0) {
            int sa = 0, ri = 0;
            uint32_t pha = 0;
            int64_t n2 = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                ri = tc_req_of(p, tile, ri);
                const TcReq &q = p.req[ri];
                const uint32_t wbytes = (uint32_t)q.Gs * KC * 4;  // this request's hi + lo chunk
                for (int kc = 0; kc < q.nkc && ok; ++kc) {
                    if (!(ok = mbar_wait(&ab_empty[sa], pha ^ 1, abort_flag, p.status))) break;
                    mbar_expect_tx(&b_full[sa], wbytes);
                    bulk_load(stB + (size_t)sa * B_BYTES, q.Wimg + (size_t)kc * (wbytes / 2), wbytes, &b_full[sa]);
                    ++n2;
                    if (++sa == p.ns2) { sa = 0; pha ^= 1; }
                }
            }
            if (!ok) drain_ring(b_full, p.ns2, n2, p.status);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int sa = 0, ri = 0;
            uint32_t pha = 0;
            int64_t it = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
                ri = tc_req_of(p, tile, ri);
                const int Gs = p.req[ri].Gs, nkc = p.req[ri].nkc, np = p.req[ri].nparts;
                const int b = (int)(it % nacc);
                const uint32_t ub = (uint32_t)((it / nacc) & 1);
                const uint32_t d_tmem = tmem + (uint32_t)(b * p.tmem_cols);
                const uint32_t idesc_full = instr_desc(BF16, BM, Gs <= 256 ? Gs : 256);
                const uint32_t idesc_tail = instr_desc(BF16, BM, Gs > 256 ? Gs - 256 : 16);
                if (!(ok = mbar_wait(&acc_empty[b], ub ^ 1, abort_flag, p.status))) break;
                tc_fence_after();
                for (int kc = 0; kc < nkc && ok; ++kc) {
                    if (!(ok = mbar_wait(&a_full[sa], pha, abort_flag, p.status))) break;
                    if (!(ok = mbar_wait(&b_full[sa], pha, abort_flag, p.status))) break;
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(stA + (size_t)sa * 2 * A_BYTES);
                    const uint32_t b_base = smem_u32(stB + (size_t)sa * B_BYTES);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
                        for (int part = 0; part < 3; ++part) {
                            // hi.hi, lo.hi, hi.lo (np = 2: the last left out)
                            if (part >= np) break;
                            const uint32_t aoff = (part == 1 ? A_BYTES : 0) + ks * 256;
                            const uint32_t boff = (part == 2 ? Gs * KC * 2 : 0) + ks * 256;
                            const uint32_t acc = (kc | ks | part) ? 1u : 0u;
                            tc_mma(d_tmem, smem_desc(a_base + aoff, 128, 512), smem_desc(b_base + boff, 128, 512),
                                   idesc_full, acc);
                            if (Gs > 256)
                                tc_mma(d_tmem + 256, smem_desc(a_base + aoff, 128, 512),
                                       smem_desc(b_base + boff + 32 * 512, 128, 512), idesc_tail, acc);
                        }
                    }
                    tc_commit(&ab_empty[sa]);
                    if (++sa == p.ns2) { sa = 0; pha ^= 1; }
                }
                if (ok) tc_commit(&acc_full[b]);
            }
            // drain every MMA still in flight before tensor memory is freed
            tc_commit(drain);
            mbar_drain(drain, 0, p.status);
        }
    } else if (warp < 7) {
        // ------------------------------------------------------------ converters
        const int r = (warp - 3) * 32 + lane;  // tile row owned by this thread
        int s1 = 0, sa = 0, ri = 0;
        uint32_t ph1 = 0, pha = 0;
        int64_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
            ri = tc_req_of(p, tile, ri);
            const TcReq &q = p.req[ri];
            int e = 0;
            if (TWO_PASS) {
                float mx = 0.f;
                for (int kc = 0; kc < q.nkc; ++kc) {
                    if (!(ok = mbar_wait(&full1[s1], ph1, abort_flag, p.status))) break;
                    const unsigned char *src = st1 + (size_t)s1 * STAGE1_BYTES + r * 128;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float4 v = *reinterpret_cast<const float4 *>(src + ((j ^ (r & 7)) << 4));
                        mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty1[s1]);
                    if (++s1 == p.ns1) { s1 = 0; ph1 ^= 1; }
                }
                if (!ok) break;
                if (mx > 0.f && mx < INFINITY) frexpf(mx, &e);
                e = min(max(e, p.j_off - 126), p.j_off + 126);  // keep 2^(j_off - e) a normal float
                // hand the exponent to the epilogue
                const int b = (int)(it % nacc);
                const uint32_t ub = (uint32_t)((it / nacc) & 1);
                if (!(ok = mbar_wait(&e_empty[b], ub ^ 1, abort_flag, p.status))) break;
                e_smem[b * BM + r] = e;
                __syncwarp();
                if (lane == 0) mbar_arrive(&e_full[b]);
            }
            const float scale = __int_as_float((127 - e + p.j_off) << 23);  // 2^(j_off - e)
            for (int kc = 0; kc < q.nkc; ++kc) {
                if (!(ok = mbar_wait(&full1[s1], ph1, abort_flag, p.status))) break;
                if (!(ok = mbar_wait(&ab_empty[sa], pha ^ 1, abort_flag, p.status))) break;
                const unsigned char *src = st1 + (size_t)s1 * STAGE1_BYTES + r * 128;
                unsigned char *dhi = stA + (size_t)sa * 2 * A_BYTES + (r >> 3) * 512 + (r & 7) * 16;
                unsigned char *dlo = dhi + A_BYTES;
#pragma unroll
                for (int cm = 0; cm < 4; ++cm) {  // 8 wavelengths = one core-matrix row
                    float4 v0 = *reinterpret_cast<const float4 *>(src + (((2 * cm) ^ (r & 7)) << 4));
                    float4 v1 = *reinterpret_cast<const float4 *>(src + (((2 * cm + 1) ^ (r & 7)) << 4));
                    uint4 h, l;
                    h.x = pack_split(v0.x * scale, v0.y * scale, BF16, l.x);
                    h.y = pack_split(v0.z * scale, v0.w * scale, BF16, l.y);
                    h.z = pack_split(v1.x * scale, v1.y * scale, BF16, l.z);
                    h.w = pack_split(v1.z * scale, v1.w * scale, BF16, l.w);
                    *reinterpret_cast<uint4 *>(dhi + cm * 128) = h;
                    *reinterpret_cast<uint4 *>(dlo + cm * 128) = l;
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) { mbar_arrive(&a_full[sa]); mbar_arrive(&empty1[s1]); }
                if (++s1 == p.ns1) { s1 = 0; ph1 ^= 1; }
                if (++sa == p.ns2) { sa = 0; pha ^= 1; }
            }
        }
    } else if constexpr (FUSED) {
        // ------------------------------------------------------------ solver groups
        // group grp owns accumulator grp and the CTA's tiles it = grp, grp + nacc, ...
        const int grp = (warp - 7) >> 2;
        const int quad = warp & 3;        // tensor-memory lane quarter of this warp
        const int r = quad * 32 + lane;   // tile row
        int ri = 0;
        int64_t it = grp;
        bool ok = true;
        for (int64_t tile = blockIdx.x + (int64_t)grp * gridDim.x; tile < ntiles && ok;
             tile += (int64_t)nacc * gridDim.x, it += nacc) {
            ri = tc_req_of(p, tile, ri);
            const TcReq &tq = p.req[ri];
            const uint32_t ub = (uint32_t)((it / nacc) & 1);
            int e = 0;
            if (TWO_PASS) {
                if (!(ok = mbar_wait(&e_full[grp], ub, abort_flag, p.status))) break;
                e = e_smem[grp * BM + r];
                __syncwarp();
                if (lane == 0) mbar_arrive(&e_empty[grp]);
            }
            if (!(ok = mbar_wait(&acc_full[grp], ub, abort_flag, p.status))) break;
            tc_fence_after();
            const int64_t cell = (tile - tq.tile_begin) * BM + r;
            const uint32_t tbase = tmem + (uint32_t)(grp * p.tmem_cols) + ((uint32_t)(quad * 32) << 16);
            solve_row(sl->req[ri], cell, cell < tq.C, e - p.j_off - p.off_exp, tbase);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[grp]);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quad = warp & 3;        // tensor-memory lane quarter of this warp
        const int r = quad * 32 + lane;   // tile row
        int ri = 0;
        int64_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
            ri = tc_req_of(p, tile, ri);
            const TcReq &q = p.req[ri];
            const int b = (int)(it % nacc);
            const uint32_t ub = (uint32_t)((it / nacc) & 1);
            int e = 0;
            if (TWO_PASS) {
                if (!(ok = mbar_wait(&e_full[b], ub, abort_flag, p.status))) break;
                e = e_smem[b * BM + r];
                __syncwarp();
                if (lane == 0) mbar_arrive(&e_empty[b]);
            }
            if (!(ok = mbar_wait(&acc_full[b], ub, abort_flag, p.status))) break;
            tc_fence_after();
            const int64_t row = (tile - q.tile_begin) * BM + r;
            const int ex = e - p.j_off - p.off_exp;
            float *dst = q.S + row * q.Gs;
            const uint32_t tbase = tmem + (uint32_t)(b * p.tmem_cols) + ((uint32_t)(quad * 32) << 16);
            for (int c0 = 0; c0 < q.Gs; c0 += 16) {
                float v[16];
                tmem_ld16(tbase + c0, v);
                if (row < q.C) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4 *>(dst + c0 + i) =
                            make_float4(scale2(v[i], ex), scale2(v[i + 1], ex), scale2(v[i + 2], ex),
                                        scale2(v[i + 3], ex));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols * nacc)
                     : "memory");
    }
}

template <bool BF16, bool TWO_PASS>
__global__ void __launch_bounds__(NTHREADS, 1) k_gemm_tc(const __grid_constant__ TcBatch p) {
    gemm_body<BF16, TWO_PASS, false>(p, nullptr);
}

// The same contraction with the temperature solve as its epilogue: S never
// leaves tensor memory.  Solver group g (warps 7 + 4g .. 10 + 4g) takes every
// nacc-th tile of the CTA from accumulator g, so nacc tiles are solved at
// once while the MMAs of the next ones run.
template <bool BF16, bool TWO_PASS>
// 80 registers: each SM sub-partition holds 16384, and 23 warps put six on some
__global__ void __launch_bounds__(NTHREADS_F, 1) k_absorb_solve(const __grid_constant__ TcBatch p,
                                                                const __grid_constant__ SolveList sl) {
    gemm_body<BF16, TWO_PASS, true>(p, &sl);
}

// Grain-major form of the same contraction for Gs <= 128: W (grains x K,
// zero rows up to 128) is the MMA's A operand and a 256-cell tile of J its B
// operand, so one MMA covers twice the cells of the cell-major kernel at
// about the same issue cost; the accumulator is 128 grain lanes x 256 cell
// columns.  Roles as in k_gemm_tc: warp 0 J producer (TMA, 256-row boxes),
// warp 1 tensor memory + MMA issuer, warp 2 W producer (two bulk copies per
// chunk: hi and lo parts into their 128-row slots), then NCV_T converter
// warps (256 / (32 NCV_T) cell rows per thread) and four epilogue warps
// (thread = grain, 32 cell columns per tensor-memory load; each store of a
// warp is 32 consecutive grains of one cell row of S).
template <bool BF16, bool TWO_PASS>
__global__ void __launch_bounds__(NTHREADS_T, 1) k_gemm_tc_t(const __grid_constant__ TcBatch p) {
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *st1 = smem;                                        // [ns1] FP32 J tiles
    unsigned char *stW = st1 + (size_t)p.ns1 * STAGE1T_BYTES;         // [ns2] W hi | lo
    unsigned char *stJ = stW + (size_t)p.ns2 * 2 * WA_PART;           // [ns2] J hi | lo
    uint64_t *bars = (uint64_t *)(stJ + (size_t)p.ns2 * 2 * JB_PART);
    uint64_t *full1 = bars, *empty1 = full1 + p.ns1;
    uint64_t *w_full = empty1 + p.ns1, *j_full = w_full + p.ns2, *ab_empty = j_full + p.ns2;
    uint64_t *acc_full = ab_empty + p.ns2, *acc_empty = acc_full + 2;
    uint64_t *e_full = acc_empty + 2, *e_empty = e_full + 2, *drain = e_empty + 2;
    int *e_smem = (int *)(drain + 1);                 // [2][BN_T] per-cell exponents
    uint32_t *tmem_slot = (uint32_t *)(e_smem + 2 * BN_T);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = p.ntiles;

    // W rows past Gs stay zero: the bulk copies write only the first Gs rows of each part
    for (int i = threadIdx.x; i < p.ns2 * 2 * WA_PART / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(stW)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async();
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.ns1; ++s) { mbar_init(&full1[s], 1); mbar_init(&empty1[s], NCV_T); }
        for (int s = 0; s < p.ns2; ++s) { mbar_init(&w_full[s], 1); mbar_init(&j_full[s], NCV_T); mbar_init(&ab_empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
            mbar_init(&e_full[b], NCV_T);
            mbar_init(&e_empty[b], 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(2 * BN_T) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ J producer
        if (lane == 0) {
            int s1 = 0, ri = 0;
            uint32_t ph1 = 0;
            int64_t n1 = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                ri = tc_req_of(p, tile, ri);
                const TcReq &q = p.req[ri];
                const CUtensorMap *tm = &p.tm[ri];
                const int row0 = (int)((tile - q.tile_begin) * BN_T);
                for (int pass = TWO_PASS ? 0 : 1; pass < 2 && ok; ++pass) {
                    for (int kc = 0; kc < q.nkc && ok; ++kc) {
                        if (!(ok = mbar_wait(&empty1[s1], ph1 ^ 1, abort_flag, p.status))) break;
                        mbar_expect_tx(&full1[s1], STAGE1T_BYTES);
                        tma_load_2d(st1 + (size_t)s1 * STAGE1T_BYTES, tm, kc * KC, row0, &full1[s1]);
                        ++n1;
                        if (++s1 == p.ns1) { s1 = 0; ph1 ^= 1; }
                    }
                }
            }
            if (!ok) drain_ring(full1, p.ns1, n1, p.status);
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------ W producer
        if (lane == 0) {
            int sa = 0, ri = 0;
            uint32_t pha = 0;
            int64_t n2 = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                ri = tc_req_of(p, tile, ri);
                const TcReq &q = p.req[ri];
                const uint32_t part = (uint32_t)q.Gs * KC * 2;  // one part of this request's chunk
                for (int kc = 0; kc < q.nkc && ok; ++kc) {
                    if (!(ok = mbar_wait(&ab_empty[sa], pha ^ 1, abort_flag, p.status))) break;
                    mbar_expect_tx(&w_full[sa], 2 * part);
                    const unsigned char *src = reinterpret_cast<const unsigned char *>(q.Wimg) + (size_t)kc * 2 * part;
                    unsigned char *dst = stW + (size_t)sa * 2 * WA_PART;
                    bulk_load(dst, src, part, &w_full[sa]);
                    bulk_load(dst + WA_PART, src + part, part, &w_full[sa]);
                    ++n2;
                    if (++sa == p.ns2) { sa = 0; pha ^= 1; }
                }
            }
            if (!ok) drain_ring(w_full, p.ns2, n2, p.status);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int sa = 0, ri = 0;
            uint32_t pha = 0;
            int64_t it = 0;
            bool ok = true;
            const uint32_t idesc = instr_desc(BF16, MW, BN_T);
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
                ri = tc_req_of(p, tile, ri);
                const int nkc = p.req[ri].nkc, np = p.req[ri].nparts;
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)((it >> 1) & 1);
                const uint32_t d_tmem = tmem + (uint32_t)(b * BN_T);
                if (!(ok = mbar_wait(&acc_empty[b], ub ^ 1, abort_flag, p.status))) break;
                tc_fence_after();
                for (int kc = 0; kc < nkc && ok; ++kc) {
                    if (!(ok = mbar_wait(&w_full[sa], pha, abort_flag, p.status))) break;
                    if (!(ok = mbar_wait(&j_full[sa], pha, abort_flag, p.status))) break;
                    tc_fence_after();
                    const uint32_t w_base = smem_u32(stW + (size_t)sa * 2 * WA_PART);
                    const uint32_t j_base = smem_u32(stJ + (size_t)sa * 2 * JB_PART);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
                        for (int part = 0; part < 3; ++part) {
                            // W hi . J hi, W hi . J lo, W lo . J hi (np = 2: the last left out)
                            if (part >= np) break;
                            const uint32_t woff = (part == 2 ? WA_PART : 0) + ks * 256;
                            const uint32_t joff = (part == 1 ? JB_PART : 0) + ks * 256;
                            const uint32_t acc = (kc | ks | part) ? 1u : 0u;
                            tc_mma(d_tmem, smem_desc(w_base + woff, 128, 512), smem_desc(j_base + joff, 128, 512),
                                   idesc, acc);
                        }
                    }
                    tc_commit(&ab_empty[sa]);
                    if (++sa == p.ns2) { sa = 0; pha ^= 1; }
                }
                if (ok) tc_commit(&acc_full[b]);
            }
            // drain every MMA still in flight before tensor memory is freed
            tc_commit(drain);
            mbar_drain(drain, 0, p.status);
        }
    } else if (warp < 3 + NCV_T) {
        // ------------------------------------------------------------ converters
        const int r0 = (warp - 3) * 32 + lane;  // cell rows r0 + h NCV_T 32 of the tile, h < RPT
        int s1 = 0, sa = 0, ri = 0;
        uint32_t ph1 = 0, pha = 0;
        int64_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
            ri = tc_req_of(p, tile, ri);
            const TcReq &q = p.req[ri];
            int e[RPT] = {};
            if (TWO_PASS) {
                float mx[RPT] = {};
                for (int kc = 0; kc < q.nkc; ++kc) {
                    if (!(ok = mbar_wait(&full1[s1], ph1, abort_flag, p.status))) break;
#pragma unroll
                    for (int h = 0; h < RPT; ++h) {
                        const int r = r0 + h * NCV_T * 32;
                        const unsigned char *src = st1 + (size_t)s1 * STAGE1T_BYTES + r * 128;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float4 v = *reinterpret_cast<const float4 *>(src + ((j ^ (r & 7)) << 4));
                            mx[h] = fmaxf(mx[h], fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty1[s1]);
                    if (++s1 == p.ns1) { s1 = 0; ph1 ^= 1; }
                }
                if (!ok) break;
#pragma unroll
                for (int h = 0; h < RPT; ++h) {
                    if (mx[h] > 0.f && mx[h] < INFINITY) frexpf(mx[h], &e[h]);
                    e[h] = min(max(e[h], p.j_off - 126), p.j_off + 126);  // keep 2^(j_off - e) a normal float
                }
                // hand the exponents to the epilogue
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)((it >> 1) & 1);
                if (!(ok = mbar_wait(&e_empty[b], ub ^ 1, abort_flag, p.status))) break;
#pragma unroll
                for (int h = 0; h < RPT; ++h) e_smem[b * BN_T + r0 + h * NCV_T * 32] = e[h];
                __syncwarp();
                if (lane == 0) mbar_arrive(&e_full[b]);
            }
            float scale[RPT];
#pragma unroll
            for (int h = 0; h < RPT; ++h) scale[h] = __int_as_float((127 - e[h] + p.j_off) << 23);  // 2^(j_off - e)
            for (int kc = 0; kc < q.nkc; ++kc) {
                if (!(ok = mbar_wait(&full1[s1], ph1, abort_flag, p.status))) break;
                if (!(ok = mbar_wait(&ab_empty[sa], pha ^ 1, abort_flag, p.status))) break;
#pragma unroll
                for (int h = 0; h < RPT; ++h) {
                    const int r = r0 + h * NCV_T * 32;
                    const unsigned char *src = st1 + (size_t)s1 * STAGE1T_BYTES + r * 128;
                    unsigned char *dhi = stJ + (size_t)sa * 2 * JB_PART + (r >> 3) * 512 + (r & 7) * 16;
                    unsigned char *dlo = dhi + JB_PART;
#pragma unroll
                    for (int cm = 0; cm < 4; ++cm) {  // 8 wavelengths = one core-matrix row
                        float4 v0 = *reinterpret_cast<const float4 *>(src + (((2 * cm) ^ (r & 7)) << 4));
                        float4 v1 = *reinterpret_cast<const float4 *>(src + (((2 * cm + 1) ^ (r & 7)) << 4));
                        uint4 hv, lv;
                        hv.x = pack_split(v0.x * scale[h], v0.y * scale[h], BF16, lv.x);
                        hv.y = pack_split(v0.z * scale[h], v0.w * scale[h], BF16, lv.y);
                        hv.z = pack_split(v1.x * scale[h], v1.y * scale[h], BF16, lv.z);
                        hv.w = pack_split(v1.z * scale[h], v1.w * scale[h], BF16, lv.w);
                        *reinterpret_cast<uint4 *>(dhi + cm * 128) = hv;
                        *reinterpret_cast<uint4 *>(dlo + cm * 128) = lv;
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) { mbar_arrive(&j_full[sa]); mbar_arrive(&empty1[s1]); }
                if (++s1 == p.ns1) { s1 = 0; ph1 ^= 1; }
                if (++sa == p.ns2) { sa = 0; pha ^= 1; }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quad = warp & 3;        // tensor-memory lane quarter of this warp
        const int g = quad * 32 + lane;   // grain row of the accumulator
        int ri = 0;
        int64_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
            ri = tc_req_of(p, tile, ri);
            const TcReq &q = p.req[ri];
            const int b = (int)(it & 1);
            const uint32_t ub = (uint32_t)((it >> 1) & 1);
            if (TWO_PASS && !(ok = mbar_wait(&e_full[b], ub, abort_flag, p.status))) break;
            if (!(ok = mbar_wait(&acc_full[b], ub, abort_flag, p.status))) break;
            tc_fence_after();
            const int Gs = q.Gs;
            const int64_t cell0 = (tile - q.tile_begin) * BN_T;
            const int nc = (int)min((int64_t)BN_T, q.C - cell0);  // cells of this tile
            const uint32_t tbase = tmem + (uint32_t)(b * BN_T) + ((uint32_t)(quad * 32) << 16);
            if (quad * 32 < Gs) {  // warp-uniform: quarters past the grains hold zeros only
                float *col = q.S + cell0 * Gs + g;  // S[cell0][g]
                const bool gok = g < Gs;
                const int ex0 = -p.j_off - p.off_exp;
                for (int c0 = 0; c0 < BN_T; c0 += 32) {
                    float v[32];
                    tmem_ld32(tbase + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int ex = (TWO_PASS ? e_smem[b * BN_T + c0 + i] : 0) + ex0;
                        if (gok && c0 + i < nc) col[(c0 + i) * Gs] = scale2(v[i], ex);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&acc_empty[b]);
                if (TWO_PASS) mbar_arrive(&e_empty[b]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN_T) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(TcBatch) + sizeof(SolveList) <= 32764, "fused launch parameters too large");

template <bool BF16, bool TWO_PASS>
int launch_t(const TcBatch &B, size_t smem, int grid, cudaStream_t st, const SolveList *sl) {
    if (B.orient == 1) {
        auto kern = k_gemm_tc_t<BF16, TWO_PASS>;
        DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, NTHREADS_T, smem, st>>>(B);
    } else if (sl) {
        auto kern = k_absorb_solve<BF16, TWO_PASS>;
        DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // the smallest shared-memory carveout that holds the rings: the rest is L1
        const int pct = (int)std::min<size_t>(100, (smem + 2048) * 100 / (228 * 1024) + 1);
        DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
        const int block = (7 + 4 * B.nacc) * 32;
        if (block > NTHREADS_F) return set_error(DUST_EINVAL, "fused kernel: %d accumulators", B.nacc);
        kern<<<grid, block, smem, st>>>(B, *sl);
    } else {
        auto kern = k_gemm_tc<BF16, TWO_PASS>;
        DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, NTHREADS, smem, st>>>(B);
    }
    DUST_CUDA_TRY(cudaGetLastError());
    return DUST_OK;
}

}  // namespace

int tc_orient(const dust_ctx *ctx) { return ctx->tb.Gs <= MW ? 1 : 0; }

int make_tc_req(const dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, float *S, TcReq &r,
                CUtensorMap &tm, int orient) {
    const bool bf16 = precision == DUST_PREC_BF16X3;
    const int K = ctx->K;
    if (C > 0x7fffffffLL - BN_T) return set_error(DUST_EINVAL, "too many cells for one tensor-core launch");
    auto encode = get_encode();
    if (!encode) return set_error(DUST_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)C};
    cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    if (orient == 1 && ctx->tb.Gs > MW) return set_error(DUST_EINVAL, "grain-major GEMM needs Gs <= %d", MW);
    cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)(orient == 1 ? BN_T : BM)};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = encode(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)J, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return set_error(DUST_EINVAL, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    r.C = C;
    r.tile_begin = 0;
    r.Gs = ctx->tb.Gs;
    r.nkc = (K + KC - 1) / KC;
    r.Wimg = ctx->Wimg[bf16 ? 0 : 1];
    r.S = S;
    r.nparts = ctx->split_products;
    return DUST_OK;
}

// Tile offsets, ring depths and tensor-memory layout of a filled batch.
int finish_tc_batch(TcBatch &B, int precision, size_t smem_optin, size_t *smem, bool fused) {
    const bool bf16 = precision == DUST_PREC_BF16X3;
    const int bm = B.orient == 1 ? BN_T : BM;
    int64_t t = 0;
    int gmax = 16;
    for (int i = 0; i < B.nreq; ++i) {
        B.req[i].tile_begin = t;
        t += (B.req[i].C + bm - 1) / bm;
        gmax = std::max(gmax, B.req[i].Gs);
    }
    B.ntiles = t;
    B.GsMax = gmax;
    const size_t budget = (smem_optin ? smem_optin : 232448) - 1024;
    if (B.orient == 1) {
        if (fused || gmax > MW) return set_error(DUST_EINVAL, "grain-major GEMM: Gs <= %d and not fused", MW);
        B.tmem_cols = BN_T;
        B.nacc = 2;
        B.j_off = bf16 ? 0 : 15;
        B.off_exp = bf16 ? 0 : 14;
        auto need_t = [&](int a, int b) {
            return (size_t)a * STAGE1T_BYTES + (size_t)b * 2 * (WA_PART + JB_PART) + (size_t)(2 * a + 3 * b + 9) * 8 +
                   2 * BN_T * 4 + 16;
        };
        int ns1 = TN_NS1, ns2 = TN_NS2;
        while (need_t(ns1, ns2) > budget && ns1 > 2) --ns1;
        while (need_t(ns1, ns2) > budget && ns2 > 2) --ns2;
        if (need_t(ns1, ns2) > budget) return set_error(DUST_EINVAL, "shared memory too small for the grain-major GEMM");
        B.ns1 = ns1;
        B.ns2 = ns2;
        *smem = need_t(ns1, ns2) + 1024;
        return DUST_OK;
    }
    int cols = 32;
    while (cols < gmax) cols <<= 1;
    B.tmem_cols = cols;
    // double-buffer the accumulator when it fits; the fused kernel takes up
    // to NACC_MAX, one per group of solver warps
    B.nacc = std::max(1, std::min(fused ? NACC_MAX : 2, 512 / cols));
    // FP16 keeps J in [2^14, 2^15) and W in (2^13, 2^14] (the W image is
    // built with 2^14 folded in); BF16 has FP32's exponent range and needs none.
    B.j_off = bf16 ? 0 : 15;
    B.off_exp = bf16 ? 0 : 14;
    const size_t b_bytes = (size_t)gmax * KC * 4;
    // the fused kernel's solver warps are latency-bound on table lookups that
    // hit in L1, so its rings stay shallow and leave L1 most of the SM's memory
    int ns2 = fused ? FUSED_NS2 : 4, ns1 = fused ? FUSED_NS1 : 6;
    auto need = [&](int a, int b) {
        return (size_t)a * STAGE1_BYTES + (size_t)b * (2 * A_BYTES + b_bytes) +
               (size_t)(2 * a + 3 * b + 4 * NACC_MAX + 1) * 8 + NACC_MAX * BM * 4 + 16;
    };
    while (need(ns1, ns2) > budget && ns1 > 3) --ns1;
    while (need(ns1, ns2) > budget && ns2 > 2) --ns2;
    while (need(ns1, ns2) > budget && ns1 > 2) --ns1;
    if (need(ns1, ns2) > budget) return set_error(DUST_EINVAL, "G too large for the tensor-core kernel");
    B.ns1 = ns1;
    B.ns2 = ns2;
    *smem = need(ns1, ns2) + 1024;
    return DUST_OK;
}

int launch_tc_batch(const TcBatch &B, int precision, size_t smem, int num_sms, cudaStream_t st,
                    const SolveList *sl) {
    if (B.ntiles <= 0) return DUST_OK;
    const int grid = (int)std::min<int64_t>(B.ntiles, num_sms);
    // BF16: the per-cell power-of-two scale is exact and leaves every product
    // unchanged, so the exponent pass runs only for FP16.
    if (precision == DUST_PREC_BF16X3) return launch_t<true, false>(B, smem, grid, st, sl);
    return launch_t<false, true>(B, smem, grid, st, sl);
}

int launch_gemm_tc(const dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, float *S,
                   cudaStream_t st) {
    if (C <= 0) return DUST_OK;
    TcBatch B;
    B.nreq = 1;
    B.status = ctx->tb.status;
    B.orient = tc_orient(ctx);
    int rc = make_tc_req(ctx, precision, C, J, ld, S, B.req[0], B.tm[0], B.orient);
    if (rc != DUST_OK) return rc;
    size_t smem = 0;
    if ((rc = finish_tc_batch(B, precision, ctx->smem_optin, &smem)) != DUST_OK) return rc;
    return launch_tc_batch(B, precision, smem, ctx->num_sms, st);
}

}  // namespace dust

// Thermally fluctuating grains: the temperature probability distribution of
// small grains and its emission.  The paper computes equilibrium temperatures
// only and names this calculation as its follow-up (Sections 1 and 6): one
// transition-matrix solve per grain species and cell, after Guhathakurta &
// Draine (1989).
//
// Per (cell c, fluctuating grain g), all in FP32:
//   1. equilibrium temperature T_eq (Eq. 7) from the context's table solve,
//      with the absorbed power S = sum_k J W32 summed in FP32;
//   2. level grid E_j = j dE, j < M, E_top = (M-1) dE =
//      min(2 (E_g(T_eq) + eps_max), E_g(T_max)), with the Einstein enthalpy
//      E_g(T) = c_g / (exp(theta_g / T) - 1) and eps_max = h c / lambda_0;
//   3. upward rates: photons of lambda_k arrive at R_k = 4 pi w_k C J / eps_k
//      and lift the grain by x_k = eps_k / dE levels, split between floor and
//      ceiling so that the energy is kept on average; the rate of jumps of at
//      least m levels from any level is
//        Phi(m) = sum_k R_k clamp(x_k - m + 1, 0, 1)
//      (landings past the top level end there), which is two prefix sums
//      over the wavelengths (x_k falls as k rises):
//        Phi(m) = Sh[kb(m)] + Sf[kb(m-1)] - Sf[kb(m)],  kb(m) = #{k : x_k >= m},
//        Sh, Sf = exclusive prefix sums of R_k and R_k frac(x_k);
//   4. thermal-continuous cooling j -> j-1 at 4 pi P_g(max(T_j, T_min)) / dE
//      (P_g from the context's Hermite table);
//   5. steady state by the balance of the probability fluxes across each cut
//      between levels j-1 and j:  P_j = sum_{i<j} P_i Phi(j-i) / cool_j,
//      computed forward: every new P_j adds P_j Phi(f-j) to the flux into
//      each level f > j (the problem's lanes own the levels: a half-warp
//      for up to 64 levels, two problems per warp, a whole warp from 128
//      levels on), so each step is M/lanes FMAs per lane and one shuffle;
//   6. emission L[c,k] = 4 pi sum_g n sum_j P_j C[g,k] B_k(T_j) (Eqs. 8-10),
//      one MUFU ex2 per (level, wavelength), the level sum accumulated as a
//      fraction with one reciprocal per 8 levels.
//
// Scaled units: energies in units of eps_ref = h c / lambda_0 (photon energies
// eps~_k = lambda_0 / lambda_k <= 1); rates in units of 4 pi P_g(T_min) /
// eps_ref 2^(f'_g + sigma), where Rhat[g,k] = w C / (eps~ P_g(T_min)) 2^-f'_g
// <= 1 and sigma is the exponent of the cell's total sum_k J Rhat; the
// cooling rate of level j is then 2^(t_j - f'_g - sigma) / dE~ with
// t_j = log2(P_g(T_j) / P_g(T_min)) the table value.  The distribution and
// the fluxes run in a common frame (a power of two), re-based exactly by a
// power of two whenever a new value would pass 2^64.
#include "dust_internal.cuh"
#include "solve_core.cuh"

#include <cmath>
#include <vector>

namespace dust {
namespace {

constexpr double H_PL = 6.62607015e-34;
constexpr double C_LI = 299792458.0;
constexpr double K_BO = 1.380649e-23;

struct FlGrain {
    int g;          // context grain index
    float ctil;     // 3 N k_B theta / eps_ref
    float theta;    // Einstein temperature [K]
    float Etop;     // E_g(T_max) / eps_ref
    float fprime;   // exponent f'_g of Rhat
    float pad[3];
};

struct FlDev {
    const float *epst;     // [K] eps_k / eps_ref
    const float *Rhat;     // [Gf][K]
    const FlGrain *gr;     // [Gf]
    int Gf, M;
};

constexpr int FL_NPL = 4;  // emission: wavelength pairs per lane per pass (256 wavelengths a pass)

__host__ __device__ constexpr int fl_k4(int K) { return (K + 3) & ~3; }
__host__ __device__ constexpr int fl_kl(int K) { return (K + 255) & ~255; }
// per-warp shared memory, every array 16-byte aligned:
//   (1/T, P) [M] pairs, M zeros then phi [M], kb [M], x [K4], Sh [K4+4],
//   Sf [K4+4], Lw [KL]
__host__ __device__ constexpr size_t fl_lw_offset(int K, int M) { return (size_t)5 * M + 3 * (size_t)fl_k4(K) + 8; }
// slot stride: 16 more than a multiple of 32 floats, so that the two problems
// of a warp (one per half) sit 16 banks apart
__host__ __device__ constexpr size_t fl_warp_floats(int K, int M) {
    return ((fl_lw_offset(K, M) + fl_kl(K) + 31) & ~(size_t)31) + 16;
}

// One level's term for two wavelengths, folded into the group's fraction
// (sum of p t/(1-t) = N/D), kept as Nn = -N and D:
//   Nn -= t (p D + Nn),  D -= t D,
// four packed operations (the sign of t is an operand modifier).  The first
// level of a group starts from Nn = -p t, D = 1 - t.
__device__ __forceinline__ void fl_term(float2 nax, float iT, float p, float2 &Nn, float2 &D) {
    const float2 a = __fmul2_rn(nax, make_float2(iT, iT));
    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    const float2 e = __ffma2_rn(make_float2(p, p), D, Nn);
    Nn = __ffma2_rn(make_float2(-t.x, -t.y), e, Nn);
    D = __ffma2_rn(make_float2(-t.x, -t.y), D, D);
}
__device__ __forceinline__ void fl_first(float2 nax, float iT, float p, float2 &Nn, float2 &D) {
    const float2 a = __fmul2_rn(nax, make_float2(iT, iT));
    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    Nn = __fmul2_rn(make_float2(-p, -p), t);
    D = __ffma2_rn(make_float2(-t.x, -t.y), make_float2(1.f, 1.f), make_float2(1.f, 1.f));
}

// One CTA per cell; its problem slots take the fluctuating grains in turn.
// Sum over the levels j0 + s i, i < n (n a multiple of 8), of P_j t/(1-t) for
// NP wavelength pairs at once: the level data is read once per level for all
// pairs; one reciprocal per pair and 8 levels.
template <int NP>
__device__ __forceinline__ void fl_levels(const float2 *LT, int j0, int s, int n, const float2 (&nx)[NP],
                                          float2 (&sum)[NP]) {
    float2 Nn[NP], D[NP];
    for (int ib = 0; ib < n; ib += 8) {
        const float2 *lp = LT + j0 + s * ib;
        float2 lt = lp[0];
#pragma unroll
        for (int u = 0; u < NP; ++u) fl_first(nx[u], lt.x, lt.y, Nn[u], D[u]);
#pragma unroll
        for (int l = 1; l < 8; ++l) {
            lt = lp[s * l];
#pragma unroll
            for (int u = 0; u < NP; ++u) fl_term(nx[u], lt.x, lt.y, Nn[u], D[u]);
        }
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            sum[u].x = fmaf(-Nn[u].x, rcp_approx(D[u].x), sum[u].x);
            sum[u].y = fmaf(-Nn[u].y, rcp_approx(D[u].y), sum[u].y);
        }
    }
}

// One pass over 2 LW NP wavelengths from k0: lane hl of the problem takes the
// pairs k0 + 2 (hl + LW u).
template <int NP, int LW>
__device__ __forceinline__ void fl_pass(const DevTables &tb, const float2 *LT, int M, int k0, int K, int g, float nq,
                                        int hl, float *Lw) {
    float2 nx[NP], sum[NP];
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        const int k = k0 + 2 * (hl + LW * u);
        nx[u] = k < tb.Kp ? *reinterpret_cast<const float2 *>(tb.nax + k) : make_float2(-1e30f, -1e30f);
        sum[u] = make_float2(0.f, 0.f);
    }
    fl_levels<NP>(LT, 0, 1, M, nx, sum);
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        const int k = k0 + 2 * (hl + LW * u);
        if (k < K) {
            const float2 ch =
                *reinterpret_cast<const float2 *>(tb.Chat + ((size_t)(k / KQ) * tb.G8 + g) * KQ + (k % KQ));
            Lw[k] = fmaf(nq * ch.x, sum[u].x, Lw[k]);
            Lw[k + 1] = fmaf(nq * ch.y, sum[u].y, Lw[k + 1]);
        }
    }
}

// Lanes per (cell, grain) problem: 16 up to 64 levels (two problems per
// warp, whose recursion chains overlap in one instruction stream; measured
// 6 % faster at M = 64), 32 above (measured faster from M = 128 on, where a
// half-warp carries 8 or more levels per lane).  Every collective below is
// scoped to the problem's lanes (mask and width), so the two halves of a
// warp may also diverge.
__host__ __device__ constexpr int fl_lanes(int M) { return M <= 64 ? 16 : 32; }
// threads per CTA at most: 8 warps (of two problems up to M = 64, of one at
// M = 128), 12 warps above
__host__ __device__ constexpr int fl_threads(int M) { return M <= 128 ? 256 : 384; }
// resident CTAs the register budget is set for.  M = 128: four 8-warp CTAs
// (64 registers, small spills) measured 84 ms against 91 ms for two 12-warp
// CTAs at 80 registers; the recursion's chains want more warps per SM.
__host__ __device__ constexpr int fl_min_ctas(int M) { return M <= 64 ? 2 : (M == 128 ? 4 : (M == 256 ? 2 : 1)); }

template <int M>
__global__ void __launch_bounds__(fl_threads(M), fl_min_ctas(M)) k_fluct(const DevTables tb, const FlDev fd,
                                                                      const float *W32, int Kw, int64_t C,
                                                                      const float *J, int64_t ld, const float *n,
                                                                      float *L, float *P, float *dE_out,
                                                                      float eps_ref) {
    constexpr int LW = fl_lanes(M);
    constexpr int MR = M / LW;    // levels per lane
    constexpr int PPW = 32 / LW;  // problems per warp
    extern __shared__ float sm[];
    const int K = tb.K, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int hl = lane % LW, slot = w * PPW + lane / LW, NPB = (blockDim.x >> 5) * PPW;
    const unsigned hmask = LW == 32 ? 0xffffffffu : (0xffffu << (lane & 16));
    const int64_t c = blockIdx.x;
    if (c >= C) return;
    const float inv_h2 = 1.f / tb.h2;
    const int Kp4 = (K + 3) & ~3;
    float *Jc = sm;
    float *base = sm + Kp4 + (size_t)slot * fl_warp_floats(K, M);
    float2 *LT = reinterpret_cast<float2 *>(base);  // level j: (1/T_j, P_j)
    float *phi = base + 3 * M;                      // phi[-M..-1] = 0
    int *kb = (int *)(phi + M);
    float *x = (float *)(kb + M), *Sh = x + fl_k4(K), *Sf = Sh + fl_k4(K) + 4;
    float *Lw = base + fl_lw_offset(K, M);

    for (int k = threadIdx.x; k < K; k += blockDim.x) Jc[k] = J[c * ld + k];
    for (int k = hl; k < fl_kl(K); k += LW) Lw[k] = 0.f;
    for (int i = hl; i < M; i += LW) phi[i - M] = 0.f;
    __syncthreads();

    for (int q = slot; q < fd.Gf; q += NPB) {
        const FlGrain gr = fd.gr[q];
        const int g = gr.g;
        // 1. equilibrium temperature of the cell's absorbed power (Eq. 7)
        float s = 0.f;
        for (int k = hl; k < K; k += LW) s = fmaf(Jc[k], __ldg(W32 + (size_t)g * Kw + k), s);
#pragma unroll
        for (int o = LW / 2; o; o >>= 1) s += __shfl_xor_sync(hmask, s, o);
        float Teq[1];
        int fl[1];
        {
            const int gg[1] = {g};
            const float ss[1] = {s};
            const GrainParam gp = tb.gp[g];
            const float4 gq[1] = {make_float4(gp.f, gp.tmax, gp.invdy, gp.pad)};
            solve_batch<1>(tb, gg, ss, gq, Teq, fl);
        }
        const float nq = n[c * fd.Gf + q];
        if (fl[0] == DUST_FLAG_INVALID) {  // NaN / negative / infinite field
            const float qnan = __int_as_float(0x7fc00000);
            if (P)
                for (int j = hl; j < M; j += LW) P[((size_t)c * fd.Gf + q) * M + j] = qnan;
            if (dE_out && hl == 0) dE_out[c * fd.Gf + q] = qnan;
            for (int k = hl; k < K; k += LW) Lw[k] = qnan;
            __syncwarp(hmask);
            continue;
        }
        // 2. level grid
        const float Eeq = gr.ctil / expm1f(gr.theta / Teq[0]);
        const float Etop = fminf(2.f * (Eeq + 1.f), gr.Etop);
        const float dEt = Etop / (float)(M - 1);
        const float idE = 1.f / dEt;
        const float cidE = gr.ctil * idE;  // level f: ctil / E_f = cidE / f
        // 3. photon landings and prefix sums over wavelength: each lane
        //    sums its own run of consecutive wavelengths (exclusive sums in
        //    place), one scan of the run totals across the lanes, then each
        //    run is offset
        const int KL = (K + LW - 1) / LW;
        const int kbeg = min(hl * KL, K), kend = min(kbeg + KL, K);
        float th = 0.f, tf = 0.f;
        for (int k = kbeg; k < kend; ++k) {
            const float xk = __ldg(fd.epst + k) * idE;
            x[k] = xk;
            const float h = Jc[k] * __ldg(fd.Rhat + (size_t)q * K + k);
            Sh[k] = th;
            Sf[k] = tf;
            th += h;
            tf = fmaf(h, xk - floorf(xk), tf);
        }
        float oh = th, of = tf;
#pragma unroll
        for (int o = 1; o < LW; o <<= 1) {
            const float a = __shfl_up_sync(hmask, oh, o, LW), b = __shfl_up_sync(hmask, of, o, LW);
            if (hl >= o) { oh += a; of += b; }
        }
        const float carry_h = __shfl_sync(hmask, oh, LW - 1, LW), carry_f = __shfl_sync(hmask, of, LW - 1, LW);
        oh -= th;
        of -= tf;
        for (int k = kbeg; k < kend; ++k) {
            Sh[k] += oh;
            Sf[k] += of;
        }
        if (hl == 0) {
            Sh[K] = carry_h;
            Sf[K] = carry_f;
        }
        __syncwarp(hmask);
        // sigma: Phi 2^-sigma <= 1 (the total rate bounds every Phi(m))
        const int sigma = (carry_h > 0.f && carry_h < INFINITY) ? ilogbf(carry_h) + 1 : 0;
        // kb(m) = #{k : x_k >= m}.  x is non-increasing, so kb = k + 1 on
        // floor(x_k+1) < m <= floor(x_k), kb = K on m <= floor(x_K-1) and 0
        // above floor(x_0): every wavelength fills its own range of m
        for (int m = hl; m < M; m += LW) kb[m] = 0;
        __syncwarp(hmask);
        for (int k = hl; k < K; k += LW) {
            const int hi = (int)fminf(floorf(x[k]), (float)(M - 1));
            const int lo = k + 1 < K ? (int)fminf(floorf(x[k + 1]), (float)M) + 1 : 0;
            for (int m = lo; m <= hi; ++m) kb[m] = k + 1;
        }
        __syncwarp(hmask);
        for (int m = hl; m < M; m += LW) {
            float v = 0.f;
            if (m > 0) {
                const int a = kb[m], b = kb[m - 1];
                v = ldexpf(Sh[a] + (Sf[b] - Sf[a]), -sigma);
            }
            phi[m] = v;
        }
        // 4. levels owned by this lane: 1/T and the cooling factor,
        //    P_f = acc_f mul_f 2^ei_f in the frame of acc; mulx = mul 2^ei
        //    where that is a normal float (NaN otherwise: exact path)
        float acc[MR], mul[MR], mulx[MR];
        int ei[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            const int f = hl + LW * r;
            acc[r] = 0.f;
            mul[r] = 0.f;
            mulx[r] = 0.f;
            ei[r] = 0;
            if (f == 0) {
                LT[0].x = PAD_INV_T;  // level 0 (T = 0) emits nothing: every t is 0
                continue;
            }
            const float T = gr.theta * rcp_approx(log1pf(cidE * rcp_approx((float)f)));
            LT[f].x = rcp_approx(T);
            // log2 of T clamped into the table: exponent split off exactly,
            // lg2.approx of the mantissa in [1/2, 1)
            const int tbits = __float_as_int(fminf(fmaxf(T, tb.Tmin), tb.Tmax));
            const float u = (float)(((tbits >> 23) & 0xff) - 126) +
                            lg2_approx(__int_as_float((tbits & 0x007fffff) | 0x3f000000));
            const float fj = (u - tb.log2Tmin) * inv_h2;
            const int j0 = min(max((int)floorf(fj), 0), tb.NT - 2);
            const float tau = fminf(fmaxf(fj - (float)j0, 0.f), 1.f);
            const float4 f4 = __ldg(tb.fw + (size_t)g * (tb.NT - 1) + j0);
            const float t = hermite(f4.x, f4.y, f4.z, f4.w, tau);
            const float e = gr.fprime + (float)sigma - t;
            const float fe = floorf(e);
            ei[r] = (int)fe;
            mul[r] = dEt * ex2_approx(e - fe);  // e - fe in [0, 1)
            // mul 2^ei where that is a normal float (the scale is 0 outside
            // the exponent range, so the test below fails there as well);
            // below the normal range the rounded (subnormal or zero) value:
            // such a level's P is below 2^-126 of the frame's, whatever its
            // last bits; above it NaN, for the exact path
            const float sc = (ei[r] >= -126 && ei[r] <= 127) ? __int_as_float((ei[r] + 127) << 23) : 0.f;
            const float mx = mul[r] * sc;
            mulx[r] = (mx >= 1.17549435e-38f && mx < INFINITY) ? mx
                    : ei[r] < 0 ? ldexpf(mul[r], ei[r]) : __int_as_float(0x7fc00000);
        }
        __syncwarp(hmask);
        // 5. forward cut-flux recursion from P_0 = 1: step j adds P_j's flux
        //    to every level above j, then reads P_{j+1} off its owner lane.
        //    Level 0 sits in lane 0's first register as acc = 1 with factor 1
        //    (its flux terms are the zero pad), so that every level's P is
        //    acc mul 2^ei in the current frame and a frame change rescales
        //    them all at once; the distribution is read off the registers
        //    at the end.
        if (hl == 0) { acc[0] = 1.f; mul[0] = 1.f; mulx[0] = 1.f; ei[0] = 0; }
        float pj = 1.f;
        const float *ph = phi + hl;
        // (registers below R0 hold levels at or below j: their updates add 0)
#define FL_STEP(J, RS, R0, OWN)                                                               \
    {                                                                                         \
        const int j_ = (J);                                                                   \
        _Pragma("unroll") for (int r = (R0); r < MR; ++r) acc[r] = fmaf(ph[LW * r - j_], pj, acc[r]); \
        const float v = __shfl_sync(hmask, acc[RS] * mulx[RS], (OWN), LW);                     \
        if (v < 0x1p64f) {                                                                    \
            pj = v;                                                                           \
        } else { /* exact path: rescale the frame, or an exponent out of float range */       \
            const float raw = __shfl_sync(hmask, acc[RS] * mul[RS], (OWN), LW);               \
            const int E = __shfl_sync(hmask, ei[RS], (OWN), LW);                              \
            const int ve = (raw > 0.f && raw < INFINITY) ? ilogbf(raw) : -1000;               \
            if (ve + E > 64) {                                                                \
                const int sh = ve + E;                                                        \
                _Pragma("unroll") for (int r = 0; r < MR; ++r) acc[r] = ldexpf(acc[r], -sh);  \
                pj = ldexpf(raw, -ve);                                                        \
            } else {                                                                          \
                pj = ldexpf(raw, E);                                                          \
            }                                                                                 \
        }                                                                                     \
    }
        // Fast form of a step: no test (a branch per step measured 12 % of
        // the kernel, a flag per step 1.4 %).  A block of LW steps is checked
        // once, at its end: a block with a value past 2^100, or a level whose
        // factor is not a normal float, is taken again from its saved state
        // with the tested step.  The check reads the block's new levels back
        // off the registers that hold them: once its level is read, a
        // register only takes zero terms (the pad below phi[1]), so it still
        // gives the value that was broadcast, or NaN where a later value
        // overflowed.  Every P of a block that passes is below 2^100, so no
        // register can pass 2^109 (at most M <= 512 terms P phi with
        // phi <= 1), and after each block the frame is moved to the newest
        // level when that is above 2^32.
#define FL_FAST(J, RS, R0, OWN)                                                               \
    {                                                                                         \
        const int j_ = (J);                                                                   \
        _Pragma("unroll") for (int r = (R0); r < MR; ++r) acc[r] = fmaf(ph[LW * r - j_], pj, acc[r]); \
        pj = __shfl_sync(hmask, acc[RS] * mulx[RS], (OWN), LW);                                \
    }
#pragma unroll
        for (int r0 = 0; r0 < MR; ++r0) {
            // block: levels LW r0 + 1 .. LW r0 + LW - 1 (this register of
            // lanes 1..LW-1), then level LW (r0 + 1) (the next register of
            // lane 0).  Saved state: the registers in the lanes' own LT[.].y
            // (free until the distribution is written), and pj.
#pragma unroll
            for (int r = 0; r < MR; ++r) LT[hl + LW * r].y = acc[r];
            const float pj0 = pj;
#pragma unroll 2
            for (int jj = 0; jj < LW - 1; ++jj) FL_FAST(LW * r0 + jj, r0, r0, jj + 1)
            if (r0 + 1 < MR) FL_FAST(LW * r0 + LW - 1, r0 + 1 < MR ? r0 + 1 : r0, r0 + 1, 0)
            // the block's levels: register r0 of lanes 1..LW-1, and register
            // r0 + 1 of lane 0 (read at the block's last step; none in the
            // last block)
            const int rb = hl > 0 ? r0 : r0 + 1;
            float vb = 0.f;
#pragma unroll
            for (int r = 0; r < MR; ++r) vb = r == rb ? acc[r] * mulx[r] : vb;
            const bool ok = __all_sync(hmask, vb < 0x1p100f);
            if (!ok) {  // the same on every lane of the problem (a vote)
#pragma unroll
                for (int r = 0; r < MR; ++r) acc[r] = LT[hl + LW * r].y;
                pj = pj0;
                for (int jj = 0; jj < LW - 1; ++jj) FL_STEP(LW * r0 + jj, r0, r0, jj + 1)
                if (r0 + 1 < MR) FL_STEP(LW * r0 + LW - 1, r0 + 1 < MR ? r0 + 1 : r0, r0 + 1, 0)
            } else {
                const int e = ((__float_as_int(pj) >> 23) & 0xff) - 127;  // pj normal, < 2^100
                if (e > 32) {
                    const float sc = __int_as_float((127 - e) << 23);
#pragma unroll
                    for (int r = 0; r < MR; ++r) acc[r] *= sc;
                    pj *= sc;
                }
            }
        }
#undef FL_FAST
#undef FL_STEP
        // the distribution in the final frame, normalised
        float pv[MR], z = 0.f;
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            const float fast = acc[r] * mulx[r];
            pv[r] = fast < 0x1p64f ? fast : ldexpf(acc[r] * mul[r], ei[r]);
            z += pv[r];
        }
#pragma unroll
        for (int o = LW / 2; o; o >>= 1) z += __shfl_xor_sync(hmask, z, o);
        const float iz = 1.f / z;
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            const int j = hl + LW * r;
            const float p = pv[r] * iz;
            LT[j].y = p;
            if (P) P[((size_t)c * fd.Gf + q) * M + j] = p;
        }
        if (dE_out && hl == 0) dE_out[c * fd.Gf + q] = dEt * eps_ref;
        __syncwarp(hmask);
        // 6. emission of the distribution, accumulated per problem slot: whole
        //    passes of 4 pairs per lane, then floor(rest / 2LW) pairs per lane,
        //    then the last < 2 LW wavelengths with the levels split between lanes
        int k0 = 0;
        for (; k0 + 8 * LW <= K; k0 += 8 * LW) fl_pass<FL_NPL, LW>(tb, LT, M, k0, K, g, nq, hl, Lw);
        switch ((K - k0) / (2 * LW)) {
            case 3: fl_pass<3, LW>(tb, LT, M, k0, K, g, nq, hl, Lw); k0 += 6 * LW; break;
            case 2: fl_pass<2, LW>(tb, LT, M, k0, K, g, nq, hl, Lw); k0 += 4 * LW; break;
            case 1: fl_pass<1, LW>(tb, LT, M, k0, K, g, nq, hl, Lw); k0 += 2 * LW; break;
            default: break;
        }
        if (k0 < K) {
            const int np = (K - k0 + 1) / 2;  // <= LW pairs
            int lp = LW;                        // lanes per pair: a power of two, >= 8 levels each
            while (lp > 1 && (lp * np > LW || M / lp < 8)) lp >>= 1;
            const int pr = hl / lp, ch0 = hl % lp, nl = M / lp;
            const int k = k0 + 2 * pr;
            float2 nx[1] = {pr < np && k < tb.Kp ? *reinterpret_cast<const float2 *>(tb.nax + k)
                                                 : make_float2(-1e30f, -1e30f)};
            float2 sum[1] = {make_float2(0.f, 0.f)};
            fl_levels<1>(LT, ch0, lp, nl, nx, sum);  // levels ch0 + lp i: the lanes of a pair read neighbours
            for (int o = 1; o < lp; o <<= 1) {
                sum[0].x += __shfl_xor_sync(hmask, sum[0].x, o);
                sum[0].y += __shfl_xor_sync(hmask, sum[0].y, o);
            }
            if (ch0 == 0 && pr < np && k < K) {
                const float2 c2 =
                    *reinterpret_cast<const float2 *>(tb.Chat + ((size_t)(k / KQ) * tb.G8 + g) * KQ + (k % KQ));
                Lw[k] = fmaf(nq * c2.x, sum[0].x, Lw[k]);
                Lw[k + 1] = fmaf(nq * c2.y, sum[0].y, Lw[k + 1]);
            }
        }
        __syncwarp(hmask);
    }
    __syncthreads();
    if (L) {
        const float *L0 = sm + Kp4 + fl_lw_offset(K, M);
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            float v = 0.f;
            for (int i = 0; i < NPB; ++i) v += L0[(size_t)i * fl_warp_floats(K, M) + k];
            L[c * ld + k] = ldexpf(v, __ldg(tb.qexp + k));
        }
    }
}

// CTA size.  Two problems per warp: the number of warps whose resident CTAs
// per SM (occupancy API) times problem slots, discounted by the idle slots of
// the last pass over the grains, is largest.  One problem per warp: up to 8
// or 12 warps, as few passes over the grains as that allows, balanced.
template <int M>
cudaError_t launch_fluct_m(const dust_ctx *ctx, const FlDev &fd, int64_t C, const float *J, int64_t ld,
                           const float *n, float *L, float *P, float *dE, cudaStream_t st, int *fw_out) {
    auto kern = k_fluct<M>;
    const int K = ctx->K, Gf = fd.Gf, ppw = 32 / fl_lanes(M);
    const size_t per_slot = sizeof(float) * fl_warp_floats(K, M);
    const size_t fixed = sizeof(float) * ((K + 3) & ~3);
    const size_t optin = ctx->smem_optin ? ctx->smem_optin : 232448;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)optin);
    if (e != cudaSuccess) return e;
    int best = 0;
    double best_score = -1.0;
    if (ppw == 1) {
        int fw = std::min(Gf, fl_threads(M) / 32);
        const int passes = (Gf + fw - 1) / fw;
        fw = (Gf + passes - 1) / passes;
        while (fw > 1 && fixed + per_slot * fw > optin) --fw;
        best = fw;
        best_score = 1.0;
    }
    for (int fw = 1; ppw == 2 && fw <= fl_threads(M) / 32; ++fw) {
        const size_t sm_b = fixed + per_slot * fw * ppw;
        if (sm_b > optin) break;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, fw * 32, sm_b) != cudaSuccess) {
            cudaGetLastError();
            nb = 0;
        }
        const int slots = fw * ppw, passes = (Gf + slots - 1) / slots;
        const double score = (double)nb * slots * ((double)Gf / ((double)slots * passes));
        if (score > best_score + 1e-9) { best_score = score; best = fw; }
    }
    if (best == 0 || best_score <= 0.0) return cudaErrorInvalidConfiguration;
    *fw_out = best;
    kern<<<(unsigned)C, best * 32, fixed + per_slot * best * ppw, st>>>(ctx->tb, fd, ctx->W32, ctx->Kw, C, J, ld, n,
                                                                       L, P, dE, ctx->fl_eps_ref);
    return cudaGetLastError();
}

int check_device_ptr(const dust_ctx *ctx, const void *p) {
    if (!p) return DUST_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DUST_EINVAL, "an argument is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error(DUST_EINVAL, "J, n, L, P and dE must be device memory");
    if (a.type == cudaMemoryTypeDevice && a.device != ctx->device)
        return set_error(DUST_EINVAL, "an argument lives on device %d, the context on device %d", a.device,
                         ctx->device);
    return DUST_OK;
}

}  // namespace
}  // namespace dust

using namespace dust;

extern "C" int dust_ctx_set_fluctuating(dust_ctx *ctx, int Gf, const int *grains, const double *n_atoms,
                                        const double *theta, int M) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (Gf < 1 || Gf > ctx->G) return set_error(DUST_EINVAL, "Gf=%d outside [1, G=%d]", Gf, ctx->G);
    if (!grains || !n_atoms || !theta) return set_error(DUST_EINVAL, "grains, n_atoms and theta must be non-NULL");
    if (M != 32 && M != 64 && M != 128 && M != 256 && M != 512)
        return set_error(DUST_EINVAL, "M=%d: levels must be 32, 64, 128, 256 or 512", M);
    const int K = ctx->K;
    if (K > 2048) return set_error(DUST_EINVAL, "K=%d > 2048", K);
    const double lam0 = ctx->lam_h[0];
    const double eps_ref = H_PL * C_LI / lam0;
    std::vector<double> P0(ctx->G);
    std::lock_guard<std::mutex> lk(ctx->mu);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DUST_ECUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    int rc = DUST_OK;
    [&] {
        if (cudaMemcpy(P0.data(), ctx->tb.P0, sizeof(double) * ctx->G, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(DUST_ECUDA, "reading P_g(T_min) failed");
            return;
        }
        std::vector<float> epst(K);
        for (int k = 0; k < K; ++k) epst[k] = (float)(lam0 / ctx->lam_h[k]);
        std::vector<float> Rhat((size_t)Gf * K);
        std::vector<FlGrain> gr(Gf);
        for (int q = 0; q < Gf; ++q) {
            const int g = grains[q];
            if (g < 0 || g >= ctx->G) { rc = set_error(DUST_EINVAL, "grains[%d]=%d outside [0, G)", q, g); return; }
            if (!(n_atoms[q] > 0.0) || !(theta[q] > 0.0) || !std::isfinite(n_atoms[q]) || !std::isfinite(theta[q])) {
                rc = set_error(DUST_EINVAL, "grain %d: n_atoms and theta must be finite and > 0", q);
                return;
            }
            const double c = 3.0 * n_atoms[q] * K_BO * theta[q] / eps_ref;
            const double Etop = c / std::expm1(theta[q] / ctx->Tmax);
            double mx = 0.0;
            std::vector<double> r(K);
            for (int k = 0; k < K; ++k) {
                r[k] = ctx->w_h[k] * ctx->C_h[(size_t)g * K + k] * (ctx->lam_h[k] / lam0) / P0[g];
                mx = std::max(mx, r[k]);
            }
            if (!(mx > 0.0) || !std::isfinite(mx) || !std::isfinite(c) || !(Etop > 0.0) || !std::isfinite(Etop) ||
                c > 1e30) {
                rc = set_error(DUST_EINVAL, "grain %d: heating or enthalpy constants out of range", q);
                return;
            }
            const int fp = (int)std::ceil(std::log2(mx));
            for (int k = 0; k < K; ++k) Rhat[(size_t)q * K + k] = (float)std::ldexp(r[k], -fp);
            gr[q] = FlGrain{g, (float)c, (float)theta[q], (float)Etop, (float)fp, {0.f, 0.f, 0.f}};
        }
        const size_t o_e = 0, o_r = (sizeof(float) * K + 255) & ~(size_t)255;
        const size_t o_g = (o_r + sizeof(float) * Rhat.size() + 255) & ~(size_t)255;
        const size_t bytes = o_g + sizeof(FlGrain) * Gf;
        void *mem = nullptr;
        if (cudaMalloc(&mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(DUST_ENOMEM, "fluctuating-grain tables: cudaMalloc(%zu) failed", bytes);
            return;
        }
        char *b = (char *)mem;
        if (cudaMemcpy(b + o_e, epst.data(), sizeof(float) * K, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b + o_r, Rhat.data(), sizeof(float) * Rhat.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b + o_g, gr.data(), sizeof(FlGrain) * Gf, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(mem);
            rc = set_error(DUST_ECUDA, "fluctuating-grain tables: copy failed");
            return;
        }
        // a solve still in flight may read the tables being replaced
        if (ctx->fl_mem && cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            cudaFree(mem);
            rc = set_error(DUST_ECUDA, "synchronising before replacing the fluctuating-grain tables failed");
            return;
        }
        cudaFree(ctx->fl_mem);
        ctx->fl_mem = mem;
        ctx->fl_Gf = Gf;
        ctx->fl_M = M;
        ctx->fl_eps_ref = (float)eps_ref;
        ctx->fl_off[0] = o_e;
        ctx->fl_off[1] = o_r;
        ctx->fl_off[2] = o_g;
    }();
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

extern "C" int dust_solve_fluct(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n,
                                float *L, float *P, float *dE, void *stream) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (n_cells < 0) return set_error(DUST_EINVAL, "n_cells < 0");
    if (ld < ctx->K) return set_error(DUST_EINVAL, "ld=%lld < K=%d", (long long)ld, ctx->K);
    if (n_cells == 0) return DUST_OK;
    if (!J || !n) return set_error(DUST_EINVAL, "J and n must be non-NULL");
    if (n_cells > 0x7fffffffLL) return set_error(DUST_EINVAL, "n_cells too large for one launch");
    for (const void *p : {(const void *)J, (const void *)n, (const void *)L, (const void *)P, (const void *)dE}) {
        const int r = check_device_ptr(ctx, p);
        if (r != DUST_OK) return r;
    }
    // the grain set (M, Gf and the tables) is read under the context's lock, in one
    // snapshot, so that a concurrent dust_ctx_set_fluctuating cannot replace it in between
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->fl_mem) return set_error(DUST_EINVAL, "no fluctuating grains: call dust_ctx_set_fluctuating");
    const int K = ctx->K, M = ctx->fl_M, Gf = ctx->fl_Gf;
    // one problem slot of shared memory per (cell, grain) in flight
    if (sizeof(float) * (((K + 3) & ~3) + fl_warp_floats(K, M)) > (ctx->smem_optin ? ctx->smem_optin : 232448))
        return set_error(DUST_EINVAL, "K=%d, M=%d need more shared memory than one CTA has", K, M);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DUST_ECUDA, "cudaGetDevice failed");
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    const char *b = (const char *)ctx->fl_mem;
    FlDev fd{(const float *)(b + ctx->fl_off[0]), (const float *)(b + ctx->fl_off[1]),
             (const FlGrain *)(b + ctx->fl_off[2]), Gf, M};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    int fw = 0;
    switch (M) {
        case 32: e = launch_fluct_m<32>(ctx, fd, n_cells, J, ld, n, L, P, dE, st, &fw); break;
        case 64: e = launch_fluct_m<64>(ctx, fd, n_cells, J, ld, n, L, P, dE, st, &fw); break;
        case 128: e = launch_fluct_m<128>(ctx, fd, n_cells, J, ld, n, L, P, dE, st, &fw); break;
        case 256: e = launch_fluct_m<256>(ctx, fd, n_cells, J, ld, n, L, P, dE, st, &fw); break;
        default: e = launch_fluct_m<512>(ctx, fd, n_cells, J, ld, n, L, P, dE, st, &fw); break;
    }
    int rc = DUST_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(DUST_ECUDA, "fluctuating-grain kernel launch failed: %s", cudaGetErrorString(e));
    } else {
        ctx->launches += 1;
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

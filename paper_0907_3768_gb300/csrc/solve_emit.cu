// Kernel (b): equilibrium-temperature solve and emission SED.  For one
// request whose emission weights fit in shared memory (dust_solve's usual
// case) they run as one warp-specialized kernel, k_solve_emit; otherwise, and
// for the server's work lists of many requests, as two kernels, k_solve and
// k_emit.  All three give the same bits.
//
// k_solve — one warp per cell, many warps per SM (the solve is a chain of
// dependent table lookups, so it wants parallelism, not shared memory):
//   the exponent m_c of max_g n[c,g] (n enters the emission as n 2^-m_c) and,
//   per grain, the root of Eq. 7 from the scaled absorbed power S
//   (A / P_g(T_min) = S 2^f_g): a guess from the inverse table u(t), then
//   Newton on the FP32 Hermite interpolant of
//   t_g(u) = log2(P_g(2^u) / P_g(T_min)) inside the bracketing table interval
//   (bisection when a step leaves it).  The paper's kernel 3 iterated Newton
//   with a fresh quadrature per step (Section 4.3); the device table removes
//   those exponentials.  Writes T, flags and, when the emission follows, the
//   pairs (1/T, n 2^-m_c) and a per-cell record (m_c, absorbed power).
// k_emit — persistent, one thread per (two cells, 8 consecutive wavelengths),
//   Eq. 10:
//     L[c,k] = 2^(m_c+q_k) sum_g (n 2^-m_c) Chat[g,k] t/(1-t),
//     t = 2^(nax_k / T[c,g])  (one MUFU ex2 per term),
//   the grain sum accumulated as a fraction N/D over groups of 8 grains so
//   that a group costs one reciprocal instead of eight:
//     N <- N + t (w D - N),  D <- D - t D   (= sum of w t/(1-t)).
//   Chat sits in shared memory ([k-group][grain][2] float4, odd row stride),
//   in grain chunks when it does not fit, as the paper staged sigma per block
//   (Section 4.4); the next tile's (1/T, n) pairs stream in with cp.async
//   while the current tile computes.  Resident weights: two CTAs of 256
//   threads per SM; streamed weights: one CTA of 512 threads, twice the cells
//   per tile and nearly all of shared memory for the chunks.
// k_solve_emit — one CTA per SM: solver warps run k_solve's per-cell code on
//   the tile after the one being emitted and leave its pairs in shared
//   memory; emission warps take one cell x 8 wavelengths per thread with
//   k_emit's arithmetic.  The latency-bound solve hides behind the emission.
// resid = sum_k w_k L[c,k] / (4 pi sum_g n Pe) - 1: both sums are kept in
//   float-float (error-free FP32 products and two-sums, ~48-bit) and their
//   quotient is taken in float-float too, so the path has no FP64 arithmetic
//   (this GPU's FP64 pipe issues two operations per clock per SM); only the
//   stored residual is widened to double.  Every reduction has a fixed order,
//   so results depend neither on the batch nor on timing.
#include "dust_internal.cuh"
#include "solve_core.cuh"
#include "mbar.cuh"

#include <algorithm>

namespace dust {
namespace {

constexpr int NTH = 256;      // emission threads per CTA (resident weights; 512 when streamed)
constexpr int EMIT_STREAM_NTH = 512;  // threads of the streamed-weights emission CTA
constexpr int SOLVE_TH = 128; // solve threads per CTA (one warp per cell)
constexpr int NB_MAX = 4;     // grains per lane per pass in the solve, at most
// temperature-only solve: CTAs of SOLVE_TH per SM (measured best: 8 at up to 3 grains per
// lane, 6 at 4)
constexpr int solve_tonly_ctas(int nb) { return nb >= 4 ? 6 : 8; }

// Energy-balance residual emitted / (4 pi absorbed) - 1 of a cell, with
// emitted = (h + l) 2^(m_c + Ew) and absorbed = (ah + al) 2^(m_c + Eg), all in
// FP32: both sums are split into mantissa and exponent, their quotient is
// taken in float-float (a reciprocal estimate corrected by an exact FMA
// remainder, ~2^-44 relative), multiplied by 2^(Ew - Eg) / (4 pi), and 1 is
// subtracted where the quotient is near 1, so that the subtraction is exact.
__device__ __forceinline__ float residual(float h, float l, float ah, float al, const DevTables &tb) {
    int he = 0, ae = 0;
    const float hm = frexpf(h, &he), am = frexpf(ah, &ae);
    const float lm = ldexpf(l, -he), alm = ldexpf(al, -ae);
    const float r0 = rcp_approx(am);
    const float q1 = hm * r0;
    const float q2 = (fmaf(-q1, am, hm) + lm - q1 * alm) * r0;
    const float p1 = q1 * tb.rc_hi;
    const float pe = fmaf(q1, tb.rc_hi, -p1) + fmaf(q1, tb.rc_lo, q2 * tb.rc_hi);
    const int E = max(-252, min(252, he - ae + tb.rc_exp));
    return (scale2(p1, E) - 1.f) + scale2(pe, E);
}

// S and (when the emission follows) n of one pass of a cell: grains
// gb + lane + 32 i.
template <int NB, bool TONLY = false>
__device__ __forceinline__ void load_pass(const EmitReq &q, int64_t cell, int gb, int lane, float (&s)[NB],
                                          float (&nv)[NB]) {
    const int G = q.tb.G;
    const bool with_n = !TONLY && (q.mode & EMIT_ON) != 0 && !(q.mode & EMIT_MASS);
    const float *Srow = q.S + cell * q.tb.Gs;
    const float *nrow = q.n + cell * G;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int g = gb + lane + 32 * i;
        s[i] = g < G ? __ldg(Srow + g) : 0.f;
        nv[i] = (with_n && g < G) ? __ldg(nrow + g) : 0.f;
    }
}

// The solve of one cell by one warp: the exponent m_c of max_g n (general
// form) or of the cell's mass (dust-mass form), then per pass of 32 NB grains
// the roots, T and flags to global memory, and (emission) the pairs
// (1/T, n 2^-m_c) and the cell record: to the request's scratch (q.prep
// [C][G8], float2 or, in the dust-mass form, 1/T only; q.cell), or with SMEM
// to `spairs` (G8 float2, or G8 floats in the dust-mass form) and `srec` in
// shared memory as well as the record to q.cell.  s0 / n0: this cell's first
// pass, loaded.
// MF: the form of n when the caller knows it (0 general, 1 dust-mass), -1 to
// read it from the request; EMIT: the emission is known to follow (the fused
// kernel, whose launch has NB = ceil(G8 / 32), so a cell is one pass when
// NB < NB_MAX).
template <int NB, bool SMEM, bool TONLY = false, int MF = -1, bool EMIT = false>
__device__ __forceinline__ void solve_cell(const EmitReq &q, int64_t cell, int lane, const float (&s0)[NB],
                                           const float (&n0)[NB], float2 *spairs, CellInfo *srec) {
    const DevTables &tb = q.tb;
    const int G = tb.G, G8 = tb.G8;
    const bool emit = EMIT || (!TONLY && (q.mode & EMIT_ON) != 0), rs = (q.mode & EMIT_RESID) != 0;
    const bool one = (EMIT && NB < NB_MAX) || G8 <= 32 * NB;  // known at compile time in the fused kernel
    const bool mass = MF >= 0 ? MF == 1 : (q.mode & EMIT_MASS) != 0;
    int mc = 0;
    float ms = 0.f;  // dust-mass form: m_c = ms 2^mc
    if (emit && mass) {
        const float m = __ldg(q.n + cell);
        ms = (m != 0.f && isfinite(m)) ? frexpf(m, &mc) : m;
    }
    if (!one && emit && !mass) {
        const float *nrow = q.n + cell * G;
        float mx = 0.f;
        for (int g = lane; g < G; g += 32) mx = fmaxf(mx, __ldg(nrow + g));
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (mx > 0.f && mx < INFINITY) frexpf(mx, &mc);
    }
    float ah = 0.f, al = 0.f;  // absorbed power n 2^-m_c Pe 2^-Eg, float-float
    for (int gb = 0; gb < G8; gb += 32 * NB) {
        int gi[NB], fl[NB];
        float s[NB], nv[NB], Tv[NB];
        float4 gq[NB];
        if (gb == 0) {
#pragma unroll
            for (int i = 0; i < NB; ++i) { s[i] = s0[i]; nv[i] = n0[i]; }
        } else {
            load_pass<NB, TONLY>(q, cell, gb, lane, s, nv);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int g = gb + lane + 32 * i;
            gi[i] = g < G ? g : 0;
            gq[i] = __ldg(reinterpret_cast<const float4 *>(tb.gp) + gi[i]);
        }
        if (one && emit && !mass) {
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < NB; ++i) mx = fmaxf(mx, nv[i]);
            for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (mx > 0.f && mx < INFINITY) frexpf(mx, &mc);
        }
        solve_batch<NB>(tb, gi, s, gq, Tv, fl);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int g = gb + lane + 32 * i;
            if (g >= G8) continue;
            float invT = PAD_INV_T, nn = 0.f;
            if (g < G) {
                q.T[cell * G + g] = Tv[i];
                if (q.flags) q.flags[cell * G + g] = (uint8_t)fl[i];
                if (!TONLY) grain_out(tb, g, Tv[i], fl[i], s[i], nv[i], mc, mass, rs, invT, nn, ah, al);
            }
            if (emit) {
                if (SMEM) {
                    if (mass) reinterpret_cast<float *>(spairs)[g] = invT;
                    else spairs[g] = make_float2(invT, nn);
                } else if (mass) {
                    reinterpret_cast<float *>(q.prep)[cell * G8 + g] = invT;
                } else {
                    q.prep[cell * G8 + g] = make_float2(invT, nn);
                }
            }
        }
    }
    if (emit) {
        if (rs)
            for (int o = 16; o; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, ah, o), ol = __shfl_xor_sync(0xffffffffu, al, o);
                ff_add(ah, al, oh, ol);
            }
        if (lane == 0) {
            CellInfo ci;
            ci.mc = mc;
            ci.ah = rs ? ah : 0.f;
            ci.al = rs ? al : 0.f;
            ci.ms_bits = __float_as_int(ms);
            q.cell[cell] = ci;
            if (SMEM) *srec = ci;
        }
    }
}

// NB grains per lane per pass: a launch takes NB = ceil(G8 / 32) of its
// widest request (at most NB_MAX), so that a cell of up to 32 NB grains is
// one pass with no idle lanes, and its n row is loaded once: the exponent
// m_c of max_g n comes from the registers of that pass.  The loop is
// software-pipelined: the next cell's first-pass loads are issued before this
// cell's two dependent table lookups, so their DRAM latency overlaps them.
// TONLY: a launch whose requests all stop at T (no n, pairs or records), with
// the emission's code compiled out and more CTAs per SM.
template <int NB, bool TONLY>
__global__ void __launch_bounds__(SOLVE_TH, TONLY ? solve_tonly_ctas(NB) : (NB >= 4 ? 5 : 6))
    k_solve(const __grid_constant__ EmitBatch B) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * SOLVE_TH) >> 5;
    int64_t u = ((int64_t)blockIdx.x * SOLVE_TH + threadIdx.x) >> 5;  // this warp's first cell
    if (u >= B.ncells) return;
    int ri = 0;
    while (ri + 1 < B.nreq && u >= B.req[ri + 1].cell_begin) ++ri;
    float s0[NB], n0[NB];  // first pass of the current cell
    load_pass<NB, TONLY>(B.req[ri], u - B.req[ri].cell_begin, 0, lane, s0, n0);
    for (;;) {
        const EmitReq &q = B.req[ri];
        const int64_t cell = u - q.cell_begin;
        // issue the next cell's first pass now
        const int64_t un = u + nw;
        const bool more = un < B.ncells;
        int rn = ri;
        float s1[NB], n1[NB];
        if (more) {
            while (rn + 1 < B.nreq && un >= B.req[rn + 1].cell_begin) ++rn;
            load_pass<NB, TONLY>(B.req[rn], un - B.req[rn].cell_begin, 0, lane, s1, n1);
        }
        solve_cell<NB, false, TONLY>(q, cell, lane, s0, n0, nullptr, nullptr);
        if (!more) break;
        u = un;
        ri = rn;
#pragma unroll
        for (int i = 0; i < NB; ++i) { s0[i] = s1[i]; n0[i] = n1[i]; }
    }
}

// One grain's term for two wavelengths of one cell, folded into the group's
// fraction N/D.  Every FP32 step is a packed (f32x2) operation: the FMA pipe,
// not the MUFU, is the limit of this loop (an f32x2 FMA costs the FMA pipe
// as much as two scalar ones, and each ex2 takes a cycle from it as well),
// so the step is kept to five packed operations per two terms.
__device__ __forceinline__ void emit_pair(float2 nax, float2 iT, float2 nn, float2 cw, float2 &N, float2 &D) {
    const float2 a = __fmul2_rn(nax, iT);
    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    const float2 w = __fmul2_rn(nn, cw);
    const float2 e = __ffma2_rn(w, D, make_float2(-N.x, -N.y));  // w D - N
    N = __ffma2_rn(t, e, N);
    D = __ffma2_rn(make_float2(-t.x, -t.y), D, D);                // D (1 - t)
}
// The dust-mass form: the weight is the table's n_g C entry itself.
__device__ __forceinline__ void emit_pair_m(float2 nax, float2 iT, float2 cw, float2 &N, float2 &D) {
    const float2 a = __fmul2_rn(nax, iT);
    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    const float2 e = __ffma2_rn(cw, D, make_float2(-N.x, -N.y));
    N = __ffma2_rn(t, e, N);
    D = __ffma2_rn(make_float2(-t.x, -t.y), D, D);
}
__device__ __forceinline__ void emit_first_m(float2 nax, float2 iT, float2 cw, float2 &N, float2 &D) {
    const float2 a = __fmul2_rn(nax, iT);
    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    N = __fmul2_rn(cw, t);
    D = __ffma2_rn(make_float2(-t.x, -t.y), make_float2(1.f, 1.f), make_float2(1.f, 1.f));
}
// The first grain of a group, from N = 0, D = 1: N = w t, D = 1 - t.
__device__ __forceinline__ void emit_first(float2 nax, float2 iT, float2 nn, float2 cw, float2 &N, float2 &D) {
    const float2 a = __fmul2_rn(nax, iT);
    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    N = __fmul2_rn(__fmul2_rn(nn, cw), t);
    D = __ffma2_rn(make_float2(-t.x, -t.y), make_float2(1.f, 1.f), make_float2(1.f, 1.f));
}

// min that returns NaN when either operand is NaN: a grain with an invalid
// temperature keeps its group on the full form, so that its NaN reaches L.
__device__ __forceinline__ float fmin_nan(float a, float b) {
    float y;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}

// Regimes of a group of RG grains x the item's 8 wavelengths, on the largest
// exponent a = nax_k / T_g in it (nax_k < 0).  Below A_ZERO every
// t = ex2.approx.ftz(a) is flushed to 0, so the group adds nothing and is
// skipped: its terms would leave N, D and the sum unchanged, so skipping it
// gives the same bits.  Below A_WIEN every t <= 2^-24, so t / (1 - t) equals
// t to within one FP32 rounding (Wien's law) and the term is w t: no
// denominator, no reciprocal, three packed operations per two terms instead
// of five.  Below A_MID every t <= 2^-12, so t / (1 - t) = t + t^2 to within
// t^3 / t = t^2 <= 2^-24 relative, and the term is w (t + t t): four packed
// operations, still no reciprocal.
constexpr float A_ZERO = -127.f;
constexpr float A_WIEN = -24.f;
constexpr float A_MID = -12.f;

// Eq. 10 for one emission item: one cell x the 8 wavelengths of one k-group,
// over grains [0, gn) (gn a multiple of RG), added to acc[p] (wavelengths
// 2p, 2p+1).  tn: the cell's (1/T, n 2^-m_c) pairs (float2; 1/T alone in the
// dust-mass form), PST floats apart from grain to grain; cp: the k-group's
// weights [g][2] float4 (Chat of 8 wavelengths per grain); nax2: its nax
// pairs; naxl: the largest of its eight nax.
//   amax = naxl * min_g 1/T_g is the largest exponent of the group (both
//   factors' extremes are taken exactly and rounding is monotone), so the
//   regime test is exact for every term of the group.
// Every lane's arithmetic depends only on its own cell, so results are the
// same in any batch, kernel or lane arrangement.
template <bool MASS, int PST>
__device__ __forceinline__ void emit_item(const float *tn, const float4 *cp, int gn, const float2 (&nax2)[4],
                                          float naxl, float2 (&acc)[4]) {
    for (int gg0 = 0; gg0 < gn; gg0 += RG) {
        float iT[RG], nv[RG];
#pragma unroll
        for (int u = 0; u < RG; ++u) {
            if (MASS) {
                iT[u] = tn[(gg0 + u) * PST];
                nv[u] = 0.f;
            } else {
                const float2 pr = *reinterpret_cast<const float2 *>(tn + (gg0 + u) * PST);
                iT[u] = pr.x;
                nv[u] = pr.y;
            }
        }
        float m = iT[0];
#pragma unroll
        for (int u = 1; u < RG; ++u) m = fmin_nan(m, iT[u]);
        const float amax = naxl * m;
        if (amax < A_ZERO) continue;  // every term is 0
        const float4 *cg = cp + 2 * gg0;
        if (amax < A_WIEN) {
#pragma unroll
            for (int u = 0; u < RG; ++u) {
                const float4 ca = cg[2 * u], cb = cg[2 * u + 1];
                const float2 cw[4] = {make_float2(ca.x, ca.y), make_float2(ca.z, ca.w), make_float2(cb.x, cb.y),
                                      make_float2(cb.z, cb.w)};
                const float2 i2 = make_float2(iT[u], iT[u]);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float2 a = __fmul2_rn(nax2[p], i2);
                    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
                    const float2 w = MASS ? cw[p] : __fmul2_rn(make_float2(nv[u], nv[u]), cw[p]);
                    acc[p] = __ffma2_rn(w, t, acc[p]);
                }
            }
        } else if (amax < A_MID) {
#pragma unroll
            for (int u = 0; u < RG; ++u) {
                const float4 ca = cg[2 * u], cb = cg[2 * u + 1];
                const float2 cw[4] = {make_float2(ca.x, ca.y), make_float2(ca.z, ca.w), make_float2(cb.x, cb.y),
                                      make_float2(cb.z, cb.w)};
                const float2 i2 = make_float2(iT[u], iT[u]);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float2 a = __fmul2_rn(nax2[p], i2);
                    const float2 t = make_float2(ex2_approx(a.x), ex2_approx(a.y));
                    const float2 w = MASS ? cw[p] : __fmul2_rn(make_float2(nv[u], nv[u]), cw[p]);
                    acc[p] = __ffma2_rn(w, __ffma2_rn(t, t, t), acc[p]);
                }
            }
        } else {
            float2 N[4], D[4];
#pragma unroll
            for (int u = 0; u < RG; ++u) {
                const float4 ca = cg[2 * u], cb = cg[2 * u + 1];
                const float2 cw[4] = {make_float2(ca.x, ca.y), make_float2(ca.z, ca.w), make_float2(cb.x, cb.y),
                                      make_float2(cb.z, cb.w)};
                const float2 i2 = make_float2(iT[u], iT[u]);
                const float2 n2 = make_float2(nv[u], nv[u]);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    if (MASS) {
                        if (u == 0) emit_first_m(nax2[p], i2, cw[p], N[p], D[p]);
                        else emit_pair_m(nax2[p], i2, cw[p], N[p], D[p]);
                    } else {
                        if (u == 0) emit_first(nax2[p], i2, n2, cw[p], N[p], D[p]);
                        else emit_pair(nax2[p], i2, n2, cw[p], N[p], D[p]);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                acc[p].x = fmaf(N[p].x, rcp_approx(D[p].x), acc[p].x);
                acc[p].y = fmaf(N[p].y, rcp_approx(D[p].y), acc[p].y);
            }
        }
    }
}

// nax pairs of k-group ikg and the largest of its eight values.
__device__ __forceinline__ float load_nax(const DevTables &tb, int ikg, float2 (&nax2)[4]) {
    float l = -INFINITY;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        nax2[p] = __ldg(reinterpret_cast<const float2 *>(tb.nax + ikg * KQ) + p);
        l = fmaxf(l, fmaxf(nax2[p].x, nax2[p].y));
    }
    return l;
}

// Cell of slot i of a request's emission order.
__device__ __forceinline__ int64_t ordered_cell(const EmitReq &q, int64_t i) {
    return q.order ? (int64_t)__ldg(q.order + i) : i;
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Epilogue of one emission item (one cell, the 8 wavelengths of k-group
// ikg) in the warp-specialized kernel, the same arithmetic in the same order
// as k_emit's inline epilogue (kept inline there: as a call it cost k_emit
// 1-3 %): the accumulators scaled by
// 2^(m_c + q_k) (times the cell's mass mantissa ms in the dust-mass form) are
// stored as L, as two 16-byte stores (one 32-byte sector) when the row allows
// it, and the item's residual partial sum_k w_k L_k is accumulated
// error-free in float-float (products split by FMA, sums by two-sum).
template <bool MASS>
__device__ __forceinline__ void emit_item_out(const EmitReq &q, int64_t cell, int ikg, const float2 (&acc)[4], int mc,
                                              float ms, bool storeL, bool vecL, bool rs) {
    const DevTables &tb = q.tb;
    const int K = tb.K;
    float sh = 0.f, sl = 0.f;
    const int kb = ikg * KQ;
    float Lv[KQ];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = min(kb + 2 * p + h, K - 1);
            const float a = h ? acc[p].y : acc[p].x;
            Lv[2 * p + h] = scale2(MASS ? a * ms : a, mc + __ldg(tb.qexp + k));
        }
    }
    if (storeL) {
        float *row = q.L + cell * q.ld + kb;
        if (vecL && kb + KQ <= K) {
            reinterpret_cast<float4 *>(row)[0] = make_float4(Lv[0], Lv[1], Lv[2], Lv[3]);
            reinterpret_cast<float4 *>(row)[1] = make_float4(Lv[4], Lv[5], Lv[6], Lv[7]);
        } else {
#pragma unroll
            for (int j = 0; j < KQ; ++j)
                if (kb + j < K) row[j] = Lv[j];
        }
    }
    if (rs) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = kb + 2 * p + h;
                if (k < K) {
                    // w_k L_k 2^-(m_c + Ew) = wq_k a: the FP32 accumulator before
                    // its power-of-two scaling (equal to the stored L unless L is subnormal)
                    const float a = h ? acc[p].y : acc[p].x;
                    const float wk = __ldg(tb.wq + k);
                    const float pr = wk * a;
                    ff_add(sh, sl, pr, fmaf(wk, a, -pr));
                }
            }
        }
    }
    if (rs) q.part[cell * tb.NKG + ikg] = make_float2(sh, sl);
}

// Request and first cell of global emission tile `tile`.
__device__ __forceinline__ int emit_req_of(const EmitBatch &B, int64_t tile, int ri) {
    while (ri + 1 < B.nreq && tile >= B.req[ri + 1].tile_begin) ++ri;
    return ri;
}

// Issue the cp.async copies of a tile's (1/T, n) pairs into the pair-major
// shared layout [pair][grain][2 cells] (padding cells of a ragged tile read
// the dummy values instead).  Tile slots follow the request's emission order.
template <bool MASS, int NT>
__device__ __forceinline__ void prefetch_tile(const EmitReq &q, int64_t local_tile, float *dstTN, int TNP, int tid) {
    const int G8 = q.tb.G8, TC = q.TC;
    const int64_t c0 = local_tile * TC;
    const int nc = (int)((q.C - c0) < (int64_t)TC ? (q.C - c0) : (int64_t)TC);
    // (c, g) of element i = tid + j NT, advanced without a division per step
    const int dc = NT / G8, dg = NT - dc * G8;
    int c = tid / G8, g = tid - c * G8;
    for (int i = tid; i < TC * G8; i += NT) {
        if (MASS) {  // 1/T only: [pair][grain][2 cells] floats
            float *dst = dstTN + (size_t)(c >> 1) * TNP + 2 * g + (c & 1);
            if (c < nc) cp_async4(dst, reinterpret_cast<const float *>(q.prep) + ordered_cell(q, c0 + c) * G8 + g);
            else *dst = PAD_INV_T;
        } else {  // (1/T, n): [pair][grain][2 cells] float2
            float *dst = dstTN + (size_t)(c >> 1) * TNP + 4 * g + 2 * (c & 1);
            if (c < nc) cp_async8(dst, q.prep + ordered_cell(q, c0 + c) * G8 + g);
            else *reinterpret_cast<float2 *>(dst) = make_float2(PAD_INV_T, 0.f);
        }
        c += dc;
        g += dg;
        if (g >= G8) { g -= G8; ++c; }
    }
    cp_async_commit();
}

template <bool MASS, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 2) k_emit(const __grid_constant__ EmitBatch B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;

    int cur = -1;
    // per-request layout: Chat [NKG][CST] float4 | two (1/T, n) tiles [NP+1][TNP]
    // The emission item of a thread is one k-group (8 wavelengths) of two
    // neighbouring cells; items run k-group-major over the threads, so the
    // lanes of a warp share few k-groups (Chat loads are near-broadcasts) and
    // one 16-byte load fetches (1/T, n) of both cells of a pair.
    int oTN = 0, TNP = 0, CST = 0, TNB = 0;
    int ipair = 0, ikg = 0, buf = 0;
    int64_t pref = -1;  // global tile whose pairs sit (or are landing) in buffer `buf`

    for (int64_t tile = blockIdx.x; tile < B.ntiles; tile += gridDim.x) {
        int ri = emit_req_of(B, tile, cur < 0 ? 0 : cur);
        const EmitReq &q = B.req[ri];
        const DevTables &tb = q.tb;
        const int G8 = tb.G8, NKG = tb.NKG, K = tb.K, TC = q.TC, NP = TC / 2;
        const bool rs = (q.mode & EMIT_RESID) != 0;
        if (ri != cur) {
            __syncthreads();  // the previous request is done with shared memory
            cp_async_wait_all();
            cur = ri;
            TNP = (MASS ? 2 : 4) * G8 + 4;
            CST = 2 * (q.resident ? G8 : q.GC) + 1;
            TNB = (NP + 1) * TNP;  // floats per (1/T, n) tile buffer
            oTN = NKG * CST * 16;
            const bool okit = tid < NP * NKG;
            ikg = okit ? tid / NP : 0;
            ipair = okit ? tid - ikg * NP : NP;  // idle threads read the dummy pair row NP
            for (int b = 0; b < 2; ++b) {
                float *dummy = reinterpret_cast<float *>(smem_raw + oTN) + (size_t)b * TNB + (size_t)NP * TNP;
                for (int g = tid; g < G8; g += NT) {
                    if (MASS) *reinterpret_cast<float2 *>(dummy + 2 * g) = make_float2(PAD_INV_T, PAD_INV_T);
                    else *reinterpret_cast<float4 *>(dummy + 4 * g) = make_float4(PAD_INV_T, 0.f, PAD_INV_T, 0.f);
                }
            }
            if (q.resident) {
                const float4 *src = reinterpret_cast<const float4 *>(tb.Chat);
                float4 *dst = reinterpret_cast<float4 *>(smem_raw);
                for (int i = tid; i < NKG * 2 * G8; i += NT) {
                    const int kg = i / (2 * G8), o = i - kg * 2 * G8;
                    dst[(size_t)kg * CST + o] = __ldg(src + i);
                }
            }
            pref = -1;
        }
        float4 *sC = reinterpret_cast<float4 *>(smem_raw);
        float *sTN0 = reinterpret_cast<float *>(smem_raw + oTN);
        const int64_t lt = tile - q.tile_begin;
        const int64_t c0 = lt * TC;
        const int nc = (int)((q.C - c0) < (int64_t)TC ? (q.C - c0) : (int64_t)TC);
        __syncthreads();  // previous tile finished with shared memory
        if (pref != tile) {  // not prefetched (first tile of a request)
            buf = 0;
            prefetch_tile<MASS, NT>(q, lt, sTN0, TNP, tid);
        }
        cp_async_wait_all();
        __syncthreads();
        float *sTN = sTN0 + (size_t)buf * TNB;
        // prefetch the next tile of this request into the other buffer
        const int64_t nt = tile + gridDim.x;
        if (nt < B.ntiles && emit_req_of(B, nt, ri) == ri) {
            prefetch_tile<MASS, NT>(q, nt - q.tile_begin, sTN0 + (size_t)(buf ^ 1) * TNB, TNP, tid);
            pref = nt;
        } else {
            pref = -1;
        }
        // ---- emission (two cells x 8 wavelengths per thread)
        float2 acc[2][4], nax2[4];
        const float naxl = load_nax(tb, ikg, nax2);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            acc[0][p] = make_float2(0.f, 0.f);
            acc[1][p] = make_float2(0.f, 0.f);
        }
        const int GC = q.resident ? G8 : q.GC;
        for (int g0 = 0; g0 < G8; g0 += GC) {
            const int gn = min(GC, G8 - g0);
            if (!q.resident) {
                __syncthreads();
                const float4 *src = reinterpret_cast<const float4 *>(tb.Chat);
                for (int i = tid; i < NKG * 2 * gn; i += NT) {
                    const int kg = i / (2 * gn), o = i - kg * 2 * gn;
                    sC[(size_t)kg * CST + o] = __ldg(src + ((size_t)kg * G8 + g0) * 2 + o);
                }
                __syncthreads();
            }
            const int goff = q.resident ? g0 : 0;
            const float *tnp = sTN + (size_t)ipair * TNP + (MASS ? 2 : 4) * g0;
            const float4 *cp = sC + (size_t)ikg * CST + 2 * goff;
            emit_item<MASS, MASS ? 2 : 4>(tnp, cp, gn, nax2, naxl, acc[0]);
            emit_item<MASS, MASS ? 2 : 4>(tnp + (MASS ? 1 : 2), cp, gn, nax2, naxl, acc[1]);
        }
        // ---- epilogue: scale, store, residual partials.  An item's 8
        // wavelengths of a cell are one 32-byte sector of L, written as two
        // 16-byte stores when the rows allow it.  The 8-term partial
        // sum_k w_k L_k of an item is accumulated error-free in float-float
        // (products split by FMA, sums by two-sum).
        const bool storeL = (q.mode & EMIT_STORE_L) != 0;
        const bool vecL = storeL && ((reinterpret_cast<uintptr_t>(q.L) & 15) == 0) && (q.ld % 4 == 0);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int c = 2 * ipair + r;
            if (c >= nc) continue;
            const int64_t cell = ordered_cell(q, c0 + c);
            const CellInfo ci = q.cell[cell];
            const int mc = ci.mc;
            const float ms = MASS ? __int_as_float(ci.ms_bits) : 1.f;  // the cell's mass mantissa
            float sh = 0.f, sl = 0.f;
            const int kb = ikg * KQ;
            float Lv[KQ];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = min(kb + 2 * p + h, K - 1);
                    const float a = h ? acc[r][p].y : acc[r][p].x;
                    Lv[2 * p + h] = scale2(MASS ? a * ms : a, mc + __ldg(tb.qexp + k));
                }
            }
            if (storeL) {
                float *row = q.L + cell * q.ld + kb;
                if (vecL && kb + KQ <= K) {
                    reinterpret_cast<float4 *>(row)[0] = make_float4(Lv[0], Lv[1], Lv[2], Lv[3]);
                    reinterpret_cast<float4 *>(row)[1] = make_float4(Lv[4], Lv[5], Lv[6], Lv[7]);
                } else {
#pragma unroll
                    for (int j = 0; j < KQ; ++j)
                        if (kb + j < K) row[j] = Lv[j];
                }
            }
            if (rs) {
#pragma unroll
                for (int p = 0; p < 4; ++p) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = kb + 2 * p + h;
                        if (k < K) {
                            // w_k L_k 2^-(m_c + Ew) = wq_k a: the FP32 accumulator before
                            // its power-of-two scaling (equal to the stored L unless L is subnormal)
                            const float a = h ? acc[r][p].y : acc[r][p].x;
                            const float wk = __ldg(tb.wq + k);
                            const float pr = wk * a;
                            ff_add(sh, sl, pr, fmaf(wk, a, -pr));
                        }
                    }
                }
            }
            if (rs) q.part[cell * NKG + ikg] = make_float2(sh, sl);
        }
        buf ^= 1;
    }
    cp_async_wait_all();
}

// Energy-balance residual of every cell of the requests that want it: one
// thread per cell sums the cell's k-group partials in ascending order, so
// the order depends only on NKG.
// Solve and emission of one request in one warp-specialized kernel, for
// either form of n (general, or the dust-mass form n_g m_c with 1/T-only
// pairs), with the emission weights resident in shared memory.
// One CTA per SM walks tiles of FSE_TC = 32 cells, taken in the request's
// emission order (cells of like temperatures together).  Its FS_W solver
// warps run k_solve's per-cell solve (solve_cell) on the tiles ahead of the
// emission, writing T and the flags to global memory and the pairs (1/T, n
// 2^-m_c) and cell records into one of FSE_NBUF shared-memory tile buffers.
// Its FE_W emission warps claim work items from a shared counter: an item is
// one k-group of one tile, its 32 cells on the 32 lanes (emit_item), items of
// a tile claimed from the longest wavelengths (the most work) down, so that
// warps stay balanced although items differ in cost by regime.  The solve is
// a latency-bound chain of table lookups and the emission is bound by the FMA
// pipe, so the two overlap on the same SM.
// Hand-over: two mbarriers per buffer (full: the solvers' writes are done,
// FS_W arrivals; empty: every item of the tile is done, NKG arrivals); every
// wait is bounded, and on expiry the kernel records DUST_ETIMEOUT and both
// roles wind down.  Buffer phases: a warp waits on full[b] for tile ti only
// once that buffer's previous tile (ti - FSE_NBUF) is filled.  Claims run in
// order and each emission warp holds at most one unfinished item, so with
// fewer than NKG (FSE_NBUF - 1) emission warps active, a claim in tile ti
// implies a finished item in tiles ti - FSE_NBUF + 1 .. ti - 1, hence (tiles
// are filled in order) a filled tile ti - FSE_NBUF.  The kernel keeps the
// active emission warps below that bound.
constexpr int FE_W = 12;  // emission warps
constexpr int FS_W = 8;   // solver warps
constexpr int FSE_TH = (FE_W + FS_W) * 32;  // 640 threads: 96 registers each
constexpr int FSE_NBUF = 3;  // pair-tile buffers: the solvers run up to FSE_NBUF tiles ahead
constexpr int FSE_TC = 32;   // cells per tile: one per lane of an emission item

// The CTA's it-th tile.  Its tiles are blockIdx.x + j gridDim.x, coldest
// cells first (the emission order); they are taken from both ends in turn
// (first, last, second, second to last, ...), so that tiles of cheap
// emission (cold cells: many groups skipped) alternate with expensive ones
// and the solve, whose cost per tile is even, stays in step.
__device__ __forceinline__ int64_t fse_tile(int64_t it, int64_t ntiles) {
    const int64_t nb = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;  // this CTA's tiles
    const int64_t j = (it & 1) ? nb - 1 - (it >> 1) : (it >> 1);
    return it < nb ? blockIdx.x + j * gridDim.x : ntiles;
}

template <int NB, bool MASS>
__global__ void __launch_bounds__(FSE_TH, 1) k_solve_emit(const __grid_constant__ EmitReq q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevTables &tb = q.tb;
    const int G8 = tb.G8, NKG = tb.NKG;
    constexpr int TC = FSE_TC;
    const int CST = 2 * G8 + 1;
    // odd row stride of a pair tile (in float2, or floats for 1/T alone): a warp's cells fall in distinct banks
    const int PS = G8 + 1;
    constexpr int PW = MASS ? 1 : 2;  // floats per pair
    float4 *sC = reinterpret_cast<float4 *>(smem_raw);                          // [NKG][CST]
    float *sP = reinterpret_cast<float *>(sC + (size_t)NKG * CST);             // [FSE_NBUF][TC][PS][PW]
    CellInfo *sI = reinterpret_cast<CellInfo *>(sP + (((size_t)FSE_NBUF * TC * PS * PW + 3) & ~(size_t)3));  // [FSE_NBUF][TC]
    uint64_t *full = reinterpret_cast<uint64_t *>(sI + FSE_NBUF * TC);         // [FSE_NBUF]
    uint64_t *empty = full + FSE_NBUF;                                         // [FSE_NBUF]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + FSE_NBUF);
    int *claim = const_cast<int *>(abort_flag) + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (q.C + TC - 1) / TC;

    {
        const float4 *src = reinterpret_cast<const float4 *>(tb.Chat);
        for (int i = tid; i < NKG * 2 * G8; i += FSE_TH) {
            const int kg = i / (2 * G8), o = i - kg * 2 * G8;
            sC[(size_t)kg * CST + o] = __ldg(src + i);
        }
    }
    if (tid == 0) {
        for (int b = 0; b < FSE_NBUF; ++b) { mbar_init(&full[b], FS_W); mbar_init(&empty[b], NKG); }
        *abort_flag = 0;
        *claim = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp >= FE_W) {
        // ------------------------------------------------------------ solvers
        const int sw = warp - FE_W;
        int it = 0;
        int64_t tile = fse_tile(0, ntiles);
        float s0[NB], n0[NB];
        int64_t pf = -1;  // the tile whose first slot of this warp s0 / n0 hold
        bool ok = true;
        for (; tile < ntiles && ok; tile = fse_tile(++it, ntiles)) {
            const int b = it % FSE_NBUF;
            const uint32_t ph = (uint32_t)((it / FSE_NBUF) & 1);
            const int nc = (int)min((int64_t)TC, q.C - tile * TC);
            // a warp with no slot in the previous tile (a ragged one) prefetched nothing
            if (sw < nc && pf != tile) load_pass<NB>(q, ordered_cell(q, tile * TC + sw), 0, lane, s0, n0);
            if (!(ok = mbar_wait(&empty[b], ph ^ 1, abort_flag, tb.status))) break;
            for (int cl = sw; cl < nc; cl += FS_W) {
                const int64_t cell = ordered_cell(q, tile * TC + cl);
                // next cell of this warp: in this tile, else its first in the next tile
                int64_t tn = tile;
                int cn = cl + FS_W;
                if (cn >= nc) { tn = fse_tile(it + 1, ntiles); cn = sw; }
                const bool more = tn < ntiles && tn * TC + cn < q.C;
                float s1[NB], n1[NB];
                if (more) load_pass<NB>(q, ordered_cell(q, tn * TC + cn), 0, lane, s1, n1);
                pf = more ? tn : -1;
                solve_cell<NB, true, false, MASS ? 1 : 0, true>(q, cell, lane, s0, n0,
                                                                reinterpret_cast<float2 *>(sP + ((size_t)b * TC + cl) * PS * PW),
                                                                sI + b * TC + cl);
#pragma unroll
                for (int i = 0; i < NB; ++i) { s0[i] = s1[i]; n0[i] = n1[i]; }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[b]);
        }
    } else {
        // ------------------------------------------------------------ emission
        if (warp >= NKG * (FSE_NBUF - 1) - 1) return;  // see the phase argument above
        const bool rs = (q.mode & EMIT_RESID) != 0, storeL = (q.mode & EMIT_STORE_L) != 0;
        const bool vecL = storeL && ((reinterpret_cast<uintptr_t>(q.L) & 15) == 0) && (q.ld % 4 == 0);
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(claim, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            const int ti = w / NKG;
            const int ikg = NKG - 1 - (w - ti * NKG);
            const int64_t tile = fse_tile(ti, ntiles);
            if (tile >= ntiles) break;
            const int b = ti % FSE_NBUF;
            const uint32_t ph = (uint32_t)((ti / FSE_NBUF) & 1);
            if (!mbar_wait(&full[b], ph, abort_flag, tb.status)) break;
            const int nc = (int)min((int64_t)TC, q.C - tile * TC);
            if (lane < nc) {
                float2 nax2[4], acc[4];
                const float naxl = load_nax(tb, ikg, nax2);
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[p] = make_float2(0.f, 0.f);
                emit_item<MASS, PW>(sP + ((size_t)b * TC + lane) * PS * PW, sC + (size_t)ikg * CST, G8, nax2, naxl, acc);
                const CellInfo ci = sI[b * TC + lane];
                emit_item_out<MASS>(q, ordered_cell(q, tile * TC + lane), ikg, acc, ci.mc,
                                    MASS ? __int_as_float(ci.ms_bits) : 1.f, storeL, vecL, rs);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
        }
    }
}

__global__ void __launch_bounds__(SOLVE_TH) k_resid(const __grid_constant__ EmitBatch E) {
    const int64_t stride = (int64_t)gridDim.x * SOLVE_TH;
    int ri = 0;
    for (int64_t u = (int64_t)blockIdx.x * SOLVE_TH + threadIdx.x; u < E.ncells; u += stride) {
        while (ri + 1 < E.nreq && u >= E.req[ri + 1].cell_begin) ++ri;
        const EmitReq &q = E.req[ri];
        if (!(q.mode & EMIT_RESID)) continue;
        const int NKG = q.tb.NKG;
        const int64_t cell = u - q.cell_begin;
        const float2 *pp = q.part + cell * NKG;
        float h = 0.f, l = 0.f;
        for (int kg = 0; kg < NKG; ++kg) {
            const float2 v = pp[kg];
            ff_add(h, l, v.x, v.y);
        }
        const CellInfo ci = q.cell[cell];
        q.resid[cell] = (double)residual(h, l, ci.ah, ci.al, q.tb);
    }
}

}  // namespace

// Emission geometry of one request: cells per tile, grain chunk, residency
// of the emission weights and the shared memory they need.
EmitPlan plan_emit(const dust_ctx *ctx, bool emit, bool mass) {
    const DevTables &tb = ctx->tb;
    EmitPlan p{};
    auto fixed_of = [&](int np) { return (size_t)2 * (np + 1) * ((mass ? 2 : 4) * tb.G8 + 4) * 4 + 64; };
    int NP = std::max(1, std::min(32, NTH / tb.NKG));  // cell pairs per tile
    p.TC = 2 * NP;
    p.nth = NTH;
    if (!emit) { p.GC = tb.G8; p.resident = 0; p.smem = 0; return p; }
    const size_t budget = 113 * 1024;  // two CTAs per SM
    const size_t full = (size_t)tb.NKG * (2 * tb.G8 + 1) * 16 + fixed_of(NP);
    if (full <= budget) { p.GC = tb.G8; p.resident = 1; p.smem = full; return p; }
    // streamed weights: one CTA of 2 NTH threads per SM, twice the cells per
    // tile and the whole shared memory for the grain chunks, so that each
    // staged chunk serves more cells and fewer barriers are paid per cell
    p.nth = EMIT_STREAM_NTH;
    const size_t budget2 = ctx->smem_optin ? ctx->smem_optin - 1024 : budget;
    NP = std::max(1, std::min(32, p.nth / tb.NKG));
    while (NP > 1 && fixed_of(NP) + (size_t)tb.NKG * (2 * RG + 1) * 16 > budget2) --NP;  // room for a chunk
    p.TC = 2 * NP;
    const size_t fixed = fixed_of(NP);
    const size_t avail = budget2 > fixed ? budget2 - fixed : 0;
    int gc = (int)((avail / ((size_t)tb.NKG * 16) - 1) / 2) / RG * RG;
    gc = std::max(RG, std::min(gc, tb.G8));
    p.GC = gc;
    p.resident = 0;
    p.smem = (size_t)tb.NKG * (2 * gc + 1) * 16 + fixed;
    return p;
}

// Scratch bytes of a request of C cells: S [C][Gs] FP32, then (emission)
// the (1/T, n) pairs [C][G8], one CellInfo per cell, the residual partials
// [C][NKG] float2, the emission order [C] int32, the cells' classes [C]
// uint16 and the class counts and cursors [2][NBK] uint32, each 16-byte
// aligned.
namespace {
inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }
}  // namespace

size_t scratch_bytes(const dust_ctx *ctx, int64_t C, bool emit) {
    size_t b = al16((size_t)C * ctx->tb.Gs * 4);
    if (emit)
        b += al16((size_t)C * ctx->tb.G8 * 8) + (size_t)C * sizeof(CellInfo) + al16((size_t)C * ctx->tb.NKG * 8) +
             al16((size_t)C * 4) + al16((size_t)C * 2) + (size_t)2 * NBK * 4;
    return b;
}

ScratchView scratch_view(const dust_ctx *ctx, int64_t C, void *base) {
    ScratchView v;
    char *p = static_cast<char *>(base);
    v.S = reinterpret_cast<float *>(p);
    p += al16((size_t)C * ctx->tb.Gs * 4);
    v.prep = reinterpret_cast<float2 *>(p);
    p += al16((size_t)C * ctx->tb.G8 * 8);
    v.cell = reinterpret_cast<CellInfo *>(p);
    p += (size_t)C * sizeof(CellInfo);
    v.part = reinterpret_cast<float2 *>(p);
    p += al16((size_t)C * ctx->tb.NKG * 8);
    v.order = reinterpret_cast<int *>(p);
    p += al16((size_t)C * 4);
    v.bkt = reinterpret_cast<uint16_t *>(p);
    p += al16((size_t)C * 2);
    v.hist = reinterpret_cast<unsigned *>(p);
    return v;
}

void fill_emit_req(const dust_ctx *ctx, const EmitPlan &p, int64_t C, const ScratchView &sv, const float *n,
                   float *T, float *L, int64_t ld, double *resid, uint8_t *flags, EmitReq &r, bool mass) {
    r.tb = mass ? ctx->tbm : ctx->tb;
    r.C = C;
    r.ld = ld;
    r.tile_begin = 0;
    r.cell_begin = 0;
    r.S = sv.S;
    r.n = n;
    r.T = T;
    r.L = L;
    r.resid = resid;
    r.flags = flags;
    r.prep = sv.prep;
    r.cell = sv.cell;
    r.part = sv.part;
    r.order = nullptr;
    r.TC = p.TC;
    r.GC = p.GC;
    r.resident = p.resident;
    r.nth = p.nth;
    r.smem = (uint32_t)p.smem;
    r.mode = ((L || resid) ? EMIT_ON : 0) | (resid ? EMIT_RESID : 0) | (L ? EMIT_STORE_L : 0) |
             ((mass && (L || resid)) ? EMIT_MASS : 0);
}

// Numbers the cells and emission tiles of a filled batch; launches the solve
// over every request, then the emission over the requests that want it.
int launch_emit_batch(EmitBatch &B, size_t smem, int num_sms, cudaStream_t st, cudaEvent_t between,
                      bool solved, int *nlaunch) {
    int nl = 0;
    int64_t cells = 0;
    for (int i = 0; i < B.nreq; ++i) {
        EmitReq &r = B.req[i];
        r.cell_begin = cells;
        cells += r.C;
    }
    B.ncells = cells;
    if (nlaunch) *nlaunch = 0;
    if (cells <= 0) return DUST_OK;
    if (!solved) {
        // one warp per cell, up to 16 CTAs of 4 warps per SM
        int g8 = 8;
        for (int i = 0; i < B.nreq; ++i) g8 = std::max(g8, B.req[i].tb.G8);
        const int nb = std::min(NB_MAX, (g8 + 31) / 32);
        const int64_t grid = std::min<int64_t>((cells * 32 + SOLVE_TH - 1) / SOLVE_TH, (int64_t)num_sms * 16);
        bool tonly = true;
        for (int i = 0; i < B.nreq; ++i) tonly = tonly && !(B.req[i].mode & EMIT_ON);
        if (tonly) {
            switch (nb) {
                case 1: k_solve<1, true><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
                case 2: k_solve<2, true><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
                case 3: k_solve<3, true><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
                default: k_solve<4, true><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
            }
        } else {
            switch (nb) {
                case 1: k_solve<1, false><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
                case 2: k_solve<2, false><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
                case 3: k_solve<3, false><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
                default: k_solve<4, false><<<(unsigned)grid, SOLVE_TH, 0, st>>>(B); break;
            }
        }
        DUST_CUDA_TRY(cudaGetLastError());
        ++nl;
    }
    if (between) DUST_CUDA_TRY(cudaEventRecord(between, st));
    // emission work lists: the requests that want L or resid, in order, one
    // list (and launch) per form of the grain numbers and CTA size
    for (int form = 0; form < 2; ++form) {
        for (int nt : {NTH, EMIT_STREAM_NTH}) {
            EmitBatch E;
            E.nreq = 0;
            int64_t tiles = 0;
            size_t lsmem = 0;
            for (int i = 0; i < B.nreq; ++i) {
                if (!(B.req[i].mode & EMIT_ON) || ((B.req[i].mode & EMIT_MASS) != 0) != (form == 1) ||
                    B.req[i].nth != nt)
                    continue;
                EmitReq &r = E.req[E.nreq++];
                r = B.req[i];
                r.tile_begin = tiles;
                tiles += (r.C + r.TC - 1) / r.TC;
                lsmem = std::max(lsmem, (size_t)r.smem);
            }
            E.ntiles = tiles;
            E.ncells = 0;
            bool resid = false;
            for (int i = 0; i < E.nreq; ++i) {  // cells of the emission list, numbered afresh
                E.req[i].cell_begin = E.ncells;
                E.ncells += E.req[i].C;
                resid = resid || (E.req[i].mode & EMIT_RESID);
            }
            if (tiles == 0) continue;
            const void *kern = form ? (nt == NTH ? reinterpret_cast<const void *>(k_emit<true, NTH>)
                                                 : reinterpret_cast<const void *>(k_emit<true, EMIT_STREAM_NTH>))
                                    : (nt == NTH ? reinterpret_cast<const void *>(k_emit<false, NTH>)
                                                 : reinterpret_cast<const void *>(k_emit<false, EMIT_STREAM_NTH>));
            DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
            int per_sm = 0;
            DUST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, lsmem));
            per_sm = std::max(per_sm, 1);
            const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)num_sms * per_sm);
            if (form) {
                if (nt == NTH) k_emit<true, NTH><<<grid, NTH, lsmem, st>>>(E);
                else k_emit<true, EMIT_STREAM_NTH><<<grid, EMIT_STREAM_NTH, lsmem, st>>>(E);
            } else {
                if (nt == NTH) k_emit<false, NTH><<<grid, NTH, lsmem, st>>>(E);
                else k_emit<false, EMIT_STREAM_NTH><<<grid, EMIT_STREAM_NTH, lsmem, st>>>(E);
            }
            DUST_CUDA_TRY(cudaGetLastError());
            ++nl;
            if (resid) {
                const int64_t rgrid = std::min<int64_t>((E.ncells + SOLVE_TH - 1) / SOLVE_TH, (int64_t)num_sms * 16);
                k_resid<<<(unsigned)rgrid, SOLVE_TH, 0, st>>>(E);
                DUST_CUDA_TRY(cudaGetLastError());
                ++nl;
            }
        }
    }
    if (nlaunch) *nlaunch = nl;
    return DUST_OK;
}

// Tile and shared memory of the warp-specialized solve + emission kernel for
// the context, or 0 where it does not apply: no emission, or emission
// weights that do not fit beside the pair tiles with room left for L1 (the
// solve's table lookups live there).
size_t plan_solve_emit(const dust_ctx *ctx, bool emit, bool mass, int *TC) {
    if (!emit || (mass && !ctx->mass_ready)) return 0;
    const DevTables &tb = mass ? ctx->tbm : ctx->tb;
    const int tc = FSE_TC;
    const size_t smem = (size_t)tb.NKG * (2 * tb.G8 + 1) * 16 + (((size_t)FSE_NBUF * tc * (tb.G8 + 1) * (mass ? 4 : 8) + 15) & ~(size_t)15) +
                        (size_t)FSE_NBUF * tc * sizeof(CellInfo) + 2 * FSE_NBUF * sizeof(uint64_t) + 16;
    if (smem > 160 * 1024) return 0;
    *TC = tc;
    return smem;
}

// The fused kernel over one request (general form), then the residual fold.
template <bool MASS>
int launch_fse(const EmitReq &r, int nb, unsigned grid, size_t smem, cudaStream_t st) {
    const void *kern = nb == 1 ? reinterpret_cast<const void *>(k_solve_emit<1, MASS>)
                     : nb == 2 ? reinterpret_cast<const void *>(k_solve_emit<2, MASS>)
                     : nb == 3 ? reinterpret_cast<const void *>(k_solve_emit<3, MASS>)
                               : reinterpret_cast<const void *>(k_solve_emit<4, MASS>);
    DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    switch (nb) {
        case 1: k_solve_emit<1, MASS><<<grid, FSE_TH, smem, st>>>(r); break;
        case 2: k_solve_emit<2, MASS><<<grid, FSE_TH, smem, st>>>(r); break;
        case 3: k_solve_emit<3, MASS><<<grid, FSE_TH, smem, st>>>(r); break;
        default: k_solve_emit<4, MASS><<<grid, FSE_TH, smem, st>>>(r); break;
    }
    DUST_CUDA_TRY(cudaGetLastError());
    return DUST_OK;
}

int launch_solve_emit_fused(const EmitReq &req, int TC, size_t smem, int num_sms, cudaStream_t st,
                            int *nlaunch) {
    if (nlaunch) *nlaunch = 0;
    if (req.C <= 0) return DUST_OK;
    EmitBatch E;
    E.nreq = 1;
    E.req[0] = req;
    EmitReq &r = E.req[0];
    r.TC = TC;
    r.cell_begin = 0;
    r.tile_begin = 0;
    E.ncells = r.C;
    E.ntiles = (r.C + TC - 1) / TC;
    const int nb = std::min(NB_MAX, (r.tb.G8 + 31) / 32);
    const bool mass = (r.mode & EMIT_MASS) != 0;
    const unsigned grid = (unsigned)std::min<int64_t>(E.ntiles, num_sms);
    int rc = mass ? launch_fse<true>(r, nb, grid, smem, st) : launch_fse<false>(r, nb, grid, smem, st);
    if (rc != DUST_OK) return rc;
    if (nlaunch) *nlaunch = 1;
    if (r.mode & EMIT_RESID) {
        const int64_t rgrid = std::min<int64_t>((r.C + SOLVE_TH - 1) / SOLVE_TH, (int64_t)num_sms * 16);
        k_resid<<<(unsigned)rgrid, SOLVE_TH, 0, st>>>(E);
        DUST_CUDA_TRY(cudaGetLastError());
        if (nlaunch) *nlaunch = 2;
    }
    return DUST_OK;
}

int launch_solve_emit(const dust_ctx *ctx, int64_t C, const ScratchView &sv, const float *n, float *T, float *L,
                      int64_t ld, double *resid, uint8_t *flags, cudaStream_t st) {
    if (C <= 0) return DUST_OK;
    const EmitPlan p = plan_emit(ctx, L || resid, false);
    EmitBatch B;
    B.nreq = 1;
    fill_emit_req(ctx, p, C, sv, n, T, L, ld, resid, flags, B.req[0], false);
    return launch_emit_batch(B, p.smem, ctx->num_sms, st);
}

}  // namespace dust

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
//   (A / P_g(T_min) = S 2^f_g): y = log2 S + f_g selects the interval of
//   the inverse table that brackets the root, and one Newton step on that
//   interval's cubic Hermite of t_g(u) = log2(P_g(2^u) / P_g(T_min)) gives
//   u = log2 T (bisection when a step leaves the bracket); one table load
//   per grain.  The paper's kernel 3 iterated Newton
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
// to `spairs` (its first gsm grains, float2 or floats in the dust-mass form)
// and `srec` in shared memory as well as the record to q.cell, and with
// also_glb the pairs of every grain to q.prep too.  s0 / n0: this cell's
// first pass, loaded.
// MF: the form of n when the caller knows it (0 general, 1 dust-mass), -1 to
// read it from the request; EMIT: the emission is known to follow (the fused
// kernel, whose launch has NB = ceil(G8 / 32), so a cell is one pass when
// NB < NB_MAX).
template <int NB, bool SMEM, bool TONLY = false, int MF = -1, bool EMIT = false>
__device__ __forceinline__ void solve_cell(const EmitReq &q, int64_t cell, int lane, const float (&s0)[NB],
                                           const float (&n0)[NB], float2 *spairs, CellInfo *srec,
                                           int gsm = 1 << 30, bool also_glb = false) {
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
                if (SMEM && g < gsm) {
                    if (mass) reinterpret_cast<float *>(spairs)[g] = invT;
                    else spairs[g] = make_float2(invT, nn);
                }
                if (!SMEM || also_glb) {
                    if (mass) reinterpret_cast<float *>(q.prep)[cell * G8 + g] = invT;
                    else q.prep[cell * G8 + g] = make_float2(invT, nn);
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
// GLB: tn is the cell's row of the solve's scratch in global memory, read
// through the read-only path (L1), instead of a shared-memory tile.
template <bool MASS, int PST, bool GLB = false>
__device__ __forceinline__ void emit_item(const float *tn, const float4 *cp, int gn, const float2 (&nax2)[4],
                                          float naxl, float2 (&acc)[4]) {
    for (int gg0 = 0; gg0 < gn; gg0 += RG) {
        float iT[RG], nv[RG];
#pragma unroll
        for (int u = 0; u < RG; ++u) {
            if (MASS) {
                iT[u] = GLB ? __ldg(tn + (gg0 + u) * PST) : tn[(gg0 + u) * PST];
                nv[u] = 0.f;
            } else {
                const float2 *pp = reinterpret_cast<const float2 *>(tn + (gg0 + u) * PST);
                const float2 pr = GLB ? __ldg(pp) : *pp;
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

// ---- the two-kernel emission: pairs from the solve kernel's scratch
// k_emit runs over a work list of requests whose temperatures are solved,
// each split into work units of up to tpu tiles (32 cells in the request's
// emission order), one CTA per unit, so that a CTA serves one request and
// loads its weights once.  Where the weights of every k-group for all grains
// do not fit in shared memory beside the pair tiles, a request is emitted
// in passes over grain chunks [g0, g1): a pass starts its sums from those
// the previous pass left in the scratch (accp) and the last one finishes
// them, so every item adds its groups in the same order as one pass would.
// Per CTA one copier warp fills KE_NBUF pair-tile buffers from the scratch
// (cp.async, 8 bytes per pair) and KE_W emission warps claim the items in
// order (one k-group of one tile, its cells on the 32 lanes, emit_item), the
// longest wavelengths of a tile first.  Hand-over through monotone counters
// per buffer: the copier adds 1 to filled[b] per tile, emission warps add 1
// to drained[b] per item; the i-th tile of the unit (buffer i % KE_NBUF) is
// emitted once filled[b] >= i / KE_NBUF + 1, and refilled once drained[b]
// counts every item of the tiles put there before it.  Waits poll with a
// short sleep, are bounded, and record DUST_ETIMEOUT.
constexpr int KE_W = 15;                // emission warps
constexpr int KE_TH = (KE_W + 1) * 32;  // and one copier warp: 512 threads, 128 registers
constexpr int KE_NBUF = 3;

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

__device__ __forceinline__ int ld_acquire_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void add_release_cta(int *p, int v) {
    asm volatile("red.release.cta.shared.add.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
// Lane 0 waits until *ctr >= target (bounded, polling with a short sleep);
// the warp learns the outcome and is ordered after the writes it waited for.
__device__ __forceinline__ bool warp_wait_geq(const int *ctr, int target, volatile int *abort_flag, int *status,
                                              int lane) {
    int ok = 1;
    if (lane == 0 && ld_acquire_cta(ctr) < target) {
        const unsigned long long t0 = globaltimer_ns();
        for (;;) {
            __nanosleep(100);
            if (ld_acquire_cta(ctr) >= target) break;
            if (*abort_flag) { ok = 0; break; }
            if (globaltimer_ns() - t0 > WAIT_NS) {
                *abort_flag = 1;
                record_status(status, DUST_ETIMEOUT);
                ok = 0;
                break;
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

template <bool MASS>
__global__ void __launch_bounds__(KE_TH, 1) k_emit(const __grid_constant__ EmitBatch B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TC = KE_TC;
    constexpr int PW = MASS ? 1 : 2;  // floats per pair
    int ri = 0;
    while (ri + 1 < B.nreq && (int64_t)blockIdx.x >= B.req[ri + 1].unit_begin) ++ri;
    const EmitReq &q = B.req[ri];
    const DevTables &tb = q.tb;
    const int G8 = tb.G8, NKG = tb.NKG, gc = q.g1 - q.g0, PS = gc + 1, CST = 2 * gc + 1;
    const int64_t ntiles = (q.C + TC - 1) / TC;
    const int64_t t0 = ((int64_t)blockIdx.x - q.unit_begin) * q.tpu;
    const int ntl = (int)min(q.tpu, ntiles - t0);
    // shared memory: counters, the pair buffers [KE_NBUF][TC][PS][PW], the weights [NKG][CST] of the grain chunk
    int *filled = reinterpret_cast<int *>(smem_raw);  // [KE_NBUF]
    int *drained = filled + 4;                        // [KE_NBUF]
    int *claim = drained + 4;
    volatile int *abort_flag = claim + 1;
    float *sP = reinterpret_cast<float *>(smem_raw + 64);
    float4 *sC = reinterpret_cast<float4 *>(sP + (((size_t)KE_NBUF * TC * PS * PW + 3) & ~(size_t)3));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const float4 *src = reinterpret_cast<const float4 *>(tb.Chat);
        for (int i = tid; i < NKG * 2 * gc; i += KE_TH) {
            const int kg = i / (2 * gc), o = i - kg * 2 * gc;
            sC[(size_t)kg * CST + o] = __ldg(src + ((size_t)kg * G8 + q.g0) * 2 + o);
        }
    }
    if (tid < 4) { filled[tid] = 0; drained[tid] = 0; }
    if (tid == 0) { *claim = 0; *abort_flag = 0; }
    __syncthreads();
    if (ntl <= 0) return;

    if (warp == KE_W) {
        // ------------------------------------------------------------ copier
        int expect[KE_NBUF] = {};  // items of the tiles put in each buffer so far
        for (int i = 0; i < ntl; ++i) {
            const int b = i % KE_NBUF;
            if (!warp_wait_geq(&drained[b], expect[b], abort_flag, tb.status, lane)) break;
            const int64_t c0 = (t0 + i) * TC;
            const int nc = (int)min((int64_t)TC, q.C - c0);
            float *dst = sP + (size_t)b * TC * PS * PW;
            // row c of the buffer <- grains [g0, g1) of the pairs of cell order[c0 + c]
            const int64_t mycell = lane < nc ? ordered_cell(q, c0 + lane) : 0;
            for (int c = 0; c < nc; ++c) {
                const int64_t cell = __shfl_sync(0xffffffffu, mycell, c);
                for (int g = lane; g < gc; g += 32) {
                    if (MASS) cp_async4(dst + (size_t)c * PS + g, reinterpret_cast<const float *>(q.prep) + cell * G8 + q.g0 + g);
                    else cp_async8(dst + ((size_t)c * PS + g) * 2, q.prep + cell * G8 + q.g0 + g);
                }
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncwarp();
            if (lane == 0) add_release_cta(&filled[b], 1);
            expect[b] += NKG;
        }
    } else {
        // ------------------------------------------------------------ emission
        const bool first = q.g0 == 0, last = q.g1 == G8;
        const bool rs = (q.mode & EMIT_RESID) != 0, storeL = (q.mode & EMIT_STORE_L) != 0;
        const bool vecL = storeL && ((reinterpret_cast<uintptr_t>(q.L) & 15) == 0) && (q.ld % 4 == 0);
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(claim, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            const int i = w / NKG;
            if (i >= ntl) break;
            const int ikg = NKG - 1 - (w - i * NKG);
            const int b = i % KE_NBUF;
            if (!warp_wait_geq(&filled[b], i / KE_NBUF + 1, abort_flag, tb.status, lane)) break;
            const int64_t c0 = (t0 + i) * TC;
            const int nc = (int)min((int64_t)TC, q.C - c0);
            if (lane < nc) {
                const int64_t cell = ordered_cell(q, c0 + lane);
                float2 nax2[4], acc[4];
                const float naxl = load_nax(tb, ikg, nax2);
                float2 *ap = q.accp + ((size_t)cell * NKG + ikg) * 4;
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[p] = first ? make_float2(0.f, 0.f) : ap[p];
                // the cell record is read now, so that its latency hides behind the sums
                CellInfo ci{};
                if (last) ci = q.cell[cell];
                emit_item<MASS, PW>(sP + ((size_t)b * TC + lane) * PS * PW, sC + (size_t)ikg * CST, gc, nax2, naxl, acc);
                if (last) {
                    emit_item_out<MASS>(q, cell, ikg, acc, ci.mc, MASS ? __int_as_float(ci.ms_bits) : 1.f, storeL, vecL,
                                        rs);
                } else {
#pragma unroll
                    for (int p = 0; p < 4; ++p) ap[p] = acc[p];
                }
            }
            __syncwarp();
            if (lane == 0) add_release_cta(&drained[b], 1);
        }
    }
}

// Residual of one cell (Eq. 6 against Eqs. 8-10, see residual()) from its
// k-group partials, summed in ascending order, and its cell record.
__device__ __forceinline__ void cell_resid(const EmitReq &q, int64_t cell) {
    const int NKG = q.tb.NKG;
    const float2 *pp = q.part + cell * NKG;
    float h = 0.f, l = 0.f;
    for (int kg = 0; kg < NKG; ++kg) {
        const float2 v = pp[kg];
        ff_add(h, l, v.x, v.y);
    }
    const CellInfo ci = q.cell[cell];
    q.resid[cell] = (double)residual(h, l, ci.ah, ci.al, q.tb);
}

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

template <int NB, bool MASS, bool PASS>
__global__ void __launch_bounds__(FSE_TH, 1) k_solve_emit(const __grid_constant__ EmitReq q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevTables &tb = q.tb;
    const int G8 = tb.G8, NKG = tb.NKG;
    // the grains of this launch, [0, gc): all of them, or (PASS) the first
    // grain pass of a request whose weights do not fit (the later passes
    // follow in k_emit)
    const int gc = PASS ? q.g1 - q.g0 : G8;
    constexpr bool whole = !PASS;
    constexpr int TC = FSE_TC;
    const int CST = 2 * gc + 1;
    // odd row stride of a pair tile (in float2, or floats for 1/T alone): a warp's cells fall in distinct banks
    const int PS = gc + 1;
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
        for (int i = tid; i < NKG * 2 * gc; i += FSE_TH) {
            const int kg = i / (2 * gc), o = i - kg * 2 * gc;
            sC[(size_t)kg * CST + o] = __ldg(src + ((size_t)kg * G8 + q.g0) * 2 + o);
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
        const bool rs = (q.mode & EMIT_RESID) != 0 && whole;  // else the fold follows the last pass
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
            // the buffer's previous tile (it - FSE_NBUF) is fully emitted: one
            // solver warp, in turn, folds its cells' residuals (lane = cell)
            if (rs && it >= FSE_NBUF && sw == it % FS_W) {
                const int64_t i = fse_tile(it - FSE_NBUF, ntiles) * TC + lane;
                if (i < q.C) cell_resid(q, ordered_cell(q, i));
            }
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
                                                                sI + b * TC + cl, PASS ? gc : 1 << 30, PASS);
#pragma unroll
                for (int i = 0; i < NB; ++i) { s0[i] = s1[i]; n0[i] = n1[i]; }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[b]);
        }
        // the residuals of the last FSE_NBUF tiles, once their emission is done
        if (rs && ok && sw == 0)
            for (int j = max(0, it - FSE_NBUF); j < it; ++j) {
                if (!mbar_wait(&empty[j % FSE_NBUF], (uint32_t)((j / FSE_NBUF) & 1), abort_flag, tb.status)) break;
                const int64_t i = fse_tile(j, ntiles) * TC + lane;
                if (i < q.C) cell_resid(q, ordered_cell(q, i));
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
                emit_item<MASS, PW>(sP + ((size_t)b * TC + lane) * PS * PW, sC + (size_t)ikg * CST, gc, nax2, naxl, acc);
                const int64_t cell = ordered_cell(q, tile * TC + lane);
                if constexpr (whole) {
                    const CellInfo ci = sI[b * TC + lane];
                    emit_item_out<MASS>(q, cell, ikg, acc, ci.mc, MASS ? __int_as_float(ci.ms_bits) : 1.f, storeL,
                                        vecL, rs);
                } else {
                    // the first pass's sums, carried to the next (k_emit's layout)
                    float2 *ap = q.accp + ((size_t)cell * NKG + ikg) * 4;
#pragma unroll
                    for (int p = 0; p < 4; ++p) ap[p] = acc[p];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
        }
    }
}

// Energy-balance residual of every cell of the requests that want it: one
// thread per cell sums the cell's k-group partials in ascending order, so
// the order depends only on NKG (cell_resid; the warp-specialized kernel
// folds its own cells with the same function).
__global__ void __launch_bounds__(SOLVE_TH) k_resid(const __grid_constant__ EmitBatch E) {
    const int64_t stride = (int64_t)gridDim.x * SOLVE_TH;
    int ri = 0;
    for (int64_t u = (int64_t)blockIdx.x * SOLVE_TH + threadIdx.x; u < E.ncells; u += stride) {
        while (ri + 1 < E.nreq && u >= E.req[ri + 1].cell_begin) ++ri;
        const EmitReq &q = E.req[ri];
        if (!(q.mode & EMIT_RESID)) continue;
        cell_resid(q, u - q.cell_begin);
    }
}

}  // namespace

// Emission geometry of one request in the two-kernel form: 32-cell tiles,
// KE_NBUF pair buffers and the weights of every k-group for a chunk of gcp
// grains in shared memory; all grains when they fit, otherwise the largest
// chunk (a multiple of RG) that does.
namespace {
size_t ke_smem(int NKG, int gc, bool mass) {
    return 64 + (((size_t)KE_NBUF * KE_TC * (gc + 1) * (mass ? 1 : 2) * 4 + 15) & ~(size_t)15) +
           (size_t)NKG * (2 * gc + 1) * 16;
}
}  // namespace

EmitPlan plan_emit(const dust_ctx *ctx, bool emit, bool mass) {
    const DevTables &tb = mass ? ctx->tbm : ctx->tb;
    EmitPlan p{};
    p.TC = KE_TC;
    p.gcp = tb.G8;
    if (!emit) { p.smem = 0; return p; }
    const size_t budget = (ctx->smem_optin ? ctx->smem_optin : 99 * 1024) - 1024;
    while (p.gcp > RG && ke_smem(tb.NKG, p.gcp, mass) > budget) p.gcp -= RG;
    p.smem = ke_smem(tb.NKG, p.gcp, mass);
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
    if (emit) {
        b += al16((size_t)C * ctx->tb.G8 * 8) + (size_t)C * sizeof(CellInfo) + al16((size_t)C * ctx->tb.NKG * 8) +
             al16((size_t)C * 4) + al16((size_t)C * 2) + (size_t)2 * NBK * 4;
        if (plan_emit(ctx, true, false).gcp < ctx->tb.G8) b += (size_t)C * ctx->tb.NKG * 32;
    }
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
    p += (size_t)2 * NBK * 4;
    v.accp = plan_emit(ctx, true, false).gcp < ctx->tb.G8 ? reinterpret_cast<float2 *>(p) : nullptr;
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
    r.accp = sv.accp;
    r.TC = p.TC;
    r.g0 = 0;
    r.g1 = p.gcp;  // the first pass; launch_emit_batch adds the others
    r.gcp = p.gcp;
    r.unit_begin = 0;
    r.tpu = 1;
    r.smem = (uint32_t)p.smem;
    r.mode = ((L || resid) ? EMIT_ON : 0) | (resid ? EMIT_RESID : 0) | (L ? EMIT_STORE_L : 0) |
             ((mass && (L || resid)) ? EMIT_MASS : 0);
}

// Numbers the cells and emission tiles of a filled batch; launches the solve
// over every request, then the emission over the requests that want it.
int launch_emit_batch(EmitBatch &B, int num_sms, cudaStream_t st, cudaEvent_t between,
                      bool solved, int *nlaunch, int pass0) {
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
    // emission work lists: the requests that want L or resid, one entry per
    // grain pass, in pass order; one list per form of the grain numbers,
    // split at MAXREQ entries.  Tiles per work unit: about two units per SM
    // over the list, at least one tile.
    for (int form = 0; form < 2; ++form) {
        const bool mass = form == 1;
        EmitBatch E;
        E.nreq = 0;
        auto flush = [&]() -> int {
            if (E.nreq == 0) return DUST_OK;
            int64_t tiles = 0;
            size_t smem = 0;
            for (int k = 0; k < E.nreq; ++k) {
                tiles += (E.req[k].C + KE_TC - 1) / KE_TC;
                smem = std::max(smem, (size_t)E.req[k].smem);
            }
            const int64_t tpu = std::max<int64_t>(1, (tiles + 2 * num_sms - 1) / (2 * num_sms));
            int64_t units = 0;
            for (int k = 0; k < E.nreq; ++k) {
                E.req[k].unit_begin = units;
                E.req[k].tpu = tpu;
                units += ((E.req[k].C + KE_TC - 1) / KE_TC + tpu - 1) / tpu;
            }
            E.ntiles = tiles;
            const void *kern = mass ? reinterpret_cast<const void *>(k_emit<true>) : reinterpret_cast<const void *>(k_emit<false>);
            DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            if (mass) k_emit<true><<<(unsigned)units, KE_TH, smem, st>>>(E);
            else k_emit<false><<<(unsigned)units, KE_TH, smem, st>>>(E);
            DUST_CUDA_TRY(cudaGetLastError());
            ++nl;
            E.nreq = 0;
            return DUST_OK;
        };
        // pass pi of every request in one list; a pass reads the sums the
        // previous one wrote, so passes are separate launches
        for (int i = 0; i < B.nreq; ++i) {
            const EmitReq &r = B.req[i];
            if ((r.mode & EMIT_ON) && r.gcp < r.tb.G8 && !r.accp)
                return set_error(DUST_EINVAL, "request %d needs grain passes but has no buffer for their sums", i);
        }
        for (int pi = pass0;; ++pi) {
            bool any = false;
            for (int i = 0; i < B.nreq; ++i) {
                const EmitReq &r = B.req[i];
                if (!(r.mode & EMIT_ON) || ((r.mode & EMIT_MASS) != 0) != mass) continue;
                const int g0 = pi * r.gcp;
                if (g0 >= r.tb.G8) continue;
                any = true;
                if (E.nreq == MAXREQ) {
                    int rc = flush();
                    if (rc != DUST_OK) return rc;
                }
                EmitReq &e = E.req[E.nreq++];
                e = r;
                e.g0 = g0;
                e.g1 = std::min(r.tb.G8, g0 + r.gcp);
            }
            int rc = flush();
            if (rc != DUST_OK) return rc;
            if (!any) break;
        }
    }
    // residual fold over the requests that want it (after every pass)
    {
        EmitBatch R;
        R.nreq = 0;
        R.ncells = 0;
        R.ntiles = 0;
        for (int i = 0; i < B.nreq; ++i) {
            if (!(B.req[i].mode & EMIT_RESID)) continue;
            EmitReq &e = R.req[R.nreq++];
            e = B.req[i];
            e.cell_begin = R.ncells;
            R.ncells += e.C;
        }
        if (R.ncells > 0) {
            const int64_t rgrid = std::min<int64_t>((R.ncells + SOLVE_TH - 1) / SOLVE_TH, (int64_t)num_sms * 16);
            k_resid<<<(unsigned)rgrid, SOLVE_TH, 0, st>>>(R);
            DUST_CUDA_TRY(cudaGetLastError());
            ++nl;
        }
    }
    if (nlaunch) *nlaunch = nl;
    return DUST_OK;
}

// Tile, grains and shared memory of the warp-specialized solve + emission
// kernel for the context, or 0 where it does not apply (no emission).  All
// grains when their weights fit beside the pair tiles; else, where the
// two-kernel form takes the grains in passes, the first of those passes (its
// grain chunk, the same as k_emit's), the later passes then following in
// k_emit.  0 where neither fits.  (A cap at 160 KB, to leave L1 to the
// solve's table lookups, measured no faster: K = 350, G = 96 took 1.00 ms in
// the two-kernel form against 0.86 ms fused at 212 KB, 131072 cells.)
size_t plan_solve_emit(const dust_ctx *ctx, bool emit, bool mass, int *TC, int *gc) {
    if (!emit || (mass && !ctx->mass_ready)) return 0;
    const DevTables &tb = mass ? ctx->tbm : ctx->tb;
    const int tc = FSE_TC;
    auto bytes = [&](int g) {
        return (size_t)tb.NKG * (2 * g + 1) * 16 + (((size_t)FSE_NBUF * tc * (g + 1) * (mass ? 4 : 8) + 15) & ~(size_t)15) +
               (size_t)FSE_NBUF * tc * sizeof(CellInfo) + 2 * FSE_NBUF * sizeof(uint64_t) + 16;
    };
    const size_t budget = (ctx->smem_optin ? ctx->smem_optin : 99 * 1024) - 1024;
    int g = tb.G8;
    size_t smem = bytes(g);
    if (smem > budget) {
        g = plan_emit(ctx, true, mass).gcp;
        if (g >= tb.G8) return 0;
        smem = bytes(g);
        if (smem > budget) return 0;
    }
    *TC = tc;
    *gc = g;
    return smem;
}

// The fused kernel over one request (general form), then the residual fold.
template <bool MASS, bool PASS>
int launch_fse(const EmitReq &r, int nb, unsigned grid, size_t smem, cudaStream_t st) {
    const void *kern = nb == 1 ? reinterpret_cast<const void *>(k_solve_emit<1, MASS, PASS>)
                     : nb == 2 ? reinterpret_cast<const void *>(k_solve_emit<2, MASS, PASS>)
                     : nb == 3 ? reinterpret_cast<const void *>(k_solve_emit<3, MASS, PASS>)
                               : reinterpret_cast<const void *>(k_solve_emit<4, MASS, PASS>);
    DUST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    switch (nb) {
        case 1: k_solve_emit<1, MASS, PASS><<<grid, FSE_TH, smem, st>>>(r); break;
        case 2: k_solve_emit<2, MASS, PASS><<<grid, FSE_TH, smem, st>>>(r); break;
        case 3: k_solve_emit<3, MASS, PASS><<<grid, FSE_TH, smem, st>>>(r); break;
        default: k_solve_emit<4, MASS, PASS><<<grid, FSE_TH, smem, st>>>(r); break;
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
    const bool pass = r.g1 - r.g0 < r.tb.G8;  // the first of several grain passes
    int rc = mass ? (pass ? launch_fse<true, true>(r, nb, grid, smem, st) : launch_fse<true, false>(r, nb, grid, smem, st))
                  : (pass ? launch_fse<false, true>(r, nb, grid, smem, st) : launch_fse<false, false>(r, nb, grid, smem, st));
    if (rc != DUST_OK) return rc;
    if (nlaunch) *nlaunch = 1;  // the residual fold runs inside the kernel
    return DUST_OK;
}

int launch_solve_emit(const dust_ctx *ctx, int64_t C, const ScratchView &sv, const float *n, float *T, float *L,
                      int64_t ld, double *resid, uint8_t *flags, cudaStream_t st, int *nlaunch) {
    if (nlaunch) *nlaunch = 0;
    if (C <= 0) return DUST_OK;
    const EmitPlan p = plan_emit(ctx, L || resid, false);
    EmitBatch B;
    B.nreq = 1;
    fill_emit_req(ctx, p, C, sv, n, T, L, ld, resid, flags, B.req[0], false);
    return launch_emit_batch(B, ctx->num_sms, st, nullptr, false, nlaunch);
}

}  // namespace dust

// Device arithmetic shared by the two temperature-solve kernels (the
// stand-alone solve and the absorption GEMM whose epilogue solves): MUFU
// wrappers, float-float accumulation and the table root solve of Eq. 7.
// Both kernels take every result through these functions, so they agree
// bit for bit.
#pragma once

#include "dust_internal.cuh"

namespace dust {

// 1/T of padding grains and cells: every t = 2^(nax_k / T) of theirs is 0
constexpr float PAD_INV_T = 1e30f;

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

// (h, l) += (a, b) in float-float (two-sum of the high parts).
__device__ __forceinline__ void ff_add(float &h, float &l, float a, float b) {
    const float t = h + a, bp = t - h;
    l += ((h - (t - bp)) + (a - bp)) + b;
    h = t;
}

// Cubic Hermite on [0,1] with end values p0, p1 and end slopes d0, d1.
__device__ __forceinline__ float hermite(float p0, float d0, float p1, float d1, float x) {
    const float d = p1 - p0;
    const float c2 = 3.f * d - 2.f * d0 - d1;
    const float c3 = d0 + d1 - 2.f * d;
    return p0 + x * (d0 + x * (c2 + x * c3));
}

// Equilibrium temperatures of NB grains at once, branch-free: every lane runs
// the table lookup on y clamped into the table, and the clamp / invalid cases
// are selected at the end.  s: scaled absorbed power (A / P_g(T_min) = s 2^f_g).
template <int NB>
__device__ __forceinline__ void solve_batch(const DevTables &tb, const int (&g)[NB], const float (&s)[NB],
                                            const float4 (&gq)[NB], float (&T)[NB], int (&fl)[NB]) {
    float y[NB], ty[NB];
    int m[NB];
    float4 rv[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        // y = log2 s + f_g = Y0 + ly: the integer Y0 (s's exponent plus f_g,
        // exact) and ly = log2 of the mantissa in [1/2, 1), where lg2.approx
        // is good to ~2^-22 absolute
        const int bits = __float_as_int(s[i]);
        const bool pos = s[i] > 0.f;  // false for 0, negatives and NaN
        const float Y0 = pos ? (float)(((bits >> 23) & 0xff) - 126) + gq[i].x : 0.f;
        const float ly = pos ? lg2_approx(__int_as_float((bits & 0x007fffff) | 0x3f000000)) : 0.f;
        y[i] = pos ? Y0 + ly : -INFINITY;
        const bool bad = !(s[i] >= 0.f) || isinf(s[i]);
        fl[i] = bad ? DUST_FLAG_INVALID : (y[i] < 0.f ? DUST_FLAG_LOW : (y[i] > gq[i].y ? DUST_FLAG_HIGH : DUST_FLAG_OK));
        // interval coordinate y invdy (node m at m): the product of the
        // integer part is split exactly (ah + al) and the interval offset
        // formed from the parts, so that it keeps ~2^-24 of an interval
        // instead of ~2^-24 of y invdy (a few thousand)
        const float ah = Y0 * gq[i].z, al = fmaf(Y0, gq[i].z, -ah), b = ly * gq[i].z;
        m[i] = min(max((int)floorf(ah + b), 0), tb.NI - 2);
        ty[i] = fminf(fmaxf(((ah - (float)m[i]) + b) + al, 0.f), 1.f);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) rv[i] = __ldg(tb.ivr + (size_t)g[i] * (tb.NI - 1) + m[i]);
    // 2^x = sum_n (x ln 2)^n / n!, five terms: |x| <= 1/8 leaves < 6e-10 (tables
    // with a wider interval take ex2)
    const float L1 = 0.69314718056f, L2 = 0.24022650695f, L3 = 0.05550410866f, L4 = 0.00961812911f,
                L5 = 0.00133335581f;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        // Newton on the interval's forward cubic, in units of the interval:
        // p(tau) = tau + tau (d0 + tau (c2 + tau c3)) = ty, p(0) = 0, p(1) = 1,
        // p'(0) = 1 + d0, p'(1) = 1 + d1, from tau = ty (the straight line
        // through the ends).  The bracket [0, 1] holds the root; a step that
        // leaves the current bracket bisects instead, and only then is a
        // second taken.  The first residual, p(ty) - ty, is the small cubic
        // term alone, so it carries no cancellation.
        const float d0 = rv[i].z, d1 = rv[i].w;
        const float c2 = -2.f * d0 - d1, c3 = d0 + d1;
        float lo = 0.f, hi = 1.f, t = ty[i];
        for (int it = 0; it < 2; ++it) {
            const float q = (t - ty[i]) + t * (d0 + t * (c2 + t * c3));
            const float dq = 1.f + d0 + t * (2.f * c2 + 3.f * t * c3);
            lo = q < 0.f ? t : lo;
            hi = q < 0.f ? hi : t;
            const float nt = t - q * rcp_approx(dq);
            const bool inside = nt >= lo && nt <= hi;
            t = inside ? nt : 0.5f * (lo + hi);
            if (inside) break;
        }
        // T = 2^u_m 2^(tau du)
        const float x = t * rv[i].y;
        const float Tv = rv[i].x * (tb.wide ? ex2_approx(x)
                                            : fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, L5, L4), L3), L2), L1), 1.f));
        T[i] = fl[i] == DUST_FLAG_OK ? Tv
             : fl[i] == DUST_FLAG_LOW ? tb.Tmin
             : fl[i] == DUST_FLAG_HIGH ? tb.Tmax : __int_as_float(0x7fc00000);
    }
}

// Emission pair and absorbed-power term of one solved grain g < G: the
// pair (1/T, n 2^-m_c) the emission reads, and (rs) the grain's share of the
// cell's absorbed power sum_g n Pe 2^-Eg added to the float-float (ah, al);
// Pe is the absorbed power of a solved grain and P_g at the clamp otherwise.
__device__ __forceinline__ void grain_out(const DevTables &tb, int g, float T, int fl, float s, float nv, int mc,
                                          bool mass, bool rs, float &invT, float &nn, float &ah, float &al) {
    invT = rcp_approx(T);
    nn = mass ? __ldg(tb.ng + g) : scale2(nv, -mc);
    if (rs) {
        const float4 gr = __ldg(tb.gres + g);
        const float se = fl == DUST_FLAG_OK ? s
                       : fl == DUST_FLAG_LOW ? gr.z
                       : fl == DUST_FLAG_HIGH ? gr.w : __int_as_float(0x7fc00000);
        const float xh = nn * se, xl = fmaf(nn, se, -xh);
        const float rh = xh * gr.x;
        ff_add(ah, al, rh, fmaf(xh, gr.x, -rh) + fmaf(xh, gr.y, xl * gr.x));
    }
}

}  // namespace dust

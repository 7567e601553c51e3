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
    float4 iv[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        // log2 s = e + log2 m with the exponent split off exactly and m in
        // [1/2, 1), where lg2.approx is good to ~2^-22 absolute; the
        // temperature error this causes is below 1e-7
        const int bits = __float_as_int(s[i]);
        const float mant = __int_as_float((bits & 0x007fffff) | 0x3f000000);
        y[i] = (s[i] > 0.f) ? (float)(((bits >> 23) & 0xff) - 126) + lg2_approx(mant) + gq[i].x : -INFINITY;
        const bool bad = !(s[i] >= 0.f) || isinf(s[i]);
        fl[i] = bad ? DUST_FLAG_INVALID : (y[i] < 0.f ? DUST_FLAG_LOW : (y[i] > gq[i].y ? DUST_FLAG_HIGH : DUST_FLAG_OK));
        const float yc = fminf(fmaxf(y[i], 0.f), gq[i].y);  // NaN -> 0
        y[i] = yc;
        const float fy = yc * gq[i].z;
        m[i] = min((int)fy, tb.NI - 2);
        ty[i] = fminf(fy - (float)m[i], 1.f);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) iv[i] = __ldg(tb.inv + (size_t)g[i] * (tb.NI - 1) + m[i]);
    int j[NB];
    float tau[NB], tn[NB];
    float4 f4[NB];
    const float inv_h2 = 1.f / tb.h2;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const float ug = hermite(iv[i].x, iv[i].y, iv[i].z, iv[i].w, ty[i]);
        const float fj = (ug - tb.log2Tmin) * inv_h2;
        j[i] = min(max((int)floorf(fj), 0), tb.NT - 2);
        tau[i] = fminf(fmaxf(fj - (float)j[i], 0.f), 1.f);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        f4[i] = __ldg(tb.fw + (size_t)g[i] * (tb.NT - 1) + j[i]);
        tn[i] = __ldg(tb.Tnode + j[i]);
    }
    const float L1 = 0.69314718056f, L2 = 0.24022650695f, L3 = 0.05550410866f;  // (ln 2)^k / k!
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        // bracketing interval t_j <= y <= t_j+1 (the guess is right unless y
        // sits within rounding of a node)
        for (int a = 0; a < 4; ++a) {
            if (y[i] < f4[i].x && j[i] > 0) { --j[i]; tau[i] = 1.f; }
            else if (y[i] > f4[i].z && j[i] < tb.NT - 2) { ++j[i]; tau[i] = 0.f; }
            else break;
            f4[i] = __ldg(tb.fw + (size_t)g[i] * (tb.NT - 1) + j[i]);
            tn[i] = __ldg(tb.Tnode + j[i]);
        }
        // Newton on the Hermite cubic q(tau) = t(u_j + tau h2) - t_j = y - t_j from
        // the inverse-table guess.  The guess is a cubic Hermite interpolant of the
        // exact inverse, so one step lands within FP32 rounding of the root; a step
        // that leaves the bracket bisects instead, and only then is a second taken
        const float r = y[i] - f4[i].x, d = f4[i].z - f4[i].x, m0 = f4[i].y, m1 = f4[i].w;
        const float c2 = 3.f * d - 2.f * m0 - m1, c3 = m0 + m1 - 2.f * d;
        float lo = 0.f, hi = 1.f, t = tau[i];
        for (int it = 0; it < 2; ++it) {
            const float q = t * (m0 + t * (c2 + t * c3)) - r;
            const float dq = m0 + t * (2.f * c2 + 3.f * t * c3);
            lo = q < 0.f ? t : lo;
            hi = q < 0.f ? hi : t;
            const float nt = t - q * rcp_approx(dq);
            const bool inside = nt >= lo && nt <= hi;
            t = inside ? nt : 0.5f * (lo + hi);
            if (inside) break;
        }
        // T = T_j 2^(tau h2), 2^x by its Taylor series (|x| <= h2, error < 1e-12)
        const float x = t * tb.h2;
        const float Tv = tn[i] * fmaf(x, fmaf(x, fmaf(x, L3, L2), L1), 1.f);
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

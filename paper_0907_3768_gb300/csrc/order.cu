// Cell ordering for the emission: a counting sort of each request's cells by
// a temperature class.
//
// The emission (Eq. 10) splits each group of 8 grains x 8 wavelengths of a
// cell by the largest exponent a = nax_k / T in it: groups whose every term
// underflows are skipped, Wien groups (t <= 2^-24) take a short form, the
// rest the full rational form.  A warp runs 32 cells of one wavelength group
// side by side, so it takes a branch when any of its lanes needs it; cells of
// unlike temperatures in one warp would run both forms.  Ordering the cells
// by the absorbed power (or the inverse temperature) of one reference grain
// puts cells of like temperatures in the same warps: every grain's
// temperature rises with the field strength of its cell, so one grain ranks
// the cells for all of them.  Only the pace depends on the order; every
// cell's arithmetic is its own, so no result does.
//
// Classes: bits 21..30 of the positive float key, i.e. its exponent and two
// mantissa bits (quarter-octave classes); keys <= 0 or NaN fall in class 0.
// The sort is a histogram (shared-memory counts per CTA, added to the
// request's global counts), then a scatter in which every CTA reserves its
// range of each class with one global atomic and places its cells with
// shared-memory atomics.  The order of cells inside a class is not fixed.
#include "dust_internal.cuh"

#include <algorithm>

namespace dust {
namespace {

constexpr int ORD_TH = 256;            // threads per CTA
constexpr int ORD_CPB = ORD_TH * 8;    // cells per CTA

__device__ __forceinline__ int key_class(float v) {
    return v > 0.f ? min(__float_as_int(v) >> 21, NBK - 1) : 0;
}

__device__ __forceinline__ int req_of_block(const OrderBatch &B, int blk) {
    int r = 0;
    while (r + 1 < B.nreq && blk >= B.req[r + 1].block_begin) ++r;
    return r;
}

__global__ void __launch_bounds__(ORD_TH) k_order_zero(const __grid_constant__ OrderBatch B) {
    unsigned *h = B.req[blockIdx.x].hist;
    for (int i = threadIdx.x; i < 2 * NBK; i += ORD_TH) h[i] = 0u;
}

// Each CTA: the classes of its ORD_CPB cells, counted in shared memory and
// added to the request's counts.
__global__ void __launch_bounds__(ORD_TH) k_order_classify(const __grid_constant__ OrderBatch B) {
    __shared__ unsigned cnt[NBK];
    const OrderReq &q = B.req[req_of_block(B, blockIdx.x)];
    const int64_t c0 = (int64_t)(blockIdx.x - q.block_begin) * ORD_CPB;
    const int64_t c1 = min(c0 + ORD_CPB, q.C);
    for (int i = threadIdx.x; i < NBK; i += ORD_TH) cnt[i] = 0u;
    __syncthreads();
    for (int64_t c = c0 + threadIdx.x; c < c1; c += ORD_TH) {
        const int b = key_class(__ldg(q.key + c * q.kstride));
        q.bkt[c] = (uint16_t)b;
        atomicAdd(&cnt[b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NBK; i += ORD_TH)
        if (cnt[i]) atomicAdd(q.hist + i, cnt[i]);
}

// Each CTA: the exclusive prefix of the request's class counts, a range of
// each class reserved for its own cells (cursor = hist + NBK), and its cells
// placed in that range.
__global__ void __launch_bounds__(ORD_TH) k_order_scatter(const __grid_constant__ OrderBatch B) {
    __shared__ unsigned base[NBK], cnt[NBK];
    __shared__ unsigned wsum[ORD_TH / 32];
    const OrderReq &q = B.req[req_of_block(B, blockIdx.x)];
    const int64_t c0 = (int64_t)(blockIdx.x - q.block_begin) * ORD_CPB;
    const int64_t c1 = min(c0 + ORD_CPB, q.C);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // exclusive scan of the NBK counts: four consecutive classes per thread
    constexpr int PER = NBK / ORD_TH;
    unsigned v[PER], s = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) { v[j] = q.hist[tid * PER + j]; s += v[j]; }
    unsigned inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    for (int i = tid; i < NBK; i += ORD_TH) cnt[i] = 0u;
    __syncthreads();
    unsigned off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    unsigned run = off + inc - s;
#pragma unroll
    for (int j = 0; j < PER; ++j) { base[tid * PER + j] = run; run += v[j]; }
    // this CTA's count per class
    for (int64_t c = c0 + tid; c < c1; c += ORD_TH) atomicAdd(&cnt[q.bkt[c]], 1u);
    __syncthreads();
    // reserve: base becomes this CTA's first slot of each class
    for (int i = tid; i < NBK; i += ORD_TH) {
        if (cnt[i]) base[i] += atomicAdd(q.hist + NBK + i, cnt[i]);
        cnt[i] = 0u;
    }
    __syncthreads();
    for (int64_t c = c0 + tid; c < c1; c += ORD_TH) {
        const int b = q.bkt[c];
        q.order[base[b] + atomicAdd(&cnt[b], 1u)] = (int)c;
    }
}

}  // namespace

int launch_order(OrderBatch &B, cudaStream_t st, int *nlaunch) {
    if (nlaunch) *nlaunch = 0;
    int blocks = 0;
    for (int i = 0; i < B.nreq; ++i) {
        B.req[i].block_begin = blocks;
        blocks += (int)((B.req[i].C + ORD_CPB - 1) / ORD_CPB);
    }
    B.nblocks = blocks;
    if (blocks == 0) return DUST_OK;
    k_order_zero<<<B.nreq, ORD_TH, 0, st>>>(B);
    DUST_CUDA_TRY(cudaGetLastError());
    k_order_classify<<<blocks, ORD_TH, 0, st>>>(B);
    DUST_CUDA_TRY(cudaGetLastError());
    k_order_scatter<<<blocks, ORD_TH, 0, st>>>(B);
    DUST_CUDA_TRY(cudaGetLastError());
    if (nlaunch) *nlaunch = 3;
    return DUST_OK;
}

}  // namespace dust

// Internal declarations shared by libdust's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cstdio>
#include <cstdarg>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/dust.h"

namespace dust {

// Wavelengths handled by one thread in the emission phase (Eq. 10's sum over
// grains is accumulated for KQ consecutive wavelengths per thread).
constexpr int KQ = 8;
// Grains folded into one rational accumulator N/D before its single division.
constexpr int RG = 8;
// Column padding of the scratch matrix of scaled absorbed powers.
constexpr int GPAD = 16;
// K-chunk (FP32 columns) of the tensor-core absorption kernel.
constexpr int KC = 32;
// Buckets of the cell ordering (order.cu): the exponent and two mantissa bits
// of a positive float key, i.e. quarter-octave classes of absorbed power.
constexpr int NBK = 1024;

// Per-grain constants of the temperature solve (float4-packed for one load).
struct GrainParam {
    float f;      // exponent f_g: A / P_g(T_min) = S * 2^f_g
    float tmax;   // t_max = log2(P_g(T_max) / P_g(T_min))
    float invdy;  // (NI - 1) / tmax: inverse-table bins per unit of log2 P
    float pad;
};

// Everything the device kernels read from a context, passed by value.
struct DevTables {
    int K, G, Kp, NKG;        // Kp = NKG * KQ >= K (emission padding)
    int G8;                   // G rounded up to RG (emission padding, zero weights)
    int Gs;                   // row stride of the absorbed-power scratch (G rounded to GPAD)
    int NT, NI;               // forward / inverse table sizes
    float log2Tmin, h2;       // u_j = log2Tmin + j h2 (u = log2 T)
    float Tmin, Tmax;
    const float4 *fw;         // [G][NT-1] (t_j, s_j h2, t_j+1, s_j+1 h2), t = log2(P/P0)
    const float4 *ivr;        // [G][NI-1] Newton records of the inverse-table intervals
                              //     (2^u_m, du = u_m+1 - u_m, d0, d1), see context.cu
    int wide;                 // some du > 1/8: 2^(tau du) by ex2 instead of its series
    const GrainParam *gp;     // [G]
    const double *gscale;     // [G] A = S * gscale (= P0 2^f)
    const double *P0;         // [G] P_g(T_min)
    const double *Pmax;       // [G] P_g(T_max)
    const float4 *gres;       // [G] residual constants: gscale 2^-Eg as float-float (x, y),
                              //     S of a grain clamped low (z = 2^-f) and high (w = Pmax / gscale)
    int Eg;
    const float *nax;         // [Kp] -log2(e) h c / (lambda_k k_B), -1e30 in the padding
    const float *Chat;        // [NKG][G8][2][4] scaled emission weights (see context.cu)
    const int *qexp;          // [Kp] per-wavelength exponent of Chat
    const double *w;          // [K] quadrature weights
    const float *wq;          // [K] w_k 2^(q_k - Ew) (residual of the scaled emission sums)
    int Ew;
    float rc_hi, rc_lo;       // 2^(Ew - Eg) / (4 pi) = (rc_hi + rc_lo) 2^rc_exp, rc_hi in [1/2, 1)
    int rc_exp;
    const float *ng;          // dust-mass form only: [G8] grains per unit mass n_g 2^-En (0 padding)
    int *status;              // device status word (dust_status)
};

// ---- work lists of the batched kernels (passed by value as kernel parameters)
constexpr int MAXREQ = 32;

// EMIT_MASS: n[c,g] = m_c n_g (the paper's n_s m_d;c, Eqs. 9-10); req.n holds m [C]
// and req.tb the dust-mass tables, whose emission weights carry n_g.
enum EmitMode { EMIT_ON = 1, EMIT_RESID = 2, EMIT_STORE_L = 4, EMIT_MASS = 8 };

// Per-cell record passed from the solve to the emission: exponent m_c of
// max_g n[c,g] and the absorbed power sum_g n Pe = (ah + al) 2^(m_c + Eg)
// as a float-float pair (the residual's denominator / 4 pi).  In the
// dust-mass form m_c is the exponent of the cell's mass m = ms 2^m_c (ms in
// [1/2, 1), stored as bits) and the absorbed power is taken per unit mass.
struct CellInfo {
    int mc;
    float ah, al;
    int ms_bits;
};

// A request's scratch: S [C][Gs] FP32, then (emission only) the pairs
// (1/T, n 2^-m_c) [C][G8], one CellInfo per cell and the residual partials
// [C][NKG] float2, each 16-byte aligned.
struct ScratchView {
    float *S;
    float2 *prep;
    CellInfo *cell;
    float2 *part;  // [C][NKG] float-float partial sums of w_k L_k (residual)
    int *order;    // [C] the cells in emission order (temperature classes)
    uint16_t *bkt; // [C] each cell's class
    unsigned *hist;  // [2][NBK] cells per class, then the scatter cursors
    float2 *accp;  // [C][NKG][4] emission sums carried between grain passes (NULL: one pass)
};

// One request of the solve / emission kernels.
struct EmitReq {
    DevTables tb;
    int64_t C, ld, tile_begin, cell_begin;
    const float *S, *n;
    float *T, *L;
    double *resid;
    uint8_t *flags;
    float2 *prep;
    CellInfo *cell;
    float2 *part;
    const int *order;  // emission order of the request's cells (NULL: ascending)
    float2 *accp;      // sums carried between grain passes, [C][NKG][4] float2
    int TC, mode;
    int g0, g1;     // grains [g0, g1) this entry emits: a pass, when the weights of every
                    // k-group for all grains exceed shared memory (multiples of RG)
    int gcp;        // grains per pass of the request's plan
    int64_t unit_begin, tpu;  // two-kernel emission: first work unit, tiles per unit
    uint32_t smem;  // its emission kernel's shared memory
};

struct EmitBatch {
    int nreq;
    int64_t ntiles, ncells;
    EmitReq req[MAXREQ];
};
// The two-kernel emission: tiles of its work units (one CTA each).
constexpr int KE_TC = 32;

// One request of the cell ordering: a positive float key per cell at
// key[c * kstride] (an absorbed power or an inverse temperature of one
// reference grain) sorted into NBK classes, then scattered into `order`.
struct OrderReq {
    const float *key;
    int64_t kstride, C;
    uint16_t *bkt;
    unsigned *hist;  // [2][NBK], zeroed by the launch
    int *order;
    int block_begin;  // first CTA of the request in the classify / scatter grids
};

struct OrderBatch {
    int nreq;
    int nblocks;
    OrderReq req[MAXREQ];
};

// Solve requests of a fused absorption + solve launch (index i belongs to
// TcBatch::req[i]).
struct SolveList {
    EmitReq req[MAXREQ];
};

// Emission geometry of a request in the two-kernel form: its grains are
// emitted in passes of gcp (all of them when the weights of every k-group
// for all grains fit in shared memory beside the pair tiles), smem bytes per
// CTA.
struct EmitPlan {
    int TC, gcp;
    size_t smem;
};

// One request of the tensor-core absorption kernel (its TMA descriptor for J
// sits in TcBatch::tm at the same index).
struct TcReq {
    int64_t C, tile_begin;
    int Gs, nkc;
    int nparts;  // split products per K step: 3 (hi.hi + lo.hi + hi.lo), or 2 without hi.lo (an ablation)
    const uint16_t *Wimg;
    float *S;
};

struct TcBatch {
    CUtensorMap tm[MAXREQ];
    TcReq req[MAXREQ];
    int nreq;
    int64_t ntiles;
    int GsMax, ns1, ns2, tmem_cols, nacc, off_exp, j_off;
    int orient;  // 0: cells are the MMA's M (128-cell tiles); 1: cells are its N (256-cell tiles, Gs <= 128)
    int *status;
};

// One request of the FP32 SIMT absorption kernel.
struct SimtReq {
    int64_t C, ld, tile_begin;
    const float *J, *W;
    float *S;
    int K, Kw, Gs, ntn;  // ntn = grain tiles per cell tile
};

struct SimtBatch {
    SimtReq req[MAXREQ];
    int nreq;
    int64_t ntiles;
};

}  // namespace dust

// The opaque context of the C ABI.
struct dust_ctx {
    int device = 0;
    int precision = DUST_PREC_FP32;
    // tensor-core precisions: absorption and temperature solve as one kernel
    // (dust_ctx_set_fused)
    bool fused = false;
    // solve and emission as one warp-specialized kernel where it applies
    // (dust_ctx_set_fused_emit)
    bool fused_emit = true;
    // split products of the tensor-core precisions (dust_ctx_set_split_products)
    int split_products = 3;
    // kernels launched by this context's solves (dust_ctx_launch_count)
    uint64_t launches = 0;
    int K = 0, G = 0, NT = 0, NI = 0;
    int Kw = 0;               // row length of the FP32 / 16-bit W copies (K rounded to KC)
    double Tmin = 0, Tmax = 0;
    dust::DevTables tb{};
    // device allocations owned by the context
    float *W32 = nullptr;     // [Gs][Kw] FP32 scaled W (SIMT path)
    uint16_t *Wimg[2] = {nullptr, nullptr};  // BF16 / FP16 hi+lo images (tensor-core path)
    size_t Wimg_bytes = 0;
    void *tables_mem = nullptr;  // one block holding every table
    size_t tables_bytes = 0;
    // per-grain constants of the paper's Newton kernel (float2 [G]; NULL until
    // dust_ctx_set_grain_sizes)
    void *newton_grain = nullptr;
    // dust-mass form (dust_ctx_set_grain_numbers): its tables and one block of
    // device memory holding its emission weights, exponents and n_g
    bool mass_ready = false;
    dust::DevTables tbm{};
    void *mass_mem = nullptr;
    size_t mass_bytes = 0;
    std::vector<double> lam_h, w_h, C_h;  // host copies of the context's inputs
    // thermally fluctuating grains (dust_ctx_set_fluctuating): one device block
    // with the photon energies, heating weights and grain constants
    void *fl_mem = nullptr;
    size_t fl_off[3] = {0, 0, 0};
    int fl_Gf = 0, fl_M = 0;
    float fl_eps_ref = 0.f;
    // working J, previous L and a change word of dust_solve_coupled
    void *cpl = nullptr;
    size_t cpl_bytes = 0;
    // scratch of scaled absorbed powers S[C][Gs]
    float *S = nullptr;
    size_t S_cap = 0;         // in cells
    // host-staging for dust_solve_host
    // a three-stage pipeline (copy in, compute, copy out) over NHB buffer sets
    static constexpr int NHB = 3;
    struct HostStage {
        cudaStream_t st[3] = {nullptr, nullptr, nullptr};  // copy in, compute, copy out
        cudaEvent_t ev_in[NHB] = {}, ev_c[NHB] = {}, ev_out[NHB] = {};
        float *J[NHB] = {}, *n[NHB] = {};
        float *T[NHB] = {}, *L[NHB] = {};
        double *r[NHB] = {};
        uint8_t *f[NHB] = {};
        void *S = nullptr;  // one scratch: the compute stream runs one chunk at a time
        int64_t cap = 0, ld = 0;
        size_t bytes = 0;
    } hs;
    int num_sms = 0;
    size_t smem_optin = 0;
    std::mutex mu;
    // per-kernel event timing (dust_ctx_profile): three events per solve
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_pool;   // reusable events
    std::vector<cudaEvent_t> prof_marks;  // recorded, not yet read (triples)
};

namespace dust {

// Thread-local error reporting.
int set_error(int code, const char *fmt, ...);
const char *cuda_err_name(cudaError_t e);

#define DUST_CUDA_TRY(expr)                                                          \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) {                                                     \
            cudaGetLastError(); /* clear it, so that it is not reported again */      \
            return ::dust::set_error(_e == cudaErrorMemoryAllocation ? DUST_ENOMEM     \
                                                                    : DUST_ECUDA,    \
                                     "%s failed: %s (%s:%d)", #expr,                 \
                                     cudaGetErrorString(_e), __FILE__, __LINE__);    \
        }                                                                            \
    } while (0)

// Kernels' entry points (host launchers), each returning a dust_status.
int launch_gemm_simt(const dust_ctx *ctx, int64_t C, const float *J, int64_t ld, float *S,
                     cudaStream_t st);
int launch_gemm_tc(const dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld,
                   float *S, cudaStream_t st);
int launch_solve_emit(const dust_ctx *ctx, int64_t C, const ScratchView &sv, const float *n, float *T,
                      float *L, int64_t ld, double *resid, uint8_t *flags, cudaStream_t st, int *nlaunch = nullptr);
EmitPlan plan_emit(const dust_ctx *ctx, bool emit, bool mass);
// Scratch bytes of a request of C cells and its layout at `base`.
size_t scratch_bytes(const dust_ctx *ctx, int64_t C, bool emit);
ScratchView scratch_view(const dust_ctx *ctx, int64_t C, void *base);
// Tensor-core batches: one request entry (encodes its TMA descriptor), the
// ring geometry of a batch, and the launch.  All requests of one launch share
// the precision.
int make_tc_req(const dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, float *S,
                TcReq &r, CUtensorMap &tm, int orient = 0);
// Orientation of the tensor-core GEMM for a context: grain-major (1) when its
// grains fit one 128-row MMA operand, cell-major (0) otherwise.
int tc_orient(const dust_ctx *ctx);
// fused: the batch feeds the kernel whose epilogue is the temperature solve
// (up to four accumulators, each with its own group of solver warps), whose
// requests `sl` holds.
int finish_tc_batch(TcBatch &B, int precision, size_t smem_optin, size_t *smem, bool fused = false);
int launch_tc_batch(const TcBatch &B, int precision, size_t smem, int num_sms, cudaStream_t st,
                    const SolveList *sl = nullptr);
// FP32 SIMT batches.
void make_simt_req(const dust_ctx *ctx, int64_t C, const float *J, int64_t ld, float *S, SimtReq &r);
int launch_simt_batch(SimtBatch &B, cudaStream_t st);
void fill_emit_req(const dust_ctx *ctx, const EmitPlan &p, int64_t C, const ScratchView &sv, const float *n,
                   float *T, float *L, int64_t ld, double *resid, uint8_t *flags, EmitReq &r, bool mass);
// Numbers cells and tiles, then launches the solve over every request and the
// emission over those that want L or resid; `between` (optional) is recorded
// on `st` between the two kernels.
// With solved = true the temperatures, pairs and cell records are already
// there (fused absorption + solve) and only the emission runs; with pass0 > 0
// the grain passes before pass0 are done too (their sums carried in accp).
int launch_emit_batch(EmitBatch &B, int num_sms, cudaStream_t st, cudaEvent_t between = nullptr,
                      bool solved = false, int *nlaunch = nullptr, int pass0 = 0);

// Orders the cells of every request of the batch by the class of its key
// (three launches: zero the counts, classify, scatter).  Cells of one class
// run together in the emission, so that the 32 lanes of a warp take the same
// regime branches; the order never changes a result.
int launch_order(OrderBatch &B, cudaStream_t st, int *nlaunch);
// Key of the ordering: the reference grain of a context.
inline int order_ref_grain(int G) { return G / 2; }

// Warp-specialized solve + emission over one request: the plan (its tile of
// TC cells, the grains [0, gc) it emits, and shared memory; 0 where it does
// not apply) and the launch (for req.g1 = gc < G8 the first grain pass only).
size_t plan_solve_emit(const dust_ctx *ctx, bool emit, bool mass, int *TC, int *gc);
int launch_solve_emit_fused(const EmitReq &req, int TC, size_t smem, int num_sms, cudaStream_t st,
                            int *nlaunch = nullptr);

// Grow the context's scratch to hold `cells` cells (synchronises `st` first).
int ensure_scratch(dust_ctx *ctx, int64_t cells, cudaStream_t st);

// The whole path on device buffers over an explicit scratch view (a
// request's, or a slice of one: order, classes and counts may be NULL, and
// the cells are then emitted in ascending order); nlaunch counts the kernels,
// ev (optional, four events) marks absorption / solve / emission boundaries.
int solve_view(dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, const float *n, float *T,
               float *L, double *resid, uint8_t *flags, const ScratchView &sv, cudaStream_t st, bool mass,
               int *nlaunch, cudaEvent_t *ev = nullptr);
// The whole path on device buffers with scratch of scratch_bytes(ctx, C, true)
// bytes at `scratch`.
int solve_device(dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld,
                 const float *n, float *T, float *L, double *resid, uint8_t *flags, void *scratch,
                 cudaStream_t st, bool mass = false);

// Bounded spin budget for device-side waits: a wait that exceeds it records
// DUST_ETIMEOUT in the status word and gives up.
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void record_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// x * 2^e for |e| <= 252 without leaving the exact power-of-two scaling
// (two steps so that each factor is a normal float).
__device__ __forceinline__ float scale2(float x, int e) {
    int e1 = e / 2, e2 = e - e1;
    return x * __int_as_float((e1 + 127) << 23) * __int_as_float((e2 + 127) << 23);
}

}  // namespace dust

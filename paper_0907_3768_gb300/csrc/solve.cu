// dust_solve and friends: argument checks, scratch management and the launch
// sequence of the hot path (absorption contraction -> fused solve/emission).
#include "dust_internal.cuh"

#include <algorithm>

namespace dust {
namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    int rc = DUST_OK;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { rc = set_error(DUST_ECUDA, "cudaGetDevice failed"); return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
            rc = set_error(DUST_ECUDA, "cudaSetDevice(%d) failed", dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int check_device_ptr(const void *p, int device, const char *name) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(DUST_EINVAL, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error(DUST_EINVAL, "%s must be device memory", name);
    if (a.type == cudaMemoryTypeDevice && a.device != device)
        return set_error(DUST_EINVAL, "%s lives on device %d, the context on device %d", name, a.device,
                         device);
    return DUST_OK;
}

int validate(const dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, const float *n,
             float *T, float *L, double *resid, uint8_t *flags, bool device_ptrs) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (C < 0) return set_error(DUST_EINVAL, "n_cells < 0");
    if (precision < DUST_PREC_FP32 || precision > DUST_PREC_FP16X3)
        return set_error(DUST_EINVAL, "unknown precision %d", precision);
    if (ld < ctx->K) return set_error(DUST_EINVAL, "ld=%lld < K=%d", (long long)ld, ctx->K);
    if (C == 0) return DUST_OK;
    if (!J || !n || !T) return set_error(DUST_EINVAL, "J, n and T must be non-NULL");
    if (precision != DUST_PREC_FP32) {
        if (ld % 4 != 0 || ((uintptr_t)J & 15) != 0)
            return set_error(DUST_EINVAL,
                             "tensor-core precisions need ld %% 4 == 0 and a 16-byte aligned J "
                             "(ld=%lld)", (long long)ld);
    }
    if (device_ptrs) {
        int rc;
        if ((rc = check_device_ptr(J, ctx->device, "J")) != DUST_OK) return rc;
        if ((rc = check_device_ptr(n, ctx->device, "n")) != DUST_OK) return rc;
        if ((rc = check_device_ptr(T, ctx->device, "T")) != DUST_OK) return rc;
        if (L && (rc = check_device_ptr(L, ctx->device, "L")) != DUST_OK) return rc;
        if (resid && (rc = check_device_ptr(resid, ctx->device, "resid")) != DUST_OK) return rc;
        if (flags && (rc = check_device_ptr(flags, ctx->device, "flags")) != DUST_OK) return rc;
    }
    return DUST_OK;
}

}  // namespace

int ensure_scratch(dust_ctx *ctx, int64_t cells, cudaStream_t st) {
    if ((size_t)cells <= ctx->S_cap) return DUST_OK;
    DUST_CUDA_TRY(cudaStreamSynchronize(st));
    if (ctx->S) { cudaFree(ctx->S); ctx->S = nullptr; ctx->S_cap = 0; }
    DUST_CUDA_TRY(cudaMalloc(&ctx->S, scratch_bytes(ctx, cells, true)));
    ctx->S_cap = (size_t)cells;
    return DUST_OK;
}

namespace {
cudaEvent_t prof_event(dust_ctx *ctx) {
    cudaEvent_t e = nullptr;
    if (!ctx->prof_pool.empty()) {
        e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    return e;
}
}  // namespace

int solve_view(dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, const float *n, float *T,
               float *L, double *resid, uint8_t *flags, const ScratchView &sv, cudaStream_t st, bool mass,
               int *nlaunch, cudaEvent_t *ev) {
    int nl_total = 0;
    if (nlaunch) *nlaunch = 0;
    if (C == 0) return DUST_OK;
    if (ev && ev[0]) DUST_CUDA_TRY(cudaEventRecord(ev[0], st));
    const EmitPlan p = plan_emit(ctx, L || resid, mass);
    EmitBatch B;
    B.nreq = 1;
    fill_emit_req(ctx, p, C, sv, n, T, L, ld, resid, flags, B.req[0], mass);
    const bool fused = ctx->fused && precision != DUST_PREC_FP32;
    int rc = DUST_OK;
    if (fused) {
        // one kernel through the temperatures: S stays in tensor memory
        TcBatch tb;
        tb.nreq = 1;
        tb.status = ctx->tb.status;
        tb.orient = 0;
        SolveList sl;
        sl.req[0] = B.req[0];
        size_t smem = 0;
        rc = make_tc_req(ctx, precision, C, J, ld, sv.S, tb.req[0], tb.tm[0]);
        if (rc == DUST_OK) rc = finish_tc_batch(tb, precision, ctx->smem_optin, &smem, true);
        if (rc == DUST_OK) rc = launch_tc_batch(tb, precision, smem, ctx->num_sms, st, &sl);
    } else {
        rc = precision == DUST_PREC_FP32 ? launch_gemm_simt(ctx, C, J, ld, sv.S, st)
                                         : launch_gemm_tc(ctx, precision, C, J, ld, sv.S, st);
    }
    if (rc == DUST_OK) nl_total += 1;
    int ftc = 0, fgc = 0;
    const size_t fsmem = !fused && ctx->fused_emit ? plan_solve_emit(ctx, L || resid, mass, &ftc, &fgc) : 0;
    if (fsmem && fgc != p.gcp) return set_error(DUST_EINVAL, "internal: grain passes of the two emission forms differ");
    // The emission order groups cells of like temperatures into the emission's
    // 32-cell tiles; it never changes a result.  A call of at most one tile per
    // SM skips it: there the ordering's three launches cost more than the
    // warp-uniform regimes save.
    const bool ordered = C > (int64_t)32 * ctx->num_sms;
    if (rc == DUST_OK && (L || resid) && ordered && sv.order && sv.bkt && sv.hist) {
        // emission order: cells classed by the absorbed power of the reference
        // grain (S), or by its inverse temperature where S stayed in tensor memory
        const int gref = order_ref_grain(ctx->G);
        OrderBatch ob;
        ob.nreq = 1;
        OrderReq &o = ob.req[0];
        if (fused) {
            const int pw = mass ? 1 : 2;
            o.key = reinterpret_cast<const float *>(sv.prep) + pw * gref;
            o.kstride = (int64_t)pw * ctx->tb.G8;
        } else {
            o.key = sv.S + gref;
            o.kstride = ctx->tb.Gs;
        }
        o.C = C;
        o.bkt = sv.bkt;
        o.hist = sv.hist;
        o.order = sv.order;
        int nl = 0;
        rc = launch_order(ob, st, &nl);
        nl_total += nl;
        B.req[0].order = sv.order;
    }
    if (rc == DUST_OK) {
        if (ev && ev[1]) DUST_CUDA_TRY(cudaEventRecord(ev[1], st));
        int nl = 0;
        if (fsmem) {
            // the solve runs inside the emission kernel: its time is reported with the emission's;
            // where the grains come in passes the kernel emits the first and k_emit the others
            if (ev && ev[2]) DUST_CUDA_TRY(cudaEventRecord(ev[2], st));
            rc = launch_solve_emit_fused(B.req[0], ftc, fsmem, ctx->num_sms, st, &nl);
            if (rc == DUST_OK && fgc < (mass ? ctx->tbm : ctx->tb).G8) {
                nl_total += nl;
                nl = 0;
                rc = launch_emit_batch(B, ctx->num_sms, st, nullptr, true, &nl, 1);
            }
        } else {
            rc = launch_emit_batch(B, ctx->num_sms, st, ev ? ev[2] : nullptr, fused, &nl);
        }
        nl_total += nl;
        if (ev && ev[3]) DUST_CUDA_TRY(cudaEventRecord(ev[3], st));
    }
    if (nlaunch) *nlaunch = nl_total;
    return rc;
}

int solve_device(dust_ctx *ctx, int precision, int64_t C, const float *J, int64_t ld, const float *n,
                 float *T, float *L, double *resid, uint8_t *flags, void *scratch, cudaStream_t st, bool mass) {
    if (C == 0) return DUST_OK;
    const ScratchView sv = scratch_view(ctx, C, scratch);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (ctx->prof_on)
        for (int i = 0; i < 4; ++i) ev[i] = prof_event(ctx);
    const bool prof = ev[0] && ev[1] && ev[2] && ev[3];
    int nl = 0;
    const int rc = solve_view(ctx, precision, C, J, ld, n, T, L, resid, flags, sv, st, mass, &nl, prof ? ev : nullptr);
    ctx->launches += (uint64_t)nl;
    for (int i = 0; i < 4; ++i) {
        if (!ev[i]) continue;
        if (prof && rc == DUST_OK) ctx->prof_marks.push_back(ev[i]);
        else ctx->prof_pool.push_back(ev[i]);
    }
    return rc;
}

}  // namespace dust

using namespace dust;

extern "C" {

int dust_solve_prec(dust_ctx *ctx, int precision, int64_t n_cells, const float *J, int64_t ld,
                    const float *n, float *T, float *L, double *resid, uint8_t *flags, void *stream) {
    int rc = validate(ctx, precision, n_cells, J, ld, n, T, L, resid, flags, true);
    if (rc != DUST_OK || n_cells == 0) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    if (dg.rc != DUST_OK) return dg.rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_scratch(ctx, n_cells, st)) != DUST_OK) return rc;
    return solve_device(ctx, precision, n_cells, J, ld, n, T, L, resid, flags, ctx->S, st);
}

int dust_solve_mass(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *m, float *T,
                    float *L, double *resid, uint8_t *flags, void *stream) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    if (!ctx->mass_ready) return set_error(DUST_EINVAL, "grain numbers not set: call dust_ctx_set_grain_numbers");
    const int precision = ctx->precision;
    // m [C] takes n's place in the checks (it is read as one float per cell)
    int rc = validate(ctx, precision, n_cells, J, ld, m, T, L, resid, flags, true);
    if (rc != DUST_OK || n_cells == 0) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    if (dg.rc != DUST_OK) return dg.rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_scratch(ctx, n_cells, st)) != DUST_OK) return rc;
    return solve_device(ctx, precision, n_cells, J, ld, m, T, L, resid, flags, ctx->S, st, true);
}

int dust_solve(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n, float *T,
               float *L, double *resid, uint8_t *flags, void *stream) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    return dust_solve_prec(ctx, ctx->precision, n_cells, J, ld, n, T, L, resid, flags, stream);
}

int dust_solve_host(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n, float *T,
                    float *L, double *resid, uint8_t *flags) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    const int precision = ctx->precision;
    int rc = validate(ctx, DUST_PREC_FP32, n_cells, J, ld, n, T, L, resid, flags, false);
    if (rc != DUST_OK || n_cells == 0) return rc;
    if (precision != DUST_PREC_FP32 && ld % 4 != 0)
        return set_error(DUST_EINVAL, "tensor-core precisions need ld %% 4 == 0");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    if (dg.rc != DUST_OK) return dg.rc;
    const int G = ctx->G;
    constexpr int NB = dust_ctx::NHB;
    // the largest chunk about an eighth of the call and at least 8192 cells:
    // every chunk costs six copies, and each copy has a fixed cost of several
    // us that, with both directions busy, outweighs the shorter pipeline fill
    // and drain of many small chunks
    int64_t chunk = std::max<int64_t>(8192, (n_cells + 7) / 8);
    chunk = (chunk + 127) / 128 * 128;
    chunk = std::min<int64_t>(chunk, n_cells);
    auto &hs = ctx->hs;
    if (hs.cap < chunk || hs.ld != ld) {
        for (int i = 0; i < NB; ++i) {
            cudaFree(hs.J[i]); cudaFree(hs.n[i]); cudaFree(hs.T[i]); cudaFree(hs.L[i]);
            cudaFree(hs.r[i]); cudaFree(hs.f[i]);
            hs.J[i] = hs.n[i] = hs.T[i] = hs.L[i] = nullptr;
            hs.r[i] = nullptr; hs.f[i] = nullptr;
        }
        cudaFree(hs.S);
        hs.S = nullptr;
        hs.cap = 0;
        for (int i = 0; i < 3; ++i)
            if (!hs.st[i]) DUST_CUDA_TRY(cudaStreamCreateWithFlags(&hs.st[i], cudaStreamNonBlocking));
        for (int i = 0; i < NB; ++i) {
            if (!hs.ev_in[i]) DUST_CUDA_TRY(cudaEventCreateWithFlags(&hs.ev_in[i], cudaEventDisableTiming));
            if (!hs.ev_c[i]) DUST_CUDA_TRY(cudaEventCreateWithFlags(&hs.ev_c[i], cudaEventDisableTiming));
            if (!hs.ev_out[i]) DUST_CUDA_TRY(cudaEventCreateWithFlags(&hs.ev_out[i], cudaEventDisableTiming));
            DUST_CUDA_TRY(cudaMalloc(&hs.J[i], sizeof(float) * chunk * ld));
            DUST_CUDA_TRY(cudaMalloc(&hs.n[i], sizeof(float) * chunk * G));
            DUST_CUDA_TRY(cudaMalloc(&hs.T[i], sizeof(float) * chunk * G));
            DUST_CUDA_TRY(cudaMalloc(&hs.L[i], sizeof(float) * chunk * ld));
            DUST_CUDA_TRY(cudaMalloc(&hs.r[i], sizeof(double) * chunk));
            DUST_CUDA_TRY(cudaMalloc(&hs.f[i], sizeof(uint8_t) * chunk * G));
        }
        DUST_CUDA_TRY(cudaMalloc(&hs.S, scratch_bytes(ctx, chunk, true)));
        hs.cap = chunk;
        hs.ld = ld;
        hs.bytes = (size_t)NB * ((size_t)chunk * ld * 4 * 2 + (size_t)chunk * G * (4 * 2 + 1) + (size_t)chunk * 8) +
                   scratch_bytes(ctx, chunk, true);
    }
    // copy in (stream 0) -> compute (stream 1) -> copy out (stream 2), chunk i in
    // buffer set i % NB: chunk i's upload, chunk i-1's compute and chunk i-2's
    // download run at the same time.  A buffer set is reused once the compute
    // that read its inputs and the download that read its outputs are done.
    // Chunk sizes: the copies back can start only once a chunk is computed, and
    // they bound the pipeline (more bytes out than in, a slower direction), so
    // the first chunk is a quarter of the largest and each next one 3/2 of the
    // one before, up to the largest: the copies back start early and stay busy
    // (measured at 2^18 cells: 2.39 ms per call against 2.49 ms with equal
    // chunks; growth 5/4 and 2 gave 2.40 and 2.45 ms).
    cudaStream_t sin = hs.st[0], scomp = hs.st[1], sout = hs.st[2];
    int64_t i = 0, cur = std::min<int64_t>(chunk, std::max<int64_t>(4096, chunk / 4));
    for (int64_t c0 = 0, cn = 0; c0 < n_cells; c0 += cn, ++i, cur = std::min<int64_t>(chunk, (cur * 3 / 2 + 127) / 128 * 128)) {
        const int b = (int)(i % NB);
        cn = std::min<int64_t>(cur, n_cells - c0);
        if (i >= NB) DUST_CUDA_TRY(cudaStreamWaitEvent(sin, hs.ev_c[b], 0));
        DUST_CUDA_TRY(cudaMemcpyAsync(hs.J[b], J + c0 * ld, sizeof(float) * cn * ld, cudaMemcpyHostToDevice, sin));
        DUST_CUDA_TRY(cudaMemcpyAsync(hs.n[b], n + c0 * G, sizeof(float) * cn * G, cudaMemcpyHostToDevice, sin));
        DUST_CUDA_TRY(cudaEventRecord(hs.ev_in[b], sin));
        DUST_CUDA_TRY(cudaStreamWaitEvent(scomp, hs.ev_in[b], 0));
        if (i >= NB) DUST_CUDA_TRY(cudaStreamWaitEvent(scomp, hs.ev_out[b], 0));
        rc = solve_device(ctx, precision, cn, hs.J[b], ld, hs.n[b], hs.T[b], L ? hs.L[b] : nullptr,
                          resid ? hs.r[b] : nullptr, flags ? hs.f[b] : nullptr, hs.S, scomp);
        if (rc != DUST_OK) {
            for (int k = 0; k < 3; ++k) cudaStreamSynchronize(hs.st[k]);
            return rc;
        }
        DUST_CUDA_TRY(cudaEventRecord(hs.ev_c[b], scomp));
        DUST_CUDA_TRY(cudaStreamWaitEvent(sout, hs.ev_c[b], 0));
        DUST_CUDA_TRY(cudaMemcpyAsync(T + c0 * G, hs.T[b], sizeof(float) * cn * G, cudaMemcpyDeviceToHost, sout));
        if (L)
            DUST_CUDA_TRY(cudaMemcpyAsync(L + c0 * ld, hs.L[b], sizeof(float) * cn * ld, cudaMemcpyDeviceToHost, sout));
        if (resid)
            DUST_CUDA_TRY(cudaMemcpyAsync(resid + c0, hs.r[b], sizeof(double) * cn, cudaMemcpyDeviceToHost, sout));
        if (flags)
            DUST_CUDA_TRY(cudaMemcpyAsync(flags + c0 * G, hs.f[b], cn * G, cudaMemcpyDeviceToHost, sout));
        DUST_CUDA_TRY(cudaEventRecord(hs.ev_out[b], sout));
    }
    for (int k = 0; k < 3; ++k) DUST_CUDA_TRY(cudaStreamSynchronize(hs.st[k]));
    return DUST_OK;
}

int dust_ctx_profile(dust_ctx *ctx, int enable) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof_on = enable != 0;
    return DUST_OK;
}

int dust_ctx_profile_read(dust_ctx *ctx, double *ms_absorb, double *ms_solve, double *ms_emit,
                          int64_t *n_solves) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    if (dg.rc != DUST_OK) return dg.rc;
    double a = 0.0, b = 0.0, c = 0.0;
    int64_t cnt = 0;
    int rc = DUST_OK;
    for (size_t i = 0; i + 3 < ctx->prof_marks.size(); i += 4) {
        cudaEvent_t *e = &ctx->prof_marks[i];
        float t01 = 0.f, t12 = 0.f, t23 = 0.f;
        if (cudaEventSynchronize(e[3]) != cudaSuccess || cudaEventElapsedTime(&t01, e[0], e[1]) != cudaSuccess ||
            cudaEventElapsedTime(&t12, e[1], e[2]) != cudaSuccess ||
            cudaEventElapsedTime(&t23, e[2], e[3]) != cudaSuccess) {
            rc = set_error(DUST_ECUDA, "profiling events could not be read");
            break;
        }
        a += t01;
        b += t12;
        c += t23;
        ++cnt;
    }
    for (cudaEvent_t e : ctx->prof_marks) ctx->prof_pool.push_back(e);
    ctx->prof_marks.clear();
    if (ms_absorb) *ms_absorb = a;
    if (ms_solve) *ms_solve = b;
    if (ms_emit) *ms_emit = c;
    if (n_solves) *n_solves = cnt;
    return rc;
}

int dust_ctx_check(dust_ctx *ctx, int *device_status) {
    if (!ctx) return set_error(DUST_EINVAL, "ctx is NULL");
    DeviceGuard dg(ctx->device);
    if (dg.rc != DUST_OK) return dg.rc;
    DUST_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    DUST_CUDA_TRY(cudaMemcpy(&v, ctx->tb.status, sizeof(int), cudaMemcpyDeviceToHost));
    DUST_CUDA_TRY(cudaMemset(ctx->tb.status, 0, sizeof(int)));
    if (device_status) *device_status = v;
    return DUST_OK;
}

}  // extern "C"

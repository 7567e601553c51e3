// Serving: continuous batching of solve requests of uneven sizes and
// wavelength / grain grids on one GPU.
//
// A scheduler thread owns one CUDA stream.  Requests are admitted in FIFO
// order (a later request may pass one that does not fit yet) while the sum of
// the device footprints of admitted requests stays within the HBM budget and
// at most `max_inflight` are active; each admitted request gets its scratch
// from a first-fit arena carved out of one allocation.  Work proceeds in
// rounds, two in flight, so requests that arrive while the GPU is busy join a
// round as soon as one retires and their work overlaps with the tail of
// earlier ones.  Rounds are sized by work, shortest remaining first: active
// requests are ranked by their remaining Planck terms discounted by how long
// they have waited (so that large requests are not starved).  A small first
// request (little work left) makes a batched round: it and the next small
// requests, whole, up to a work budget and 32 parts, through one launch per
// kernel (absorption GEMM per precision and orientation, the cell ordering,
// the batched solve, the emission in work units, the residual).  A large one
// runs alone, a chunk of cells per round, through dust_solve's own path (the
// fused solve + emission where it applies).  A cell's arithmetic does not
// depend on its chunk, its batch or its place in the emission order, so a
// request's results are bitwise those of dust_solve on the same context.
#include "dust_internal.cuh"

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>

using namespace dust;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { RS_QUEUED = 0, RS_ACTIVE = 1, RS_DONE = 2, RS_CANCELLED = 3, RS_FAILED = 4 };

struct ServeReq {
    uint64_t ticket = 0;
    dust_ctx *ctx = nullptr;
    int precision = 0;
    int64_t C = 0, ld = 0;
    const float *J = nullptr, *n = nullptr;
    float *T = nullptr, *L = nullptr;
    double *resid = nullptr;
    uint8_t *flags = nullptr;
    size_t footprint = 0, s_bytes = 0, s_off = 0;
    float *S = nullptr;
    int64_t next = 0, done = 0;
    int inflight_parts = 0;
    int state = RS_QUEUED;
    int status = DUST_OK;
    double t_submit = 0, t_done = 0;
    cudaEvent_t ready = nullptr;  // recorded on the producer's stream at submit
    bool ready_waited = false;    // the server stream waits on it once
};

// First-fit allocator over one device allocation (offsets in bytes).
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> size
    void reset(size_t bytes) { free_.clear(); if (bytes) free_[0] = bytes; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, o = it->first + bytes;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Part {
    ServeReq *r;
    int64_t c0, cn;
};

struct Round {
    cudaEvent_t ev = nullptr;
    int slot = 0;  // its part of the server's class-count workspace
    std::vector<Part> parts;
};

// Rounds in flight at once, each with its own class counts for the parts' cell order.
constexpr int NSLOT = 2;

}  // namespace

struct dust_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_inflight = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    cudaStream_t st = nullptr;
    char *arena_mem = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeReq *> queue;
    std::vector<ServeReq *> active;
    std::unordered_map<uint64_t, ServeReq *> by_ticket;
    std::deque<Round> inflight;
    std::vector<cudaEvent_t> ev_pool;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    unsigned *hist_ws = nullptr;    // [NSLOT][MAXREQ][2 NBK] class counts of the rounds' parts
    bool slot_busy[NSLOT] = {};
    // scheduling: shortest remaining work first, the remaining work of a request
    // discounted by 1 + wait / age_ms so that large requests are not starved;
    // requests of at most small_terms Planck terms go whole into batched rounds of
    // up to batch_terms, larger ones run alone in chunks of about chunk_terms
    double small_terms = 1.0e9, batch_terms = 5.0e9, chunk_terms = 1.0e10, age_ms = 20.0;
    // statistics
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, cells_done = 0, rounds = 0, launches = 0;
    double t_first = -1, t_last = -1;
};

namespace {

size_t footprint_of(const dust_ctx *ctx, int64_t C, int64_t ld, bool L, bool resid, bool flags) {
    const size_t G = ctx->G;
    size_t b = (size_t)C * ld * 4 + (size_t)C * G * 4 * 2 + scratch_bytes(ctx, C, L || resid);  // J, n, T, scratch
    if (L) b += (size_t)C * ld * 4;
    if (resid) b += (size_t)C * 8;
    if (flags) b += (size_t)C * G;
    return b;
}

void finish_req(dust_server *s, ServeReq *r, int state, int status) {
    if (r->ready) {  // the server stream is past its wait (or never reached it)
        s->ev_pool.push_back(r->ready);
        r->ready = nullptr;
    }
    r->state = state;
    r->status = status;
    r->t_done = now_ms();
    if (r->s_bytes) {
        s->arena.release(r->s_off, r->s_bytes);
        r->s_bytes = 0;
    }
    s->used -= r->footprint;
    r->footprint = 0;
    auto it = std::find(s->active.begin(), s->active.end(), r);
    if (it != s->active.end()) s->active.erase(it);
    if (state == RS_DONE) {
        s->completed++;
        s->cells_done += r->C;
        s->lat_ms.push_back(r->t_done - r->t_submit);
        s->t_last = r->t_done;
    } else if (state == RS_CANCELLED) {
        s->cancelled++;
    } else {
        s->failed++;
    }
}

void admit(dust_server *s) {
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        ServeReq *r = *it;
        if ((int)s->active.size() >= s->max_inflight) break;
        const size_t fp = footprint_of(r->ctx, r->C, r->ld, r->L, r->resid, r->flags);
        size_t off = 0;
        if (s->used + fp <= s->budget && s->arena.alloc(r->s_bytes, &off)) {
            r->s_off = off;
            r->S = reinterpret_cast<float *>(s->arena_mem + off);
            r->footprint = fp;
            s->used += fp;
            r->state = RS_ACTIVE;
            s->active.push_back(r);
            it = s->queue.erase(it);
        } else {
            ++it;
        }
    }
}

// Build one round.  Active requests are ranked by remaining Planck terms
// discounted by their wait, (C - next) K G / (1 + wait / age_ms), smallest
// first.  If the first is small (at most small_terms left), the round takes
// it and the next small ones whole, up to batch_terms and MAXREQ parts, for
// the batched kernels; otherwise it takes a chunk of about chunk_terms of the
// first alone (a multiple of 128 cells, at least 4096), for dust_solve's path.
std::vector<Part> build_round(dust_server *s) {
    std::vector<Part> parts;
    std::vector<std::pair<double, ServeReq *>> cand;
    const double t = now_ms();
    auto terms = [](const ServeReq *r) { return (double)(r->C - r->next) * r->ctx->K * r->ctx->G; };
    for (ServeReq *r : s->active)
        if (r->state == RS_ACTIVE && r->next < r->C)
            cand.push_back({terms(r) / (1.0 + (t - r->t_submit) / s->age_ms), r});
    if (cand.empty()) return parts;
    std::stable_sort(cand.begin(), cand.end(),
                     [](const std::pair<double, ServeReq *> &a, const std::pair<double, ServeReq *> &b) { return a.first < b.first; });
    ServeReq *top = cand[0].second;
    if (terms(top) <= s->small_terms) {
        double sum = 0.0;
        for (const auto &c : cand) {
            ServeReq *r = c.second;
            const double w = terms(r);
            if (w > s->small_terms || (!parts.empty() && sum + w > s->batch_terms)) continue;
            parts.push_back({r, r->next, r->C - r->next});
            r->next = r->C;
            r->inflight_parts++;
            sum += w;
            if (parts.size() == (size_t)MAXREQ) break;
        }
        return parts;
    }
    const double per_cell = (double)top->ctx->K * top->ctx->G;
    int64_t cn = (int64_t)(s->chunk_terms / per_cell);
    cn = std::max<int64_t>(cn, 4096);
    cn = (cn + 127) / 128 * 128;
    cn = std::min<int64_t>(cn, top->C - top->next);
    parts.push_back({top, top->next, cn});
    top->next += cn;
    top->inflight_parts++;
    return parts;
}

// Scratch of one part: rows c0.. of its request's S, (1/T, n) pairs, cell
// records, residual partials, grain-pass sums, emission order and classes,
// and the round slot's class counts for part index k.
ScratchView part_view(const dust_server *s, const Part &p, int slot, int k) {
    const ScratchView v = scratch_view(p.r->ctx, p.r->C, p.r->S);
    const DevTables &tb = p.r->ctx->tb;
    ScratchView w{};
    w.S = v.S + p.c0 * tb.Gs;
    w.prep = v.prep + p.c0 * tb.G8;
    w.cell = v.cell + p.c0;
    w.part = v.part + p.c0 * tb.NKG;
    w.accp = v.accp ? v.accp + p.c0 * tb.NKG * 4 : nullptr;
    w.order = v.order + p.c0;
    w.bkt = v.bkt + p.c0;
    w.hist = s->hist_ws + ((size_t)slot * MAXREQ + k) * 2 * NBK;
    return w;
}

int launch_round(dust_server *s, const Round &rd) {
    const std::vector<Part> &parts = rd.parts;
    // a request's first round waits (on the device) for the work its
    // producer had queued before submitting
    for (const Part &p : parts) {
        ServeReq *r = p.r;
        if (r->ready && !r->ready_waited) {
            if (cudaStreamWaitEvent(s->st, r->ready, 0) != cudaSuccess)
                return set_error(DUST_ECUDA, "cudaStreamWaitEvent on a request's input event failed");
            r->ready_waited = true;
        }
    }
    if (parts.size() == 1) {
        // one chunk of one request: dust_solve's own path over its cells
        const Part &p = parts[0];
        ServeReq *r = p.r;
        const int G = r->ctx->G;
        int nl = 0;
        const int rc = solve_view(r->ctx, r->precision, p.cn, r->J + p.c0 * r->ld, r->ld, r->n + p.c0 * G,
                                  r->T + p.c0 * G, r->L ? r->L + p.c0 * r->ld : nullptr, r->resid ? r->resid + p.c0 : nullptr,
                                  r->flags ? r->flags + p.c0 * G : nullptr, part_view(s, p, rd.slot, 0), s->st, false, &nl);
        s->launches += (uint64_t)nl;
        return rc;
    }
    // absorption GEMMs, one launch per precision
    for (int prec = DUST_PREC_FP32; prec <= DUST_PREC_FP16X3; ++prec) {
        if (prec == DUST_PREC_FP32) {
            SimtBatch B;
            B.nreq = 0;
            for (size_t k = 0; k < parts.size(); ++k) {
                const Part &p = parts[k];
                if (p.r->precision != prec) continue;
                ServeReq *r = p.r;
                make_simt_req(r->ctx, p.cn, r->J + p.c0 * r->ld, r->ld, part_view(s, p, rd.slot, (int)k).S, B.req[B.nreq++]);
            }
            if (B.nreq) {
                int rc = launch_simt_batch(B, s->st);
                if (rc != DUST_OK) return rc;
                s->launches++;
            }
        } else {
            // one launch per orientation, each request in the one dust_solve uses for
            // its context, so that results are bitwise those of a solve alone
            for (int orient = 0; orient < 2; ++orient) {
                TcBatch B;
                B.nreq = 0;
                B.status = nullptr;
                B.orient = orient;
                for (size_t k = 0; k < parts.size(); ++k) {
                    const Part &p = parts[k];
                    if (p.r->precision != prec || tc_orient(p.r->ctx) != orient) continue;
                    ServeReq *r = p.r;
                    if (!B.status) B.status = r->ctx->tb.status;
                    int rc = make_tc_req(r->ctx, prec, p.cn, r->J + p.c0 * r->ld, r->ld, part_view(s, p, rd.slot, (int)k).S,
                                         B.req[B.nreq], B.tm[B.nreq], orient);
                    if (rc != DUST_OK) return rc;
                    B.nreq++;
                }
                if (B.nreq) {
                    size_t smem = 0;
                    int rc = finish_tc_batch(B, prec, s->smem_optin, &smem);
                    if (rc == DUST_OK) rc = launch_tc_batch(B, prec, smem, s->num_sms, s->st);
                    if (rc != DUST_OK) return rc;
                    s->launches++;
                }
            }
        }
    }
    // emission order of every part that emits (classes of the reference grain's absorbed power)
    EmitBatch E;
    E.nreq = 0;
    OrderBatch ob;
    ob.nreq = 0;
    for (size_t k = 0; k < parts.size(); ++k) {
        const Part &p = parts[k];
        ServeReq *r = p.r;
        dust_ctx *ctx = r->ctx;
        const int G = ctx->G;
        const ScratchView v = part_view(s, p, rd.slot, (int)k);
        const EmitPlan pl = plan_emit(ctx, r->L || r->resid, false);
        EmitReq &e = E.req[E.nreq++];
        fill_emit_req(ctx, pl, p.cn, v, r->n + p.c0 * G, r->T + p.c0 * G, r->L ? r->L + p.c0 * r->ld : nullptr, r->ld,
                      r->resid ? r->resid + p.c0 : nullptr, r->flags ? r->flags + p.c0 * G : nullptr, e, false);
        if (r->L || r->resid) {
            OrderReq &o = ob.req[ob.nreq++];
            o.key = v.S + order_ref_grain(G);
            o.kstride = ctx->tb.Gs;
            o.C = p.cn;
            o.bkt = v.bkt;
            o.hist = v.hist;
            o.order = v.order;
            e.order = v.order;
        }
    }
    int nl = 0;
    if (ob.nreq) {
        int rc = launch_order(ob, s->st, &nl);
        if (rc != DUST_OK) return rc;
        s->launches += (uint64_t)nl;
    }
    int rc = launch_emit_batch(E, s->num_sms, s->st, nullptr, false, &nl);
    if (rc != DUST_OK) return rc;
    s->launches += (uint64_t)nl;
    return DUST_OK;
}

void retire_round(dust_server *s, Round &rd, int status) {
    for (const Part &p : rd.parts) {
        ServeReq *r = p.r;
        r->inflight_parts--;
        if (status != DUST_OK) {
            if (r->state == RS_ACTIVE || r->state == RS_CANCELLED) r->status = status;
            r->state = RS_FAILED;
        } else {
            r->done += p.cn;
        }
        if (r->inflight_parts == 0) {
            if (r->state == RS_FAILED) finish_req(s, r, RS_FAILED, r->status);
            else if (r->state == RS_CANCELLED && r->footprint) finish_req(s, r, RS_CANCELLED, DUST_OK);
            else if (r->done == r->C) finish_req(s, r, RS_DONE, DUST_OK);
        }
    }
    s->ev_pool.push_back(rd.ev);
    s->slot_busy[rd.slot] = false;
    s->cv_done.notify_all();
}

void scheduler(dust_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        while (!s->inflight.empty() && cudaEventQuery(s->inflight.front().ev) != cudaErrorNotReady) {
            Round rd = std::move(s->inflight.front());
            s->inflight.pop_front();
            cudaError_t e = cudaEventQuery(rd.ev);
            retire_round(s, rd, e == cudaSuccess ? DUST_OK : DUST_ECUDA);
        }
        admit(s);
        if (s->inflight.size() < (size_t)NSLOT) {
            std::vector<Part> parts = build_round(s);
            if (!parts.empty()) {
                Round rd;
                if (!s->ev_pool.empty()) { rd.ev = s->ev_pool.back(); s->ev_pool.pop_back(); }
                else cudaEventCreateWithFlags(&rd.ev, cudaEventDisableTiming);
                rd.parts = std::move(parts);
                while (s->slot_busy[rd.slot]) ++rd.slot;  // a free slot exists: fewer than NSLOT in flight
                s->slot_busy[rd.slot] = true;
                int rc = launch_round(s, rd);
                if (rc == DUST_OK && cudaEventRecord(rd.ev, s->st) == cudaSuccess) {
                    s->rounds++;
                    s->inflight.push_back(std::move(rd));
                } else {
                    retire_round(s, rd, rc == DUST_OK ? DUST_ECUDA : rc);
                }
                continue;
            }
        }
        if (!s->inflight.empty()) {
            cudaEvent_t ev = s->inflight.front().ev;
            lk.unlock();
            cudaEventSynchronize(ev);
            lk.lock();
            continue;
        }
        if (s->stop) break;
        s->cv_work.wait(lk);
    }
}

int check_dev(const void *p, int device, const char *name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DUST_EINVAL, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error(DUST_EINVAL, "%s must be device memory", name);
    if (a.type == cudaMemoryTypeDevice && a.device != device)
        return set_error(DUST_EINVAL, "%s lives on device %d, the server on device %d", name, a.device, device);
    return DUST_OK;
}

}  // namespace

extern "C" {

int dust_server_create(dust_server **out, size_t hbm_budget_bytes, int max_inflight, int device) {
    if (!out) return set_error(DUST_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes < (1u << 20)) return set_error(DUST_EINVAL, "budget below 1 MiB");
    if (max_inflight < 1 || max_inflight > 4096) return set_error(DUST_EINVAL, "max_inflight outside [1, 4096]");
    int ndev = 0;
    DUST_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_error(DUST_EINVAL, "device %d of %d", device, ndev);
    int prev = 0;
    DUST_CUDA_TRY(cudaGetDevice(&prev));
    DUST_CUDA_TRY(cudaSetDevice(device));
    dust_server *s = new dust_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->max_inflight = max_inflight;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_mem, hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->hist_ws, sizeof(unsigned) * NSLOT * MAXREQ * 2 * NBK);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        if (s->st) cudaStreamDestroy(s->st);
        if (s->arena_mem) cudaFree(s->arena_mem);
        delete s;
        return set_error(e == cudaErrorMemoryAllocation ? DUST_ENOMEM : DUST_ECUDA, "server setup failed: %s",
                         cudaGetErrorString(e));
    }
    s->num_sms = prop.multiProcessorCount;
    s->smem_optin = prop.sharedMemPerBlockOptin;
    s->arena.reset(hbm_budget_bytes);
    s->th = std::thread(scheduler, s);
    *out = s;
    return DUST_OK;
}

int dust_serve_submit(dust_server *s, dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n,
                      float *T, float *L, double *resid, uint8_t *flags, void *stream, uint64_t *ticket) {
    if (!s || !ctx || !ticket) return set_error(DUST_EINVAL, "server, ctx and ticket must be non-NULL");
    if (ctx->device != s->device) return set_error(DUST_EINVAL, "context and server on different devices");
    if (n_cells < 0) return set_error(DUST_EINVAL, "n_cells < 0");
    if (ld < ctx->K) return set_error(DUST_EINVAL, "ld=%lld < K=%d", (long long)ld, ctx->K);
    const int prec = ctx->precision;
    if (n_cells > 0) {
        if (!J || !n || !T) return set_error(DUST_EINVAL, "J, n and T must be non-NULL");
        if (prec != DUST_PREC_FP32 && (ld % 4 != 0 || ((uintptr_t)J & 15) != 0))
            return set_error(DUST_EINVAL, "tensor-core precisions need ld %% 4 == 0 and a 16-byte aligned J");
        int rc;
        if ((rc = check_dev(J, s->device, "J")) || (rc = check_dev(n, s->device, "n")) ||
            (rc = check_dev(T, s->device, "T")) || (L && (rc = check_dev(L, s->device, "L"))) ||
            (resid && (rc = check_dev(resid, s->device, "resid"))) ||
            (flags && (rc = check_dev(flags, s->device, "flags"))))
            return rc;
    }
    const size_t fp = footprint_of(ctx, n_cells, ld, L, resid, flags);
    if (fp > s->budget)
        return set_error(DUST_EBUSY, "request footprint %zu B exceeds the server budget %zu B", fp, s->budget);
    ServeReq *r = new ServeReq();
    r->ctx = ctx;
    r->precision = prec;
    r->C = n_cells;
    r->ld = ld;
    r->J = J; r->n = n; r->T = T; r->L = L; r->resid = resid; r->flags = flags;
    r->s_bytes = scratch_bytes(ctx, std::max<int64_t>(n_cells, 1), L || resid);
    if (n_cells > 0) {
        // mark the producer's position: J and n are complete once the work
        // queued on `stream` so far has run
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (!s->ev_pool.empty()) { r->ready = s->ev_pool.back(); s->ev_pool.pop_back(); }
        }
        int prev = -1;
        cudaError_t e = cudaGetDevice(&prev);
        if (e == cudaSuccess && prev != s->device) e = cudaSetDevice(s->device);
        if (e == cudaSuccess && !r->ready) e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r->ready, (cudaStream_t)stream);
        if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (r->ready) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->ev_pool.push_back(r->ready);
            }
            delete r;
            return set_error(DUST_ECUDA, "recording the input event on the producer stream failed: %s",
                             cudaGetErrorString(e));
        }
    }
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            if (r->ready) s->ev_pool.push_back(r->ready);
            delete r;
            return set_error(DUST_EINVAL, "server is shutting down");
        }
        r->ticket = s->next_ticket++;
        s->by_ticket[r->ticket] = r;
        s->submitted++;
        if (s->t_first < 0) s->t_first = r->t_submit;
        if (n_cells == 0) {
            r->state = RS_DONE;
            r->t_done = r->t_submit;
            s->completed++;
            s->lat_ms.push_back(0.0);
        } else {
            s->queue.push_back(r);
        }
    }
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return DUST_OK;
}

int dust_serve_poll(dust_server *s, uint64_t ticket, int *state, double *latency_ms) {
    if (!s) return set_error(DUST_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return set_error(DUST_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    ServeReq *r = it->second;
    const bool fin = r->state == RS_DONE || r->state == RS_CANCELLED || (r->state == RS_FAILED && !r->footprint);
    if (state) *state = fin ? r->state : (r->state == RS_FAILED ? RS_ACTIVE : r->state);
    if (latency_ms) *latency_ms = fin ? r->t_done - r->t_submit : now_ms() - r->t_submit;
    if (fin) {
        const int st = r->state, status = r->status;
        s->by_ticket.erase(it);
        delete r;
        if (st == RS_FAILED) return set_error(status ? status : DUST_ECUDA, "request failed");
    }
    return DUST_OK;
}

int dust_serve_wait(dust_server *s, uint64_t ticket, double timeout_ms, double *latency_ms) {
    if (!s) return set_error(DUST_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double, std::milli>(timeout_ms);
    for (;;) {
        auto it = s->by_ticket.find(ticket);
        if (it == s->by_ticket.end())
            return set_error(DUST_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        ServeReq *r = it->second;
        const bool fin = r->state == RS_DONE || r->state == RS_CANCELLED || (r->state == RS_FAILED && !r->footprint);
        if (fin) {
            if (latency_ms) *latency_ms = r->t_done - r->t_submit;
            const int st = r->state, status = r->status;
            s->by_ticket.erase(it);
            delete r;
            if (st == RS_FAILED) return set_error(status ? status : DUST_ECUDA, "request failed");
            if (st == RS_CANCELLED) return set_error(DUST_ENOTFOUND, "request was cancelled");
            return DUST_OK;
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout)
            return set_error(DUST_ETIMEOUT, "request %llu not finished after %.1f ms", (unsigned long long)ticket,
                             timeout_ms);
    }
}

int dust_serve_cancel(dust_server *s, uint64_t ticket) {
    if (!s) return set_error(DUST_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return set_error(DUST_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    ServeReq *r = it->second;
    if (r->state == RS_QUEUED) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        if (r->ready) {  // never waited on: free to be recorded again
            s->ev_pool.push_back(r->ready);
            r->ready = nullptr;
        }
        r->state = RS_CANCELLED;
        r->t_done = now_ms();
        s->cancelled++;
    } else if (r->state == RS_ACTIVE) {
        // no further chunks are scheduled; chunks already on the GPU finish
        r->state = RS_CANCELLED;
        r->next = r->C;
        if (r->inflight_parts == 0) finish_req(s, r, RS_CANCELLED, DUST_OK);
    }
    s->cv_done.notify_all();
    return DUST_OK;
}

int dust_server_stats(dust_server *s, dust_serve_stats *out) {
    if (!s || !out) return set_error(DUST_EINVAL, "server and out must be non-NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        double x = p * (v.size() - 1);
        size_t i = (size_t)x;
        double f = x - i;
        return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
    };
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->cancelled = s->cancelled;
    out->failed = s->failed;
    out->queued = (int64_t)s->queue.size();
    out->active = (int64_t)s->active.size();
    out->cells_completed = s->cells_done;
    out->rounds = s->rounds;
    out->launches = s->launches;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.empty() ? 0.0 : v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = v.empty() ? 0.0 : sum / v.size();
    out->span_ms = (s->t_first >= 0 && s->t_last >= 0) ? s->t_last - s->t_first : 0.0;
    out->hbm_in_use = s->used;
    return DUST_OK;
}

int dust_server_set_policy(dust_server *s, double small_terms, double batch_terms, double chunk_terms, double age_ms) {
    if (!s) return set_error(DUST_EINVAL, "server is NULL");
    if (!(small_terms >= 0.0) || !(batch_terms > 0.0) || !(chunk_terms > 0.0) || !(age_ms > 0.0) ||
        !std::isfinite(small_terms) || !std::isfinite(batch_terms) || !std::isfinite(chunk_terms) || !std::isfinite(age_ms))
        return set_error(DUST_EINVAL, "policy values must be finite, small_terms >= 0 and the others > 0");
    std::lock_guard<std::mutex> lk(s->mu);
    s->small_terms = small_terms;
    s->batch_terms = batch_terms;
    s->chunk_terms = chunk_terms;
    s->age_ms = age_ms;
    return DUST_OK;
}

int dust_server_reset_stats(dust_server *s) {
    if (!s) return set_error(DUST_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->submitted = s->completed = s->cancelled = s->failed = s->cells_done = s->rounds = s->launches = 0;
    s->t_first = s->t_last = -1;
    return DUST_OK;
}

void dust_server_destroy(dust_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (ServeReq *r : s->queue) {  // never admitted: cancelled
            r->state = RS_CANCELLED;
            s->cancelled++;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();  // finishes every admitted request
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->st);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (auto &kv : s->by_ticket)
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    cudaStreamDestroy(s->st);
    cudaFree(s->arena_mem);
    cudaFree(s->hist_ws);
    cudaSetDevice(prev);
    for (auto &kv : s->by_ticket) delete kv.second;
    delete s;
}

}  // extern "C"

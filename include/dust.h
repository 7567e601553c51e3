/*
 * dust.h -- C ABI of libdust, a GB300 (sm_103a) engine for dust-grain
 * equilibrium temperatures and the resulting infrared emission SED.
 *
 * Method: Jonsson & Primack, "Accelerating Dust Temperature Calculations with
 * Graphics Processing Units".  For every cell c of a radiation-transfer grid
 * and every grain g (species x size), with wavelengths lambda_k and quadrature
 * weights w_k:
 *
 *   A[c,g] = sum_k w_k C_abs[g,k] J[c,k]                   absorbed power (Eq. 6)
 *   P_g(T) = sum_k w_k C_abs[g,k] B_k(T)                   emitted power  (Eq. 7)
 *   T[c,g] : P_g(T[c,g]) = A[c,g], T in [T_min, T_max]     equilibrium    (Eqs. 1, 7)
 *   L[c,k] = 4 pi sum_g n[c,g] C_abs[g,k] B_k(T[c,g])      emission SED   (Eqs. 8-10)
 *
 * with B_k(T) = 2 h c^2 lambda_k^-5 / (exp(h c / (lambda_k k_B T)) - 1)
 * (Eq. 1) and n[c,g] the number of grains g in cell c (the paper's
 * n_s m_d;c of Eqs. 9-10, generalised to any per-cell, per-grain value).
 *
 * Conventions shared by every entry point:
 *  - Status: every function returning int returns a dust_status code; a
 *    non-zero code leaves a thread-local message for dust_last_error().
 *    Nothing throws or aborts across this boundary.
 *  - Argument checks happen on the host before anything is enqueued; a call
 *    that fails them has no effect.
 *  - Units are the caller's, but must be consistent: with lambda and w in m,
 *    C_abs in m^2 and J in W m^-2 m^-1 sr^-1, A and P are in W sr^-1 and L
 *    in W m^-1 (per unit n).
 *  - Device pointers are plain CUDA device addresses on the context's device
 *    (e.g. torch tensor data pointers); "stream" is a cudaStream_t passed as
 *    void* (NULL = the legacy default stream).
 */
#ifndef DUST_H
#define DUST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dust_ctx dust_ctx;
typedef struct dust_server dust_server;

enum dust_status {
    DUST_OK = 0,
    DUST_EINVAL = 1,     /* invalid argument                                   */
    DUST_ENOMEM = 2,     /* device or host allocation failed                   */
    DUST_ECUDA = 3,      /* a CUDA runtime / driver call failed                */
    DUST_EBUSY = 4,      /* request can never be admitted (over the budget)    */
    DUST_ETIMEOUT = 5,   /* a bounded device-side wait gave up                 */
    DUST_ENOTFOUND = 6   /* unknown ticket                                     */
};

/* Arithmetic of the absorption contraction A = J W^T (Eq. 6).  The
 * temperature solve and the emission always run in FP32; FP64 is used only
 * to build the context tables and for the energy-balance residual. */
enum dust_precision {
    DUST_PREC_FP32 = 0,   /* FP32 FMA on the CUDA cores                          */
    DUST_PREC_BF16X3 = 1, /* tensor cores: BF16 hi+lo split, 3 products, FP32 acc */
    DUST_PREC_FP16X3 = 2  /* tensor cores: FP16 hi+lo split, 3 products, FP32 acc */
};

/* Per-grain solve flags written to the optional flags output. */
enum dust_flag {
    DUST_FLAG_OK = 0,      /* T solved inside the bracket                          */
    DUST_FLAG_LOW = 1,     /* A < P_g(T_min) (includes A = 0): T = T_min           */
    DUST_FLAG_HIGH = 2,    /* A > P_g(T_max): T = T_max                            */
    DUST_FLAG_INVALID = 4, /* A negative or not finite (bad J): T = NaN            */
    DUST_FLAG_NOCONV = 8   /* dust_solve_T_newton only: no convergence in 64 steps */
};

/* Create a context for one wavelength grid and one set of grains on `device`.
 *
 *  K, lambda[K], w[K]  host FP64, 2 <= K <= 2048: wavelengths (strictly increasing, > 0) and
 *                      quadrature weights (>= 0) such that sum_k w_k f(lambda_k)
 *                      approximates the integral over wavelength (the paper's
 *                      Delta lambda_l, Eqs. 6-8).
 *  G, c_abs[G*K]       host FP64, row-major [g][k]: absorption cross sections
 *                      (the paper's sigma_a;s,l), >= 0, every row with some
 *                      w_k C_abs[g,k] > 0.  1 <= G <= 512.
 *  T_min, T_max        temperature bracket, 0 < T_min < T_max.
 *  n_table             points of the P_g(T) table (uniform in log T), 64..65536;
 *                      0 selects 4096.
 *  precision           default dust_precision of dust_solve (changeable later).
 *
 * The context copies every input (the caller may free them on return), keeps
 * all tables resident in device memory, and owns a scratch buffer for the
 * absorbed powers that dust_solve grows on demand.  The P_g(T) table, its
 * slope and an inverse table (the roots of the table at n_table uniform steps
 * of log2 P, with the table's cubic on each interval between them) are built
 * on the device in FP64, replacing the per-iteration quadrature of the
 * paper's Newton kernel (Section 4.3) by the table lookup its production code
 * uses (Section 6); a solve is one lookup and one Newton step.  Also fails
 * with DUST_EINVAL when P_g(T) is not strictly increasing in FP64.
 * Also fails with DUST_EINVAL when h c / (lambda_max k_B T_max) < 1e-3 (the
 * emission kernel's rational accumulation needs 1 - exp(-x) >= 1e-3).
 * Synchronous; returns DUST_OK and *out, or an error and *out = NULL. */
int dust_ctx_create(dust_ctx **out, int K, const double *lambda, const double *w, int G,
                    const double *c_abs, double T_min, double T_max, int n_table,
                    int precision, int device);

/* Free a context and all its device memory (synchronises the device first).
 * NULL is a no-op. */
void dust_ctx_destroy(dust_ctx *ctx);

/* Change the default precision of later dust_solve calls. */
int dust_ctx_set_precision(dust_ctx *ctx, int precision);

/* Kernel layout of later solves at the tensor-core precisions (Eqs. 6-7):
 * fused != 0 runs the absorption contraction and the temperature solve as one
 * kernel whose epilogue solves each cell straight from the tensor-memory
 * accumulator, so the absorbed powers S[C][G] never go to device memory;
 * fused == 0 runs them as two kernels with S in the context's scratch.  T,
 * flags and L are bitwise the same either way; the residual differs by the
 * summation order of the cell's absorbed power (rounding only).  FP32 solves
 * ignore the setting.  Takes the context's lock; returns DUST_OK, or
 * DUST_EINVAL for a NULL context. */
int dust_ctx_set_fused(dust_ctx *ctx, int fused);

/* Kernel layout of the temperature solve and the emission (Eqs. 7-10) in
 * later dust_solve calls: fused != 0 runs them as one warp-specialized kernel
 * where it applies (L or resid wanted), in dust_solve and dust_solve_mass
 * alike.  Its solver warps solve the next tile of cells into shared memory
 * while its emission warps emit the current one.  Where the emission weights
 * do not fit in shared memory beside three tiles of (1/T, n) pairs, the
 * emission runs in grain passes: the fused kernel solves every grain and
 * emits the first pass, a second kernel the others.  T, flags, L and resid
 * are bitwise the same either way.  On by default; ignored when
 * dust_ctx_set_fused is on.  Takes the context's lock; returns DUST_OK, or
 * DUST_EINVAL for a NULL context. */
int dust_ctx_set_fused_emit(dust_ctx *ctx, int fused);

/* Ablation of the split precisions' third product: later tensor-core solves
 * of this context take `products` split products per K step, 3 (the default:
 * J_hi W_hi + J_lo W_hi + J_hi W_lo, FP32 accumulation, Eq. 6) or 2 (the
 * last left out: J is split, W rounded to 16 bits once, a relative error of
 * up to 2^-9 in W).  With 2 the results are not held to the mixed
 * tolerances; the FP32 path ignores the setting.  Takes the context's lock;
 * DUST_EINVAL for a NULL context or another count. */
int dust_ctx_set_split_products(dust_ctx *ctx, int products);

/* Number of kernels that this context's solves (dust_solve and the entry
 * points built on it) have launched since it was created; the server's own
 * launches are counted by dust_server_stats.  Takes the context's lock;
 * DUST_EINVAL for a NULL argument. */
int dust_ctx_launch_count(dust_ctx *ctx, uint64_t *count);

/* Shape and capability query: any output pointer may be NULL.  device_bytes
 * is the device memory the context holds now: its tables and W images, the
 * grown scratch, the host-buffer staging, and the tables or buffers of the
 * optional entry points once they have been used. */
int dust_ctx_info(const dust_ctx *ctx, int *K, int *G, int *n_table, int *precision,
                  int *device, size_t *device_bytes);

/* Solve one batch of cells: the whole hot path of Eqs. 6-10, enqueued on
 * `stream`; returns after enqueueing (the results are ready when the stream
 * reaches that point).
 *
 *  n_cells   number of cells C >= 0 (0 is a no-op).
 *  J         device FP32 [C x ld], row-major: mean intensity J[c,k] at
 *            lambda_k (the paper's I_c,l), >= 0.  Columns K..ld-1 are ignored.
 *  ld        row stride of J and L in elements, ld >= K.  The tensor-core
 *            precisions also need ld % 4 == 0 and J 16-byte aligned (rows
 *            read with the Tensor Memory Accelerator).
 *  n         device FP32 [C x G] row-major: number of grains g in cell c, >= 0.
 *  T         device FP32 [C x G] out: equilibrium temperatures.
 *  L         device FP32 [C x ld] out, or NULL: emission SED L[c,k] (columns
 *            K..ld-1 are not written).  With L = NULL and resid = NULL the
 *            call stops after the temperatures.
 *  resid     device FP64 [C] out, or NULL: per-cell energy-balance residual
 *            r_c = sum_k w_k L[c,k] / (4 pi sum_g n[c,g] Pe[c,g]) - 1, where
 *            Pe = A for solved grains and P_g(T_clamp) for clamped ones; it
 *            vanishes for the exact solution (Eqs. 6, 7 and 10 together).
 *  flags     device uint8 [C x G] out, or NULL: dust_flag per grain.
 *  stream    cudaStream_t as void*.
 *
 * Ownership: all buffers belong to the caller and must stay valid until the
 * stream passes this call.  Outputs must not overlap inputs.  One context may
 * be used by one stream at a time (its scratch buffer is shared).  If the
 * scratch buffer must grow, the call first synchronises `stream`.
 * Errors: DUST_EINVAL (bad pointer / size / alignment), DUST_ENOMEM,
 * DUST_ECUDA (launch failure; asynchronous faults surface at the next
 * synchronisation). */
int dust_solve(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n,
               float *T, float *L, double *resid, uint8_t *flags, void *stream);

/* Same as dust_solve, with an explicit precision for this call only. */
int dust_solve_prec(dust_ctx *ctx, int precision, int64_t n_cells, const float *J, int64_t ld,
                    const float *n, float *T, float *L, double *resid, uint8_t *flags,
                    void *stream);

/* dust_solve on HOST buffers (same shapes; ld applies to J and L): the cells
 * are processed in chunks whose host->device copies, kernels and
 * device->host copies overlap on two internal streams.  Host buffers should
 * be page-locked for the copies to overlap.  Blocks until every output is
 * in host memory.  Device staging buffers are owned by the context. */
int dust_solve_host(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n,
                    float *T, float *L, double *resid, uint8_t *flags);

/* dust_solve without any device allocation (the paper has no counterpart).
 * For callers that may not allocate device memory: device memory owned by a
 * host framework's pool, real-time loops that cannot take cudaMalloc's
 * implicit device synchronisation, memory-capped embeddings.  Same arguments,
 * layouts, ownership and errors as dust_solve with the context's current
 * precision; the caller still provides every input and output buffer.  The
 * scratch (absorbed powers, then the solve's per-grain and per-cell results,
 * the residual's partial sums and the emission order: 4 Gs + 8 G8 + 16 +
 * 8 NKG + 6 bytes per cell and 8 KiB of class counts, Gs = G rounded up to
 * 16, G8 to 8, NKG = K / 8 rounded up; 32 NKG more per cell for contexts
 * whose emission weights do not fit in shared memory at once) lives in one
 * fixed 64 MiB array in the library's device data, which every GPU that
 * loads the library holds until the process exits, so n_cells may not
 * exceed dust_noalloc_max_cells(ctx) (48836 cells for 96 grains and 200
 * wavelengths): larger batches get DUST_EINVAL and must be split.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress, no allocation) and keeps it for the life of the
 * process: make that first call before any stream capture, and do not reset
 * the device (cudaDeviceReset reloads the module; a reset device is not
 * supported).  All calls share the array: calls whose work overlaps on the
 * GPU (different streams, or different contexts on one device) race on it
 * and must be serialised by the caller.  Nothing is left to clear between
 * calls (every scratch value a call reads, it writes first).  Its kernel
 * launches count in dust_ctx_launch_count. */
int dust_solve_noalloc(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n,
                       float *T, float *L, double *resid, uint8_t *flags, void *stream);

/* Largest n_cells dust_solve_noalloc accepts for this context (0 if ctx is NULL). */
size_t dust_noalloc_max_cells(const dust_ctx *ctx);

/* Read and clear the context's device status word (a dust_status: DUST_OK,
 * or DUST_ETIMEOUT if a bounded wait inside a kernel gave up since the last
 * call).  Synchronises the device. */
int dust_ctx_check(dust_ctx *ctx, int *device_status);

/* Per-kernel device timing.  While enabled, every solve on this context
 * records CUDA events on its stream before the absorption kernel (Eq. 6),
 * before the temperature solve (Eq. 7), before the emission and residual
 * (Eqs. 8-10; empty when neither L nor resid is wanted) and after it.
 * dust_ctx_profile_read synchronises on the recorded events and returns the
 * summed milliseconds of each of the three stages and the number of solves
 * since the last read (any output may be NULL), then forgets them. */
int dust_ctx_profile(dust_ctx *ctx, int enable);
int dust_ctx_profile_read(dust_ctx *ctx, double *ms_absorb, double *ms_solve, double *ms_emit,
                          int64_t *n_solves);

/* ------------------------------------------------------------------ serving
 * Continuous batching of solve requests (many snapshots / sub-grids, uneven
 * cell counts, different contexts) on one GPU.  A scheduler thread admits
 * requests in FIFO order (later ones may pass one that does not fit yet)
 * while the summed device footprint of admitted requests (J, n, T, L, resid,
 * flags and the scratch the solve needs) stays within `hbm_budget_bytes` and
 * at most `max_inflight` are active; it then runs them in rounds of work
 * sized by priority, with two rounds in flight: active requests are
 * ranked by remaining Planck terms discounted by their wait (shortest first,
 * large ones not starved); small ones go whole into batched rounds (one
 * launch per kernel for up to 32 of them), large ones run alone a chunk at a
 * time through dust_solve's path.  Requests arriving while the GPU is busy
 * join a round as soon as one retires.  A request's results are bitwise
 * those of dust_solve on the same context with the context's precision at
 * submit time.  The paper
 * processes one grid per call (Section 5); serving has no counterpart there.
 *
 * dust_server_create: the server allocates `hbm_budget_bytes` (>= 1 MiB) of
 * device memory for scratch up front.  max_inflight in [1, 4096].
 * dust_serve_submit: arguments as dust_solve (device buffers, caller-owned,
 * valid until the request finishes).  `stream` is the stream that produced J
 * and n (NULL = the legacy default stream): the call records an event there,
 * and the request's first launch waits for it on the device, so inputs still
 * being written when submit is called are safe and the caller need not
 * synchronise.  Returns a ticket; DUST_EBUSY when the request's footprint
 * exceeds the whole budget (it could never be admitted).
 * dust_serve_poll: *state = 0 queued, 1 active, 2 done, 3 cancelled (and
 * *latency_ms = submit-to-completion time, or the time so far).  A poll that
 * reports 2 or 3 releases the ticket (a later call returns DUST_ENOTFOUND);
 * a failed request returns its error code and is released.
 * dust_serve_wait: blocks up to timeout_ms; DUST_ETIMEOUT if still running,
 * DUST_OK when done (ticket released).
 * dust_serve_cancel: a queued request is dropped; an active one gets no
 * further chunks (chunks already launched finish; its outputs are partial).
 * dust_server_destroy: cancels queued requests, finishes active ones, frees
 * everything. */
typedef struct {
    int64_t submitted, completed, cancelled, failed, queued, active;
    int64_t cells_completed, rounds, launches;
    double p50_ms, p99_ms, max_ms, mean_ms;  /* submit-to-completion latency */
    double span_ms;                          /* first submit to last completion */
    size_t hbm_in_use;                       /* footprint of admitted requests */
} dust_serve_stats;

int dust_server_create(dust_server **out, size_t hbm_budget_bytes, int max_inflight, int device);
int dust_serve_submit(dust_server *srv, dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld,
                      const float *n, float *T, float *L, double *resid, uint8_t *flags,
                      void *stream, uint64_t *ticket);
int dust_serve_poll(dust_server *srv, uint64_t ticket, int *state, double *latency_ms);
int dust_serve_wait(dust_server *srv, uint64_t ticket, double timeout_ms, double *latency_ms);
int dust_serve_cancel(dust_server *srv, uint64_t ticket);
int dust_server_stats(dust_server *srv, dust_serve_stats *out);
/* The round policy (defaults 1e9, 5e9, 1e10, 20): requests with at most
 * small_terms Planck terms (cells x K x G) left go whole into batched rounds
 * of up to batch_terms; larger ones run alone in chunks of about chunk_terms
 * (at least 4096 cells); the ranking divides remaining terms by
 * 1 + wait / age_ms.  Applies from the next round.  DUST_EINVAL for a NULL
 * server or values that are not finite, small_terms < 0, or the others <= 0. */
int dust_server_set_policy(dust_server *srv, double small_terms, double batch_terms, double chunk_terms,
                           double age_ms);
int dust_server_reset_stats(dust_server *srv);
void dust_server_destroy(dust_server *srv);

/* ------------------------------------------------------- dust-mass form
 * The paper writes the grain numbers of a cell as n_s m_d;c (Eqs. 9-10): a
 * fixed number of grains of each kind per unit dust mass times the cell's
 * dust mass.  With n[c,g] = n_g m_c the emission weights can carry n_g, so
 * each Planck term of the emission sum needs one FP32 operation less.
 *
 * dust_ctx_set_grain_numbers: n_g[G] host FP64 >= 0 (not all 0), grains per
 *   unit mass; builds the dust-mass emission tables (synchronous; may be
 *   called again to replace them).
 * dust_solve_mass: as dust_solve with n replaced by m[C] FP32 device, the
 *   cells' dust masses (>= 0); the result is that of dust_solve with
 *   n[c,g] = n_g m_c up to FP32 rounding.  resid is computed per unit mass
 *   (it does not depend on m_c; 0 / 0 does not arise for m_c = 0).
 *   DUST_EINVAL before dust_ctx_set_grain_numbers. */
int dust_ctx_set_grain_numbers(dust_ctx *ctx, const double *n_g);
int dust_solve_mass(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *m, float *T,
                    float *L, double *resid, uint8_t *flags, void *stream);

/* ------------------------------------------------------- self-absorption
 * Dust that is optically thick to its own emission is heated by it as well,
 * so the paper's radiative-transfer code iterates the radiation field and the
 * temperatures together (Section 2).  dust_solve_coupled is the local form of
 * that iteration around the hot path:
 *   J^(0) = J_ext,  J^(i) = J_ext + E (.) L^(i),  L^(i) = emission of a solve on J^(i-1),
 * stopping when max_c max_k |L^(i) - L^(i-1)| / max_k L^(i)[c,k] <= tol, or
 * after max_iters solves (1 <= max_iters <= 10000).
 *
 *  J_ext [C,ld], E [C,ld]  FP32 device: the external mean intensity and the
 *                      coupling E[c,k] >= 0 (the part of the cell's own
 *                      emission L[c,k], in L's units, that returns to J[c,k]).
 *                      The iteration converges when the self-absorbed fraction
 *                      of the emitted power stays below 1.
 *  n, T, L, resid, flags  as dust_solve; T, L, resid and flags hold the last
 *                      solve.  L is required.
 *  *iters_done         solves run; *last_change the last measured change
 *                      (infinite until two solves have run).  Either may be NULL.
 * Synchronises `stream` once per iteration (the stop test is read on the
 * host).  The context keeps a working J and the previous L (8 C ld bytes). */
int dust_solve_coupled(dust_ctx *ctx, int64_t n_cells, const float *J_ext, int64_t ld, const float *E,
                       const float *n, int max_iters, double tol, float *T, float *L, double *resid,
                       uint8_t *flags, int *iters_done, double *last_change, void *stream);

/* ------------------------------------------------------- paper's kernel 3
 * The paper's own temperature method (Section 4.3), kept as an ablation of
 * the table solve on the same GPU.  Per (cell, grain) it runs Newton-Raphson
 * in T on Eq. 7, evaluating P_g(T) and dP_g/dT by the full wavelength sum at
 * every iterate, from the fitted initial guess of Eqs. 11-12 (SI units,
 * log10; floored at 5 K) until |P_g(T) - A| <= 1e-3 A (the paper's 0.1 %
 * energy non-conservation).  Costs two MUFU operations per wavelength per
 * iterate, which is the work the table removes.
 *
 * dust_ctx_set_grain_sizes: a_m[G] host FP64 grain radii in metres (> 0), the
 *   `a` of Eqs. 11-12; required before dust_solve_T_newton.  The guess formula
 *   assumes SI units for lambda, C_abs and J (it was fitted in them).
 * dust_solve_T_newton: J as in dust_solve (the absorbed power uses the
 *   context's precision); T [C,G] FP32 out; iters [C,G] uint8 out (Newton
 *   steps taken, saturating at 255) or NULL; flags [C,G] uint8 out or NULL,
 *   as dust_solve plus DUST_FLAG_NOCONV.  Device pointers, async on `stream`.
 *   Returns DUST_EINVAL when the grain sizes were not set. */
int dust_ctx_set_grain_sizes(dust_ctx *ctx, const double *a_m);
int dust_solve_T_newton(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, float *T,
                        uint8_t *iters, uint8_t *flags, void *stream);

/* ------------------------------------------------ fluctuating grains
 * The temperature probability distribution of small grains, which a single
 * photon heats far above their equilibrium temperature, and its emission.
 * The paper names this calculation as its follow-up (Sections 1 and 6): per
 * grain species and cell a transition-matrix problem between the grain's
 * energy levels, after Guhathakurta & Draine (1989).  The method here:
 *  - enthalpy of grain g: an Einstein solid of N_g atoms with characteristic
 *    temperature theta_g, E_g(T) = 3 N_g k_B theta_g / (exp(theta_g/T) - 1);
 *  - per (cell, grain) M levels E_j = j dE, E_top = (M-1) dE =
 *    min(2 (E_g(T_eq) + h c / lambda_0), E_g(T_max)), T_eq the equilibrium
 *    temperature of Eq. 7 and T_j = E_g^-1(E_j);
 *  - heating: photons of lambda_k are absorbed at 4 pi w_k C[g,k] J[c,k] /
 *    (h c / lambda_k) per second and move the grain to the two levels around
 *    E_i + h c / lambda_k with the weights that keep the energy on average;
 *    landings past the top level end on it (that energy is lost);
 *  - cooling: j -> j-1 only, at 4 pi P_g(max(T_j, T_min)) / dE (P_g of Eq. 7);
 *  - steady state: the probability flux up across each cut between two
 *    levels equals the flux down, solved level by level from P_0;
 *  - emission L[c,k] = 4 pi sum_g n[c,g] sum_j P_j C[g,k] B_k(T_j).
 * FP32 throughout (the equilibrium temperature uses the context's tables
 * with an FP32 absorbed power whatever the context's precision).
 *
 * dust_ctx_set_fluctuating: Gf >= 1 grains (indices into the context's
 *   grains, host int[Gf]), their atom counts n_atoms[Gf] and Einstein
 *   temperatures theta[Gf] (host FP64, > 0), and the number of levels M
 *   (32, 64, 128, 256 or 512).  Synchronous; may be called again to replace
 *   the set.  Needs K <= 2048.
 * dust_solve_fluct: J [C x ld] device FP32 as in dust_solve; n [C x Gf]
 *   device FP32, the numbers of the fluctuating grains (row stride Gf);
 *   L [C x ld] device FP32 out or NULL, their emission (columns K..ld-1 not
 *   written); P [C x Gf x M] device FP32 out or NULL, the normalised level
 *   probabilities; dE [C x Gf] device FP32 out or NULL, the level spacing in
 *   joules.  A cell whose J gives an invalid equilibrium solve (NaN,
 *   negative, infinite) gets NaN in P, dE and L.  Asynchronous on `stream`.
 *   DUST_EINVAL before dust_ctx_set_fluctuating, or when K and M need more
 *   shared memory than one CTA has. */
int dust_ctx_set_fluctuating(dust_ctx *ctx, int Gf, const int *grains, const double *n_atoms,
                             const double *theta, int M);
int dust_solve_fluct(dust_ctx *ctx, int64_t n_cells, const float *J, int64_t ld, const float *n, float *L,
                     float *P, float *dE, void *stream);

/* Failure-detection probe (no counterpart in the paper): one thread waits on
 * an mbarrier phase that nothing completes, through the same bounded wait the
 * tensor-core absorption kernel uses for every pipeline hand-off, with a
 * limit of limit_ms (0 < limit_ms <= 2000; kernels use 2000).  The wait gives
 * up, records DUST_ETIMEOUT in a device status word and returns, so the
 * context stays usable.  *device_status receives the status word (DUST_ETIMEOUT
 * when the bound works) and *elapsed_ms the device time the wait took (either
 * may be NULL).  Synchronises the device.  Returns DUST_EINVAL for a bad
 * device or limit, DUST_ECUDA if the launch failed. */
int dust_diag_wait_timeout(int device, double limit_ms, int *device_status, double *elapsed_ms);

/* Diagnostics (no counterpart in the paper): measured issue rates on `device`
 * of the two pipes the emission kernel uses, MUFU ex2.approx and FP32 FMA, in
 * operations per second (lane operations), from compute-only kernels with 8
 * independent chains per thread.  Used as roofline denominators. */
int dust_diag_throughput(int device, double *ex2_per_s, double *ffma_per_s);

/* Message of the last failure on the calling thread ("" if none). */
const char *dust_last_error(void);

/* Library version string. */
const char *dust_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DUST_H */

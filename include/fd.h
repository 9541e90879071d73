/*
 * fd.h -- C ABI of the GB300 (sm_103a) fractional reaction-diffusion engine.
 *
 * The library advances the explicit Grunwald-Letnikov scheme of Sprouse,
 * MacDonald & Silva for d^g u/dt^g = alpha Lap u + f(u) (eq. fracdiff):
 *
 *     u^{k+1} = u^k + dt f(u^k) + S sum_{(m,c) in sched(k)} c delta^{k-m},
 *     S = alpha dt^g / dx^2,  delta^r = L u^r  (eq. frac_final, eq. deltasimp),
 *
 * where sched(k) is the full memory (m = 0..k, c = psi(g,m); eq. frac_norxn),
 * the short memory (m <= min(L, k); eq. frac_shortmemory) or the adaptive
 * memory (Definitions 3.1/3.2, Proposition 3.1, eq. eq:adapttime).  The GL
 * weights psi(g,m) follow the recurrence of Section 2.1.  f is a cubic
 * polynomial, applied as an explicit term outside the memory sum (the reading
 * of eq. frac_final).
 *
 * Conventions for every entry point:
 *  - Return value: FD_OK (0) or a negative FD_ERR_* code; nothing throws,
 *    asserts or traps across this boundary.  fd_strerror() names a code.
 *  - Device memory: the caller owns every buffer.  The library never calls
 *    cudaMalloc; all device state lives in a caller-provided workspace whose
 *    size fd_workspace_bytes() reports (256-byte aligned base required).
 *    A handle owns host memory only.
 *  - Streams: all device work is enqueued on the cudaStream_t passed to
 *    fd_init (NULL = legacy default stream).  Calls returning only after the
 *    stream drains say so.
 *  - Field layout: N = nx*ny*nz points, row-major with x fastest
 *    (point (x, y, z) at index (z*ny + y)*nx + x), in the problem's state_dtype.
 *  - State pointers may be device or host memory (cudaMemcpyDefault under
 *    unified addressing; pinned host memory keeps copies asynchronous).
 */
#ifndef FD_H
#define FD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FD_OK 0
#define FD_ERR_INVALID_ARG (-1) /* a field or pointer is out of range */
#define FD_ERR_UNSTABLE (-2)    /* S above the von Neumann bound 2^g/(4 ndim) */
#define FD_ERR_WORKSPACE (-3)   /* workspace missing, misaligned or too small */
#define FD_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define FD_ERR_NONFINITE (-5)   /* a NaN/Inf appeared in the state (sticky) */
#define FD_ERR_TIMEOUT (-6)     /* a device-side wait ran past timeout_ms */
#define FD_ERR_STATE (-7)       /* call out of order (e.g. adjoint without tape) */
#define FD_ERR_UNSUPPORTED (-8) /* valid but not implemented combination */

/* ---- enumerations ---- */
enum { FD_BC_DIRICHLET0 = 0, FD_BC_NOFLUX = 1 };           /* ghosts: 0 | mirror u_-1=u_0 */
enum { FD_MEM_FULL = 0, FD_MEM_SHORT = 1, FD_MEM_ADAPTIVE = 2 };
enum { FD_ADAPT_PAPER = 0, FD_ADAPT_PARTITION = 1 };
enum { FD_F64 = 0, FD_F32 = 1, FD_BF16 = 2, FD_F16 = 3 };

#define FD_FLAG_KAHAN 1u           /* compensated FP32 accumulation of the memory sum */
#define FD_FLAG_ALLOW_UNSTABLE 2u  /* skip the stability pre-check */
#define FD_FLAG_KEEP_TAPE 4u       /* keep what fd_adjoint needs (u checkpoints, adjoint buffers) */
#define FD_FLAG_PLAIN_STATE 16u   /* F32 state without the hi/lo compensation (see fd_problem) */
#define FD_FLAG_INJECT_STALL 8u    /* fault injection: the first tile's first update waits on a
                                      counter nothing advances, so the wait times out and the
                                      launch ends with FD_ERR_TIMEOUT (GPU stays usable) */
#define FD_FLAG_STEP_UPDATES 32u   /* time_block: one update unit per step and tile even where
                                      block-long update units would fit (see time_block) */
#define FD_FLAG_FMA_FAR 64u        /* time_block with BF16 / F16 history: multiply the far rows on
                                      the CUDA cores instead of the tensor cores (see time_block) */
#define FD_FLAG_CLOSED_LOOP 128u   /* adaptive memory with feedback from the history (see mem_tau) */

typedef struct fd_problem {
    int ndim;            /* 1, 2 or 3 (3-D: the 7-point analogue of eq. deltasimp) */
    int nx, ny;          /* interior points per axis (ny = 1 in 1-D), N = nx*ny*nz >= 1 */
    double gamma;        /* anomalous exponent, 0 < gamma < 2 */
    double alpha;        /* diffusivity > 0 */
    double dt, dx;       /* time step and grid spacing > 0 */
    int bc;              /* FD_BC_DIRICHLET0 | FD_BC_NOFLUX (cell-centred mirror) */
    double react[4];     /* f(u) = react[0] + react[1] u + react[2] u^2 + react[3] u^3 */
    int mem_mode;        /* FD_MEM_FULL | FD_MEM_SHORT | FD_MEM_ADAPTIVE */
    int mem_L;           /* short memory window in steps: lags 0..min(mem_L, k), mem_L >= 1 */
    int mem_a;           /* adaptive base interval [0, a], a >= 2 */
    int adaptive_rule;   /* FD_ADAPT_PAPER (literal Prop. 3.1) | FD_ADAPT_PARTITION */
    int state_dtype;     /* FD_F64 | FD_F32.  An F32 state is kept as a compensated hi + lo pair
                            (TwoSum update), so per-step increments far below half an ulp of u
                            still accumulate; FD_FLAG_PLAIN_STATE turns this off.  Values read
                            and written through the ABI are the hi part. */
    int hist_dtype;      /* FD_F64 (with F64 state) | FD_F32 | FD_BF16 | FD_F16 (F32 state) */
    int accum_dtype;     /* FD_F64 (with F64 state) | FD_F32 */
    unsigned flags;      /* FD_FLAG_* */
    int max_steps;       /* capacity: total steps this handle may advance (>= 1) */
    int ckpt_every;      /* adjoint checkpoint interval in steps (0 = 200) */
    int timeout_ms;      /* limit on any device-side wait (0 = 10000) */
    /* launch geometry (0 = automatic) */
    int tile_threads;    /* threads per CTA: 64..512, multiple of 32; tile = threads*16/elt bytes */
    int chunk_terms;     /* memory terms per work unit */
    int stage_rows;      /* history rows per TMA stage */
    int stages;          /* stages in the shared-memory ring */
    int ctas_per_sm;     /* resident CTAs per SM for the persistent grid */
    int head_lags;       /* lags 1..head_lags are summed by the per-tile update from rows kept in
                            state precision (0 = 8 for F32/F64 history, 32 for BF16/F16) */
    int nz;              /* points along the third axis when ndim == 3, else 1 */
    int time_block;      /* 0, or 4 / 8 / 16 / 32 / 64: temporally blocked sum (F32 state and
                            accumulation, F32 / BF16 / F16 history, no Kahan; with
                            FD_FLAG_KEEP_TAPE F32 history, full or short memory and 4 or 8).
                            Rows older than the current block are read once per block into
                            time_block accumulators (the Toeplitz structure of eq. frac_norxn);
                            the newest rows are summed per step.  Far rows on the tensor cores
                            (tcgen05, FP32 accumulation in tensor memory, weights split into
                            16-bit hi + lo halves; tile_threads 128 or 256, stage_rows 16 or 32
                            dividing time_block) unless FD_FLAG_FMA_FAR: BF16 / F16 history at
                            16, 32 and 64; F32 history at 32 and 64, stored as FP16 hi + lo
                            planes with a power-of-two scale per (row, tile).  4 / 8 / 16 on
                            F32 history, and BF16 / F16 with FD_FLAG_FMA_FAR, use the CUDA
                            cores.  Low-precision and paired history keep the newest
                            2 time_block rows in FP32 as well.  Adaptive memory: the older rows
                            carry the weights that the medians settle on (psi on the base
                            interval, d psi at a median, 0 between, Definition 3.2) and each
                            step's tail rows (Proposition 3.1) are summed per step.  Same terms,
                            grouped differently; history traffic drops by about time_block
                            (adaptive: all rows are read once per block).  When the tiles are
                            few against the grid (at most a quarter of its CTAs) and the far rows
                            run on the CUDA cores, one unit per tile carries a whole block's
                            updates and keeps the block's newest rows in on-chip memory, unless
                            FD_FLAG_STEP_UPDATES is set. */
    double mem_tau;      /* FD_FLAG_CLOSED_LOOP: threshold tau >= 0 (+inf allowed) of closed-loop
                            adaptive memory, a reading of the Discussion (Section 4: the backward
                            sum's spacing follows the derivative of the past history).  At step k
                            a median m of Proposition 3.1, standing for the d = 2i-1 lags
                            m-(i-1) .. m+(i-1), keeps the weight d psi_m while
                            V = sum_{r = k-m-(i-1)+1}^{k-m+(i-1)} D_r / M_{k-m} < tau, with
                            D_r = max_j |delta^r_j - delta^{r-1}_j| and M_r = max_j |delta^r_j|
                            over the whole field (one schedule for every point); otherwise its d
                            lags are summed one by one with weight psi (M = 0: kept only when
                            V = 0 and tau > 0).  tau = +inf is the open-loop rule; tau = 0 with
                            FD_ADAPT_PARTITION is full memory.  Requires FD_MEM_ADAPTIVE,
                            hist_dtype == state_dtype (F32 or F64), time_block 0 and no
                            FD_FLAG_KEEP_TAPE (FD_ERR_UNSUPPORTED otherwise); single handles only
                            (fd_batch_*, fd_run_batch and fd_run_static: FD_ERR_UNSUPPORTED).
                            Ignored without the flag. */
} fd_problem;

typedef struct fd_handle fd_handle;
typedef struct fd_batch fd_batch;

/* Host, FP64: GL weights psi(g, m) for m = 0..n-1 by the recurrence of Section 2.1
 * (psi(g,0) = 1, psi(g,m) = psi(g,m-1) (m-2+g)/m) and, if dpsi != NULL, their
 * derivative in g by differentiating the recurrence.  n >= 1. */
int fd_weights(double gamma, int64_t n, double *psi, double *dpsi);

/* Host: the memory terms sched(k) as the engine uses them (ascending lag; lag 0
 * included, weight multiplicity 1 or d_i = 2i-1 for an adaptive median).  Writes
 * at most cap entries into lags/mult and the term count into *n.  Defined by
 * eq. frac_final, eq. frac_shortmemory and Proposition 3.1. */
int fd_schedule(const fd_problem *p, int64_t k, int64_t *lags, int64_t *mult, int64_t cap,
                int64_t *n);

/* Host: bytes of device workspace a handle for *p needs (includes the adjoint's
 * buffers when FD_FLAG_KEEP_TAPE is set). */
int fd_workspace_bytes(const fd_problem *p, size_t *bytes);

/* Bind a handle for the scheme of eq. frac_final (Section 2.2) with the memory of p (eq.
 * frac_norxn, eq. frac_shortmemory or Proposition 3.1) to a caller-owned device workspace and
 * stream.  Validates p,
 * checks stability (unless FD_FLAG_ALLOW_UNSTABLE), builds the weight and
 * schedule tables on the host and uploads them.  The handle is at step 0 with
 * an all-zero state until fd_set_state.  Synchronises the stream once. */
int fd_init(const fd_problem *p, void *workspace, size_t ws_bytes, void *cuda_stream,
            fd_handle **out);

/* Copy u^0 (N values of state_dtype; device or host pointer), the initial field of eq. fracdiff,
 * and reset to step 0 (empty history). */
int fd_set_state(fd_handle *h, const void *u0);

/* Enqueue nsteps steps of eq. frac_final, u^{k+1} = u^k + dt f(u^k) + S sum c delta^{k-m}, each
 * appending delta^k = L u^k (eq. deltasimp) to the history (one persistent launch); returns
 * without synchronising.
 * Fails with FD_ERR_STATE if the total would exceed max_steps. */
int fd_step(fd_handle *h, int nsteps);

/* fd_step(nsteps) (eq. frac_final), then copy u^k to u_out (device or host; NULL = no copy),
 * synchronise the stream and return the device status (FD_ERR_NONFINITE,
 * FD_ERR_TIMEOUT, ...). */
int fd_run(fd_handle *h, int nsteps, void *u_out);

/* Enqueue a copy of the current state u^k of eq. frac_final to u_out (device or host). */
int fd_get_state(fd_handle *h, void *u_out);

/* Current step k of the handle. */
int64_t fd_current_step(fd_handle *h);

/* Reverse-time adjoint of J(u^K) for the K steps taken since fd_set_state: the transpose of
 * the linearised eq. frac_final, lambda^r = lambda^{r+1} + dt f'(u^r) lambda^{r+1} + S L^T g^r,
 * g^r = sum_m w_{r+m}(m) psi_m lambda^{r+1+m} (w: lag m's multiplicity in step r+m's schedule).
 * F32 or F64 state/history, FD_FLAG_KEEP_TAPE required.  Short memory transposes its window
 * (delta^r reaches the steps r+m with m <= L, eq. frac_shortmemory); adaptive memory sums every
 * lag with the weight the medians settle on (Definitions 3.1/3.2) and corrects each step's tail
 * terms (Proposition 3.1), which reach only the rows below the longest tail.
 * dJ_duK: N values (state dtype, device or host) = dJ/du^K.  Outputs dJ/du^0
 * (N values, device or host; may be NULL) and the scalar gradients with respect
 * to gamma (through psi and dt^g), alpha and react[0..3] (each may be NULL).
 * Recomputes u between checkpoints every ckpt_every steps.  Synchronises. */
int fd_adjoint(fd_handle *h, const void *dJ_duK, void *dJ_du0, double *dJ_dgamma,
               double *dJ_dalpha, double dJ_dreact[4]);

/* Memory terms (lag, weight) used by the steps run since fd_set_state (or restored by fd_load),
 * lag 0 included: the sum over those steps of |sched(k)| + 1.  Closed-loop adaptive memory
 * (FD_FLAG_CLOSED_LOOP) counts them on the device as the steps run (synchronises the stream);
 * the other modes take them from the schedule.  The count the paper compares its memory forms by
 * (Section 3.2). */
int fd_memory_terms(fd_handle *h, int64_t *terms);

/* Sticky device status of the last launches (synchronises the stream). */
int fd_get_status(fd_handle *h);

/* Where a bounded device wait gave up (after FD_ERR_TIMEOUT), for diagnosis; the paper has
 * no counterpart.  info[0] is the site: 0 none, 1 blocked far unit waiting for its history
 * rows, 2 blocked far unit's bulk copy, 3 blocked update waiting for the far count, 4 blocked
 * update waiting for its own rows, 5 blocked update waiting for a halo tile, 6 per-step chunk
 * waiting for its rows, 7 per-step chunk's bulk copy, 8 per-step fixup waiting for a halo
 * tile, 9 the stall injected by FD_FLAG_INJECT_STALL, 10 blocked far unit waiting for the
 * previous chunk's running sum, 11 tensor-core far unit waiting for a copy, its coefficient
 * block or its MMAs (operands as for site 2), 12 near unit waiting for the previous block's
 * rows, 13 mid unit waiting for its block's earlier rows, 14 closed-loop chunk waiting for its
 * step's decisions (operands: step, tile, chunk, the decision word read, the step + 1 it waits for).
 * info[1..6] are the site's operands
 * (step or block, tile, the counter target and the value last read, the launch's first step;
 * site 2 packs pairs into the high and low 32 bits), info[7] the CTA.  Only the first failure
 * since fd_set_state is kept.  Synchronises the stream. */
int fd_get_error_info(fd_handle *h, int64_t info[8]);

/* Checkpoint of a handle at its current step k, for resuming a run of eq. frac_final later
 * (the paper has no counterpart): the step count, u^k (with the compensation part of an F32
 * state), the history rows written so far (both planes where the history keeps two), the newest
 * rows kept in state precision and the row scales.  Partial sums are not saved: every launch
 * recomputes those of the blocks it starts in.  fd_save_bytes gives the size; fd_save writes it to
 * buf (host or device memory, `bytes` at least that size) and synchronises the stream; fd_load
 * restores it into a handle initialised for the same problem and launch geometry (the stored
 * geometry is checked: FD_ERR_INVALID_ARG on a mismatch or a short buffer), after which fd_step /
 * fd_run continue from step k with the bits an uninterrupted run gives.  Handles with
 * FD_FLAG_KEEP_TAPE: FD_ERR_UNSUPPORTED. */
int fd_save_bytes(fd_handle *h, size_t *bytes);
int fd_save(fd_handle *h, void *buf, size_t bytes);
int fd_load(fd_handle *h, const void *buf, size_t bytes);

/* Release the handle (host memory only; the workspace stays the caller's). */
int fd_destroy(fd_handle *h);

/* Launch geometry the handle resolved (for tuning and reports). */
typedef struct fd_geometry {
    int tile_threads, tile_points, tiles, chunk_terms, stage_rows, stages, ctas_per_sm, grid;
    int head_lags;
    int64_t units_total;     /* work units for max_steps steps */
    int64_t hist_rows_total; /* sum_k n(k): history rows read over max_steps steps (lags >= 1) */
    int64_t terms_total;     /* sum_k N (n(k) + 1): GL terms over max_steps steps, lag 0 included */
    int64_t stream_rows_total; /* history rows the chosen kernel reads over max_steps steps: equal
                                  to hist_rows_total per step; with time_block, far rows once per
                                  block plus every step's newest (head) rows */
    int time_block;
    int block_updates;       /* time_block: 1 when one unit per tile carries a whole block's updates */
    int far_tensor_cores;    /* time_block: 1 when the far rows are multiplied on the tensor cores */
    int64_t head_rows_total; /* time_block: of stream_rows_total, the rows of the newest 2 time_block
                                steps that the update units read (FP32, also for 16-bit history) */
    int64_t smem_bytes;      /* dynamic shared memory per CTA */
} fd_geometry;
int fd_get_geometry(fd_handle *h, fd_geometry *g);

/* ---- batches: many independent instances in one persistent launch ----
 * Each instance is its own problem of eq. frac_final (own grid, gamma, alpha, f, memory and step
 * count).  Instance i runs probs[i].max_steps steps (a batch takes each instance's step count
 * from its max_steps, not from a separate array); all instances share one device
 * work queue ordered by step, so uneven sizes and step counts balance across
 * the GPU.  The launch is recorded once as a CUDA graph (workspace reset +
 * persistent kernel) and replayed by fd_batch_run.  Histories and geometry
 * follow each problem's fields; all instances must share state/history/accum
 * dtypes and flags. */
int fd_batch_workspace_bytes(const fd_problem *probs, int count, size_t *bytes);
int fd_batch_init(const fd_problem *probs, int count, void *workspace, size_t ws_bytes,
                  void *cuda_stream, fd_batch **out);
int fd_batch_set_state(fd_batch *b, int i, const void *u0);   /* device or host */
int fd_batch_run(fd_batch *b);                                 /* enqueue all steps */
int fd_batch_get_state(fd_batch *b, int i, void *u_out);       /* enqueue copy of u^{K_i} */
int fd_batch_get_status(fd_batch *b);                          /* synchronises */
int fd_batch_get_geometry(fd_batch *b, int i, fd_geometry *g);  /* instance i's resolved geometry */
int fd_batch_destroy(fd_batch *b);

/* One-shot batch of eq. frac_final instances: init, set u_io[i] as u^0, run probs[i].max_steps
 * steps, write u^{K_i} back to u_io[i] (device or host pointers), synchronise, destroy. */
int fd_run_batch(const fd_problem *probs, int count, void *const *u_io, void *workspace,
                 size_t ws_bytes, void *cuda_stream);

const char *fd_strerror(int code);

/* ---- allocation-free forward run ----
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory at all (a plugin inside a host application that owns the GPU's
 * allocator and passes in only a stream, or a control loop that must not allocate after it
 * starts).  fd_run_static advances nsteps steps from u0 (N values of state_dtype, device or
 * host) and writes u^nsteps to u_out (device or host), using the same engine kernel as fd_run
 * but with all scratch -- state buffers, delta history, partial sums, counters and the weight /
 * schedule tables -- taken from one static device array of FD_STATIC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine, and uses no host heap.
 *  - Problems needing more scratch than FD_STATIC_SCRATCH_BYTES are rejected with
 *    FD_ERR_WORKSPACE before any device work.  p->max_steps is ignored (nsteps is the length);
 *    FD_FLAG_KEEP_TAPE is rejected with FD_ERR_UNSUPPORTED (forward only).
 *  - Each call looks up the array's address on the current device (cudaGetSymbolAddress), so
 *    the call works on whichever device is current and after a context reset.
 *  - Every call shares the one array and overwrites what the previous call left in it; calls
 *    whose work overlaps on the GPU (other streams, other host threads) race and must be
 *    serialised by the caller.
 *  - Synchronises the stream; returns FD_OK or the device status (as fd_run). */
#define FD_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
int fd_run_static(const fd_problem *p, const void *u0, int nsteps, void *u_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FD_H */

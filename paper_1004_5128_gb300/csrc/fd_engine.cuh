// fd_engine.cuh -- persistent dataflow engine for the Grunwald-Letnikov memory sum.
//
// One launch advances one or many problem instances by a range of steps of
// the explicit scheme (eq. frac_final):
//     u^{k+1} = u^k + dt f(u^k) + S ( delta^k + H^k ),
//     H^k     = sum_{(m,c) in sched(k), m >= 1} c delta^{k-m}        (the memory sum)
// with delta^r = L u^r (eq. deltasimp) kept in a history ring, one row per step.
//
// Work decomposition.  For each (instance, step k) the N points are cut into
// tiles of P points (P = threads x one 16-byte vector) and the memory terms of
// sched(k) (ascending lag) into chunks of R terms.  A work unit is one
// (tile, chunk); units are numbered step-major and claimed from a global
// counter, so every unit waits only on units with smaller numbers and the
// persistent grid cannot deadlock.  Within a step the oldest-lag chunks come
// first; the chunk holding lag 1 (the only one needing the row written by the
// previous step) comes last.
//
// Per unit: the CTA's elected thread streams the chunk's history row segments
// (one cp.async.bulk per row, 16-byte aligned, no multicast) into a ring of
// shared-memory stages completed by mbarrier transaction counts; every thread
// owns one 16-byte vector column and accumulates c * row (optionally Kahan)
// from shared memory.  A unit writes its partial sum; the last unit of a
// (step, tile) to arrive (atomic arrival counter) sums the partials in fixed
// chunk order (deterministic), evaluates the stencil on u^k, appends
// delta^k to the history, applies the update and publishes the tile's step
// counter.  Dependencies are per tile: a unit needs the rows it reads, the
// fixup needs the halo tiles of u^k.  Every spin-wait is bounded by a
// globaltimer limit after which the launch records FD_ERR_TIMEOUT and exits.
//
// Adjoint mode (ADJ) runs the same machinery on the reverse-time recursion
//     mu^{r+1} = L lambda^{r+1},
//     lambda^r = lambda^{r+1} + dt f'(u^r) lambda^{r+1} + S sum_{m>=0} psi_m mu^{r+1+m}
// (L is symmetric for both boundary rules, so L^T g^r = sum psi_m L lambda),
// with a second accumulator for psi' = d psi / d gamma and per-tile FP64 dot
// products for the parameter gradients.
//
// Closed-loop adaptive memory (forward): each update also publishes its tile's
// share of the row maxima D_k = max |delta^k - delta^{k-1}| and M_k = max |delta^k|;
// the update completing row r on the last tile decides step r + a + 1 for the
// field (which medians stand for their increments); units stream their terms as
// scheduled and add correction passes for the expanded increments.
#pragma once

#include "fd_common.cuh"

namespace fdk {

struct Unit {
    int valid, inst, k, tile, chunk, C, tau0, tau1;
    int4 sc;
    int last;  // set for the arrival election
    unsigned long long clw;  // closed loop: the chunk's decision word as read at the claim
};

// Term tau of sched(k) (lags >= 1, ascending): lag and coefficient(s).
template <class TA, bool ADJ>
__device__ __forceinline__ void term_of(const Inst &I, const int4 sc, int tau, int &lag, TA &c, TA &c2)
{
    const TA *psi = reinterpret_cast<const TA *>(I.psi);
    if (tau < sc.x) {
        lag = tau + 1;
        c = psi[lag];
        if (ADJ) c2 = reinterpret_cast<const TA *>(I.dpsi)[lag];
    } else if (tau < sc.x + sc.y) {
        const int g = tau - sc.x;
        lag = I.g_lag[g];
        c = reinterpret_cast<const TA *>(I.g_coef)[g];
        c2 = TA(0);
    } else {
        lag = sc.z + (tau - sc.x - sc.y);
        c = psi[lag];
        if (ADJ) c2 = reinterpret_cast<const TA *>(I.dpsi)[lag];
    }
}

// Closed-loop adaptive memory: does the median at lag m of step k stand for its increment of d
// lags?  Reads the maxima of rows k-m-(d-1)/2+1 .. k-m+(d-1)/2, which the caller has waited for.
// Ascending rows, FP64, the rule's comparison as written (tau = +inf keeps every median; a zero
// reference keeps it only for zero variation and tau > 0).
__device__ __forceinline__ bool cl_smooth(const Inst &I, int k, int m, int d)
{
    const int h = (d - 1) / 2, r1 = k - m + h;
    const double ref = __ldcg(I.cl_M + (k - m));
    double var = 0.0;
    for (int r = k - m - h + 1; r <= r1; r += 8) {  // eight loads in flight, added in row order
        double x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = (r + i <= r1) ? __ldcg(I.cl_D + r + i) : 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (r + i <= r1) var += x[i];
    }
    if (isinf(I.cl_tau)) return true;
    return (ref > 0.0) ? (var / ref < I.cl_tau) : (var == 0.0 && I.cl_tau > 0.0);
}

template <class TS, class TH, class TA, bool KAHAN, bool ADJ>
__global__ void __launch_bounds__(512, 1) engine_kernel(const Launch L)
{
    constexpr int V = HVec<TH>::V;
    constexpr int PLANES = ADJ ? 2 : 1;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int RS = L.stage_rows, NS = L.stages;
    const int row_bytes = nthr * 16;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *stages = smem;
    TA *coef = reinterpret_cast<TA *>(smem + (size_t)NS * RS * row_bytes);  // per-unit term tables
    TA *coef2 = coef + L.rmax;
    int *toff = reinterpret_cast<int *>(coef2 + L.rmax);                   // history slot per term
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(toff + L.rmax) + 15) & ~uintptr_t(15));
    // closed loop: entry offsets of a unit's terms (rmax + 1), then the per-warp row maxima
    int *eoff = reinterpret_cast<int *>(bars + NS);
    double *clmax = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(eoff + L.rmax + 1) + 7) & ~uintptr_t(7));

    __shared__ Inst I;
    __shared__ Unit U;
    __shared__ int s_cur_inst;
    __shared__ int s_ok, s_ok2;
    __shared__ int s_nexp;    // closed loop: expanded medians of the unit
    __shared__ int s_decide;  // closed loop: the step this update decides for the field, or -1
    __shared__ int s_pipe;
    __shared__ float s_red[32];
    __shared__ double s_dred[32][6];

    if (tid == 0) {
        for (int b = 0; b < NS; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_cur_inst = -1;
    }
    __syncthreads();

    uint32_t n_issued = 0, n_used = 0;  // ring counters (identical in all threads)
    int ghint = L.g_begin;
    const long long u_base = L.g_off[L.g_begin];
    const long long u_end = L.g_off[L.g_end];
    unsigned long long next = 0;
    if (tid == 0) next = atomicAdd(L.queue, 1ull);

    for (;;) {
        // ---------------------------------------------------------- claim
        if (tid == 0) {
            const long long u = u_base + (long long)next;
            int ok = (u < u_end) && (ld_volatile(L.err) == ERR_NONE);
            if (ok) {
                next = atomicAdd(L.queue, 1ull);
                const int g = find_group(L.g_off, ghint, L.g_end, u);
                ghint = g;
                const int2 gi = L.g_info[g];
                if (gi.x != s_cur_inst) {
                    I = L.inst[gi.x];
                    s_cur_inst = gi.x;
                }
                const long long local = u - L.g_off[g];
                const int C = (int)((L.g_off[g + 1] - L.g_off[g]) / I.T);
                U.inst = gi.x;
                U.k = gi.y;
                U.tile = (int)(local % I.T);
                U.C = C;
                U.chunk = C - 1 - (int)(local / I.T);
                const int4 sc = I.sched[gi.y];
                U.sc = sc;
                const int n = sc.x + sc.y + (sc.w >= sc.z ? sc.w - sc.z + 1 : 0);
                U.tau0 = min(I.head, sc.x) + U.chunk * I.R;
                U.tau1 = min(n, U.tau0 + I.R);
                // dependencies: rows read (newest row k - lag_min) and partial-buffer reuse
                const int rel = gi.y - L.k0;
                int need = 0;
                if (U.tau1 > U.tau0) {
                    int lag;
                    TA c, c2;
                    term_of<TA, ADJ>(I, sc, U.tau0, lag, c, c2);
                    const int r_hi = gi.y - lag;
                    if (r_hi >= L.k0) need = r_hi - L.k0 + 1;
                }
                // partial rows of step k-npar consumed by its fixup
                if (C > 1 && rel - I.npar + 1 > need) need = rel - I.npar + 1;
                // closed loop: the chunk's decision word, read now (relaxed) and used after the
                // chunk has streamed, so that its latency hides behind the waits and copies
                unsigned long long clw = 0;
                if (!ADJ && I.cl_D && U.tau0 < sc.x + sc.y && U.tau1 > sc.x)
                    clw = ld_relaxed_u64(I.cl_word + (size_t)(gi.y % I.cl_slots) * I.maxC + U.chunk);
                if (need > 0) {
                    const int w = wait_until(&I.done[U.tile], (unsigned)need, L, 512);
                    if (w < 0) note_failure(L, 6, gi.y, U.tile, need, ld_acquire(&I.done[U.tile]), L.k0, 0);
                    if (w <= 0) ok = 0;
                }
                U.clw = clw;
            }
            U.valid = ok;
        }
        __syncthreads();
        if (!U.valid) break;

        const int tile = U.tile, k = U.k, C = U.C;
        const int tau0 = U.tau0, tau1 = U.tau1;
        const int nterm = tau1 - tau0;
        const int j0 = tile * I.P + tid * V;  // first point of this thread's vector
        long long tile_bytes = (long long)min(I.P, I.N - tile * I.P) * (long long)sizeof(TH);
        tile_bytes = (tile_bytes + 15) & ~15ll;

        TA acc[V], cmp[V], acc2[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = cmp[v] = acc2[v] = TA(0);

        // ------------------------------------------------- stream the chunk
        // Pass 0 streams the chunk's terms as scheduled.  Closed loop: then the chunk's decision
        // word (read at the claim; acquired again if it was not yet written or shows expanded
        // medians) says whether every median stands for its increment.  Where one does not, the
        // step's expanded lengths give eoff[0..nterm] (warp 0 prefix-sums them) and correction
        // passes stream, in rounds of at most rmax entries, each such increment's lags with weight
        // psi (psi_m - d psi_m at the median itself, whose d psi_m pass 0 already added).
        const bool cl_chunk = !ADJ && I.cl_D && nterm > 0 && tau0 < U.sc.x + U.sc.y && tau1 > U.sc.x;  // holds medians
        const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
        int aborted = 0, ncorr = 0, nexp = 0;
        for (int pass = 0, e0 = 0;;) {
            const int ne = pass ? min(L.rmax, ncorr - e0) : nterm;
            const int nst = (ne + RS - 1) / RS;
            // term tables of this round, built by the whole CTA: coefficient(s) and history slot
            for (int t = tid; t < ne; t += nthr) {
                int lag;
                TA c, c2;
                if (!pass) {
                    term_of<TA, ADJ>(I, U.sc, tau0 + t, lag, c, c2);
                } else {
                    const int e = e0 + t;
                    int lo = 0, hi = nterm;  // the term holding entry e: eoff[lo] <= e < eoff[lo + 1]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (eoff[mid] <= e) lo = mid;
                        else hi = mid;
                    }
                    int m;
                    TA cm;
                    term_of<TA, ADJ>(I, U.sc, tau0 + lo, m, cm, c2);
                    const int cnt = eoff[lo + 1] - eoff[lo];
                    lag = m - (cnt - 1) / 2 + (e - eoff[lo]);
                    c = reinterpret_cast<const TA *>(I.psi)[lag];
                    if (lag == m) c -= cm;
                }
                const int slot = (k - lag) % I.cap;
                if (I.hscale) c = c * (TA)__ldcg(I.hscale + (size_t)slot * I.T + tile);
                coef[t] = c;
                if (ADJ) coef2[t] = c2;
                toff[t] = slot;
            }
            __syncthreads();
            // Stage s of this round into ring slot `slot` % NS, by warp s mod (warps), one lane per
            // row: the copies of a stage go out together and the issue work rotates over the warps
            // instead of delaying one warp at every stage barrier.  All lanes of the warp call it.
            auto issue = [&](int s, uint32_t slot) {
                const int b = (int)(slot % (uint32_t)NS);
                const int t0 = s * RS;
                const int t1 = min(ne, t0 + RS);
                if (lane == 0) mbar_expect_tx(&bars[b], (uint32_t)(tile_bytes * (t1 - t0)));
                __syncwarp();
                const char *col = I.hist + (size_t)tile * I.P * sizeof(TH);
                for (int t = t0 + lane; t < t1; t += 32)
                    bulk_g2s(stages + ((size_t)b * RS + (t - t0)) * row_bytes, col + (size_t)toff[t] * I.pitch,
                             (uint32_t)tile_bytes, &bars[b]);
            };
            // every lane that issues copies orders the rows it acquired before the async proxy
            if (lane < RS) fence_proxy_async_global();
            {
                const int pre = min(NS, nst);
                for (int s = 0; s < pre; ++s)
                    if (warp == s % nwarp) issue(s, n_issued + (uint32_t)s);
                n_issued += (uint32_t)pre;
            }
            for (int s = 0; s < nst; ++s) {
                const int b = (int)(n_used % (uint32_t)NS);
                const uint32_t par = (n_used / (uint32_t)NS) & 1u;
                int tmo = 0;
                if (!mbar_try_wait(&bars[b], par)) {
                    const long long t0 = globaltimer();
                    while (!mbar_try_wait(&bars[b], par)) {
                        if (globaltimer() - t0 > L.timeout_ns) {
                            if (atomicCAS(L.err, ERR_NONE, ERR_PIPE) == ERR_NONE) note_failure(L, 7, U.k, U.tile, 0, 0, 0, 0);
                            tmo = 1;  // the copy is still owed to this slot; see below
                            break;
                        }
                    }
                }
                const int rows = tmo ? 0 : min(RS, ne - s * RS);
                const unsigned char *base = stages + (size_t)b * RS * row_bytes + (size_t)tid * 16;
                for (int r = 0; r < rows; ++r) {
                    const uint4 w = *reinterpret_cast<const uint4 *>(base + (size_t)r * row_bytes);
                    TA x[V];
                    HVec<TH>::unpack(w, x);
                    const TA c = coef[s * RS + r];
                    if (KAHAN) {
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const TA y = c * x[v] - cmp[v];
                            const TA t = acc[v] + y;
                            cmp[v] = (t - acc[v]) - y;
                            acc[v] = t;
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = fma(c, x[v], acc[v]);
                    }
                    if (ADJ) {
                        const TA c2 = coef2[s * RS + r];
#pragma unroll
                        for (int v = 0; v < V; ++v) acc2[v] = fma(c2, x[v], acc2[v]);
                    }
                }
                // slot b fully read by every thread.  A stage that any thread gave up on stops the
                // unit: nothing more is issued, and the stage stays owed (n_used not advanced) for
                // the drain below.
                if (__syncthreads_or(tmo)) {
                    aborted = 1;
                    break;
                }
                ++n_used;
                if (s + NS < nst) {
                    if (warp == (s + NS) % nwarp) issue(s + NS, n_issued);
                    ++n_issued;
                }
            }
            if (aborted) break;
            if (!pass) {
                if (!cl_chunk) break;
                if (tid == 0) {
                    const unsigned gen = (unsigned)k + 1u;
                    unsigned long long w = U.clw;
                    if ((unsigned)(w >> 32) != gen || (unsigned)w != 0u) {
                        // not decided when claimed, or expanded medians to read: acquire the word
                        const unsigned long long *wp = I.cl_word + (size_t)(k % I.cl_slots) * I.maxC + U.chunk;
                        w = wait_word(wp, gen, L);
                        if (!w) note_failure(L, 14, k, tile, U.chunk, (long long)ld_acquire_u64(wp), gen, 0);
                    }
                    s_nexp = (int)(unsigned)w;  // 0 after a failed wait: the launch ends with its error
                }
                __syncthreads();
                nexp = s_nexp;
                if (!nexp) break;
                {
                    const unsigned char *cnt = I.cl_cnt + (size_t)(k % I.cl_slots) * I.cl_gmax;
                    for (int t = tid; t < nterm; t += nthr) {
                        const int tau = tau0 + t;
                        eoff[t + 1] = (tau >= U.sc.x && tau < U.sc.x + U.sc.y) ? (int)__ldcg(cnt + (tau - U.sc.x)) : 0;
                    }
                }
                __syncthreads();
                if (tid < 32) {  // exclusive offsets of the correction entries; expanded medians
                    const int seg = (nterm + 31) / 32, a = min(nterm, tid * seg), b = min(nterm, a + seg);
                    int sum = 0, cntx = 0;
                    for (int t = a; t < b; ++t) {
                        sum += eoff[t + 1];
                        cntx += eoff[t + 1] > 0;
                    }
                    int pre = sum;  // inclusive warp scan of the segment sums
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, pre, o);
                        if (tid >= o) pre += y;
                    }
                    int run = pre - sum;
                    for (int t = a; t < b; ++t) {
                        run += eoff[t + 1];
                        eoff[t + 1] = run;
                    }
                    cntx = __reduce_add_sync(0xffffffffu, cntx);
                    if (tid == 0) {
                        eoff[0] = 0;
                        s_nexp = cntx;
                    }
                }
                __syncthreads();
                ncorr = eoff[nterm];
                nexp = s_nexp;
                pass = 1;
                e0 = 0;
            } else {
                e0 += ne;
                if (e0 >= ncorr) break;
                __syncthreads();  // this round's tables are read
            }
        }
        // closed loop: terms used = the chunk's terms, each expanded median counted d times
        if (!ADJ && I.cl_D && tid == 0 && tile == 0 && nterm > 0 && !aborted)
            atomicAdd(I.cl_terms, (unsigned long long)(nterm + ncorr - nexp));
        if (tid == 0) s_pipe = aborted || (ld_volatile(L.err) == ERR_PIPE);
        __syncthreads();
        if (s_pipe) {
            // A stage never completed: drain what is owed (bounded) and stop.
            if (tid == 0) {
                const long long t0 = globaltimer();
                while (n_used < n_issued && globaltimer() - t0 < L.timeout_ns) {
                    const int b = (int)(n_used % (uint32_t)NS);
                    if (mbar_try_wait(&bars[b], (n_used / (uint32_t)NS) & 1u)) ++n_used;
                }
            }
            break;
        }
        if (KAHAN) {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] -= cmp[v];
        }

        // ------------------------------------------- partials and arrival
        const int par = k % I.npar;
        auto prow = [&](int c, int plane) -> TA * {
            return reinterpret_cast<TA *>(I.part + ((size_t)((par * I.maxC + c) * PLANES + plane)) * I.part_pitch);
        };
        if (C > 1) {
            if (j0 < I.N) {
                TA *p0 = prow(U.chunk, 0) + j0;
#pragma unroll
                for (int v = 0; v < V; ++v) p0[v] = acc[v];
                if (ADJ) {
                    TA *p1 = prow(U.chunk, 1) + j0;
#pragma unroll
                    for (int v = 0; v < V; ++v) p1[v] = acc2[v];
                }
            }
            // CTA barrier, then one acq_rel atomic: its release half is cumulative over every
            // thread's partial-row stores ordered before the barrier
            __syncthreads();
            if (tid == 0) {
                unsigned *ar = &I.arrive[par * I.T + tile];
                const unsigned old = atom_add_acq_rel(ar, 1u);
                U.last = (old == (unsigned)(C - 1));
                if (U.last) *ar = 0u;  // reset for step k+npar (published by the done release below)
            }
            __syncthreads();
            if (!U.last) continue;
        }

        // ------------------------------------------------------- fixup
        // Phase A, before the halo is needed: the partial rows (this unit is the step's last
        // arrival, so they are complete) and head lags h..2 (this tile's rows up to k-2, i.e. its
        // own step k-2).  Phase B waits for u^k on the halo tiles, adds lag 1 and updates.  The
        // summation order is that of one pass: partials by chunk, then lags h..1.
        const int rel = k - L.k0;
        if (tid < 32) {
            int ok = 1;
            if (tid == 0 && rel > 1) {
                const int w = wait_until(&I.done[tile], (unsigned)(rel - 1), L, 32);
                if (w < 0) note_failure(L, 8, k, tile, tile, rel - 1, ld_acquire(&I.done[tile]), L.k0);
                ok = w > 0;
            }
            ok = __all_sync(0xffffffffu, ok);
            if (tid == 0) s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;

        TA H[V], H2[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            H[v] = TA(0);
            H2[v] = TA(0);
        }
        if (C > 1) {
            if (j0 < I.N) {
                // partial rows in fixed chunk order (this unit's own row holds the same bits as
                // its registers); 16-byte loads, 4 rows at a time so the L2 round trips overlap
                constexpr int B = 4;
                for (int c0 = 0; c0 < C; c0 += B) {
                    TA w[B][V], w2[B][V];
#pragma unroll
                    for (int i = 0; i < B; ++i)
                        if (c0 + i < C) {
                            load_vec<TA, V>(prow(c0 + i, 0) + j0, w[i]);
                            if (ADJ) load_vec<TA, V>(prow(c0 + i, 1) + j0, w2[i]);
                        }
#pragma unroll
                    for (int i = 0; i < B; ++i)
                        if (c0 + i < C) {
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                H[v] += w[i][v];
                                if (ADJ) H2[v] += w2[i][v];
                            }
                        }
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                H[v] = acc[v];
                H2[v] = acc2[v];
            }
        }

        // head lags h..1 from the most recent rows (state precision), fixed order
        const int hh = min(I.head, U.sc.x);
        const TA *psi = reinterpret_cast<const TA *>(I.psi);
        const TA *dpsi = reinterpret_cast<const TA *>(I.dpsi);
        TA hs[V], hc[V], hs2[V];
#pragma unroll
        for (int v = 0; v < V; ++v) hs[v] = hc[v] = hs2[v] = TA(0);
        auto head_row = [&](int m) -> const TS * {
            return reinterpret_cast<const TS *>(I.hring + (size_t)((k - m) % I.hring_cap) * I.hring_pitch) + j0;
        };
        auto head_add = [&](int m, const TS *x) {
            const TA c = psi[m];
            if (KAHAN) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const TA y = c * (TA)x[v] - hc[v];
                    const TA t = hs[v] + y;
                    hc[v] = (t - hs[v]) - y;
                    hs[v] = t;
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) hs[v] = fma(c, (TA)x[v], hs[v]);
            }
            if (ADJ) {
                const TA c2 = dpsi[m];
#pragma unroll
                for (int v = 0; v < V; ++v) hs2[v] = fma(c2, (TA)x[v], hs2[v]);
            }
        };
        if (j0 < I.N) {  // lags h..2, several rows in flight
            constexpr int HB = (V > 4) ? 2 : 4;
            int m = hh;
            for (; m - (HB - 1) >= 2; m -= HB) {
                TS x[HB][V];
#pragma unroll
                for (int i = 0; i < HB; ++i) load_vec<TS, V>(head_row(m - i), x[i]);
#pragma unroll
                for (int i = 0; i < HB; ++i) head_add(m - i, x[i]);
            }
            for (; m >= 2; --m) {
                TS x[V];
                load_vec<TS, V>(head_row(m), x);
                head_add(m, x);
            }
        }

        // Phase B: u^k on this tile and its halo tiles (one lane per tile), and row k-1
        if (tid < 32) {
            int ok = 1;
            const int h = (I.ndim == 3) ? I.nx * I.ny : (I.ndim == 2) ? I.nx : 1;
            const int lo = max(0, tile * I.P - h) / I.P;
            const int hi = min(I.N - 1, tile * I.P + I.P - 1 + h) / I.P;
            for (int t = lo + tid; t <= hi && ok; t += 32)
                if (rel > 0) {
                    const int w = wait_until(&I.done[t], (unsigned)rel, L, 32);
                    if (w < 0) note_failure(L, 8, k, tile, t, rel, ld_acquire(&I.done[t]), L.k0);
                    if (w <= 0) ok = 0;
                }
            if (tid == 0 && ok && I.stall && rel == 0 && tile == 0) {
                // fault injection: nothing ever raises a step counter to 2^31
                const int w = wait_until(&I.done[tile], 0x80000000u, L, 512);
                if (w < 0) note_failure(L, 9, k, tile, 0x80000000ll, ld_acquire(&I.done[tile]), L.k0, 0);
                if (w <= 0) ok = 0;
            }
            ok = __all_sync(0xffffffffu, ok);
            if (tid == 0) s_ok2 = ok;
        }
        __syncthreads();
        if (!s_ok2) break;

        // stencil on u^k (eq. deltasimp), ghosts: 0 (Dirichlet) or mirror (no-flux).  Every
        // operand is loaded before any is used: the centre as one vector, x-neighbours inside
        // the vector from it, y/z-neighbours as one vector where the row (plane) length keeps
        // the points in one row (plane) and the vector aligned.
        const TS *uk = reinterpret_cast<const TS *>(I.ubuf[k & 1]);
        TS *un = reinterpret_cast<TS *>(I.ubuf[(k + 1) & 1]);
        const bool mirror = (I.bc == 1);
        const int pl = I.nx * I.ny;
        TS d[V], uc[V], up[V], dn[V], fw[V], bk[V];
        TS xr = TS(0), xl = TS(0);  // x-neighbours of the vector's last and first point
        unsigned inb[V];
        TS x1[V];
        const bool lag1 = (hh >= 1) && (j0 < I.N);
        if (lag1) load_vec<TS, V>(head_row(1), x1);
        grid_masks<V>(I, j0, inb);
#pragma unroll
        for (int v = 0; v < V; ++v) d[v] = uc[v] = up[v] = dn[v] = fw[v] = bk[v] = TS(0);
        if (j0 < I.N) {
            const bool full = (j0 + V <= I.N);
            if (full) {
                load_vec<TS, V>(uk + j0, uc);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (j0 + v < I.N) uc[v] = __ldcg(uk + j0 + v);
            }
            // x-neighbours inside the vector come from uc (a set mask bit means the same row)
            if (inb[V - 1] & 1u) xr = __ldcg(uk + j0 + V);
            if (inb[0] & 2u) xl = __ldcg(uk + j0 - 1);
            auto vert = [&](TS *o, unsigned bit, int off, int len) {
                if (full && len % V == 0) {  // the V points share a row (plane): one mask, one vector
                    if (inb[0] & bit) load_vec<TS, V>(uk + j0 + off, o);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (inb[v] & bit) o[v] = __ldcg(uk + j0 + v + off);
                }
            };
            if (I.ndim >= 2) {
                vert(up, 4u, I.nx, I.nx);
                vert(dn, 8u, -I.nx, I.nx);
            }
            if (I.ndim == 3) {
                vert(fw, 16u, pl, pl);
                vert(bk, 32u, -pl, pl);
            }
        }
        if (lag1) head_add(1, x1);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            H[v] += KAHAN ? (hs[v] - hc[v]) : hs[v];
            if (ADJ) H2[v] += hs2[v];
        }
        if (ADJ) adjoint_tail<TS, TA, V>(I, k, j0, H, H2);
        float amax = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (j0 + v >= I.N) continue;
            const TS c = uc[v];
            const TS g = mirror ? c : TS(0);
            const unsigned m = inb[v];
            const TS r = (m & 1u) ? ((v + 1 < V) ? uc[(v + 1) % V] : xr) : g;
            const TS l = (m & 2u) ? ((v > 0) ? uc[(v + V - 1) % V] : xl) : g;
            if (I.ndim == 1) {
                d[v] = r - TS(2) * c + l;
            } else {
                const TS u_ = (m & 4u) ? up[v] : g, dn_ = (m & 8u) ? dn[v] : g;
                if (I.ndim == 2) {
                    d[v] = r + l - TS(4) * c + u_ + dn_;
                } else {
                    // 7-point analogue of eq. deltasimp for the N-dimensional x of eq. fracdiff
                    const TS f_ = (m & 16u) ? fw[v] : g, b_ = (m & 32u) ? bk[v] : g;
                    d[v] = r + l - TS(6) * c + u_ + dn_ + f_ + b_;
                }
            }
            amax = fmaxf(amax, fabsf((float)d[v]));
        }

        // closed loop (forward only): this tile's share of the row maxima D_k and M_k (published
        // with the step)
        if (!ADJ && I.cl_D) {
            double dm = 0.0, mm = 0.0;
            if (j0 < I.N) {
                TS xp[V];
#pragma unroll
                for (int v = 0; v < V; ++v)
                    xp[v] = lag1 ? x1[v] : (k >= 1 && j0 + v < I.N) ? __ldcg(head_row(1) + v) : TS(0);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (j0 + v < I.N) {
                        mm = fmax(mm, fabs((double)d[v]));
                        if (k >= 1) dm = fmax(dm, fabs((double)d[v] - (double)xp[v]));
                    }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                mm = fmax(mm, __shfl_xor_sync(0xffffffffu, mm, o));
            }
            if ((tid & 31) == 0) {
                clmax[2 * (tid >> 5)] = dm;
                clmax[2 * (tid >> 5) + 1] = mm;
            }
        }

        // history row k (FP16: per (row, tile) power-of-two scale)
        float hsc = 1.f;
        const int slot = k % I.cap;
        if (I.hist_write) {
            if (I.hscale) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                if ((tid & 31) == 0) s_red[tid >> 5] = amax;
                __syncthreads();
                if (tid == 0) {
                    float m = 0.f;
                    for (int w = 0; w < (nthr + 31) / 32; ++w) m = fmaxf(m, s_red[w]);
                    int e = 0;
                    if (m > 0.f && isfinite(m)) {
                        int ex;
                        frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
                        e = max(-100, min(100, 15 - ex));
                    }
                    s_red[0] = ldexpf(1.f, e);
                    I.hscale[(size_t)slot * I.T + tile] = ldexpf(1.f, -e);
                }
                __syncthreads();
                hsc = s_red[0];
            }
            if (j0 < I.N) {
                TS dz[V];
#pragma unroll
                for (int v = 0; v < V; ++v) dz[v] = (j0 + v < I.N) ? d[v] : TS(0);
                *reinterpret_cast<uint4 *>(I.hist + (size_t)slot * I.pitch + (size_t)j0 * sizeof(TH)) =
                    HVec<TH>::pack(dz, hsc);
                if (I.hring_sep)
                    store_vec<TS, V>(reinterpret_cast<TS *>(I.hring + (size_t)(k % I.hring_cap) * I.hring_pitch) + j0, dz);
            }
        }

        // update (eq. frac_final; adjoint: reverse-time recursion)
        const TS S = (TS)I.S, dt = (TS)I.dt;
        const TS r0 = (TS)I.react[0], r1 = (TS)I.react[1], r2 = (TS)I.react[2], r3 = (TS)I.react[3];
        double dl[6] = {0, 0, 0, 0, 0, 0};
        bool bad = false;
        const TS *ua = nullptr;
        if (ADJ) ua = reinterpret_cast<const TS *>(I.uadj) + (size_t)((I.adj_K - 1 - k) - I.uadj_r0) * I.N;
        const TS *lo_k = I.ulo[0] ? reinterpret_cast<const TS *>(I.ulo[k & 1]) : nullptr;
        TS *lo_n = I.ulo[0] ? reinterpret_cast<TS *>(I.ulo[(k + 1) & 1]) : nullptr;
        const bool tape_row = I.tape && (k + 1 - I.tape_k0) >= 0 && ((k + 1 - I.tape_k0) % I.tape_every) == 0 &&
                              ((k + 1 - I.tape_k0) / I.tape_every) < I.tape_rows;
        TS *tp = tape_row ? reinterpret_cast<TS *>(I.tape) + (size_t)((k + 1 - I.tape_k0) / I.tape_every) * I.N
                          : nullptr;
        TS nvv[V], nlv[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = j0 + v;
            nvv[v] = nlv[v] = TS(0);
            if (j >= I.N) continue;
            const TA G = (TA)d[v] + H[v];  // psi_0 delta^k + memory sum
            TS nv, inc;
            const TS x = uc[v];
            if (!ADJ) {
                const TS f = r0 + x * (r1 + x * (r2 + x * r3));
                inc = dt * f + S * (TS)G;
            } else {
                const TS ur = __ldcg(ua + j);
                const TS fp = r1 + ur * (TS(2) * r2 + ur * TS(3) * r3);
                inc = dt * fp * x + S * (TS)G;
            }
            if (lo_k) {
                // state kept as hi + lo: TwoSum of hi and (increment + lo) (Knuth), so increments
                // far below half an ulp of the state still accumulate
                const TS y = inc + __ldcg(lo_k + j);
                const TS sum = x + y;
                const TS bb = sum - x;
                nlv[v] = (x - (sum - bb)) + (y - bb);
                nv = sum;
            } else {
                nv = x + inc;
            }
            if (ADJ) {
                const TS lam = x;
                const TS ur = __ldcg(ua + j);
                dl[0] += (double)ur * (double)G;
                dl[1] += (double)ur * (double)H2[v];
                double pw = 1.0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    dl[2 + i] += (double)lam * pw;
                    pw *= (double)ur;
                }
            }
            bad |= !finite_(nv);
            nvv[v] = nv;
        }
        if (j0 + V <= I.N) {  // 16-byte stores where all V points exist
            store_vec<TS, V>(un + j0, nvv);
            if (lo_n) store_vec<TS, V>(lo_n + j0, nlv);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (j0 + v < I.N) {
                    un[j0 + v] = nvv[v];
                    if (lo_n) lo_n[j0 + v] = nlv[v];
                }
        }
        if (tp) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (j0 + v < I.N) tp[j0 + v] = nvv[v];
        }
        if (bad) atomicOr(L.nonfinite, 1u);
        if (ADJ) {
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dl[i] += __shfl_xor_sync(0xffffffffu, dl[i], o);
            if ((tid & 31) == 0)
#pragma unroll
                for (int i = 0; i < 6; ++i) s_dred[tid >> 5][i] = dl[i];
        }
        // history rows are read later by bulk copies (async proxy): order this thread's generic
        // stores before them, then publish the tile's step with one release store after the
        // CTA barrier (cumulative over all threads' stores)
        fence_proxy_async_global();
        __syncthreads();
        if (tid == 0) {
            if (ADJ) {
                double *dd = I.dots + (size_t)tile * 8;
                for (int i = 0; i < 6; ++i) {
                    double s = 0.0;
                    for (int w = 0; w < (nthr + 31) / 32; ++w) s += s_dred[w][i];
                    dd[i] += s;
                }
            }
            st_release(&I.done[tile], (unsigned)(rel + 1));
            if (!ADJ && I.cl_D) {  // off the step chain: nothing waits on these before the next steps' units
                double dm = 0.0, mm = 0.0;
                for (int w = 0; w < (nthr + 31) / 32; ++w) {
                    dm = fmax(dm, clmax[2 * w]);
                    mm = fmax(mm, clmax[2 * w + 1]);
                }
                atomicMax(reinterpret_cast<unsigned long long *>(I.cl_D + k), (unsigned long long)__double_as_longlong(dm));
                atomicMax(reinterpret_cast<unsigned long long *>(I.cl_M + k), (unsigned long long)__double_as_longlong(mm));
                if (tile == 0) atomicAdd(I.cl_terms, (unsigned long long)(1 + hh));  // lag 0 and the head lags
                // releases the maxima (row k done on this tile); the last tile acquires every
                // tile's, and decides step k + cl_lo, the first to read row k
                const unsigned old = atom_add_acq_rel(&I.cl_rows[k], 1u);
                const int kd = k + I.cl_lo;
                s_decide = (old + 1u == (unsigned)I.T && kd < I.ksteps) ? kd : -1;
            }
        }
        if (!ADJ && I.cl_D) {
            __syncthreads();
            const int kd = s_decide;
            if (kd >= 0) {
                // Step kd's decisions for the whole field, once: each median's expanded length
                // and, per chunk, the number of expanded medians (tallied in the stage ring, idle
                // between units; the host keeps a step's chunks within it).
                const int4 sc = I.sched[kd];
                const int hd = min(I.head, sc.x);
                const int n = sc.x + sc.y + (sc.w >= sc.z ? sc.w - sc.z + 1 : 0);
                const int Ck = max(1, (n - hd + I.R - 1) / I.R);
                int *tally = reinterpret_cast<int *>(stages);
                for (int c = tid; c < Ck; c += nthr) tally[c] = 0;
                __syncthreads();
                unsigned char *cnt = I.cl_cnt + (size_t)(kd % I.cl_slots) * I.cl_gmax;
                for (int g = tid; g < sc.y; g += nthr) {
                    const int d = I.g_d[g];
                    const int e = (d > 1 && !cl_smooth(I, kd, I.g_lag[g], d)) ? d : 0;
                    cnt[g] = (unsigned char)e;
                    if (e) atomicAdd(&tally[(sc.x + g - hd) / I.R], 1);
                }
                __syncthreads();
                if (tid == 0) {
                    __threadfence();  // every thread's lengths (behind the barrier) before the words
                    unsigned long long *word = I.cl_word + (size_t)(kd % I.cl_slots) * I.maxC;
                    const unsigned long long gen = (unsigned long long)(unsigned)(kd + 1) << 32;
                    for (int c = 0; c < Ck; ++c) st_relaxed_u64(word + c, gen | (unsigned)tally[c]);
                }
                // the ring's next writes come from bulk copies (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
            }
        }
    }
}

}  // namespace fdk

// fd_common.cuh -- what the per-step engine (fd_engine.cuh) and the temporally blocked engine
// (fd_engine_tb.cuh) share: the instance descriptor a launch reads (one per problem of eq.
// frac_final), the launch descriptor, the adjoint's tail-term table of adaptive memory, the PTX
// helpers (mbarriers, bulk copies, acquire / release words), the bounded waits and their error
// record, the history vector formats, the stencil's neighbour masks and the unit queue's group
// search.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdk {

enum { ERR_NONE = 0, ERR_TIMEOUT = 1, ERR_PIPE = 2 };

// One problem instance as the device sees it (copied to shared memory per unit).
struct Inst {
    int ndim, nx, ny, nz, bc;
    int N, T, P, R;          // points, tiles, points per tile, terms per chunk
    int hist_write;          // 0: history rows already hold delta (adjoint recompute pass)
    int cap;                 // history ring rows
    int maxC;                // partial rows per parity
    int npar;                // partial-row parities: steps k and k+npar share rows
    int stall;               // fault injection: first fixup waits on a counter nothing advances
    int head;                // lags 1..head are summed by the fixup from the head rows
    int hring_cap;           // rows in the head ring (== cap when it is the history itself)
    int hring_sep;           // 1: separate state-precision ring (low-precision history)
    int tb;                  // temporal block (steps per block) of the blocked kernel, else 0
    int mem_mode, mem_L;     // memory mode and short window (blocked kernel)
    int ksteps;              // steps the instance runs (its max_steps); bounds a batch launch
    int ub;                  // blocked kernel: 1 = one update unit per (block, tile)
    int cmax;                // blocked kernel: most far chunks per block (0 = no limit)
    int ralign;              // blocked kernel: far chunks start on multiples of ralign rows (0, 1: any)
    int near;                // blocked kernel: one near unit per (block, tile) adds the previous block's rows
    int ug;                  // blocked kernel: tiles per per-step update unit
    int mid;                 // blocked kernel: mid units per (block, tile): sub-blocks 1 .. mid of 16 steps
                             // get the block's earlier rows as one partial row
    int tc_cols;             // blocked tensor-core kernel: tensor-memory columns per CTA
    int tmap_rank;           // blocked tensor-core kernel: 3 = one box per stage, 2 = one per 64 points
    const void *tmap;        // blocked tensor-core kernel: tensor map of the history rows
    const void *tmap2;       // tensor-core near / mid units over 16-bit history: both planes, 16-row boxes
    int tmap2_rank;
    int lo_plane;            // the history has a lo plane cap rows after its rows (16-bit: fp16/bf16 of
                             // the rounding remainder), read by tensor-core near and mid units
    int tape_k0, tape_every, tape_rows;
    int adj_K, uadj_r0;      // adjoint: u^r is row (adj_K-1-k) - uadj_r0 of uadj
    double S, dt;
    double react[4];
    long long pitch;         // history row pitch (bytes, multiple of 256)
    long long part_pitch;    // partial row pitch (bytes)
    long long hring_pitch;   // head ring row pitch (bytes)
    char *hring;             // head rows in state precision (the history itself when TH == TS)
    char *hist;
    float *hscale;           // [cap][T] row-tile scales (FP16 history) or null
    char *ubuf[2];           // state double buffer: u^k lives in ubuf[k & 1]
    char *ulo[2];            // compensated state: low parts (null = plain state)
    char *part;              // [npar][maxC][planes] partial rows
    unsigned *arrive;        // [npar][T]
    unsigned *done;          // [T] steps completed by each tile in this launch
    const char *psi;         // weights in accumulator type
    const char *dpsi;        // d psi / d gamma (adjoint)
    const int4 *sched;       // per step: (nb, ng, tail_lo, tail_hi)
    const int *g_lag;        // adaptive medians (prefix-ordered)
    const char *g_coef;      // d * psi at the medians
    const char *gw;          // blocked kernel, adaptive memory: settled weight g(m) of every lag
    const int *br0;          // blocked kernel, adaptive memory: first far row of each block
    char *tape;              // optional u rows (checkpoints / recompute segment)
    const char *uadj;        // adjoint: forward states u^r
    double *dots;            // adjoint: [T][8] per-tile gradient partials
    const int *acorr_off;    // adjoint of adaptive memory: tail terms of row r at [off[r], off[r+1])
    const struct AdjTail *acorr;
    int acorr_rows;          // rows r = 0 .. acorr_rows-1 have tail terms
    // Closed-loop adaptive memory (per-step kernel; null = open loop).  Per history row r the
    // field-wide largest change from row r-1, D_r = max_j |delta^r_j - delta^{r-1}_j|, and largest
    // magnitude M_r = max_j |delta^r_j| (doubles, raised with integer atomics on their bits: for
    // non-negative doubles the order of the bits is the order of the values), and the tiles that
    // have added row r to them.  A median stands for its increment while
    // V = sum_{rows of the increment but its oldest} D / M_{k-m} < cl_tau, else the increment's
    // lags are summed one by one with weight psi.
    double *cl_D, *cl_M;
    unsigned *cl_rows;
    unsigned long long *cl_terms;  // memory terms used, lag 0 included (counted by tile 0)
    const int *g_d;                // increment length d of each median
    double cl_tau;
    int cl_lo;                     // smallest lag of any median's increment (the first one's)
    // Step k's decisions, made once for the field by the update that completes row k - cl_lo on
    // the last tile, in slot k % cl_slots (cl_slots = cl_lo: step k's units have all finished
    // when row k is complete, before step k + cl_slots is decided): per median its expanded
    // length (0 = it stands for its increment), per chunk one word (k + 1) << 32 | expanded
    // medians in the chunk, stored after the lengths with release semantics.
    unsigned char *cl_cnt;         // [cl_slots][cl_gmax]
    unsigned long long *cl_word;   // [cl_slots][maxC]
    int cl_slots, cl_gmax;
};

// Adjoint of adaptive memory.  The adjoint sums every (step k, lag m) pair with the weight g(m)
// that the medians settle on (Definitions 3.1/3.2: psi_m on the base interval, d psi_m at a
// median, 0 between), which is the forward weight of every lag up to the step's settled end e(k).
// A tail lag m > e(k) has forward weight psi_m instead; such a term reaches adjoint row r = k - m,
// and only rows below the longest tail have any.  Row r's list holds (k, psi_m - g(m),
// d/dgamma of the same), ascending in k.
struct AdjTail {
    int k, pad;
    double w, w2;
};

// Adds row r's tail terms to the adjoint memory sums H, H2 of adjoint step q (r = adj_K-1-q): the
// term of step k reads mu^{k+1}, the row of adjoint step adj_K-1-k, from the adjoint history.
// Eight rows in flight per thread.
template <class TS, class TA, int V>
__device__ __forceinline__ void adjoint_tail(const Inst &I, int q, int j0, TA *H, TA *H2)
{
    const int r = I.adj_K - 1 - q;
    if (!I.acorr || r < 0 || r >= I.acorr_rows || j0 >= I.N) return;
    const int e0 = I.acorr_off[r], e1 = I.acorr_off[r + 1];
    constexpr int G = 8;
    for (int e = e0; e < e1; e += G) {
        TS x[G][V];
        TA w[G], w2[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const bool on = e + i < e1 && I.acorr[e + i].k < I.adj_K;
            w[i] = on ? (TA)I.acorr[e + i].w : TA(0);
            w2[i] = on ? (TA)I.acorr[e + i].w2 : TA(0);
            const int row = on ? I.adj_K - 1 - I.acorr[e + i].k : 0;
            const TS *src = reinterpret_cast<const TS *>(I.hist + (size_t)(row % I.cap) * I.pitch) + j0;
#pragma unroll
            for (int v = 0; v < V; ++v) x[i][v] = (on && j0 + v < I.N) ? __ldcg(src + v) : TS(0);
        }
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                H[v] = fma(w[i], (TA)x[i][v], H[v]);
                H2[v] = fma(w2[i], (TA)x[i][v], H2[v]);
            }
    }
}

struct Launch {
    const Inst *inst;
    const long long *g_off;  // unit offset of each (instance, step) group, +1 sentinel
    const int2 *g_info;      // (instance, step) of each group
    int g_begin, g_end;
    int k0;                  // first step of the launch: tile step counters count from it
    int k_end;               // one past the last step of the launch (blocked kernel)
    int stage_rows, stages;
    int rmax;                // largest chunk (terms) over the launch's instances
    int smem_half;           // tensor-core kernels: dynamic shared memory of each half of a CTA
    int fsub;                // tensor-core kernels: far units per (chunk, tile), each of P/fsub points
    int nm_tc;               // tensor-core kernels: near and mid units on the tensor cores (one per sub-tile)
    unsigned long long *queue;
    int *err;
    unsigned *nonfinite;
    long long timeout_ns;
    long long *err_info;     // first wait that gave up: site code, operands, CTA (8 words) or null
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return static_cast<long long>(t);
}
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ int ld_volatile(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

// Bounded wait until *p >= need, with a sleep between polls that doubles up to max_sleep ns.
// Returns 1 when satisfied, 0 when another wait has already recorded an error, and -1 when
// this wait ran out of time (it then records FD_ERR_TIMEOUT).
__device__ __forceinline__ int wait_until(const unsigned *p, unsigned need, const Launch &L, unsigned max_sleep)
{
    if (ld_acquire(p) >= need) return 1;
    const long long t0 = globaltimer();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < max_sleep) ns <<= 1;
        if (ld_acquire(p) >= need) return 1;
        if (ld_volatile(L.err) != ERR_NONE) return 0;
        if (globaltimer() - t0 > L.timeout_ns) {
            atomicCAS(L.err, ERR_NONE, ERR_TIMEOUT);
            return -1;
        }
    }
}

// Bounded wait until the word's high half holds `gen`; returns the word (acquired), or 0 after the
// launch's error flag is set or the limit passes (which sets FD_ERR_TIMEOUT).
__device__ __forceinline__ unsigned long long wait_word(const unsigned long long *p, unsigned gen, const Launch &L)
{
    unsigned long long w = ld_acquire_u64(p);
    if ((unsigned)(w >> 32) == gen) return w;
    const long long t0 = globaltimer();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        w = ld_acquire_u64(p);
        if ((unsigned)(w >> 32) == gen) return w;
        if (ld_volatile(L.err) != ERR_NONE) return 0;
        if (globaltimer() - t0 > L.timeout_ns) {
            atomicCAS(L.err, ERR_NONE, ERR_TIMEOUT);
            return 0;
        }
    }
}

__device__ __forceinline__ bool wait_counter(const unsigned *p, unsigned need, const Launch &L)
{
    return wait_until(p, need, L, 512) > 0;
}

// Records the first wait that gave up: a site code, six operands and the CTA, for the host's
// error report.  Later failures (usually consequences of the first) leave it unchanged.
__device__ __forceinline__ void note_failure(const Launch &L, long long site, long long a, long long b, long long c,
                                             long long d, long long e, long long f)
{
    if (!L.err_info) return;
    if (atomicCAS(reinterpret_cast<unsigned long long *>(L.err_info), 0ull, (unsigned long long)site) != 0ull)
        return;
    L.err_info[1] = a;
    L.err_info[2] = b;
    L.err_info[3] = c;
    L.err_info[4] = d;
    L.err_info[5] = e;
    L.err_info[6] = f;
    L.err_info[7] = blockIdx.x;
    __threadfence();
}

// ------------------------------------------------------- history vector traits
template <class TH> struct HVec;
template <> struct HVec<double> {
    static constexpr int V = 2;
    template <class TA> __device__ static void unpack(uint4 w, TA *x)
    {
        x[0] = (TA)__hiloint2double((int)w.y, (int)w.x);
        x[1] = (TA)__hiloint2double((int)w.w, (int)w.z);
    }
    __device__ static uint4 pack(const double *d, float)
    {
        uint4 w;
        w.x = (unsigned)__double2loint(d[0]);
        w.y = (unsigned)__double2hiint(d[0]);
        w.z = (unsigned)__double2loint(d[1]);
        w.w = (unsigned)__double2hiint(d[1]);
        return w;
    }
};
template <> struct HVec<float> {
    static constexpr int V = 4;
    template <class TA> __device__ static void unpack(uint4 w, TA *x)
    {
        x[0] = (TA)__uint_as_float(w.x);
        x[1] = (TA)__uint_as_float(w.y);
        x[2] = (TA)__uint_as_float(w.z);
        x[3] = (TA)__uint_as_float(w.w);
    }
    template <class TS> __device__ static uint4 pack(const TS *d, float)
    {
        return make_uint4(__float_as_uint((float)d[0]), __float_as_uint((float)d[1]),
                          __float_as_uint((float)d[2]), __float_as_uint((float)d[3]));
    }
};
template <> struct HVec<__nv_bfloat16> {
    static constexpr int V = 8;
    template <class TA> __device__ static void unpack(uint4 w, TA *x)
    {
        const unsigned a[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = (TA)__uint_as_float(a[i] << 16);
            x[2 * i + 1] = (TA)__uint_as_float(a[i] & 0xffff0000u);
        }
    }
    template <class TS> __device__ static uint4 pack(const TS *d, float)
    {
        unsigned a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn((float)d[2 * i], (float)d[2 * i + 1]);
            a[i] = *reinterpret_cast<unsigned *>(&h);
        }
        return make_uint4(a[0], a[1], a[2], a[3]);
    }
};
template <> struct HVec<__half> {
    static constexpr int V = 8;
    template <class TA> __device__ static void unpack(uint4 w, TA *x)
    {
        const unsigned a[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = *reinterpret_cast<const __half2 *>(&a[i]);
            float2 f = __half22float2(h);
            x[2 * i] = (TA)f.x;
            x[2 * i + 1] = (TA)f.y;
        }
    }
    // scale = 2^e chosen per (row, tile) so the largest |delta| lands in [2^14, 2^15)
    template <class TS> __device__ static uint4 pack(const TS *d, float scale)
    {
        unsigned a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = __floats2half2_rn((float)d[2 * i] * scale, (float)d[2 * i + 1] * scale);
            a[i] = *reinterpret_cast<unsigned *>(&h);
        }
        return make_uint4(a[0], a[1], a[2], a[3]);
    }
};

template <class T> __device__ __forceinline__ bool finite_(T x) { return isfinite(x); }

// V consecutive state values (16-byte aligned groups), loaded bypassing L1 / stored.
template <class TS, int V> __device__ __forceinline__ void load_vec(const TS *p, TS *x)
{
    if constexpr (sizeof(TS) == 8) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
            const double2 w = __ldcg(reinterpret_cast<const double2 *>(p + i));
            x[i] = (TS)w.x;
            x[i + 1] = (TS)w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < V; i += 4) {
            const float4 w = __ldcg(reinterpret_cast<const float4 *>(p + i));
            x[i] = (TS)w.x;
            x[i + 1] = (TS)w.y;
            x[i + 2] = (TS)w.z;
            x[i + 3] = (TS)w.w;
        }
    }
}
template <class TS, int V> __device__ __forceinline__ void store_vec(TS *p, const TS *x)
{
    if constexpr (sizeof(TS) == 8) {
#pragma unroll
        for (int i = 0; i < V; i += 2)
            *reinterpret_cast<double2 *>(p + i) = make_double2((double)x[i], (double)x[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < V; i += 4)
            *reinterpret_cast<float4 *>(p + i) =
                make_float4((float)x[i], (float)x[i + 1], (float)x[i + 2], (float)x[i + 3]);
    }
}

// Unit descriptor broadcast from thread 0.

// Neighbour masks of the V consecutive points j0 .. j0+V-1: bit e set when neighbour e (+x, -x,
// +y, -y, +z, -z) lies inside the grid.  One division of j0, then a running (x, y, z).
template <int V> __device__ __forceinline__ void grid_masks(const Inst &I, int j0, unsigned *inb)
{
    int x = j0 % I.nx;
    const int r = j0 / I.nx;
    int y = (I.ndim >= 2) ? r % I.ny : 0, z = (I.ndim == 3) ? r / I.ny : 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const bool in = j0 + v < I.N;
        unsigned m = 0;
        if (in && x + 1 < I.nx) m |= 1u;
        if (in && x > 0) m |= 2u;
        if (in && I.ndim >= 2 && y + 1 < I.ny) m |= 4u;
        if (in && I.ndim >= 2 && y > 0) m |= 8u;
        if (in && I.ndim == 3 && z + 1 < I.nz) m |= 16u;
        if (in && I.ndim == 3 && z > 0) m |= 32u;
        inb[v] = m;
        if (++x == I.nx) {
            x = 0;
            if (++y == I.ny) {
                y = 0;
                ++z;
            }
        }
    }
}

__device__ __forceinline__ int find_group(const long long *off, int g, int g_end, long long u)
{
    if (u < off[g + 1]) return g;
    int lo = g + 1, step = 1, hi = lo + 1;
    while (hi < g_end && off[hi] <= u) {
        lo = hi;
        step <<= 1;
        hi = lo + step;
    }
    if (hi > g_end) hi = g_end;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace fdk
